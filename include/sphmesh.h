/*
 * sphmesh.h -- C ABI of the GB300 feature-aware SPH relaxation library (libsphmesh.so).
 *
 * The library evolves mesh-vertex particles of every feature type (singular points, feature
 * curves, feature surfaces, volume) concurrently under the SPH pressure-like interaction
 * forces of Ji, Fu, Hu and Adams, "A Feature-aware SPH for Isotropic Unstructured Mesh
 * Generation" (arXiv 2003.01061), towards a target feature-size field h_t(x), driven by the
 * paper's two-phase controller.  All per-step work runs in the library's own CUDA kernels on
 * one GPU; the host only marshals descriptors and copies states in and out.
 *
 * Conventions shared by every entry point
 *  - Every function returns sph_status and never aborts or exits.  On failure
 *    sph_last_error() returns a message describing the most recent failure of the calling
 *    thread.  Inputs that fail validation give SPH_E_INVALID and change no state.
 *  - Positions, velocities and normals are arrays of 3 doubles per particle in host memory,
 *    row-major [n][3]; in 2D the third entry is ignored on input and written as 0.
 *  - "Original order" is the order of the particles passed to sph_mesh_set_state; every
 *    per-particle output is returned in that order.
 *  - The library never keeps caller pointers past the call.  Device memory is owned by the
 *    handle and released by sph_mesh_destroy.
 *  - Work is enqueued on the handle's CUDA stream (the one passed to sph_mesh_create, or a
 *    stream the library created).  Functions that return host data synchronise that stream.
 *  - A handle may be used by one thread at a time.
 */
#ifndef SPHMESH_H
#define SPHMESH_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPH_OK = 0,
    SPH_E_INVALID = 1,        /* a descriptor, size or pointer failed validation            */
    SPH_E_NOMEM = 2,          /* device or host allocation failed                            */
    SPH_E_CUDA = 3,           /* a CUDA call failed (the message names it)                   */
    SPH_E_DIVERGED = 4,       /* a non-finite acceleration or position was detected          */
    SPH_E_NOT_CONVERGED = 5,  /* run_until_converged reached max_iters; the state is valid   */
    SPH_E_OVERFLOW = 6        /* a particle left the cell grid or a debug buffer was short   */
} sph_status;

#define SPH_MAX_FEATURES 64
#define SPH_MAX_HOLES 8
#define SPH_MAX_LEVELS 8

/* Feature kinds (Sec. 3.2, "feature definition"): particles carry the type and index of the
 * feature they belong to.  The intrinsic dimension d of each kind is given in brackets. */
typedef enum {
    SPH_FEAT_VOLUME = 0,   /* [D] the positive phase phi > 0 of the level set (Eq. 1)          */
    SPH_FEAT_POINT = 1,    /* [0] singularity point; its particle never moves                  */
    SPH_FEAT_SEGMENT = 2,  /* [1] straight feature curve from geom[0..2] to geom[3..5]         */
    SPH_FEAT_CIRCLE = 3,   /* [1] 2D circle, centre geom[0..1], radius geom[2]                  */
    SPH_FEAT_RECT = 4,     /* [2] 3D planar face: origin geom[0..2], unit axes geom[3..5] and
                                  geom[6..8], extents geom[9], geom[10]                         */
    SPH_FEAT_SPHERE = 5    /* [2] 3D sphere surface, centre geom[0..2], radius geom[3]          */
} sph_feature_kind;

typedef struct {
    int32_t kind;        /* sph_feature_kind                                                   */
    int32_t dim;         /* intrinsic dimension (0..3); must match the kind (VOLUME: D)        */
    double geom[12];     /* geometry, see sph_feature_kind                                     */
    double normal[3];    /* POINT, SEGMENT, RECT: unit outward normal of the domain at the
                            feature (edges and corners: bisector of the incident faces).  It is
                            the n_b of the boundary term of Eq. 19 when this feature's particles
                            act as boundary particles.                                         */
    double orient;       /* CIRCLE, SPHERE: +1 when the domain is inside (outer boundary),
                            -1 when it is outside (a hole)                                     */
} sph_feature;

/* The domain (Sec. 2.1, Sec. 3.1): phi > 0 is the volume.  phi is given analytically as a box
 * (base 0, the bounding box itself) or a ball (base 1) minus up to SPH_MAX_HOLES balls. */
typedef struct {
    int32_t dim;                       /* ambient dimension D: 2 or 3                          */
    int32_t base;                      /* 0: box [bbox_lo, bbox_hi]; 1: ball (ball_center, r)  */
    double bbox_lo[3], bbox_hi[3];     /* bounding box of every particle position              */
    double ball_center[3];
    double ball_radius;
    int32_t n_holes;
    double hole_center[SPH_MAX_HOLES][3];
    double hole_radius[SPH_MAX_HOLES];
    int32_t n_features;                /* 1..SPH_MAX_FEATURES; a particle's group = its index  */
    sph_feature features[SPH_MAX_FEATURES];
} sph_domain_desc;

/* Target feature size h_t(x) (Eq. 2, rho_t = h_t^-d), analytic:
 *   kind 0 CONST:      h = a
 *   kind 1 HOLE_DIST:  h = clamp(a + b * min_k | |x - ref_center_k| - ref_radius_k |, lo, hi)
 *   kind 2 RADIAL:     h = clamp(a + b * |x - center|, lo, hi)      (the form of Eqs. 25-28)
 * lo and hi must bound h everywhere (they size the cell grid). */
typedef struct {
    int32_t kind;
    double a, b, lo, hi;
    double center[3];
    int32_t n_ref;
    double ref_center[SPH_MAX_HOLES][3];
    double ref_radius[SPH_MAX_HOLES];
} sph_sizing_desc;

/* Method parameters.  Defaults in brackets are the paper's (see each field). */
typedef struct {
    double kappa;          /* support radius r_c = kappa*h of the Wendland C2 kernel, h the
                              target size (the paper leaves r_c/h open: 2.6 = twice a
                              smoothing length of 1.3 h)                                  [2.6]*/
    double p0;             /* EOS constant P0, Eq. 6                                     [1]  */
    double visc;           /* nu = visc * r_c * |v|, Eq. 8; 0 disables viscosity         [0.1]*/
    double cfl_a;          /* Eq. 24 acceleration constant                               [0.25]*/
    double cfl_v;          /* Eq. 24 velocity constant                                   [1/40]*/
    double eps1;           /* Phase-One damping epsilon, Eq. 23 (paper: 0..0.2)          [0]  */
    double dt_cap;         /* step size of a group with no acceleration and no velocity  [1e30]*/
    double dt_collapse;    /* nullify velocities when dt drops below this factor of the
                              previous step (Sec. 3.4.3: "an order of magnitude")         [0.1]*/
    double threshold;      /* E_sys threshold of Sec. 3.4.2                              [5e-6]*/
    int32_t reset_period;  /* Phase-One nullification period, Sec. 3.4.3                 [100]*/
    int32_t sample_every;  /* steps between samples of V-bar, Sec. 3.4.2                 [20] */
    int32_t window;        /* samples per averaging window, Sec. 3.4.2                   [10] */
    int32_t ramp_len;      /* steps of the Phase-One -> Phase-Two transition, Sec. 3.4.4 [200]*/
    int32_t boundary_rho;  /* 1: boundary sum of Eq. 19 carries rho_b (units-consistent);
                              0: the sum exactly as printed                              [1]  */
    int32_t precision;     /* 32: FP32 pair sums (FP64 projection and reductions);
                              64: FP64 everywhere                                         [32] */
    int32_t cells_per_support;  /* cell grid refinement m (see sph_grid_spec): 1, 2 or 4;
                              0: the library's choice for the dimension (not a paper
                              parameter; it changes no result beyond rounding)          [0]  */
    int32_t boundary_correction;  /* 1: the feature-boundary sum of Eq. 19 (this paper's
                              correction, Sec. 3.2) acts on every particle; 0: it is left out,
                              as in the earlier method compared in Sec. 4.1              [1]  */
    int32_t group_convergence;  /* 0: the instance changes phase when E_sys (the largest
                              group error) passes the threshold (Sec. 3.4.2); 1: every group
                              runs its own phases on its own error and stops moving once it
                              has converged (Algorithm 1 skips a converged feature); the
                              instance is then in the phase of its least advanced group   [0]  */
    int32_t feature_order;  /* 0: every group reads the state at the start of the step (the
                              data-parallel reading of Algorithm 1's feature loop); 1: the loop
                              in sequence: a step advances the curves, then the surfaces, then
                              the volume, each reading the positions the lower-dimensional
                              features reached in the step (they act on it through Eq. 19).
                              Requires group_convergence = 1 (the loop checks each feature's
                              own convergence)                                             [0]  */
} sph_params;

/* Method presets of the comparison in Sec. 4.1 (Square, its table of N_iter): the improved
 * method of this paper, the earlier SPH mesh generator it is compared with (velocities set to
 * zero every step, no feature-boundary correction) and that method's variant "v2" (velocities
 * set to zero every 100 steps, as in the improved method). */
typedef enum { SPH_METHOD_IMPROVED = 0, SPH_METHOD_FU2019 = 1, SPH_METHOD_FU2019_V2 = 2 } sph_method;

/* Controller phases (Sec. 3.4) */
typedef enum { SPH_PHASE1 = 1, SPH_RAMP = 2, SPH_PHASE2 = 3, SPH_DONE = 4 } sph_phase;

typedef struct {
    int32_t phase;                     /* sph_phase                                           */
    int32_t n_groups;
    int64_t iteration;                 /* completed steps                                      */
    int64_t ramp_start;                /* step at which Phase One ended (RAMP began)           */
    int64_t escapes;                   /* volume particles moved back inside the domain        */
    uint32_t status;                   /* bit 0: non-finite value seen; bit 1: particle outside
                                          the cell grid; bit 2: h outside [lo, hi]; bit 3: the
                                          cell scan gave up waiting (internal error)           */
    uint32_t pad;
    double E_t, E_avg, E_sys;          /* convergence errors of the last evaluated sample       */
    double vbar[SPH_MAX_FEATURES];     /* last sampled V-bar per group (Eq. 22, V_ref = 1)     */
    double dt[SPH_MAX_FEATURES];       /* step size of each group in the last step (Eq. 24)    */
    int32_t reset[SPH_MAX_FEATURES];   /* 1 if the group's velocities were nullified            */
    int32_t group_phase[SPH_MAX_FEATURES];  /* each group's phase (the instance's unless
                                          group_convergence = 1)                               */
    double group_E[SPH_MAX_FEATURES];  /* each group's last error E_g (group_convergence = 1)  */
} sph_report;

typedef struct sph_mesh sph_mesh;

/* Creates a relaxation instance: checks the descriptors, derives the cell grid from the
 * bounding box and [sizing.lo, sizing.hi] and allocates device memory for up to
 * max_particles particles.  stream: a cudaStream_t to enqueue work on, or NULL for a stream
 * owned by the library.  Problem statement: Sec. 2.1-2.2 and Sec. 3.1-3.2 (geometry, target
 * feature size, feature tags).  Errors: SPH_E_INVALID, SPH_E_NOMEM, SPH_E_CUDA. */
sph_status sph_mesh_create(const sph_domain_desc* domain, const sph_sizing_desc* sizing,
                           const sph_params* params, int64_t max_particles, void* stream,
                           sph_mesh** out);

/* Fills params with the paper's defaults (bracketed values above). */
sph_status sph_params_default(sph_params* params);

/* Sets the fields that distinguish the methods of Sec. 4.1 (reset_period and
 * boundary_correction) for method (a sph_method) and leaves every other field as it is:
 * IMPROVED 100 / 1, FU2019 1 / 0, FU2019_V2 100 / 0.  The controller and the step size
 * rules are the same for all three.  Errors: SPH_E_INVALID (NULL params, unknown method). */
sph_status sph_params_preset(sph_params* params, int32_t method);

/* Loads a particle set (Algorithm 1, "allocate particles ... initial particle sampling") and
 * resets the controller to Phase One, step 0.  x: [n][3] positions; group: feature index of
 * each particle; v: [n][3] velocities or NULL for zero; h: per-particle smoothing length or
 * NULL for h_t(x).  Positions must lie inside the bounding box and h in (0, hi*(1+2^-11)].
 * The host arrays (pinned or pageable; pinned ones are copied fastest) are copied as they are
 * into a device staging buffer, allocated on the first call and grown when a larger set
 * comes, then checked and converted on the device; a rejected set leaves the loaded state as
 * it was, and the message names the first offending particle (its checks taken in the order
 * group, position, h, velocity).  Errors: SPH_E_INVALID (n > max_particles, bad group,
 * position or h out of range, non-finite velocity), SPH_E_NOMEM (staging buffer). */
sph_status sph_mesh_set_state(sph_mesh* m, int64_t n, const double* x, const int32_t* group,
                              const double* v, const double* h);

/* ---- initial particles on the device (Sec. 3.6; Algorithm 1: "calculate the target
 * information (Eqs. 10, 11)", "allocate particles ... initial particle sampling") ---- */

/* Quadrature points of the target counts: the midpoint rule on a grid of SPH_QUAD_AREA^2 (2D) or
 * SPH_QUAD_VOLUME^3 (3D) cells of the bounding box (cells whose centre has phi > 0 count),
 * SPH_QUAD_CURVE points per curve, SPH_QUAD_FACE^2 per face, SPH_QUAD_SPHERE x 2 SPH_QUAD_SPHERE
 * (polar x azimuthal) per sphere. */
#define SPH_QUAD_AREA 2048
#define SPH_QUAD_VOLUME 256
#define SPH_QUAD_CURVE 65536
#define SPH_QUAD_FACE 1024
#define SPH_QUAD_SPHERE 512

/* Target particle count of every feature: N_k = the integral of rho_t = h_t^-d over feature k
 * (Eqs. 10, 11) with the quadrature above, computed on the device of `stream` (a point feature:
 * 1).  integral_out[k] (may be NULL) receives the integral, count_out[k] (may be NULL) its
 * nearest integer; both hold domain->n_features entries.  Errors: SPH_E_INVALID (descriptors,
 * as for sph_mesh_create; no output), SPH_E_CUDA. */
sph_status sph_feature_counts(const sph_domain_desc* domain, const sph_sizing_desc* sizing, void* stream,
                              double* integral_out, int64_t* count_out);

/* Draws counts[k] particles on every feature k with probability proportional to rho_t (Sec.
 * 3.6), on the device of `stream`, by rejection: candidate c of feature k takes the four words of
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011) for counter (c, c >> 32, k, 0) and key
 * (seed, seed >> 32) as uniforms u = (w + 1/2) 2^-32 and is accepted with probability
 * (h_min / h_t(x))^d, h_min = sizing->lo; a volume candidate is uniform in the bounding box and
 * also needs phi(x) > h_t(x)/4, a curve candidate is uniform along the segment or (circle) in
 * angle, a face candidate uniform on the face at least h_t(x)/4 inside its edges, a sphere
 * candidate uniform in direction; a point feature gives its point (counts[k] <= 1).  Feature k
 * keeps its first counts[k] accepted candidates in candidate order, so the result is a
 * function of (problem, seed, counts) alone.  Caller-owned host outputs: x_out
 * [sum counts][3] and group_out [sum counts] in feature order.  Errors: SPH_E_INVALID
 * (descriptors; negative counts; a feature whose acceptance is too small to reach its count
 * within 2^36 candidates), SPH_E_CUDA. */
sph_status sph_sample_particles(const sph_domain_desc* domain, const sph_sizing_desc* sizing, uint64_t seed,
                                const int64_t* counts, void* stream, double* x_out, int32_t* group_out);

/* sph_feature_counts + sph_sample_particles for the mesh's problem on its stream, then the
 * particles are loaded as by sph_mesh_set_state (v = 0, h = h_t(x)).  n_out (may be NULL)
 * receives the particle count.  Errors: SPH_E_NOMEM (more particles than max_particles), and
 * those of the two calls. */
sph_status sph_mesh_sample(sph_mesh* m, uint64_t seed, int64_t* n_out);

/* Enqueues n_steps relaxation steps (Algorithm 1, one pass of the while loop each: cell-list
 * rebuild, pressure pass with the feature-boundary correction of Eq. 19, per-group step size
 * of Eq. 24 and the two-phase controller of Sec. 3.4, viscous pass, update and projection).
 * Returns without waiting for the GPU.  The step sequence is captured once into a CUDA
 * graph.  Errors: SPH_E_CUDA. */
sph_status sph_mesh_step(sph_mesh* m, int32_t n_steps);

/* Waits for all work enqueued on the handle and checks the device status word.
 * Errors: SPH_E_CUDA, SPH_E_DIVERGED (non-finite value), SPH_E_OVERFLOW (left the grid). */
sph_status sph_mesh_sync(sph_mesh* m);

/* Steps until the controller reports the end of Phase Two (Sec. 3.4: Phase One until E_sys
 * falls below the threshold, transition, Phase Two until the criterion holds again) or until
 * max_iters steps have run.  iters_out (may be NULL) receives the completed step count.
 * Errors: SPH_E_NOT_CONVERGED when max_iters was reached, plus those of sph_mesh_sync. */
sph_status sph_mesh_run_until_converged(sph_mesh* m, int64_t max_iters, int64_t* iters_out);

/* Copies the current state to host buffers in original order (any pointer may be NULL):
 * x_out [n][3], group_out [n], v_out [n][3], h_out [n].  capacity is the number of particles
 * the buffers hold.  The outputs are assembled in input order on the device (FP64 positions
 * origin + cell c0 + offset) in the staging buffer of sph_mesh_set_state, then copied out one
 * array each.  Errors: SPH_E_INVALID (capacity < n), SPH_E_NOMEM (staging buffer). */
sph_status sph_mesh_positions(sph_mesh* m, double* x_out, int32_t* group_out, double* v_out,
                              double* h_out, int64_t capacity, int64_t* n_out);

/* Copies the controller state (Sec. 3.4) and the device status word. */
sph_status sph_mesh_report(sph_mesh* m, sph_report* out);

/* Checkpoint and resume.  sph_mesh_snapshot writes the state into buf: the particles exactly
 * as stored on the device (cell, offset, velocity, h, feature tag, input index, in the order
 * of the last sort), the controller (Sec. 3.4) and a fingerprint of the problem and its grid.
 * With buf NULL (or cap too small: SPH_E_OVERFLOW) it only stores the size needed in *used.
 * sph_mesh_restore loads such a snapshot into a handle of the same problem (same descriptors,
 * same cells per support, same precision; SPH_E_INVALID otherwise) with room for its
 * particles; the run then continues bit for bit as if it had not been interrupted.  The
 * format is the host's native byte order.  Both wait for the handle's stream. */
sph_status sph_mesh_snapshot(sph_mesh* m, void* buf, size_t cap, size_t* used);
sph_status sph_mesh_restore(sph_mesh* m, const void* buf, size_t len);

/* Releases the handle and its device memory.  NULL is ignored. */
void sph_mesh_destroy(sph_mesh* m);

/* Message of the last failure on the calling thread ("" if none). */
const char* sph_last_error(void);

/* ------------------------------------------------------------------------------------------
 * Cell grid (Algorithm 1, "update the multi-level data structure").  Pure host function.
 * Level l has cubic cells of edge c0 * 2^l; a particle goes to the first level whose
 * threshold thr[l] is >= its h.  Keys number the cells of all levels consecutively
 * (row-major within a level, x fastest).  With m = cells_per_support (1, 2 or 4: a level's
 * cell edge is 1/m of the largest support it holds; smaller cells visit fewer candidates and
 * more cell rows), the specification is:
 *   c0 = kappa*h_lo*(1+2^-10)/m rounded up to float; L = the least count with
 *   m*c0*2^(L-1) >= kappa*h_hi*(1+2^-10) (at most SPH_MAX_LEVELS); thr[l] = m*c0*2^l /
 *   (kappa*(1+2^-10)) rounded down to float for l < L-1, +inf for the top level;
 *   with M = m*c0*2^(L-1): origin = bbox_lo - M rounded down to float; dims[l] =
 *   ceil((bbox_hi + M - origin) / (c0*2^l)) + 1 per axis (1 for unused axes).
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    int32_t dim, levels;
    int32_t cells_per_support;
    float c0;
    float origin[3];
    float thr[SPH_MAX_LEVELS];
    int64_t dims[SPH_MAX_LEVELS][3];
    int64_t base[SPH_MAX_LEVELS];
    int64_t n_cells;
} sph_grid_info;

sph_status sph_grid_spec(int32_t dim, const double* bbox_lo, const double* bbox_hi, double h_lo,
                         double h_hi, double kappa, int32_t cells_per_support, sph_grid_info* out);
sph_status sph_mesh_grid(const sph_mesh* m, sph_grid_info* out);

/* ------------------------------------------------------------------------------------------
 * Inspection entry points, for parity checks.  Each runs parts of one step on the GPU on
 * the current state without advancing it (the controller state is left untouched).
 * ------------------------------------------------------------------------------------------ */

/* Rebuilds the cell lists of the current state (Algorithm 1, Verlet list construction by
 * cell key + stable counting sort).  key_out [n]: cell key of each particle in the order the
 * state is currently stored (right after set_state that is the original order);
 * cell_start_out [n_cells + 1]: first sorted slot of every cell; perm_out [n]: for every
 * sorted slot, the index of the particle in the stored order.  Any pointer may be NULL. */
sph_status sph_debug_rebuild(sph_mesh* m, int64_t* key_out, int64_t* cell_start_out,
                             int64_t* perm_out);

/* Neighbour sets seen by the pair sums, for every particle in original order.
 * mode 0: all j != i with |x_i - x_j| < kappa*(h_i+h_j)/2, any group (Eq. 7, Eq. 19);
 * mode 1: all j (i included) with |x_i - x_j| < kappa*h_i, any group (Eq. 18, Eq. 20).
 * counts_out [n]; lists_out receives the concatenated lists (original indices, ascending)
 * for particles in original order, up to list_capacity entries; total_out the total.
 * Errors: SPH_E_OVERFLOW when list_capacity < total (counts are still complete). */
sph_status sph_debug_neighbors(sph_mesh* m, int32_t mode, int64_t* counts_out, int32_t* lists_out,
                               int64_t list_capacity, int64_t* total_out);

/* Pressure pass of the current state (Eqs. 18-20, Eq. 24), per particle in original order:
 * a_p [n][3] (Eq. 19 after the map onto the feature), sigma [n] (kernel sum of Eq. 20),
 * gamma [n] (Eq. 18), and per group dta/dtv [n_groups] (the minima of 0.25 sqrt(r_c/|a|) and
 * r_c/(40|v|) of Eq. 24).  Any pointer may be NULL. */
sph_status sph_debug_interact(sph_mesh* m, double* a_p, double* sigma, double* gamma, double* dta,
                              double* dtv);

/* One full update of the current state with the step parameters given explicitly instead of
 * the controller's: per group dt[g] and reset[g] (velocity nullification), damping eps and
 * velocity attenuation f (Algorithm 1: mid-point velocity, viscous force, update, map).
 * Outputs in original order: x_out [n][3], v_out [n][3], h_out [n], a_v [n][3] (the viscous
 * acceleration after the map).  The stored state is NOT changed.  Any pointer may be NULL. */
sph_status sph_debug_update(sph_mesh* m, const double* dt, const int32_t* reset, double eps,
                            double f, double* x_out, double* v_out, double* h_out, double* a_v);

/* Per-kernel timing.  When enabled, sph_mesh_step records CUDA events around every kernel
 * launch; sph_mesh_kernel_times returns, for each kernel name, the launch count and the
 * summed device time in milliseconds since timing was enabled (up to cap entries). */
typedef struct {
    char name[32];
    int64_t launches;
    double total_ms;
} sph_kernel_time;

sph_status sph_mesh_set_timing(sph_mesh* m, int32_t enable);
sph_status sph_mesh_kernel_times(sph_mesh* m, sph_kernel_time* out, int32_t cap, int32_t* n_out);

/* Pair statistics of the current state's neighbour search (for the FLOP account): number of
 * candidate pairs visited and pairs inside the support, over one pressure pass. */
sph_status sph_debug_pair_counts(sph_mesh* m, int64_t* candidates, int64_t* accepted);

/* ------------------------------------------------------------------------------------------
 * Batches: many independent relaxation problems advanced together.  Every problem ("instance")
 * runs Algorithm 1 with its own domain, sizing, parameters and two-phase controller (Sec. 3.4),
 * exactly as a sph_mesh would; the batch packs all instances into one particle array and one
 * cell-key range so that each kernel of a step serves every instance in one launch.  This is
 * how small problems fill the GPU (the paper relaxes one problem at a time).
 *
 * All instances of a batch share the ambient dimension and the precision.  The batch allocates
 * particle slots for the sum of the max_particles given at creation (each rounded up to
 * SPH_SLOT_CHUNK); any instance may hold any count as long as the loaded instances' counts, each
 * rounded up to SPH_SLOT_CHUNK, fit that total.  Loaded instances occupy consecutive slot
 * ranges; loading or emptying one moves the others on the device and makes the next step
 * re-capture its graph.  A freshly
 * created instance is empty and idle (controller DONE).  An empty instance costs nothing per
 * step; a converged (DONE) one costs a pass over its slots and no pair work.  Instance results
 * do not depend on the other instances of the batch: a particle only interacts with particles
 * of its own instance, and every sum runs in the same order as for the instance alone.
 * Indices `inst` run from 0 to n_inst-1; out-of-range indices give SPH_E_INVALID.
 * ------------------------------------------------------------------------------------------ */
#define SPH_MAX_INSTANCES 4096
#ifndef SPH_SLOT_CHUNK
#define SPH_SLOT_CHUNK 128   /* an instance's slots are its particle count rounded up to this */
#endif
typedef struct sph_batch sph_batch;

/* Creates a batch of n_inst instances; domains, sizings, params and max_particles are arrays of
 * n_inst entries, validated as by sph_mesh_create.  stream as for sph_mesh_create.
 * Errors: SPH_E_INVALID (a descriptor, mixed dims or precisions, too many cells or slots in
 * total), SPH_E_NOMEM, SPH_E_CUDA. */
sph_status sph_batch_create(int32_t n_inst, const sph_domain_desc* domains, const sph_sizing_desc* sizings,
                            const sph_params* params, const int64_t* max_particles, void* stream,
                            sph_batch** out);

/* Number of instances, particle slots in use (the work of one step is proportional to it) and
 * slots allocated.  Any pointer may be NULL. */
sph_status sph_batch_size(const sph_batch* b, int32_t* n_inst, int64_t* n_slots, int64_t* slot_capacity);

/* Replaces the problem of instance inst (domain, sizing, parameters; same dim and precision)
 * and leaves it empty and idle.  Waits for the batch's stream.  The other instances keep their
 * state. */
sph_status sph_batch_set_problem(sph_batch* b, int32_t inst, const sph_domain_desc* domain,
                                 const sph_sizing_desc* sizing, const sph_params* params);

/* sph_mesh_set_state for instance inst: loads its particles and resets its controller to
 * Phase One, step 0; n = 0 empties the instance (controller DONE).  Waits for the batch's
 * stream.  The other instances keep their state.  Errors: those of sph_mesh_set_state, and
 * SPH_E_NOMEM when the loaded instances would not fit the batch's slots (nothing changes). */
sph_status sph_batch_set_state(sph_batch* b, int32_t inst, int64_t n, const double* x,
                               const int32_t* group, const double* v, const double* h);

/* Enqueues n_steps steps of every instance (idle and DONE instances stay frozen). */
sph_status sph_batch_step(sph_batch* b, int32_t n_steps);

/* Waits for the batch's stream and checks every instance's status word; the first instance
 * with a problem names itself in the message.  Errors as for sph_mesh_sync. */
sph_status sph_batch_sync(sph_batch* b);

/* Steps until every loaded instance is DONE or has run max_iters steps (checking every
 * sample_every steps); iters_out receives the largest step count.  Errors as for
 * sph_mesh_run_until_converged (SPH_E_NOT_CONVERGED names the first unfinished instance). */
sph_status sph_batch_run_until_converged(sph_batch* b, int64_t max_iters, int64_t* iters_out);

/* sph_mesh_positions for instance inst (original order of its last sph_batch_set_state). */
sph_status sph_batch_positions(sph_batch* b, int32_t inst, double* x_out, int32_t* group_out,
                               double* v_out, double* h_out, int64_t capacity, int64_t* n_out);

/* Controller reports of all instances (out: cap >= n_inst entries), from one device copy. */
sph_status sph_batch_reports(sph_batch* b, sph_report* out, int32_t cap);

/* Per-stage timing over the whole batch, as sph_mesh_set_timing / sph_mesh_kernel_times. */
sph_status sph_batch_set_timing(sph_batch* b, int32_t enable);
sph_status sph_batch_kernel_times(sph_batch* b, sph_kernel_time* out, int32_t cap, int32_t* n_out);

/* sph_mesh_snapshot / sph_mesh_restore for instance inst. */
sph_status sph_batch_snapshot(sph_batch* b, int32_t inst, void* buf, size_t cap, size_t* used);
sph_status sph_batch_restore(sph_batch* b, int32_t inst, const void* buf, size_t len);

/* Cell-size autotuning: runs trial_steps steps (after two untimed ones) of the loaded state
 * with 1, 2 and 4 cells per support (see sph_grid_spec), keeps the fastest for every instance,
 * and leaves the batch holding the state it had before the call -- re-represented on the
 * chosen grid, so later results change only by rounding -- with the controllers as they were.
 * cells_per_support receives the choice; trial_ms (3 entries, may be NULL) the trial times in
 * milliseconds (-1: that grid was not possible, e.g. too many cells).  Waits for the stream.
 * Errors: SPH_E_INVALID (nothing loaded), SPH_E_NOMEM, SPH_E_CUDA. */
sph_status sph_batch_autotune(sph_batch* b, int32_t trial_steps, int32_t* cells_per_support, float* trial_ms);

/* Releases the batch and its device memory.  NULL is ignored. */
void sph_batch_destroy(sph_batch* b);

/* Device bytes per particle slot of a batch of the given dimension and precision (the
 * per-cell arrays, which grow with the loaded problems' grids, come on top).  For sizing a
 * batch or a server from the free device memory. */
sph_status sph_batch_slot_bytes(int32_t dim, int32_t precision, int64_t* bytes_per_slot);

/* ------------------------------------------------------------------------------------------
 * Serving: a continuous-batching request loop over two batches (2D and 3D jobs, on two CUDA
 * streams so that their steps overlap).  The paper has no counterpart (it relaxes one problem
 * at a time).  A job is a problem (domain, sizing, parameters) with its initial particles and
 * an iteration limit.  sph_server_poll runs one scheduling round:
 *   1. retire every resident job whose controller is DONE (SPH_JOB_DONE), whose iteration count
 *      reached its max_iters (SPH_JOB_NOT_CONVERGED) or whose status word shows a non-finite
 *      value or a particle outside the grid (SPH_JOB_FAILED): its particles are copied to host
 *      memory and its instance and slots are freed;
 *   2. admit queued jobs in arrival order while an instance is free and the job's particles
 *      (rounded up to SPH_SLOT_CHUNK) fit the free slots -- a job that does not fit waits, later smaller
 *      jobs may pass it;
 *   3. advance every resident job by steps_per_poll steps and wait for them.
 * A job's result does not depend on the other jobs resident with it: it equals the result of
 * the same problem run alone through sph_mesh_run_until_converged with the same limit, as long
 * as steps_per_poll divides the number of steps the job needs (otherwise the job runs up to
 * steps_per_poll - 1 steps past its end, with its state frozen once it is DONE).
 * Times are seconds since sph_server_create (host steady clock).
 * ------------------------------------------------------------------------------------------ */
typedef struct sph_server sph_server;

typedef enum {
    SPH_JOB_QUEUED = 1,
    SPH_JOB_RUNNING = 2,
    SPH_JOB_DONE = 3,           /* both phases finished (Sec. 3.4)                              */
    SPH_JOB_NOT_CONVERGED = 4,  /* max_iters reached first; the result is the state at that step */
    SPH_JOB_FAILED = 5          /* non-finite value or particle outside the grid; or admission
                                   failed for a reason other than memory                       */
} sph_job_state;

typedef struct {
    int32_t precision;          /* 32 or 64, for every job                                       */
    int32_t max_jobs;           /* resident jobs per dimension (1..SPH_MAX_INSTANCES)            */
    int64_t slot_capacity[2];   /* particle slots for 2D and 3D jobs (0: no jobs of that
                                   dimension; -1: hbm_fraction of the free device memory,
                                   shared by the dimensions asking for it)                     */
    double hbm_fraction;        /* used with slot_capacity -1, in (0, 1)                         */
    int32_t steps_per_poll;     /* steps per scheduling round (20 = the paper's sample period)   */
} sph_server_config;

typedef struct {
    int32_t state;              /* sph_job_state                                                 */
    int32_t dim;
    int64_t n;                  /* particles                                                     */
    int64_t iterations;         /* steps run (at retirement)                                     */
    int32_t phase;              /* controller phase at retirement                                */
    uint32_t status_word;       /* device status word at retirement (sph_report.status)         */
    int64_t escapes;
    double E_sys;
    double t_submit, t_admit, t_finish;
} sph_job_info;

typedef struct {
    int64_t submitted, finished, running, queued, rounds;
    double particle_steps;      /* sum over rounds of resident particles x steps_per_poll        */
} sph_server_stats;

/* Creates the server and allocates its batches.  Errors: SPH_E_INVALID, SPH_E_NOMEM, SPH_E_CUDA. */
sph_status sph_server_create(const sph_server_config* cfg, sph_server** out);

/* Queues a job (inputs are copied; h may be NULL for h_t(x)); job_id receives its id.
 * Errors: SPH_E_INVALID (no capacity for its dimension, other precision, n < 1, more
 * particles than the server's slots).  Problem descriptors are validated at admission: a job
 * whose descriptors are invalid ends as SPH_JOB_FAILED. */
sph_status sph_server_submit(sph_server* s, const sph_domain_desc* domain, const sph_sizing_desc* sizing,
                             const sph_params* params, int64_t n, const double* x, const int32_t* group,
                             const double* h, int64_t max_iters, int64_t* job_id);

/* Queues a job given by its problem alone: its target counts are computed at submission
 * (sph_feature_counts) and its particles are drawn on the device when it is admitted
 * (sph_sample_particles with this seed), so that its latency includes its initialisation.
 * Errors: SPH_E_INVALID (descriptors, as for sph_feature_counts; no capacity for its
 * dimension; other precision; a problem with no particle or more than the server's slots),
 * SPH_E_CUDA. */
sph_status sph_server_submit_sampled(sph_server* s, const sph_domain_desc* domain, const sph_sizing_desc* sizing,
                                     const sph_params* params, uint64_t seed, int64_t max_iters, int64_t* job_id);

/* One scheduling round (see above); stats (may be NULL) receives the counters after it. */
sph_status sph_server_poll(sph_server* s, sph_server_stats* stats);

/* Polls until no job is queued or resident, at most max_rounds rounds.
 * Errors: SPH_E_NOT_CONVERGED when work is left after max_rounds, plus those of poll. */
sph_status sph_server_drain(sph_server* s, int64_t max_rounds, sph_server_stats* stats);

/* State and timing of a job; for a finished job also its particles in submission order
 * (x_out [n][3], group_out [n], h_out [n]; any may be NULL; capacity >= n). */
sph_status sph_server_job(sph_server* s, int64_t job_id, sph_job_info* info, double* x_out,
                          int32_t* group_out, double* h_out, int64_t capacity);

/* Forgets a finished job (its results are freed). */
sph_status sph_server_release(sph_server* s, int64_t job_id);

void sph_server_destroy(sph_server* s);

/* ------------------------------------------------------------------------------------------
 * Cell-list rebuild that allocates nothing.  The paper has no counterpart: this entry point
 * serves callers that are not allowed to allocate device memory -- for example an application
 * that reserves all of the GPU's memory for its own pool at start-up and forbids libraries from
 * allocating afterwards (so that its budget stays fixed), or a latency-critical loop in which a
 * cudaMalloc/cudaFree could synchronise the device or fail under memory pressure.
 *
 * It computes the same cell keys, cell starts and stable permutation as sph_debug_rebuild of an
 * FP32 mesh (precision 32), for positions x_dev, y_dev, z_dev (device arrays of n doubles each;
 * z_dev may be NULL in 2D) and smoothing lengths h_dev (n floats) on the grid `grid` (from
 * sph_grid_spec or sph_mesh_grid).  The level of a particle is chosen by comparing its float h
 * with the grid's thresholds; an FP64 mesh compares its double h, so for an FP64 mesh the
 * results agree only where every h is exactly representable as a float.  A grid whose coarser
 * levels do not cover its finest level (each dims[l][a] >= ((dims[0][a] - 1) >> l) + 1, as
 * sph_grid_spec makes them) is rejected with SPH_E_INVALID.
 * Outputs, all caller-owned device arrays: key_dev [n], cell_start_dev [n_cells + 1], perm_dev [n].
 * Work is enqueued on `stream` (a cudaStream_t, NULL for the default stream); the call does not
 * wait for it.
 *
 * Its only scratch is a fixed array in device memory, SPH_NOALLOC_MAX_CELLS + 256 ints
 * (4 MiB + 1 KiB), that every GPU which loads the library holds until the process exits.
 * The first call on a device looks up that array's device address with the device current
 * (a one-time set-up per device); make that first call before any stream capture.  Grids with
 * more than SPH_NOALLOC_MAX_CELLS cells are rejected with SPH_E_INVALID.  All calls share the
 * array: the counters are cleared at the start of each call, and calls whose work overlaps on
 * the GPU (other streams or other threads) race and give wrong results.  Positions outside
 * the grid are clamped into its border cells without a report.  The call itself never
 * allocates or frees memory.  The CUDA runtime, however, may load the library's device code
 * lazily (the default since CUDA 12.2): the first call on a device may then load the module,
 * and that load reserves the fixed array.  A caller that reserves the GPU's memory for its own
 * pool should therefore make its first call at start-up, before it reserves the pool, or run
 * with CUDA_MODULE_LOADING=EAGER.  Errors: SPH_E_INVALID, SPH_E_CUDA (message in
 * sph_last_error()).
 * ------------------------------------------------------------------------------------------ */
#define SPH_NOALLOC_MAX_CELLS (1 << 20)
sph_status sph_cell_sort_noalloc(const sph_grid_info* grid, int64_t n, const double* x_dev,
                                 const double* y_dev, const double* z_dev, const float* h_dev,
                                 int32_t* key_dev, int32_t* cell_start_dev, int32_t* perm_dev,
                                 void* stream);

#ifdef __cplusplus
}
#endif
#endif
