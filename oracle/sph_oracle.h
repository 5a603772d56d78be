/*
 * sph_oracle.h -- plain FP64 CPU oracle of the feature-aware SPH relaxation step
 * (Ji, Fu, Hu, Adams, "A Feature-aware SPH for Isotropic Unstructured Mesh Generation").
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously-correct restatement of the
 * method that the CUDA path is checked against.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header, table or helper
 * with the CUDA library; both are written independently from the paper and from the readings
 * listed in the design notes.
 *
 * Conventions
 *  - D is the ambient dimension (2 or 3).  Positions, velocities and normals are arrays of
 *    3 doubles per particle even in 2D (the z entry is ignored and kept at 0).
 *  - A particle's "group" is the index k of the feature it belongs to.  A feature has a type
 *    (point / curve / surface / volume), i.e. an intrinsic dimension d (0,1,2,D).
 *    Section 3.2 (feature definition) and Fig. 1: particles of the same type and index form a
 *    group; groups of equal type but different index do not interact; lower-dimensional
 *    particles act one-sidedly as boundary particles for higher-dimensional ones.
 *  - Every function is pure with respect to its inputs unless it says otherwise.
 */
#ifndef SPH_ORACLE_H
#define SPH_ORACLE_H
#include <stdint.h>

#define ORC_MAX_FEAT 64
#define ORC_MAX_HOLES 8
#define ORC_MAX_LEVELS 8

/* feature kinds (intrinsic dimension in brackets) */
enum { ORC_VOLUME = 0,  /* [D]  the positive phase phi > 0 (Eq. 1)                        */
       ORC_POINT = 1,   /* [0]  singularity particle, never moves                          */
       ORC_SEGMENT = 2, /* [1]  straight feature curve a->b                                */
       ORC_CIRCLE = 3,  /* [1]  2D circle (outer rim or hole boundary)                     */
       ORC_RECT = 4,    /* [2]  3D planar face: origin, axes u,w, extents                  */
       ORC_SPHERE = 5   /* [2]  3D sphere surface (outer or hole)                          */ };

typedef struct {
    int32_t kind;
    int32_t dim;        /* intrinsic dimension d of the feature                                 */
    double p[12];       /* geometry.  POINT: p[0..2] position.  SEGMENT: a=p[0..2], b=p[3..5].
                           CIRCLE: centre p[0..1], radius p[2].  SPHERE: centre p[0..2], radius p[3].
                           RECT: origin p[0..2], unit axis u p[3..5], unit axis w p[6..8],
                           extent along u p[9], along w p[10].                                   */
    double nb[3];       /* POINT, SEGMENT, RECT: outward unit normal of the domain at the feature
                           (for edges and corners: the normalised bisector of the incident faces) */
    double orient;      /* CIRCLE, SPHERE: +1 if the domain lies inside (outer boundary),
                           -1 if the domain lies outside (a hole)                                */
} orc_feature;

enum { ORC_BASE_BOX = 0, ORC_BASE_BALL = 1 };

typedef struct {
    int32_t D;
    int32_t base;                 /* ORC_BASE_BOX: box [lo,hi]; ORC_BASE_BALL: ball (bc, br)      */
    double lo[3], hi[3];          /* bounding box of the domain (box base: the box itself)        */
    double bc[3], br;
    int32_t n_holes;              /* spherical / circular holes subtracted from the base          */
    double hc[ORC_MAX_HOLES][3];
    double hr[ORC_MAX_HOLES];
    int32_t n_feat;
    orc_feature feat[ORC_MAX_FEAT];
} orc_domain;

/* target feature size h_t(x) (Eq. 2 with rho_t = h^-d) as an analytic input */
enum { ORC_H_CONST = 0,      /* h = a                                                  */
       ORC_H_HOLE_DIST = 1,  /* h = clamp(a + b * min_k | |x-c_k| - r_k |, lo, hi)     */
       ORC_H_RADIAL = 2      /* h = clamp(a + b * |x - q|, lo, hi)   (form of Eq. 25)  */ };
typedef struct {
    int32_t kind;
    double a, b, lo, hi;
    double q[3];                        /* RADIAL: centre                                   */
    int32_t n_ref;                      /* HOLE_DIST: reference spheres / circles            */
    double rc[ORC_MAX_HOLES][3];
    double rr[ORC_MAX_HOLES];
} orc_sizing;

typedef struct {
    double kappa;          /* support radius r_c = kappa * h                                   */
    double p0;             /* EOS constant pressure P0 (Eq. 6)                                 */
    double visc;           /* nu = visc * r_c * |v| (Eq. 8); 0 switches viscosity off          */
    double cfl_a, cfl_v;   /* Eq. 9 / Eq. 24 constants 0.25 and 1/40                           */
    double eps1;           /* Phase-One damping factor epsilon (Eq. 23)                        */
    double dt_cap;         /* step used when a group has neither acceleration nor velocity     */
    double dt_collapse;    /* reset velocities when dt < dt_collapse * previous dt (Sec. 3.4.3)*/
    double threshold;      /* convergence threshold on E_sys (Sec. 3.4.2)                      */
    int32_t reset_period;  /* Phase-One velocity nullification period (Sec. 3.4.3)             */
    int32_t sample_every;  /* steps between samples of V-bar (Sec. 3.4.2)                      */
    int32_t window;        /* samples per averaging window (Sec. 3.4.2)                        */
    int32_t ramp_len;      /* length of the Phase-One -> Phase-Two transition (Sec. 3.4.4)     */
    int32_t boundary_rho;  /* 1: boundary term carries rho_b (units-consistent reading of
                              Eq. 19); 0: Eq. 19 as printed                                    */
    int32_t max_newton;    /* projection iterations onto the domain for escaped particles       */
    int32_t boundary_correction;  /* 1: the feature-boundary sum of Eq. 19 (Sec. 3.2) is applied;
                              0: it is left out (the earlier method compared in Sec. 4.1)       */
    int32_t group_convergence;    /* 0: the instance changes phase on E_sys (Sec. 3.4.2);
                              1: every group runs its own phases on its own E_g and stops when
                              it has converged (Algorithm 1: "if V-bar_k is not converged")     */
    int32_t feature_order;        /* 0: every group reads the state at the start of the step
                              (Jacobi); 1: Algorithm 1's feature loop in sequence (Gauss-Seidel):
                              the groups are advanced class by class in increasing intrinsic
                              dimension, each class reading the positions the lower classes
                              reached in this step (requires group_convergence = 1)            */
} orc_params;

/* two-phase controller state (Sec. 3.4) */
enum { ORC_PHASE1 = 1, ORC_RAMP = 2, ORC_PHASE2 = 3, ORC_DONE = 4 };
typedef struct {
    int32_t phase;
    int32_t wcount;        /* samples in the current (open) window                              */
    int32_t nwin;          /* completed windows since the phase (re)started                     */
    int32_t pad;
    int64_t n;             /* step counter                                                      */
    int64_t ramp_start;
    int64_t escapes;       /* volume particles re-projected into the domain                     */
    double wsum[ORC_MAX_FEAT];
    double A_last[ORC_MAX_FEAT], A_prev[ORC_MAX_FEAT];
    double Vbar[ORC_MAX_FEAT];
    double dt_prev[ORC_MAX_FEAT];
    double dt[ORC_MAX_FEAT];      /* step size used by each group in the last step            */
    int32_t reset[ORC_MAX_FEAT];  /* velocity reset applied to each group in the last step    */
    double E_t, E_avg, E_sys;
    double eps, ramp_f;           /* damping and velocity attenuation used in the last step   */
    /* per group: phase, window counters, switch step, last error, and the damping and
       attenuation used in the last step (the instance's values when group_convergence = 0) */
    int32_t gphase[ORC_MAX_FEAT], gwcount[ORC_MAX_FEAT], gnwin[ORC_MAX_FEAT];
    int64_t gramp_start[ORC_MAX_FEAT];
    double gE[ORC_MAX_FEAT], geps[ORC_MAX_FEAT], gf[ORC_MAX_FEAT];
} orc_ctrl;

/* cell-list representation used by the data-parallel neighbour search (multi-level grid) */
typedef struct {
    int32_t D, L;
    int32_t cps;                    /* cells per support: 1, 2 or 4                          */
    float c0;                       /* finest cell edge (exactly representable in float)     */
    float origin[3];
    float thr[ORC_MAX_LEVELS];      /* level l holds particles with thr[l-1] < h <= thr[l]  */
    int64_t dims[ORC_MAX_LEVELS][3];
    int64_t base[ORC_MAX_LEVELS];   /* first key of each level                              */
    int64_t ncell;                  /* total cells over all levels                          */
} orc_grid;

#ifdef __cplusplus
extern "C" {
#endif

/* ---- smoothing kernel (Wendland C2, support kappa*h) and its radial derivative ---- */
double orc_W(int d, double r, double h, double kappa);
double orc_dW(int d, double r, double h, double kappa);

/* ---- geometry and sizing ---- */
double orc_h(const orc_sizing* s, const double* x);
double orc_phi(const orc_domain* dom, const double* x, double* grad /* may be NULL */);
void orc_project(const orc_domain* dom, int k, double* x);
void orc_frame(const orc_domain* dom, int k, const double* x, double* nb, double* tg);
void orc_tangent(const orc_domain* dom, int k, const double* x, double* v);
double orc_feature_measure_density(const orc_domain* dom, const orc_sizing* s, int k, int n_quad);

/* ---- neighbour search ---- */
int64_t orc_neighbors_brute(int64_t n, int D, const double* x, const double* h, double kappa,
                            int64_t i, int32_t* out, int64_t cap);
void orc_grid_spec(int D, const double* lo, const double* hi, double h_lo, double h_hi,
                   double kappa, int cells_per_support, orc_grid* g);
void orc_grid_repr(const orc_grid* g, int64_t n, const double* x, const double* h, int32_t prec,
                   int32_t* level, int64_t* cell, double* off, int64_t* key, int32_t* clamped);
int64_t orc_neighbors_repr(const orc_grid* g, int64_t n, const double* x, const double* h,
                           int32_t prec, double kappa, int32_t self_radius, int64_t i,
                           int32_t* out, int64_t cap);
void orc_counting_sort(int64_t n, const int64_t* key, int64_t ncell,
                       int64_t* cell_start, int64_t* perm);

/* ---- one step of the relaxation, split into the stages of Algorithm 1 ---- */
void orc_interact(int64_t n, const orc_domain* dom, const orc_params* prm,
                  const double* x, const double* h, const int32_t* grp, const double* v,
                  int64_t n_sub, const int64_t* sub, int32_t use_grid,
                  double* sigma, double* gamma, double* F, double* a_p, double* S,
                  double* dta, double* dtv);
void orc_control(const orc_params* prm, int n_groups, const int32_t* gdim,
                 const double* Vsum, const double* dta, const double* dtv, orc_ctrl* c);
void orc_integrate(int64_t n, const orc_domain* dom, const orc_sizing* siz, const orc_params* prm,
                   const orc_ctrl* c, const double* x, const double* h, const int32_t* grp,
                   const double* v, const double* a_p, int64_t n_sub, const int64_t* sub,
                   int32_t use_grid, double* x_out, double* v_out, double* h_out, double* a_v,
                   int64_t* escapes);
void orc_ctrl_init(orc_ctrl* c);

/* ---- initial particle sampling (Sec. 3.6) ---- */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC 2011). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* The first n accepted candidates of feature k for seed (positions x_out[n][3]); returns the
 * number of candidates examined. */
int64_t orc_sample_feature(const orc_domain* dom, const orc_sizing* s, int k, uint64_t seed, int64_t n,
                           double* x_out);
void orc_step(int64_t n, const orc_domain* dom, const orc_sizing* siz, const orc_params* prm,
              orc_ctrl* c, double* x, double* v, double* h, const int32_t* grp,
              int32_t use_grid, int32_t n_steps);

#ifdef __cplusplus
}
#endif
#endif
