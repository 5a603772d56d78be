// sph_internal.cuh -- device pointers of a batch of instances and the kernel launchers shared by
// the translation units of libsphmesh.so.  Not part of the public ABI.
//
// A batch packs NI independent instances (same dimension and precision) into one particle
// array.  Instance i owns the slots [inst_off[i], inst_off[i+1]) -- its particle count rounded up
// to a multiple of CHUNK, none while it is empty -- of which the first inst_n[i] hold its
// particles in the current order; the rest are padding (hashed to the instance's dummy cell,
// which sorts last and is never searched).  Its cells are the global keys grids[i].base[0] ..
// grids[i].base[MAXL]-1, followed by its dummy key grids[i].base[MAXL].  Every kernel serves all
// instances in one launch over the n slots in use.
#pragma once
#include "../../include/sphmesh.h"
#include "sph_device.cuh"

namespace sph {

constexpr int CHUNK = SPH_SLOT_CHUNK;   // slot alignment of instances (a multiple of every pair-pass block)

template <typename T> struct State {
    int n;             // total slots of the batch
    int NI;            // instances
    const int* inst_off;    // [NI+1]
    const int* inst_n;      // [NI]
    const int* chunk_inst;  // [n / CHUNK] instance of every chunk of slots
    const Grid* grids;      // [NI]
    const Params* params;   // [NI]
    const Domain* doms;     // [NI]
    const Sizing* sizs;     // [NI]
    Ctrl* ctrls;            // [NI]
    // stored state (order of the previous sort): position = finest cell C + offset O
    int* C[3];
    T* O[3];
    T* V[3];
    T* H;
    unsigned* G;
    int* ID;           // index of the particle in its instance's input order (-1: padding)
    int* K;            // cell key of every stored particle (written by the hash)
    // sorted state
    int* Cs[3];
    T* Os[3];
    Vec4<T>* VH;       // (v.x, v.y, v.z, h): one 16-byte (FP64: 32-byte) load per neighbour
    unsigned* Ms;
    int* IDs;
    int* Ks;
    Vec4<T>* P;
    Vec4<T>* A;
    // rebuild scratch: per-cell counts (also the scatter cursors), cell starts, scan block
    // sums, and the sorted-slot -> stored-index permutation
    int* count;
    int* cell_start;
    int* bsum;
    // one-pass scan: per-tile status words (flag << 62 | value) and the tile ticket, cleared by
    // whichever kernel produces the histogram
    unsigned long long* tstate;
    int* ticket;
    int ntile;
    int* perm;         // slot -> stored index as left by the scatter (unordered inside a cell)
    int* sperm;        // slot -> stored index, stable (ordered inside a cell; written by the gather)
    int ncell;         // total keys (all instances' cells and dummy cells)
    // per occupancy cell, OCCW words: per level the largest h of its particles in the cell
    // (float bits, 0 for none; built by the gather)
    unsigned* occ;
    int nocc;
    // same-group pairs found by the pressure pass, handed to the viscous pass: for lane
    // g = k*LPP + r of particle k, entry c is (vj, vr)[c * n*LPP + g] (index, and the pair's
    // kernel factor of Eq. 7, (rho_i^-2 + rho_j^-2) W'(r, h_ij) / r);
    // vcnt[g] counts them (> VCAP: the list overflowed and the viscous pass walks the cells)
    int* vj;
    T* vr;
    int* vcnt;
    // per-block, per-group partial sums of V~ (sample steps); nblk = blocks of the pair passes.
    // The last pressure-pass block of every chunk of CHUNK slots (counted in pticket) adds the
    // chunk's block rows in block order into partials2 [chunk][MAXF], which the controller reads
    double* partials;
    int nblk;
    double* partials2;
    int* pticket;
};

// The grid and parameters of a batch of one, passed to the kernels by value so that they are
// read as constant-bank operands; with more instances the kernels read the per-instance tables.
struct One {
    Grid g;
    Params p;
};

// output set of the update kernel (the stored state, or scratch for inspection calls)
template <typename T> struct Out {
    int* C[3];
    T* O[3];
    T* V[3];
    T* H;
    unsigned* G;
    int* ID;
    T* av[3];          // optional: viscous acceleration (inspection only)
    int* K;            // optional (stored state): the next rebuild's cell keys ...
    int* count;        // ... and per-cell histogram, so that the next step needs no hash pass
};

// (measured with the 2.6h support: 12 / 20 / 24 make the whole 2D step 22 % slower / 1 % slower /
// 5 % slower than 16, and the 1.2M cube's 33 % / 2 % / 11 %)
// the pressure pass's per-block Eq. 24 minima and V~ partial sums in the memory of its
// candidate buffers once the walk is done (1) or in arrays of their own (0) (measured: 3D
// pressure pass on the 1.2M cube 3.36 ms against 3.42, 2D on the 120k disk 80.1 us against 79.0)
#ifndef SPH_ALIAS_TAIL_2D
#define SPH_ALIAS_TAIL_2D 0
#endif
#ifndef SPH_ALIAS_TAIL_3D
#define SPH_ALIAS_TAIL_3D 1
#endif
#ifndef SPH_BUF_CAP
#define SPH_BUF_CAP 16
#endif
constexpr int BUF_CAP = SPH_BUF_CAP;   // kept candidates per lane between flushes of the walk (shared memory)
// lanes per particle in the pair passes (measured with a 2.6h support, 5 steps after the start,
// whole step in ms for disks of 1k / 20k / 120k / 1M particles: 2 lanes 0.134 / 0.123 / 0.183 /
// 0.829, 4 lanes with 64 hand-over slots 0.096 / 0.093 / 0.153 / 0.828; 1 lane 1.7-2.5x slower;
// cubes of 20k / 200k / 1.2M: 8 lanes 0.229 / 1.018 / 4.92, 4 lanes 0.50 / 1.79 / 9.44, 16 lanes
// 0.48 / 1.60 / 7.54, 16 faster only at 1k (0.166 against 0.199); fewer lanes repeat less of
// the per-particle stencil work, more lanes balance the candidates)
#ifndef SPH_LPP_2D
#define SPH_LPP_2D 4
#endif
#ifndef SPH_LPP_3D
#define SPH_LPP_3D 8
#endif
template <int D> struct Lpp {
    static constexpr int v = D == 2 ? SPH_LPP_2D : SPH_LPP_3D;
};
// same-group pair slots per particle (SPH_VCAP_2D/3D) and per lane (Vcap) in the
// pressure-to-viscous hand-over list (measured with a 2.6h support, whose overflowing particles
// walk the cells again: in 2D with 4 lanes per particle 64 slots make the 120k disk's step 5 %
// faster than 48, 96 no faster; in 3D 192 slots are 4.5x faster than 96 on the viscous pass,
// 128 make the 1.2M cube's step 11 % slower and 256 no faster)
#ifndef SPH_VCAP_2D
#define SPH_VCAP_2D 64
#endif
#ifndef SPH_VCAP_3D
#define SPH_VCAP_3D 192
#endif
template <int D> struct Vcap {
    static constexpr int v = D == 2 ? SPH_VCAP_2D / Lpp<2>::v : SPH_VCAP_3D / Lpp<3>::v;
};
// lanes per particle in the viscous pass; each lane reads Lpp/ILpp of the pressure pass's
// hand-over columns, and the list-overflow fallback walks with ILpp lanes (measured: one lane
// in 2D, 2 % faster than 2; in 3D with the 2.6h support and 192 list slots per particle, on the
// 1.2M cube after 5 steps, 2 lanes make the pass 0.854 ms against 1.177 ms with one lane (27 %
// faster; with 5 blocks per SM 0.891 ms), and 3 entries fetched together instead of 2 are 74 %
// slower)
#ifndef SPH_ILPP_2D
#define SPH_ILPP_2D 1
#endif
#ifndef SPH_ILPP_3D
#define SPH_ILPP_3D 2
#endif
template <int D> struct ILpp {
    static constexpr int v = D == 2 ? SPH_ILPP_2D : SPH_ILPP_3D;
};
static_assert(CHUNK % (BLOCK / Lpp<2>::v) == 0 && CHUNK % (BLOCK / Lpp<3>::v) == 0 &&
                  CHUNK % (BLOCK / ILpp<2>::v) == 0 && CHUNK % (BLOCK / ILpp<3>::v) == 0,
              "a pair-pass block must lie in one chunk");
static_assert(Lpp<2>::v % ILpp<2>::v == 0 && Lpp<3>::v % ILpp<3>::v == 0,
              "the viscous lanes split the pressure pass's columns evenly");

// 3D occupancy cells finer than the cells-per-support top-level cells by 2^SPH_OCC_FINER per axis
// (measured on the 3D cube: 1 and 2 make the pressure pass 5 % and 21 % slower than 0; with the
// search radius from the cells' largest h, 6 % and 16 %)
#ifndef SPH_OCC_FINER
#define SPH_OCC_FINER 0
#endif

// minimum resident blocks per SM asked of the compiler for the two pair passes (FP32 build;
// the FP64 build asks for 4): it bounds the registers per thread, trading spills for occupancy
// (measured on the pressure pass: 10 and 12 spill and are 17 % and 40 % slower than 8; with
// the 2.6h support and 8 lanes per particle in 3D, on a 1.2M cube, 5 / 6 / 7 / 9 / 10 were
// 24 / 13 / 8 / 10 / 46 % slower than 8 although 8 spills a few words in the batched form,
// and 9 in 2D 4 % slower; on the viscous pass with one lane per particle 7 is 3 % faster than
// 8 in 2D, and 6 is 5 % faster than 7 in 3D but 26 % slower in 2D; again with the 2.6h support:
// 2D 6 / 8 30 % / 3 % slower than 7, 3D 5 2 % faster than 6 on the pass (0.3 % on the step)
// and 7 12 % slower)
#ifndef SPH_INTERACT_MINB
#define SPH_INTERACT_MINB 8
#endif
#ifndef SPH_INTERACT_MINB_3D
#define SPH_INTERACT_MINB_3D SPH_INTERACT_MINB
#endif
// the viscous pass and the update as two kernels (each with its own register budget) instead
// of one (measured on the 1.2M cube: 0.73 ms against 0.86 for the fused kernel, the viscous
// kernel at 8 blocks/SM, 7 and 6 being 3 % and 7 % slower; with the kernel factor in the
// hand-over list 0.64 ms, 9 blocks/SM 0.70; on the 120k disk, with one viscous lane per
// particle, 47 us against 39.5 us fused)
#ifndef SPH_SPLIT_INTEGRATE_2D
#define SPH_SPLIT_INTEGRATE_2D 0
#endif
#ifndef SPH_SPLIT_INTEGRATE_3D
#define SPH_SPLIT_INTEGRATE_3D 1
#endif
#ifndef SPH_VISC_MINB_2D
#define SPH_VISC_MINB_2D 8
#endif
#ifndef SPH_VISC_MINB_3D
#define SPH_VISC_MINB_3D 8
#endif
#ifndef SPH_UPDATE_MINB
#define SPH_UPDATE_MINB 6
#endif
#ifndef SPH_INTEGRATE_MINB_2D
#define SPH_INTEGRATE_MINB_2D 7
#endif
#ifndef SPH_INTEGRATE_MINB_3D
#define SPH_INTEGRATE_MINB_3D 6
#endif
// cells per support of the cell grid when the parameters leave the choice to the library
// (measured with a 2.6h support: 2 in 2D are 9 % faster than 1; 1 in 3D is 45 % slower than 2)
#ifndef SPH_DEFAULT_CPS_2D
#define SPH_DEFAULT_CPS_2D 2
#endif
#ifndef SPH_DEFAULT_CPS_3D
#define SPH_DEFAULT_CPS_3D 2
#endif
// entries of the pressure-to-viscous hand-over list fetched together by the viscous pass
#ifndef SPH_VISC_BATCH
#define SPH_VISC_BATCH 2
#endif

// Whether a particle of intrinsic dimension di takes part in the step pass for dimension class
// cls: 0 is the whole step at once; with Algorithm 1's feature loop in sequence (feature_order)
// a step runs the passes cls = 1 .. D in turn and each moves the particles of its class, and an
// instance without it (batched with one that has it) takes its whole step in the last pass.
__device__ __forceinline__ bool in_pass(const Params& p, int cls, int di, int D) {
    if (cls == 0) return true;
    return p.feature_order ? di == cls : cls == D;
}

// instance of slot k, and whether the slot holds a particle
template <typename T> __device__ __forceinline__ int inst_of(const State<T>& s, int k) {
    return __ldg(s.chunk_inst + k / CHUNK);
}
template <typename T> __device__ __forceinline__ bool live(const State<T>& s, int i, int k) {
    return k - __ldg(s.inst_off + i) < __ldg(s.inst_n + i);
}

// the one-pass scan's tile states back to "nothing published" (grid-stride over any grid)
template <typename T> __device__ __forceinline__ void reset_scan_state(const State<T>& s) {
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    for (int t = t0; t < s.ntile; t += stride) s.tstate[t] = 0ull;
    if (t0 == 0) *s.ticket = 0;
}

// copy a struct into shared memory with the whole block (one round trip)
template <typename S> __device__ __forceinline__ void block_copy(S* dst, const S* src) {
    const unsigned* a = reinterpret_cast<const unsigned*>(src);
    unsigned* b = reinterpret_cast<unsigned*>(dst);
    for (int t = threadIdx.x; t < (int)(sizeof(S) / 4); t += blockDim.x) b[t] = a[t];
}

// level and level-cell of sorted particle k (from its h and stored finest cell; the same as
// decoding its key, without the integer divisions)
template <typename T, int D>
__device__ __forceinline__ void own_cell(const Grid& g, const State<T>& s, int k, T h, int& l, int c[3]) {
    l = level_of(g, h);
    for (int a = 0; a < 3; ++a) c[a] = a < D ? (s.Cs[a][k] >> l) : 0;
}

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
// cells per thread and threads per tile of the step's one-pass scan (measured: 2 is 6 % faster
// than 4 in the rebuild, 8 and 16 are 27 % and 86 % slower; again with the 2.6h support and its
// 1.41M-cell 2D grid: 1 / 4 / 8 per thread 20 / 9 / 65 % slower than 2; 512 x 2 and 256 x 4
// threads x cells equal to 1024 x 2 within 1 %, 512 x 4 and 256 x 8 9 % and 35 % slower)
#ifndef SPH_SCAN1_ITEMS
#define SPH_SCAN1_ITEMS 2
#endif
#ifndef SPH_SCAN1_THREADS
#define SPH_SCAN1_THREADS 1024
#endif
constexpr int SCAN1_ITEMS = SPH_SCAN1_ITEMS;
constexpr int SCAN1_THREADS = SPH_SCAN1_THREADS;
constexpr int SCAN1_TILE = SCAN1_THREADS * SCAN1_ITEMS;

inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }

// Programmatic dependent launch between the kernels of a step.  A kernel launched with
// pdl = true may be scheduled while its predecessor in the stream is still running (once every
// block of the predecessor has started); its blocks then wait in dep_wait() until the
// predecessor has completed and its writes are visible.  Every step kernel calls dep_wait()
// before its first access to device memory other than its kernel parameters, so the order of
// the stream is kept; without the attribute dep_wait() returns at once.  dep_launch() lets
// the successor be scheduled as soon as every block of this kernel is running.
__device__ __forceinline__ void dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

#ifndef SPH_PDL
#define SPH_PDL 1
#endif
template <typename... K, typename... A>
inline void launch_k(void (*kern)(K...), int grid, int block, cudaStream_t st, bool pdl, A&&... args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = (pdl && SPH_PDL) ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kern, static_cast<A&&>(args)...);
}

// rebuild.cu
// `one`: the descriptors of a batch of one (nullptr: read the per-instance tables)
template <typename T, int D> void launch_hash(const State<T>& s, const One* one, cudaStream_t st);
void launch_scan(int ncell, int* count, int* cell_start, int* bsum, cudaStream_t st, unsigned* occ = nullptr,
                 int nocc = 0, bool relative = false);
// relative one-pass scan of the step (decoupled look-back over tiles taken in ticket order)
template <typename T> void launch_scan_onepass(const State<T>& s, cudaStream_t st);
template <typename T> void launch_scatter(const State<T>& s, cudaStream_t st, bool pdl = false);
void launch_cellsort(int ncell, int n, const int* cell_start, int* perm, int* count, cudaStream_t st);
template <typename T, int D> void launch_gather(const State<T>& s, const One* one, cudaStream_t st, bool pdl = false);
template <typename T, int D> void launch_init_h(const State<T>& s, int inst, cudaStream_t st);
template <typename T, int D> void launch_repack(const State<T>& s, const int* old_off, const int* move_n, cudaStream_t st);

// state_io.cu: an instance's slots from and to the caller's FP64 arrays (staged on the device)
struct IoCheck {      // accepted ranges: positions inside [lo, hi] per axis, h in (0, hmax]
    double lo[3], hi[3];
    double hmax;
    int G, D;
};
struct IoGrid {       // finest-level cell geometry of an instance, and each group's dimension
    double origin[3];
    double c0, inv_c0;
    int dims0[3];
    unsigned char fdim[MAXF];
};
template <typename T> struct SlotArrays {   // an instance's stored state, from its first slot
    int* C[3];
    T* O[3];
    T* V[3];
    T* H;
    unsigned* G;
    int* ID;
};
template <typename T> struct ConstSlotArrays {
    const int* C[3];
    const T* O[3];
    const T* V[3];
    const T* H;
    const unsigned* G;
    const int* ID;
};
// first offending particle as (index << 2) | check (0 group, 1 position, 2 h, 3 velocity) by
// atomicMin into *first (the caller sets it to all ones)
void launch_check_state(const IoCheck& c, int n, const double* x, const int* group, const double* v, const double* h,
                        unsigned long long* first, cudaStream_t st);
// slots [0, n) from the arrays (v, h may be null: zero), [n, ns) padding
template <typename T, int D>
void launch_load_state(const SlotArrays<T>& s, const IoGrid& g, int ns, int n, const double* x, const int* group,
                       const double* v, const double* h, cudaStream_t st);
// slots [0, ns) to the arrays in input order (any may be null); cnt[0] counts the particles
// written, cnt[1] is set when a slot holds an index >= n (both zeroed by the caller)
template <typename T, int D>
void launch_store_state(const ConstSlotArrays<T>& s, const IoGrid& g, int ns, int n, double* x, int* group, double* v,
                        double* h, int* cnt, cudaStream_t st);

// interact.cu
template <typename T, int D>
void launch_interact(const State<T>& s, const One* one, T* dbg_sigma, T* dbg_gamma, cudaStream_t st,
                     bool pdl = false, int cls = 0);
template <typename T, int D>
void launch_neighbors(const State<T>& s, int mode, int* counts, const long long* offsets, int* lists, cudaStream_t st);
template <typename T, int D> void launch_pair_counts(const State<T>& s, unsigned long long* out2, cudaStream_t st);

// integrate.cu
template <typename T, int D>
void launch_control(const State<T>& s, const One* one, cudaStream_t st, bool pdl = false, int cls = 0);
template <typename T, int D>
void launch_integrate(const State<T>& s, const One* one, const Ctrl* use, const Out<T>& o, cudaStream_t st,
                      bool pdl = false, int cls = 0);

// sample.cu: midpoint-rule integrals of rho_t over every feature of dm (Eqs. 10, 11), and the
// rejection sampling of counts[k] particles per feature into d_out[n][3] in feature order
// (d_dom / d_siz: device copies of dm and its sizing)
int quad_points(int kind, int D, long long* npts);
cudaError_t feature_integrals(const Domain& dm, const Domain* d_dom, const Sizing* d_siz, cudaStream_t st,
                              double* integral);
cudaError_t sample_features(const Domain& dm, const Sizing& z, const Domain* d_dom, const Sizing* d_siz,
                            unsigned long long seed, const int64_t* counts, cudaStream_t st, double* d_out);

// sets the message returned by sph_last_error() on the calling thread (capi.cu)
void set_last_error(const char* msg);

}  // namespace sph
