// capi.cu -- host side of libsphmesh.so: descriptor validation, the cell-grid specification,
// the layout of a batch of instances in device memory, the per-step launch sequence (captured
// once into a CUDA graph), and the inspection entry points.  See include/sphmesh.h for the
// contract of every function.
//
// Every handle is a batch: NI independent instances, each with its own domain, sizing,
// parameters and controller, packed into one particle array and one cell-key range.  The loaded
// instances occupy consecutive slot ranges in index order (each its particle count rounded up
// to CHUNK); loading or emptying an instance re-packs the others (a device-side move) and
// re-captures the step graph.  Every kernel serves all instances in one launch.  A sph_mesh is
// a batch of one.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sphmesh.h"
#include "sph_internal.cuh"

using namespace sph;

namespace {

thread_local std::string g_err;

sph_status fail(sph_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return fail(SPH_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_));  \
    } while (0)

float round_up_f(double v) {
    float f = (float)v;
    if ((double)f < v) f = std::nextafter(f, INFINITY);
    return f;
}
float round_down_f(double v) {
    float f = (float)v;
    if ((double)f > v) f = std::nextafter(f, -INFINITY);
    return f;
}

// Cell-grid specification (documented with sph_grid_spec in the header).
sph_status grid_spec(int D, const double* lo, const double* hi, double h_lo, double h_hi, double kappa, int cps,
                     sph_grid_info* out) {
    if (D != 2 && D != 3) return fail(SPH_E_INVALID, "grid: dim must be 2 or 3");
    if (!(h_lo > 0) || !(h_hi >= h_lo) || !(kappa > 0)) return fail(SPH_E_INVALID, "grid: need 0 < h_lo <= h_hi, kappa > 0");
    if (cps != 1 && cps != 2 && cps != 4) return fail(SPH_E_INVALID, "grid: cells_per_support must be 1, 2 or 4");
    for (int a = 0; a < D; ++a)
        if (!(hi[a] > lo[a])) return fail(SPH_E_INVALID, "grid: empty bounding box on axis %d", a);
    const double m = 1.0 + std::ldexp(1.0, -10);
    const double cm = (double)cps;
    sph_grid_info g;
    std::memset(&g, 0, sizeof g);
    g.dim = D;
    g.cells_per_support = cps;
    g.c0 = round_up_f(kappa * h_lo * m / cm);
    int L = 1;
    while (cm * std::ldexp((double)g.c0, L - 1) < kappa * h_hi * m) {
        if (L == SPH_MAX_LEVELS) return fail(SPH_E_INVALID, "grid: h_hi/h_lo too large for %d levels", SPH_MAX_LEVELS);
        ++L;
    }
    g.levels = L;
    for (int l = 0; l < SPH_MAX_LEVELS; ++l)
        g.thr[l] = l < L - 1 ? round_down_f(cm * std::ldexp((double)g.c0, l) / (kappa * m)) : INFINITY;
    const double top = cm * std::ldexp((double)g.c0, L - 1);
    for (int a = 0; a < 3; ++a) g.origin[a] = a < D ? round_down_f(lo[a] - top) : 0.0f;
    int64_t base = 0;
    for (int l = 0; l < L; ++l) {
        const double cl = std::ldexp((double)g.c0, l);
        int64_t cells = 1;
        for (int a = 0; a < 3; ++a) {
            g.dims[l][a] = a < D ? (int64_t)std::ceil((hi[a] + top - (double)g.origin[a]) / cl) + 1 : 1;
            cells *= g.dims[l][a];
        }
        g.base[l] = base;
        base += cells;
    }
    g.n_cells = base;
    *out = g;
    return SPH_OK;
}

}  // namespace

void sph::set_last_error(const char* msg) { g_err = msg; }

namespace {

struct KTime {
    const char* name;
    int kernels;   // kernel launches per step in this stage
};
// the step graph: rebuild = one-pass scan, scatter, gather (the keys and histogram come from
// the previous step's update); the update also computes the next keys, and is two kernels
// (viscous sum, update) where SPH_SPLIT_INTEGRATE_2D/3D says so
constexpr int NSTAGE = 4;
const KTime kStages[NSTAGE] = {{"rebuild", 3}, {"interact", 1}, {"control", 1}, {"integrate", 1}};
int stage_kernels(int k, int D) {
    if (k == 3) return (D == 2 ? SPH_SPLIT_INTEGRATE_2D : SPH_SPLIT_INTEGRATE_3D) ? 2 : 1;
    return kStages[k].kernels;
}

// host copy of one instance
struct Inst {
    Grid grid;            // base[] and occ_base are global (set by relayout)
    int lbase[MAXL];      // first key of each level within the instance
    int ncell = 0;        // cells of the instance
    int nocc = 0;         // its top-level cells
    Params params;
    Domain dom;
    Sizing siz;
    double h_lo = 0, h_hi = 0;
    int64_t cap = 0;      // max_particles given at creation
    int off = 0, slots = 0;   // current slot range [off, off + slots) (slots = 0 while empty)
    int n = 0;            // particles loaded
    // the descriptors as given (to derive the grid again with other cells per support)
    sph_domain_desc dd;
    sph_sizing_desc sz;
    sph_params pp;
};

}  // namespace

struct sph_batch {
    int D = 2, prec = 32, NI = 0;
    std::vector<Inst> in;
    int nslots = 0;                   // slots in use (all loaded instances)
    int slot_cap = 0;                 // slots allocated
    int ncell = 0, nocc = 0;          // keys (cells + one dummy key per loaded instance), top-level cells
    size_t cell_cap = 0, occ_cap = 0; // allocated entries of the cell arrays
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    void* pool = nullptr;             // per-slot arrays
    void* cpool = nullptr;            // per-cell arrays
    void* stage = nullptr;            // the caller's arrays on the device (set_state, positions)
    size_t stage_cap = 0;
    State<float> sf;
    State<double> sd;
    Grid* d_grids = nullptr;
    Params* d_params = nullptr;
    Domain* d_doms = nullptr;
    Sizing* d_sizs = nullptr;
    Ctrl* d_ctrl = nullptr;
    Ctrl* d_ctrl_dbg = nullptr;
    int* d_inst_off = nullptr;
    int* d_inst_n = nullptr;
    int* d_chunk_inst = nullptr;
    int* d_old_off = nullptr;         // re-packing: previous offsets and slots to move, per instance
    int* d_move_n = nullptr;
    One one;                          // descriptors passed by value when NI == 1
    bool hashed = false;              // keys and histogram of the stored state are in place
    bool mesh = false;                // created by sph_mesh_create
    // CUDA graph of one step; rebuilt when the layout or the timing mode changes
    cudaGraphExec_t gexec = nullptr;
    long long layout_version = 0, graph_version = -1;
    bool graph_timed = false;
    // stage timing
    bool timing = false;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    bool ev_pending = false;
    double stage_ms[4] = {0, 0, 0, 0};   // NSTAGE entries used
    int64_t stage_steps = 0;
};

struct sph_mesh : sph_batch {};

namespace {

#define DISPATCH(b, fn, ...)                                              \
    ((b)->prec == 32 ? ((b)->D == 2 ? fn<float, 2>(__VA_ARGS__) : fn<float, 3>(__VA_ARGS__)) \
                     : ((b)->D == 2 ? fn<double, 2>(__VA_ARGS__) : fn<double, 3>(__VA_ARGS__)))

template <typename T> State<T>& st(sph_batch* b);
template <> State<float>& st<float>(sph_batch* b) { return b->sf; }
template <> State<double>& st<double>(sph_batch* b) { return b->sd; }

// cell keys of a batch (int32 keys and cell starts; the one-pass scan has no other bound)
constexpr long long MAX_KEYS = 1ll << 30;

int lpp_of(int D) { return D == 2 ? Lpp<2>::v : Lpp<3>::v; }
// cells per support when the parameters leave it to the library (measured per dimension)
int default_cps(int D) { return D == 2 ? SPH_DEFAULT_CPS_2D : SPH_DEFAULT_CPS_3D; }
int vcap_of(int D) { return D == 2 ? Vcap<2>::v : Vcap<3>::v; }

// Validates one instance's descriptors and fills its host copy (grid bases instance-relative).
sph_status make_instance(const sph_domain_desc* dd, const sph_sizing_desc* sz, const sph_params* pp,
                         int64_t max_particles, Inst& I) {
    if (!dd || !sz || !pp) return fail(SPH_E_INVALID, "create: NULL argument");
    if (dd->dim != 2 && dd->dim != 3) return fail(SPH_E_INVALID, "domain: dim must be 2 or 3");
    if (dd->n_features < 1 || dd->n_features > SPH_MAX_FEATURES) return fail(SPH_E_INVALID, "domain: n_features out of range");
    if (dd->n_holes < 0 || dd->n_holes > SPH_MAX_HOLES) return fail(SPH_E_INVALID, "domain: n_holes out of range");
    if (dd->base != 0 && dd->base != 1) return fail(SPH_E_INVALID, "domain: base must be 0 (box) or 1 (ball)");
    if (pp->precision != 32 && pp->precision != 64) return fail(SPH_E_INVALID, "params: precision must be 32 or 64");
    if (!(pp->kappa > 0) || !(pp->p0 > 0) || pp->visc < 0 || !(pp->cfl_a > 0) || !(pp->cfl_v > 0) || pp->eps1 < 0 ||
        !(pp->dt_cap > 0) || pp->dt_collapse < 0 || !(pp->threshold > 0) || pp->reset_period < 1 ||
        pp->sample_every < 1 || pp->window < 1 || pp->ramp_len < 1 || (pp->boundary_rho != 0 && pp->boundary_rho != 1) ||
        (pp->boundary_correction != 0 && pp->boundary_correction != 1) ||
        (pp->group_convergence != 0 && pp->group_convergence != 1) || (pp->feature_order != 0 && pp->feature_order != 1))
        return fail(SPH_E_INVALID, "params: value out of range");
    if (pp->feature_order == 1 && pp->group_convergence != 1)
        return fail(SPH_E_INVALID, "params: feature_order = 1 (Algorithm 1's loop in sequence) needs group_convergence = 1");
    if (max_particles < 0 || max_particles > (int64_t)1 << 30) return fail(SPH_E_INVALID, "max_particles out of range");
    if (sz->kind < 0 || sz->kind > 2 || !(sz->lo > 0) || !(sz->hi >= sz->lo) || sz->n_ref < 0 || sz->n_ref > SPH_MAX_HOLES)
        return fail(SPH_E_INVALID, "sizing: need kind 0..2, 0 < lo <= hi, n_ref <= %d", SPH_MAX_HOLES);
    if (sz->kind == 0 && !(sz->a >= sz->lo && sz->a <= sz->hi)) return fail(SPH_E_INVALID, "sizing: constant h outside [lo, hi]");
    const int D = dd->dim;
    for (int k = 0; k < dd->n_features; ++k) {
        const sph_feature& f = dd->features[k];
        int want = -1;
        switch (f.kind) {
            case SPH_FEAT_VOLUME: want = D; break;
            case SPH_FEAT_POINT: want = 0; break;
            case SPH_FEAT_SEGMENT: want = 1; break;
            case SPH_FEAT_CIRCLE: want = D == 2 ? 1 : -1; break;
            case SPH_FEAT_RECT: want = D == 3 ? 2 : -1; break;
            case SPH_FEAT_SPHERE: want = D == 3 ? 2 : -1; break;
            default: break;
        }
        if (want < 0 || f.dim != want) return fail(SPH_E_INVALID, "feature %d: kind/dim mismatch for a %dD domain", k, D);
        if (f.kind == SPH_FEAT_SEGMENT) {
            const double d0 = f.geom[3] - f.geom[0], d1 = f.geom[4] - f.geom[1], d2 = f.geom[5] - f.geom[2];
            if (!(d0 * d0 + d1 * d1 + d2 * d2 > 0)) return fail(SPH_E_INVALID, "feature %d: zero-length segment", k);
        }
    }
    int cps = pp->cells_per_support;
    if (cps == 0) cps = default_cps(D);
    sph_grid_info gi;
    sph_status r = grid_spec(D, dd->bbox_lo, dd->bbox_hi, sz->lo, sz->hi, pp->kappa, cps, &gi);
    if (r != SPH_OK) return r;
    if (gi.n_cells > MAX_KEYS)
        return fail(SPH_E_INVALID, "grid: %lld cells is more than the %lld cell keys supported", (long long)gi.n_cells,
                    (long long)MAX_KEYS);
    for (int l = 0; l < gi.levels; ++l)
        if (gi.dims[l][0] >= ((int64_t)1 << 23) || gi.dims[l][1] >= ((int64_t)1 << 14) || gi.dims[l][2] >= ((int64_t)1 << 14))
            return fail(SPH_E_INVALID, "grid: too many cells (x < 2^23, y and z < 2^14 per level)");

    I = Inst();
    I.dd = *dd;
    I.sz = *sz;
    I.pp = *pp;
    I.cap = max_particles;
    I.h_lo = sz->lo;
    I.h_hi = sz->hi;
    Grid& g = I.grid;
    std::memset(&g, 0, sizeof g);
    g.D = D;
    g.L = gi.levels;
    g.c0 = gi.c0;
    for (int a = 0; a < 3; ++a) g.origin[a] = gi.origin[a];
    for (int l = 0; l < MAXL; ++l) {
        g.c[l] = std::ldexp((double)gi.c0, l);
        g.inv_c[l] = 1.0 / g.c[l];
        g.cf[l] = (float)g.c[l];
        g.thr[l] = gi.thr[l];
        for (int a = 0; a < 3; ++a) g.dims[l][a] = l < gi.levels ? (int)gi.dims[l][a] : 1;
        I.lbase[l] = l < gi.levels ? (int)gi.base[l] : (int)gi.n_cells;
    }
    I.ncell = (int)gi.n_cells;
    g.ncell = I.ncell;
    g.sm = cps == 1 ? 0 : (cps == 2 ? 1 : 2);
    // occupancy cells: cps top-level cells per axis (a search window spans at most one of them
    // on each side), in 3D divided SPH_OCC_FINER times in two.  A level's search is skipped when
    // the occupancy cells covering its own cell box hold none of its particles, and its radius
    // is taken from the largest h they hold.
    const int t = gi.levels - 1;
    const int fin = D == 3 ? std::min(SPH_OCC_FINER, t + g.sm) : 0;
    g.osh = t + g.sm - fin;
    int64_t nocc = 1;
    for (int a = 0; a < 3; ++a) {
        g.od[a] = a < D ? (int)((((int64_t)gi.dims[t][a] << fin) + cps - 1) / cps) : 1;
        nocc *= g.od[a];
    }
    I.nocc = (int)nocc;
    Params& p = I.params;
    std::memset(&p, 0, sizeof p);
    p.kappa = pp->kappa;
    p.p0 = pp->p0;
    p.visc = pp->visc;
    p.cfl_a = pp->cfl_a;
    p.cfl_v = pp->cfl_v;
    p.eps1 = pp->eps1;
    p.dt_cap = pp->dt_cap;
    p.dt_collapse = pp->dt_collapse;
    p.threshold = pp->threshold;
    p.reset_period = pp->reset_period;
    p.sample_every = pp->sample_every;
    p.window = pp->window;
    p.ramp_len = pp->ramp_len;
    p.boundary_rho = pp->boundary_rho;
    p.boundary_corr = pp->boundary_correction;
    p.group_conv = pp->group_convergence;
    p.feature_order = pp->feature_order;
    p.kappa_f = (float)p.kappa;
    p.p0_f = (float)p.p0;
    p.visc_f = (float)p.visc;
    p.cfl_a_f = (float)p.cfl_a;
    p.cfl_v_f = (float)p.cfl_v;
    p.G = dd->n_features;
    for (int k = 0; k < MAXF; ++k) p.gdim[k] = k < dd->n_features ? dd->features[k].dim : 0;
    Domain& dm = I.dom;
    std::memset(&dm, 0, sizeof dm);
    dm.D = D;
    dm.base = dd->base;
    for (int a = 0; a < 3; ++a) {
        dm.lo[a] = dd->bbox_lo[a];
        dm.hi[a] = dd->bbox_hi[a];
        dm.bc[a] = dd->ball_center[a];
    }
    dm.br = dd->ball_radius;
    dm.nh = dd->n_holes;
    for (int k = 0; k < dd->n_holes; ++k) {
        for (int a = 0; a < 3; ++a) dm.hc[k][a] = dd->hole_center[k][a];
        dm.hr[k] = dd->hole_radius[k];
    }
    dm.nf = dd->n_features;
    for (int k = 0; k < dd->n_features; ++k) {
        const sph_feature& f = dd->features[k];
        Feat& F = dm.f[k];
        F.kind = f.kind;
        F.dim = f.dim;
        for (int a = 0; a < 12; ++a) F.g[a] = f.geom[a];
        for (int a = 0; a < 3; ++a) {
            F.nb[a] = f.normal[a];
            F.fnb[a] = (float)f.normal[a];
        }
        F.orient = f.orient;
        F.forient = (float)f.orient;
        if (f.kind == SPH_FEAT_SEGMENT) {
            double ab[3] = {f.geom[3] - f.geom[0], f.geom[4] - f.geom[1], f.geom[5] - f.geom[2]};
            double L = std::sqrt(ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2]);
            for (int a = 0; a < 3; ++a) F.ftg[a] = (float)(ab[a] / L);
        } else if (f.kind == SPH_FEAT_RECT) {
            for (int a = 0; a < 3; ++a) F.ftg[a] = (float)f.normal[a];
        }
        if (f.kind == SPH_FEAT_CIRCLE || f.kind == SPH_FEAT_SPHERE)
            for (int a = 0; a < 3; ++a) F.fc[a] = (float)f.geom[a];
        if (f.kind == SPH_FEAT_CIRCLE) F.fc[2] = 0.0f;
    }
    Sizing& zs = I.siz;
    std::memset(&zs, 0, sizeof zs);
    zs.kind = sz->kind;
    zs.a = sz->a;
    zs.b = sz->b;
    zs.lo = sz->lo;
    zs.hi = sz->hi;
    for (int a = 0; a < 3; ++a) zs.q[a] = sz->center[a];
    zs.nref = sz->n_ref;
    for (int k = 0; k < sz->n_ref; ++k) {
        for (int a = 0; a < 3; ++a) zs.rc[k][a] = sz->ref_center[k][a];
        zs.rr[k] = sz->ref_radius[k];
    }
    // float copies used by the FP32 evaluation of h_t and of the level set
    zs.fa = (float)zs.a;
    zs.fb = (float)zs.b;
    zs.flo = (float)zs.lo;
    zs.fhi = (float)zs.hi;
    for (int a = 0; a < 3; ++a) zs.fq[a] = (float)zs.q[a];
    for (int k = 0; k < MAXH; ++k) {
        for (int a = 0; a < 3; ++a) zs.frc[k][a] = (float)zs.rc[k][a];
        zs.frr[k] = (float)zs.rr[k];
    }
    for (int a = 0; a < 3; ++a) {
        dm.flo[a] = (float)dm.lo[a];
        dm.fhi[a] = (float)dm.hi[a];
        dm.fbc[a] = (float)dm.bc[a];
    }
    dm.fbr = (float)dm.br;
    for (int k = 0; k < MAXH; ++k) {
        for (int a = 0; a < 3; ++a) dm.fhc[k][a] = (float)dm.hc[k][a];
        dm.fhr[k] = (float)dm.hr[k];
    }
    return SPH_OK;
}

// the instance's phase, damping and attenuation, copied to every group
void host_ctrl_phase(Ctrl* c, int phase, double eps, double f) {
    c->phase = phase;
    c->eps = eps;
    c->f = f;
    c->eps_f = (float)eps;
    c->f_f = (float)f;
    for (int g = 0; g < MAXF; ++g) {
        c->gphase[g] = phase;
        c->geps[g] = eps;
        c->gf[g] = f;
        c->geps_f[g] = (float)eps;
        c->gf_f[g] = (float)f;
    }
}

void host_ctrl_init(Ctrl* c) {
    std::memset(c, 0, sizeof *c);
    c->sample_now = 1;
    host_ctrl_phase(c, PH1, 0.0, 1.0);
}

template <typename T> void ctrl_inf_bits(Ctrl* c) {
    for (int g = 0; g < MAXF; ++g) {
        c->dta_bits[g] = inf_bits<T>();
        c->dtv_bits[g] = inf_bits<T>();
    }
}

void ctrl_inf_bits(int prec, Ctrl* c) {
    if (prec == 32) ctrl_inf_bits<float>(c);
    else ctrl_inf_bits<double>(c);
}

// carve the per-slot arrays out of one allocation (256-byte aligned pieces)
template <typename T> size_t slot_layout(sph_batch* b, char* base, bool assign) {
    const size_t cap = (size_t)std::max(b->slot_cap, 1);
    const size_t nlanes = cap * (size_t)lpp_of(b->D);
    const size_t nblk = (size_t)div_up((long long)nlanes, BLOCK);
    const size_t vcap = (size_t)vcap_of(b->D);
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        off = (off + 255) & ~(size_t)255;
        char* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    State<T> s;
    std::memset(&s, 0, sizeof s);
    for (int a = 0; a < 3; ++a) {
        s.C[a] = (int*)take(cap * 4);
        s.O[a] = (T*)take(cap * sizeof(T));
        s.V[a] = (T*)take(cap * sizeof(T));
        s.Cs[a] = (int*)take(cap * 4);
        s.Os[a] = (T*)take(cap * sizeof(T));
    }
    s.VH = (Vec4<T>*)take(cap * sizeof(Vec4<T>));
    s.H = (T*)take(cap * sizeof(T));
    s.G = (unsigned*)take(cap * 4);
    s.ID = (int*)take(cap * 4);
    s.K = (int*)take(cap * 4);
    s.Ms = (unsigned*)take(cap * 4);
    s.IDs = (int*)take(cap * 4);
    s.Ks = (int*)take(cap * 4);
    s.P = (Vec4<T>*)take(cap * sizeof(Vec4<T>));
    s.A = (Vec4<T>*)take(cap * sizeof(Vec4<T>));
    s.perm = (int*)take(cap * 4);
    s.sperm = (int*)take(cap * 4);
    s.partials = (double*)take(nblk * MAXF * sizeof(double));
    s.partials2 = (double*)take((cap / CHUNK + 1) * MAXF * sizeof(double));
    s.pticket = (int*)take((cap / CHUNK + 1) * sizeof(int));
    s.vj = (int*)take(nlanes * vcap * 4);
    s.vr = (T*)take(nlanes * vcap * sizeof(T));
    s.vcnt = (int*)take(nlanes * 4);
    if (assign) {
        s.n = b->nslots;
        s.NI = b->NI;
        s.nblk = div_up((long long)b->nslots * lpp_of(b->D), BLOCK);
        s.inst_off = b->d_inst_off;
        s.inst_n = b->d_inst_n;
        s.chunk_inst = b->d_chunk_inst;
        s.grids = b->d_grids;
        s.params = b->d_params;
        s.doms = b->d_doms;
        s.sizs = b->d_sizs;
        s.ctrls = b->d_ctrl;
        st<T>(b) = s;
    }
    return off + 256;
}

template <typename T> void set_cell_arrays(sph_batch* b) {
    State<T>& s = st<T>(b);
    char* base = (char*)b->cpool;
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        off = (off + 255) & ~(size_t)255;
        char* p = base + off;
        off += bytes;
        return p;
    };
    s.count = (int*)take(b->cell_cap * 4);
    s.cell_start = (int*)take((b->cell_cap + 1) * 4);
    s.bsum = (int*)take((size_t)SCAN_TILE * 4);
    s.tstate = (unsigned long long*)take((size_t)div_up((long long)b->cell_cap, SCAN1_TILE) * 8);
    s.ticket = (int*)take(4);
    s.ntile = div_up(b->ncell, SCAN1_TILE);
    s.occ = (unsigned*)take(b->occ_cap * 4 * OCCW);
    s.ncell = b->ncell;
    s.nocc = b->nocc;
}

template <typename T, int D> void repack(sph_batch* b) { launch_repack<T, D>(st<T>(b), b->d_old_off, b->d_move_n, b->stream); }
template <typename T> void set_slots(sph_batch* b) {
    State<T>& s = st<T>(b);
    s.n = b->nslots;
    s.nblk = div_up((long long)b->nslots * lpp_of(b->D), BLOCK);
}

// Lays the batch out again after instance `changed` gets `new_n` particles (changed < 0: no
// count changes).  Slot ranges: the loaded instances in index order, each its count rounded up
// to CHUNK; the stored state of every other loaded instance is moved to its new range on the
// device.  Key ranges: each loaded instance's cells and its dummy key.  The per-cell arrays are
// reallocated if too small and cleared (the relative scan then starts from zero counts).
// Uploads the grids and the descriptors of instance `desc` (all instances for desc < 0).
// Fails with SPH_E_NOMEM, changing nothing, when the slots do not fit the allocation.
sph_status relayout(sph_batch* b, int changed, int new_n, int desc) {
    const int NI = b->NI;
    std::vector<int> old_off(NI), move(NI, 0), noff(NI + 1), nsl(NI), nn(NI);
    long long total = 0;
    for (int i = 0; i < NI; ++i) {
        const Inst& I = b->in[i];
        nn[i] = i == changed ? new_n : I.n;
        nsl[i] = (nn[i] + CHUNK - 1) / CHUNK * CHUNK;
        noff[i] = (int)total;
        total += nsl[i];
        old_off[i] = I.off;
        if (i != changed && I.slots > 0 && I.off != noff[i]) move[i] = I.slots;
    }
    noff[NI] = (int)total;
    if (total > b->slot_cap)
        return fail(SPH_E_NOMEM, "batch: %lld particle slots needed, %d allocated", total, b->slot_cap);
    long long keys = 0, occ = 0;
    for (int i = 0; i < NI; ++i)
        if (nn[i] > 0) {
            keys += b->in[i].ncell + 1;
            occ += b->in[i].nocc;
        }
    if (keys > MAX_KEYS)
        return fail(SPH_E_INVALID, "batch: %lld cell keys is more than the %lld supported", keys, (long long)MAX_KEYS);
    if (!b->cpool || (size_t)keys > b->cell_cap || (size_t)occ > b->occ_cap) {
        const size_t kc = std::max({(size_t)keys, b->cell_cap, (size_t)1});
        const size_t oc = std::max({(size_t)occ, b->occ_cap, (size_t)1});
        const size_t bytes = kc * 4 + (kc + 1) * 4 + (size_t)SCAN_TILE * 4 + oc * 4 * OCCW +
                             (size_t)div_up((long long)kc, SCAN1_TILE) * 8 + 4 + 6 * 256;
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess)
            return fail(SPH_E_NOMEM, "device allocation of %zu bytes of cell arrays failed", bytes);
        if (b->cpool) {
            CK(cudaStreamSynchronize(b->stream));
            cudaFree(b->cpool);
        }
        b->cpool = p;
        b->cell_cap = kc;
        b->occ_cap = oc;
    }
    // slots: chunk table, offsets, counts; then the moves
    std::vector<int> chunk((size_t)(total / CHUNK));
    for (int i = 0; i < NI; ++i)
        for (int c = noff[i] / CHUNK; c < (noff[i] + nsl[i]) / CHUNK; ++c) chunk[c] = i;
    if (!chunk.empty())
        CK(cudaMemcpyAsync(b->d_chunk_inst, chunk.data(), 4 * chunk.size(), cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(b->d_inst_off, noff.data(), 4 * (size_t)(NI + 1), cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(b->d_inst_n, nn.data(), 4 * (size_t)NI, cudaMemcpyHostToDevice, b->stream));
    b->nslots = (int)total;
    if (b->prec == 32) set_slots<float>(b);
    else set_slots<double>(b);
    if (std::any_of(move.begin(), move.end(), [](int v) { return v > 0; })) {
        CK(cudaMemcpyAsync(b->d_old_off, old_off.data(), 4 * (size_t)NI, cudaMemcpyHostToDevice, b->stream));
        CK(cudaMemcpyAsync(b->d_move_n, move.data(), 4 * (size_t)NI, cudaMemcpyHostToDevice, b->stream));
        DISPATCH(b, repack, b);
        CK(cudaGetLastError());
    }
    for (int i = 0; i < NI; ++i) {
        Inst& I = b->in[i];
        I.off = noff[i];
        I.slots = nsl[i];
        I.n = nn[i];
    }
    // keys
    long long kb = 0, ob = 0;
    for (Inst& I : b->in) {
        const bool loaded = I.n > 0;
        for (int l = 0; l < MAXL; ++l) I.grid.base[l] = (int)kb + (loaded ? I.lbase[l] : 0);
        I.grid.base[MAXL] = (int)kb + (loaded ? I.ncell : 0);   // the instance's dummy key (padding slots)
        I.grid.ncell = loaded ? I.ncell : 0;
        I.grid.occ_base = (int)ob;
        if (loaded) {
            kb += I.ncell + 1;
            ob += I.nocc;
        }
    }
    b->ncell = (int)keys;
    b->nocc = (int)occ;
    b->one.g = b->in[0].grid;
    b->one.p = b->in[0].params;
    if (b->prec == 32) set_cell_arrays<float>(b);
    else set_cell_arrays<double>(b);
    const State<float>& sf = b->sf;
    const State<double>& sd = b->sd;
    CK(cudaMemsetAsync(b->prec == 32 ? sf.count : sd.count, 0, (size_t)std::max<long long>(keys, 1) * 4, b->stream));
    CK(cudaMemsetAsync(b->prec == 32 ? sf.cell_start : sd.cell_start, 0, (size_t)(keys + 1) * 4, b->stream));
    CK(cudaMemsetAsync(b->prec == 32 ? sf.occ : sd.occ, 0, (size_t)std::max<long long>(occ, 1) * 4 * OCCW, b->stream));
    CK(cudaMemsetAsync(b->prec == 32 ? sf.tstate : sd.tstate, 0, (size_t)div_up(std::max<long long>(keys, 1), SCAN1_TILE) * 8,
                       b->stream));
    CK(cudaMemsetAsync(b->prec == 32 ? sf.ticket : sd.ticket, 0, 4, b->stream));
    std::vector<Grid> g(NI);
    for (int i = 0; i < NI; ++i) g[i] = b->in[i].grid;
    CK(cudaMemcpyAsync(b->d_grids, g.data(), sizeof(Grid) * NI, cudaMemcpyHostToDevice, b->stream));
    std::vector<Params> p;
    std::vector<Domain> d;
    std::vector<Sizing> z;
    const int d0 = desc < 0 ? 0 : desc, d1 = desc < 0 ? NI : desc + 1;
    for (int i = d0; i < d1; ++i) {
        p.push_back(b->in[i].params);
        d.push_back(b->in[i].dom);
        z.push_back(b->in[i].siz);
    }
    const size_t nd = (size_t)(d1 - d0);
    CK(cudaMemcpyAsync(b->d_params + d0, p.data(), sizeof(Params) * nd, cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(b->d_doms + d0, d.data(), sizeof(Domain) * nd, cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(b->d_sizs + d0, z.data(), sizeof(Sizing) * nd, cudaMemcpyHostToDevice, b->stream));
    CK(cudaStreamSynchronize(b->stream));   // the host vectors above go out of scope
    b->layout_version += 1;
    b->hashed = false;
    return SPH_OK;
}

void batch_free(sph_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    for (int k = 0; k < 5; ++k)
        if (b->ev[k]) cudaEventDestroy(b->ev[k]);
    cudaFree(b->pool);
    cudaFree(b->cpool);
    cudaFree(b->stage);
    cudaFree(b->d_grids);
    cudaFree(b->d_params);
    cudaFree(b->d_doms);
    cudaFree(b->d_sizs);
    cudaFree(b->d_ctrl);
    cudaFree(b->d_ctrl_dbg);
    cudaFree(b->d_inst_off);
    cudaFree(b->d_inst_n);
    cudaFree(b->d_chunk_inst);
    cudaFree(b->d_old_off);
    cudaFree(b->d_move_n);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

// Device side of a batch whose host instances are filled in: allocations for the sum of the
// instances' max_particles (each rounded up to CHUNK), descriptors, every instance empty.
sph_status batch_init(sph_batch* b, void* stream) {
    b->NI = (int)b->in.size();
    long long cap = 0;
    for (Inst& I : b->in) {
        I.off = 0;
        I.slots = 0;
        I.n = 0;
        cap += std::max<int64_t>(CHUNK, (I.cap + CHUNK - 1) / CHUNK * CHUNK);
    }
    if (cap * 12 >= ((long long)1 << 31))   // lane-indexed arrays hold slots * LPP * VCAP entries
        return fail(SPH_E_INVALID, "batch: %lld particle slots in total is too many", cap);
    b->slot_cap = (int)cap;
    b->nslots = 0;
    if (cudaGetDevice(&b->device) != cudaSuccess) return fail(SPH_E_CUDA, "no CUDA device");
    if (stream) b->stream = (cudaStream_t)stream;
    else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(SPH_E_CUDA, "cudaStreamCreate failed");
        b->own_stream = true;
    }
    const int NI = b->NI;
    if (cudaMalloc(&b->d_grids, sizeof(Grid) * NI) != cudaSuccess ||
        cudaMalloc(&b->d_params, sizeof(Params) * NI) != cudaSuccess ||
        cudaMalloc(&b->d_doms, sizeof(Domain) * NI) != cudaSuccess ||
        cudaMalloc(&b->d_sizs, sizeof(Sizing) * NI) != cudaSuccess ||
        cudaMalloc(&b->d_ctrl, sizeof(Ctrl) * NI) != cudaSuccess ||
        cudaMalloc(&b->d_ctrl_dbg, sizeof(Ctrl) * NI) != cudaSuccess ||
        cudaMalloc(&b->d_inst_off, sizeof(int) * (NI + 1)) != cudaSuccess ||
        cudaMalloc(&b->d_inst_n, sizeof(int) * NI) != cudaSuccess ||
        cudaMalloc(&b->d_old_off, sizeof(int) * NI) != cudaSuccess ||
        cudaMalloc(&b->d_move_n, sizeof(int) * NI) != cudaSuccess ||
        cudaMalloc(&b->d_chunk_inst, sizeof(int) * (size_t)(b->slot_cap / CHUNK)) != cudaSuccess)
        return fail(SPH_E_NOMEM, "device allocation of descriptors failed");
    const size_t bytes = b->prec == 32 ? slot_layout<float>(b, nullptr, false) : slot_layout<double>(b, nullptr, false);
    if (cudaMalloc(&b->pool, bytes) != cudaSuccess)
        return fail(SPH_E_NOMEM, "device allocation of %zu bytes failed", bytes);
    if (b->prec == 32) slot_layout<float>(b, (char*)b->pool, true);
    else slot_layout<double>(b, (char*)b->pool, true);
    CK(cudaMemsetAsync(b->pool, 0, bytes, b->stream));
    std::vector<Ctrl> c(NI);
    for (int i = 0; i < NI; ++i) {
        host_ctrl_init(&c[i]);
        ctrl_inf_bits(b->prec, &c[i]);
    }
    CK(cudaMemcpyAsync(b->d_ctrl, c.data(), sizeof(Ctrl) * NI, cudaMemcpyHostToDevice, b->stream));
    sph_status r = relayout(b, -1, 0, -1);   // synchronises the stream
    if (r != SPH_OK) return r;
    for (int k = 0; k < 5; ++k)
        if (cudaEventCreate(&b->ev[k]) != cudaSuccess) return fail(SPH_E_CUDA, "cudaEventCreate failed");
    return SPH_OK;
}

const One* one_of(const sph_batch* b) { return b->NI == 1 ? &b->one : nullptr; }

// keys + histogram of the stored state, unless the last update already computed them
template <typename T, int D> void ensure_hashed(sph_batch* b, const State<T>& s, cudaStream_t stream) {
    if (b->hashed) return;
    launch_hash<T, D>(s, one_of(b), stream);
    b->hashed = true;
}

// the rebuild after the keys and histogram are in place (they are consumed by the scatter)
template <typename T, int D> void enqueue_rebuild(const sph_batch* b, const State<T>& s, cudaStream_t stream) {
    launch_scan_onepass<T>(s, stream);
    launch_scatter<T>(s, stream, true);
    launch_gather<T, D>(s, one_of(b), stream, true);
}

template <typename T> Out<T> out_stored(const State<T>& s) {
    Out<T> o;
    for (int a = 0; a < 3; ++a) {
        o.C[a] = s.C[a];
        o.O[a] = s.O[a];
        o.V[a] = s.V[a];
        o.av[a] = nullptr;
    }
    o.H = s.H;
    o.G = s.G;
    o.ID = s.ID;
    o.K = s.K;
    o.count = s.count;
    return o;
}

template <typename T, int D> void enqueue_step(sph_batch* b, bool timed) {
    const State<T>& s = st<T>(b);
    cudaStream_t stream = b->stream;
    bool seq = false;
    for (const Inst& I : b->in) seq = seq || (I.n > 0 && I.params.feature_order != 0);
    if (seq) {
        // Algorithm 1's feature loop in sequence: one pass per dimension class (curves, surfaces,
        // volume), each re-sorting the state the previous pass left (the update writes the next
        // keys and histogram) and moving its class; the stage events bracket the first pass and
        // the step's end
        for (int cls = 1; cls <= D; ++cls) {
            const bool first = cls == 1;
            if (timed && first) cudaEventRecordWithFlags(b->ev[0], stream, cudaEventRecordExternal);
            enqueue_rebuild<T, D>(b, s, stream);
            if (timed && first) cudaEventRecordWithFlags(b->ev[1], stream, cudaEventRecordExternal);
            launch_interact<T, D>(s, one_of(b), nullptr, nullptr, stream, !timed, cls);
            if (timed && first) cudaEventRecordWithFlags(b->ev[2], stream, cudaEventRecordExternal);
            launch_control<T, D>(s, one_of(b), stream, !timed, cls);
            if (timed && first) cudaEventRecordWithFlags(b->ev[3], stream, cudaEventRecordExternal);
            launch_integrate<T, D>(s, one_of(b), s.ctrls, out_stored<T>(s), stream, !timed, cls);
        }
        if (timed) cudaEventRecordWithFlags(b->ev[4], stream, cudaEventRecordExternal);
        return;
    }
    if (timed) cudaEventRecordWithFlags(b->ev[0], stream, cudaEventRecordExternal);
    enqueue_rebuild<T, D>(b, s, stream);
    if (timed) cudaEventRecordWithFlags(b->ev[1], stream, cudaEventRecordExternal);
    // kernel-to-kernel edges start the successor early (programmatic dependent launch); an
    // event between two kernels makes the edge an ordinary one
    launch_interact<T, D>(s, one_of(b), nullptr, nullptr, stream, !timed);
    if (timed) cudaEventRecordWithFlags(b->ev[2], stream, cudaEventRecordExternal);
    launch_control<T, D>(s, one_of(b), stream, !timed);
    if (timed) cudaEventRecordWithFlags(b->ev[3], stream, cudaEventRecordExternal);
    launch_integrate<T, D>(s, one_of(b), s.ctrls, out_stored<T>(s), stream, !timed);
    if (timed) cudaEventRecordWithFlags(b->ev[4], stream, cudaEventRecordExternal);
}

sph_status collect_timing(sph_batch* b) {
    if (!b->ev_pending) return SPH_OK;
    CK(cudaEventSynchronize(b->ev[NSTAGE]));
    for (int k = 0; k < NSTAGE; ++k) {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, b->ev[k], b->ev[k + 1]));
        b->stage_ms[k] += ms;
    }
    b->stage_steps += 1;
    b->ev_pending = false;
    return SPH_OK;
}

template <typename T, int D> sph_status build_graph(sph_batch* b) {
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    enqueue_step<T, D>(b, b->timing);
    cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
    if (e != cudaSuccess) return fail(SPH_E_CUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(SPH_E_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    b->graph_version = b->layout_version;
    b->graph_timed = b->timing;
    return SPH_OK;
}

template <typename T, int D> sph_status step_impl(sph_batch* b, int32_t n_steps) {
    if (b->nslots == 0) return SPH_OK;   // nothing loaded
    CK(cudaSetDevice(b->device));
    if (!b->gexec || b->graph_version != b->layout_version || b->graph_timed != b->timing) {
        sph_status r = build_graph<T, D>(b);
        if (r != SPH_OK) return r;
    }
    if (n_steps > 0) ensure_hashed<T, D>(b, st<T>(b), b->stream);
    for (int i = 0; i < n_steps; ++i) {
        if (b->timing) {
            sph_status r = collect_timing(b);
            if (r != SPH_OK) return r;
        }
        CK(cudaGraphLaunch(b->gexec, b->stream));
        if (b->timing) b->ev_pending = true;
    }
    return SPH_OK;
}


// a device buffer of at least `bytes` for the caller's arrays (grown on demand, kept)
char* stage_buf(sph_batch* b, size_t bytes) {
    if (b->stage_cap < bytes) {
        if (b->stage) {
            cudaStreamSynchronize(b->stream);
            cudaFree(b->stage);
            b->stage = nullptr;
            b->stage_cap = 0;
        }
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        b->stage = p;
        b->stage_cap = bytes;
    }
    return static_cast<char*>(b->stage);
}

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

IoGrid io_grid(const Inst& I) {
    IoGrid g;
    std::memset(&g, 0, sizeof g);
    for (int a = 0; a < 3; ++a) {
        g.origin[a] = I.grid.origin[a];
        g.dims0[a] = I.grid.dims[0][a];
    }
    g.c0 = I.grid.c[0];
    g.inv_c0 = I.grid.inv_c[0];
    for (int k = 0; k < MAXF; ++k) g.fdim[k] = (unsigned char)I.dom.f[k].dim;
    return g;
}

// one instance's slots in device memory -> host arrays in its original order (arrays indexed
// by global slot; the instance's range is read).  A kernel writes the outputs in input order
// into the staging buffer, then each requested array is copied out once.
template <typename T>
sph_status download(sph_batch* b, int inst, int* const Cd[3], T* const Od[3], T* const V[3], T* H, unsigned* G,
                    int* ID, double* x_out, int32_t* group_out, double* v_out, double* h_out) {
    const Inst& I = b->in[inst];
    const int ns = I.slots, o0 = I.off, n = I.n, D = b->D;
    const size_t nx = up256((size_t)n * 24), nh = up256((size_t)n * 8), ng = up256((size_t)n * 4);
    char* p = stage_buf(b, 256 + 2 * nx + nh + ng);
    if (!p) return fail(SPH_E_NOMEM, "device allocation of the positions' staging buffer failed");
    int* cnt = reinterpret_cast<int*>(p);
    double* dx = x_out ? reinterpret_cast<double*>(p + 256) : nullptr;
    double* dv = v_out ? reinterpret_cast<double*>(p + 256 + nx) : nullptr;
    double* dh = h_out ? reinterpret_cast<double*>(p + 256 + 2 * nx) : nullptr;
    int* dg = group_out ? reinterpret_cast<int*>(p + 256 + 2 * nx + nh) : nullptr;
    ConstSlotArrays<T> sa;
    std::memset(&sa, 0, sizeof sa);
    for (int a = 0; a < D; ++a) {
        sa.C[a] = Cd[a] + o0;
        sa.O[a] = Od[a] + o0;
        sa.V[a] = V[a] + o0;
    }
    sa.H = H + o0;
    sa.G = G + o0;
    sa.ID = ID + o0;
    CK(cudaMemsetAsync(cnt, 0, 8, b->stream));
    if (D == 2) launch_store_state<T, 2>(sa, io_grid(I), ns, n, dx, dg, dv, dh, cnt, b->stream);
    else launch_store_state<T, 3>(sa, io_grid(I), ns, n, dx, dg, dv, dh, cnt, b->stream);
    CK(cudaGetLastError());
    int hc[2] = {0, 0};
    CK(cudaMemcpyAsync(hc, cnt, 8, cudaMemcpyDeviceToHost, b->stream));
    if (x_out) CK(cudaMemcpyAsync(x_out, dx, (size_t)n * 24, cudaMemcpyDeviceToHost, b->stream));
    if (v_out) CK(cudaMemcpyAsync(v_out, dv, (size_t)n * 24, cudaMemcpyDeviceToHost, b->stream));
    if (h_out) CK(cudaMemcpyAsync(h_out, dh, (size_t)n * 8, cudaMemcpyDeviceToHost, b->stream));
    if (group_out) CK(cudaMemcpyAsync(group_out, dg, (size_t)n * 4, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    if (hc[1] != 0 || hc[0] != n) return fail(SPH_E_CUDA, "corrupt particle index on the device");
    return SPH_OK;
}

sph_status check_args(const sph_batch* b, int inst, int64_t n, const double* x, const int32_t* group, const double*,
                      const double*) {
    const Inst& I = b->in[inst];
    const int64_t cap = b->mesh ? I.cap : (int64_t)b->slot_cap;
    if (n < 0 || n > cap) return fail(SPH_E_INVALID, "set_state: n=%lld outside [0, %lld]", (long long)n, (long long)cap);
    if (n > 0 && (!x || !group)) return fail(SPH_E_INVALID, "set_state: x and group are required");
    return SPH_OK;   // the particles themselves are checked on the device by set_state_impl
}

// Loads one instance's particles into its slots (live first, padding after) and resets its
// controller: Phase One at step 0, or, for an empty batch instance, the idle state DONE.
template <typename T, int D> sph_status set_state_impl(sph_batch* b, int inst, int64_t n, const double* x,
                                                       const int32_t* group, const double* v, const double* h,
                                                       bool idle_when_empty, const Ctrl* keep = nullptr) {
    State<T>& s = st<T>(b);
    Inst& I = b->in[inst];
    const int nn = (int)n;
    CK(cudaSetDevice(b->device));
    // the caller's arrays as they are, on the device: checked there before anything changes
    const size_t nx = up256((size_t)nn * 24), ng = up256((size_t)nn * 4), nh = up256((size_t)nn * 8);
    char* p = stage_buf(b, 256 + 2 * nx + ng + nh);
    if (!p) return fail(SPH_E_NOMEM, "device allocation of the particles' staging buffer failed");
    unsigned long long* first = reinterpret_cast<unsigned long long*>(p);
    double* dx = reinterpret_cast<double*>(p + 256);
    int* dg = reinterpret_cast<int*>(p + 256 + nx);
    double* dv = v ? reinterpret_cast<double*>(p + 256 + nx + ng) : nullptr;
    double* dh = h ? reinterpret_cast<double*>(p + 256 + 2 * nx + ng) : nullptr;
    if (nn > 0) {
        CK(cudaMemcpyAsync(dx, x, (size_t)nn * 24, cudaMemcpyHostToDevice, b->stream));
        CK(cudaMemcpyAsync(dg, group, (size_t)nn * 4, cudaMemcpyHostToDevice, b->stream));
        if (v) CK(cudaMemcpyAsync(dv, v, (size_t)nn * 24, cudaMemcpyHostToDevice, b->stream));
        if (h) CK(cudaMemcpyAsync(dh, h, (size_t)nn * 8, cudaMemcpyHostToDevice, b->stream));
        IoCheck c;
        std::memset(&c, 0, sizeof c);
        for (int a = 0; a < D; ++a) {
            const double lo = I.dom.lo[a], hi = I.dom.hi[a];
            c.lo[a] = lo - 1e-9 * (1 + std::fabs(lo));
            c.hi[a] = hi + 1e-9 * (1 + std::fabs(hi));
        }
        // the grid's top level covers kappa*h_hi*(1+2^-10); h up to h_hi*(1+2^-11) is accepted so
        // that values rounded to the working precision pass
        c.hmax = I.h_hi * (1 + 1.0 / 2048.0);
        c.G = I.params.G;
        c.D = D;
        CK(cudaMemsetAsync(first, 0xff, 8, b->stream));
        launch_check_state(c, nn, dx, dg, dv, dh, first, b->stream);
        CK(cudaGetLastError());
        unsigned long long f = 0;
        CK(cudaMemcpyAsync(&f, first, 8, cudaMemcpyDeviceToHost, b->stream));
        CK(cudaStreamSynchronize(b->stream));
        if (f != ~0ull) {
            const long long i = (long long)(f >> 2);
            switch ((int)(f & 3)) {
            case 0: return fail(SPH_E_INVALID, "set_state: particle %lld has group %d", i, group[i]);
            case 1: return fail(SPH_E_INVALID, "set_state: particle %lld outside the bounding box", i);
            case 2: return fail(SPH_E_INVALID, "set_state: h of particle %lld outside [lo, hi]", i);
            default: return fail(SPH_E_INVALID, "set_state: non-finite velocity");
            }
        }
    }
    sph_status r = relayout(b, inst, nn, inst);   // makes room (moving the other instances)
    if (r != SPH_OK) return r;
    const int ns = I.slots, o0 = I.off;
    SlotArrays<T> sa;
    std::memset(&sa, 0, sizeof sa);
    for (int a = 0; a < D; ++a) {
        sa.C[a] = s.C[a] + o0;
        sa.O[a] = s.O[a] + o0;
        sa.V[a] = s.V[a] + o0;
    }
    sa.H = s.H + o0;
    sa.G = s.G + o0;
    sa.ID = s.ID + o0;
    launch_load_state<T, D>(sa, io_grid(I), ns, nn, dx, dg, dv, dh, b->stream);
    if (!h && nn > 0) launch_init_h<T, D>(s, inst, b->stream);
    Ctrl c;
    host_ctrl_init(&c);
    ctrl_inf_bits<T>(&c);
    if (nn == 0 && idle_when_empty) {
        host_ctrl_phase(&c, PH_DONE, 0.0, 0.0);
        c.sample_now = 0;
    }
    if (keep) c = *keep;   // re-representation of the same state: the controller carries on
    CK(cudaMemcpyAsync(b->d_ctrl + inst, &c, sizeof c, cudaMemcpyHostToDevice, b->stream));
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(b->stream));
    b->stage_steps = 0;
    for (double& t : b->stage_ms) t = 0;
    b->ev_pending = false;
    return SPH_OK;
}

// a copy of the state whose controllers are the scratch controllers (inspection calls never
// touch the real ones)
template <typename T> sph_status dbg_state(sph_batch* b, State<T>& out, const Ctrl* init) {
    out = st<T>(b);
    std::vector<Ctrl> c(b->NI);
    if (init) std::fill(c.begin(), c.end(), *init);
    else {
        CK(cudaMemcpyAsync(c.data(), b->d_ctrl, sizeof(Ctrl) * b->NI, cudaMemcpyDeviceToHost, b->stream));
        CK(cudaStreamSynchronize(b->stream));
    }
    for (Ctrl& x : c) {
        ctrl_inf_bits<T>(&x);
        x.sample_now = 0;
        if (!init && x.phase == PH_DONE) x.phase = PH2;   // inspect a converged state as well
        for (int g = 0; g < MAXF; ++g)
            if (!init && x.gphase[g] == PH_DONE) x.gphase[g] = PH2;
    }
    CK(cudaMemcpyAsync(b->d_ctrl_dbg, c.data(), sizeof(Ctrl) * b->NI, cudaMemcpyHostToDevice, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    out.ctrls = b->d_ctrl_dbg;
    return SPH_OK;
}

template <typename T, int D> sph_status dbg_prepare(sph_batch* b, State<T>& s, const Ctrl* init) {
    sph_status r = dbg_state<T>(b, s, init);
    if (r != SPH_OK) return r;
    ensure_hashed<T, D>(b, s, b->stream);
    enqueue_rebuild<T, D>(b, s, b->stream);
    b->hashed = false;   // the scatter consumed the histogram; the stored state is unchanged
    CK(cudaGetLastError());
    return SPH_OK;
}

// The inspection entry points serve a mesh (a batch of one: instance 0, slots from 0).
template <typename T, int D> sph_status dbg_rebuild_impl(sph_batch* b, int64_t* key_out, int64_t* cs_out, int64_t* perm_out) {
    State<T> s;
    sph_status r = dbg_prepare<T, D>(b, s, nullptr);
    if (r != SPH_OK) return r;
    const int n = b->in[0].n, nc = b->in[0].ncell;
    std::vector<int> k(n), cs(nc + 1), p(n);
    CK(cudaMemcpyAsync(k.data(), s.K, 4 * (size_t)n, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaMemcpyAsync(cs.data(), s.cell_start, 4 * (size_t)(nc + 1), cudaMemcpyDeviceToHost, b->stream));
    CK(cudaMemcpyAsync(p.data(), s.sperm, 4 * (size_t)n, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    for (int i = 0; i < n; ++i) {
        if (key_out) key_out[i] = k[i];
        if (perm_out) perm_out[i] = p[i];
    }
    if (cs_out)
        for (int c = 0; c <= nc; ++c) cs_out[c] = cs[c];
    return SPH_OK;
}

template <typename T, int D>
sph_status dbg_neighbors_impl(sph_batch* b, int32_t mode, int64_t* counts_out, int32_t* lists_out, int64_t cap,
                              int64_t* total_out) {
    State<T> s;
    sph_status r = dbg_prepare<T, D>(b, s, nullptr);
    if (r != SPH_OK) return r;
    const int ns = s.n, n = b->in[0].n;
    int* d_counts = nullptr;
    long long* d_off = nullptr;
    int* d_lists = nullptr;
    CK(cudaMalloc(&d_counts, 4 * (size_t)std::max(ns, 1)));
    launch_neighbors<T, D>(s, mode, d_counts, nullptr, nullptr, b->stream);
    std::vector<int> cnt(ns), ids(ns);
    CK(cudaMemcpyAsync(cnt.data(), d_counts, 4 * (size_t)ns, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaMemcpyAsync(ids.data(), s.IDs, 4 * (size_t)ns, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    std::vector<long long> off(ns + 1, 0);
    for (int k = 0; k < ns; ++k) off[k + 1] = off[k] + cnt[k];
    const long long total = off[ns];
    CK(cudaMalloc(&d_off, sizeof(long long) * (size_t)(ns + 1)));
    CK(cudaMalloc(&d_lists, 4 * (size_t)std::max<long long>(total, 1)));
    CK(cudaMemcpyAsync(d_off, off.data(), sizeof(long long) * (size_t)(ns + 1), cudaMemcpyHostToDevice, b->stream));
    launch_neighbors<T, D>(s, mode, d_counts, d_off, d_lists, b->stream);
    std::vector<int> lists((size_t)std::max<long long>(total, 1));
    CK(cudaMemcpyAsync(lists.data(), d_lists, 4 * (size_t)total, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    cudaFree(d_counts);
    cudaFree(d_off);
    cudaFree(d_lists);
    // regroup by original index, map sorted slots to original indices, ascending
    std::vector<int> slot_of(n, -1);
    for (int k = 0; k < ns; ++k)
        if (ids[k] >= 0 && ids[k] < n) slot_of[ids[k]] = k;
    long long w = 0;
    bool overflow = false;
    for (int i = 0; i < n; ++i) {
        const int k = slot_of[i];
        if (k < 0) return fail(SPH_E_CUDA, "corrupt particle index on the device");
        std::vector<int> li(lists.begin() + off[k], lists.begin() + off[k + 1]);
        for (int& j : li) j = ids[j];
        std::sort(li.begin(), li.end());
        if (counts_out) counts_out[i] = (int64_t)li.size();
        for (int j : li) {
            if (lists_out && w < cap) lists_out[w] = j;
            else if (lists_out) overflow = true;
            ++w;
        }
    }
    if (total_out) *total_out = w;
    if (overflow) return fail(SPH_E_OVERFLOW, "neighbour list capacity %lld < %lld", (long long)cap, (long long)w);
    return SPH_OK;
}

template <typename T, int D>
sph_status dbg_interact_impl(sph_batch* b, double* a_p, double* sigma, double* gamma, double* dta, double* dtv) {
    State<T> s;
    sph_status r = dbg_prepare<T, D>(b, s, nullptr);
    if (r != SPH_OK) return r;
    const int ns = s.n, n = b->in[0].n, G = b->in[0].params.G;
    T *d_sig = nullptr, *d_gam = nullptr;
    CK(cudaMalloc(&d_sig, sizeof(T) * (size_t)std::max(ns, 1)));
    CK(cudaMalloc(&d_gam, sizeof(T) * (size_t)std::max(ns, 1)));
    launch_interact<T, D>(s, one_of(b), d_sig, d_gam, b->stream);
    CK(cudaGetLastError());
    std::vector<Vec4<T>> A(ns);
    std::vector<T> sg(ns), gm(ns);
    std::vector<int> ids(ns);
    Ctrl c;
    CK(cudaMemcpyAsync(A.data(), s.A, sizeof(Vec4<T>) * (size_t)ns, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaMemcpyAsync(sg.data(), d_sig, sizeof(T) * (size_t)ns, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaMemcpyAsync(gm.data(), d_gam, sizeof(T) * (size_t)ns, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaMemcpyAsync(ids.data(), s.IDs, 4 * (size_t)ns, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaMemcpyAsync(&c, b->d_ctrl_dbg, sizeof c, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    cudaFree(d_sig);
    cudaFree(d_gam);
    for (int k = 0; k < ns; ++k) {
        const int i = ids[k];
        if (i < 0 || i >= n) continue;
        if (a_p) {
            a_p[(size_t)i * 3 + 0] = (double)A[k].x;
            a_p[(size_t)i * 3 + 1] = (double)A[k].y;
            a_p[(size_t)i * 3 + 2] = D == 3 ? (double)A[k].z : 0.0;
        }
        if (sigma) sigma[i] = (double)sg[k];
        if (gamma) gamma[i] = (double)gm[k];
    }
    for (int g = 0; g < G; ++g) {
        T a, bb;
        if (sizeof(T) == 4) {
            unsigned ua = (unsigned)c.dta_bits[g], ub = (unsigned)c.dtv_bits[g];
            float fa, fb;
            std::memcpy(&fa, &ua, 4);
            std::memcpy(&fb, &ub, 4);
            a = (T)fa;
            bb = (T)fb;
        } else {
            double fa, fb;
            std::memcpy(&fa, &c.dta_bits[g], 8);
            std::memcpy(&fb, &c.dtv_bits[g], 8);
            a = (T)fa;
            bb = (T)fb;
        }
        if (dta) dta[g] = (double)a;
        if (dtv) dtv[g] = (double)bb;
    }
    return SPH_OK;
}

template <typename T, int D>
sph_status dbg_update_impl(sph_batch* b, const double* dt, const int32_t* reset, double eps, double f, double* x_out,
                           double* v_out, double* h_out, double* a_v) {
    const int G = b->in[0].params.G;
    Ctrl c;
    host_ctrl_init(&c);
    for (int g = 0; g < G; ++g) {
        c.dt[g] = dt[g];
        c.dt_f[g] = (float)dt[g];
        c.reset[g] = reset[g];
    }
    host_ctrl_phase(&c, PH1, eps, f);
    State<T> s;
    sph_status r = dbg_prepare<T, D>(b, s, &c);
    if (r != SPH_OK) return r;
    launch_interact<T, D>(s, one_of(b), nullptr, nullptr, b->stream);
    // scratch output arrays
    Out<T> o;
    void* buf = nullptr;
    const size_t nn = (size_t)std::max(s.n, 1);
    const size_t bytes = nn * (3 * 4 + 9 * sizeof(T) + sizeof(T) + 8) + 20 * 256;
    CK(cudaMalloc(&buf, bytes));
    char* p = (char*)buf;
    auto take = [&](size_t sz) {
        char* q = p;
        p += (sz + 255) & ~(size_t)255;
        return q;
    };
    for (int a = 0; a < 3; ++a) o.C[a] = (int*)take(nn * 4);
    for (int a = 0; a < 3; ++a) o.O[a] = (T*)take(nn * sizeof(T));
    for (int a = 0; a < 3; ++a) o.V[a] = (T*)take(nn * sizeof(T));
    for (int a = 0; a < 3; ++a) o.av[a] = (T*)take(nn * sizeof(T));
    o.H = (T*)take(nn * sizeof(T));
    o.G = (unsigned*)take(nn * 4);
    o.ID = (int*)take(nn * 4);
    o.K = nullptr;       // scratch output: no keys for a next step
    o.count = nullptr;
    launch_integrate<T, D>(s, one_of(b), b->d_ctrl_dbg, o, b->stream);
    CK(cudaGetLastError());
    r = download<T>(b, 0, o.C, o.O, o.V, o.H, o.G, o.ID, x_out, nullptr, v_out, h_out);
    if (r == SPH_OK && a_v) {
        T* const avs[3] = {o.av[0], o.av[1], o.av[2]};
        r = download<T>(b, 0, o.C, o.O, avs, o.H, o.G, o.ID, nullptr, nullptr, a_v, nullptr);
    }
    cudaFree(buf);
    return r;
}

template <typename T, int D> sph_status pair_counts_impl(sph_batch* b, int64_t* cand, int64_t* accd) {
    State<T> s;
    sph_status r = dbg_prepare<T, D>(b, s, nullptr);
    if (r != SPH_OK) return r;
    unsigned long long* d = nullptr;
    CK(cudaMalloc(&d, 16));
    CK(cudaMemsetAsync(d, 0, 16, b->stream));
    launch_pair_counts<T, D>(s, d, b->stream);
    unsigned long long h[2];
    CK(cudaMemcpyAsync(h, d, 16, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    cudaFree(d);
    if (cand) *cand = (int64_t)h[0];
    if (accd) *accd = (int64_t)h[1];
    return SPH_OK;
}

template <typename T, int D>
sph_status positions_impl(sph_batch* b, int inst, double* x_out, int32_t* group_out, double* v_out, double* h_out) {
    State<T>& s = st<T>(b);
    return download<T>(b, inst, s.C, s.O, s.V, s.H, s.G, s.ID, x_out, group_out, v_out, h_out);
}

sph_status read_ctrls(sph_batch* b, std::vector<Ctrl>& c) {
    c.resize(b->NI);
    CK(cudaMemcpyAsync(c.data(), b->d_ctrl, sizeof(Ctrl) * b->NI, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    return SPH_OK;
}

// ---- checkpoint / resume ----
// A snapshot holds one instance's particles exactly as stored (finest cell, offset, velocity,
// h, meta, input index, in stored order, padding included), its controller, and a fingerprint
// of its problem and grid, so that a restored instance continues bit for bit.
struct SnapHeader {
    char magic[8];
    int32_t version, dim, precision, n, slots, pad;
    uint64_t fingerprint;
    uint64_t payload;
};
constexpr char kSnapMagic[8] = {'S', 'P', 'H', 'S', 'N', 'A', 'P', '1'};

uint64_t fnv(uint64_t h, const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
        h ^= c[i];
        h *= 1099511628211ull;
    }
    return h;
}

// the instance's problem and grid, independent of where the batch put it
uint64_t fingerprint(const Inst& I, int prec) {
    Grid g = I.grid;
    for (int l = 0; l <= MAXL; ++l) g.base[l] = 0;
    g.occ_base = 0;
    g.ncell = I.ncell;
    uint64_t h = 14695981039346656037ull;
    h = fnv(h, &prec, sizeof prec);
    h = fnv(h, &g, sizeof g);
    h = fnv(h, I.lbase, sizeof I.lbase);
    h = fnv(h, &I.params, sizeof I.params);
    h = fnv(h, &I.dom, sizeof I.dom);
    h = fnv(h, &I.siz, sizeof I.siz);
    return h;
}

template <typename T> size_t slot_bytes_of(int D) { return (size_t)D * (4 + 2 * sizeof(T)) + sizeof(T) + 8; }

template <typename T, int D>
sph_status snapshot_impl(sph_batch* b, int inst, void* buf, size_t cap, size_t* used) {
    const Inst& I = b->in[inst];
    const size_t payload = sizeof(Ctrl) + (size_t)I.slots * slot_bytes_of<T>(D);
    const size_t need = sizeof(SnapHeader) + payload;
    if (used) *used = need;
    if (!buf) return SPH_OK;
    if (cap < need) return fail(SPH_E_OVERFLOW, "snapshot: %zu bytes needed, %zu given", need, cap);
    SnapHeader hd;
    std::memset(&hd, 0, sizeof hd);
    std::memcpy(hd.magic, kSnapMagic, 8);
    hd.version = 1;
    hd.dim = D;
    hd.precision = b->prec;
    hd.n = I.n;
    hd.slots = I.slots;
    hd.fingerprint = fingerprint(I, b->prec);
    hd.payload = payload;
    char* p = static_cast<char*>(buf);
    std::memcpy(p, &hd, sizeof hd);
    p += sizeof hd;
    State<T>& s = st<T>(b);
    const int o0 = I.off, ns = I.slots;
    CK(cudaMemcpyAsync(p, b->d_ctrl + inst, sizeof(Ctrl), cudaMemcpyDeviceToHost, b->stream));
    p += sizeof(Ctrl);
    for (int a = 0; a < D; ++a) {
        CK(cudaMemcpyAsync(p, s.C[a] + o0, 4 * (size_t)ns, cudaMemcpyDeviceToHost, b->stream));
        p += 4 * (size_t)ns;
        CK(cudaMemcpyAsync(p, s.O[a] + o0, sizeof(T) * ns, cudaMemcpyDeviceToHost, b->stream));
        p += sizeof(T) * ns;
        CK(cudaMemcpyAsync(p, s.V[a] + o0, sizeof(T) * ns, cudaMemcpyDeviceToHost, b->stream));
        p += sizeof(T) * ns;
    }
    CK(cudaMemcpyAsync(p, s.H + o0, sizeof(T) * ns, cudaMemcpyDeviceToHost, b->stream));
    p += sizeof(T) * ns;
    CK(cudaMemcpyAsync(p, s.G + o0, 4 * (size_t)ns, cudaMemcpyDeviceToHost, b->stream));
    p += 4 * (size_t)ns;
    CK(cudaMemcpyAsync(p, s.ID + o0, 4 * (size_t)ns, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    return SPH_OK;
}

template <typename T, int D> sph_status restore_impl(sph_batch* b, int inst, const void* buf, size_t len) {
    SnapHeader hd;
    if (len < sizeof hd) return fail(SPH_E_INVALID, "restore: buffer shorter than a snapshot header");
    std::memcpy(&hd, buf, sizeof hd);
    if (std::memcmp(hd.magic, kSnapMagic, 8) != 0 || hd.version != 1)
        return fail(SPH_E_INVALID, "restore: not a snapshot of this library");
    if (hd.dim != D || hd.precision != b->prec)
        return fail(SPH_E_INVALID, "restore: snapshot of a %dD, precision %d instance", hd.dim, hd.precision);
    Inst& I = b->in[inst];
    if (hd.fingerprint != fingerprint(I, b->prec))
        return fail(SPH_E_INVALID, "restore: the snapshot is of another problem or grid");
    const int64_t cap = b->mesh ? I.cap : (int64_t)b->slot_cap;
    if (hd.n < 0 || hd.n > cap || hd.slots != (hd.n + CHUNK - 1) / CHUNK * CHUNK)
        return fail(SPH_E_INVALID, "restore: particle count out of range");
    const size_t payload = sizeof(Ctrl) + (size_t)hd.slots * slot_bytes_of<T>(D);
    if (hd.payload != payload || len < sizeof hd + payload) return fail(SPH_E_INVALID, "restore: truncated snapshot");
    const char* p = static_cast<const char*>(buf) + sizeof hd;
    Ctrl c;
    std::memcpy(&c, p, sizeof c);
    p += sizeof c;
    // host copies: the device reads them after this function returns the stream synchronised
    const int ns = hd.slots;
    std::vector<char> data(p, p + (payload - sizeof(Ctrl)));
    CK(cudaSetDevice(b->device));
    sph_status r = relayout(b, inst, hd.n, inst);
    if (r != SPH_OK) return r;
    State<T>& s = st<T>(b);
    const int o0 = I.off;
    const char* q = data.data();
    for (int a = 0; a < D; ++a) {
        CK(cudaMemcpyAsync(s.C[a] + o0, q, 4 * (size_t)ns, cudaMemcpyHostToDevice, b->stream));
        q += 4 * (size_t)ns;
        CK(cudaMemcpyAsync(s.O[a] + o0, q, sizeof(T) * ns, cudaMemcpyHostToDevice, b->stream));
        q += sizeof(T) * ns;
        CK(cudaMemcpyAsync(s.V[a] + o0, q, sizeof(T) * ns, cudaMemcpyHostToDevice, b->stream));
        q += sizeof(T) * ns;
    }
    CK(cudaMemcpyAsync(s.H + o0, q, sizeof(T) * ns, cudaMemcpyHostToDevice, b->stream));
    q += sizeof(T) * ns;
    CK(cudaMemcpyAsync(s.G + o0, q, 4 * (size_t)ns, cudaMemcpyHostToDevice, b->stream));
    q += 4 * (size_t)ns;
    CK(cudaMemcpyAsync(s.ID + o0, q, 4 * (size_t)ns, cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(b->d_ctrl + inst, &c, sizeof c, cudaMemcpyHostToDevice, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    b->stage_steps = 0;
    for (double& t : b->stage_ms) t = 0;
    b->ev_pending = false;
    return SPH_OK;
}

// ---- cell-size autotuning ----
// The state of every loaded instance in host memory (positions, velocities, h, groups in
// original order) and every controller, to re-represent it on another grid.
struct Snapshot {
    std::vector<std::vector<double>> x, v, h;
    std::vector<std::vector<int32_t>> g;
    std::vector<Ctrl> ctrl;
};

template <typename T, int D> sph_status snapshot(sph_batch* b, Snapshot& sn) {
    sph_status r = read_ctrls(b, sn.ctrl);
    if (r != SPH_OK) return r;
    State<T>& s = st<T>(b);
    const int NI = b->NI;
    sn.x.assign(NI, {});
    sn.v.assign(NI, {});
    sn.h.assign(NI, {});
    sn.g.assign(NI, {});
    for (int i = 0; i < NI; ++i) {
        const int n = b->in[i].n;
        if (n == 0) continue;
        sn.x[i].resize((size_t)n * 3);
        sn.v[i].resize((size_t)n * 3);
        sn.h[i].resize(n);
        sn.g[i].resize(n);
        r = download<T>(b, i, s.C, s.O, s.V, s.H, s.G, s.ID, sn.x[i].data(), sn.g[i].data(), sn.v[i].data(),
                        sn.h[i].data());
        if (r != SPH_OK) return r;
    }
    return SPH_OK;
}

// Every instance's grid with `cps` cells per support, and the snapshot loaded onto it (the
// controllers carry on).  Fails, leaving the batch on the snapshot's grids, when a grid is
// invalid or does not fit.
template <typename T, int D> sph_status regrid(sph_batch* b, int cps, const Snapshot& sn) {
    std::vector<Inst> next(b->in);
    for (int i = 0; i < b->NI; ++i) {
        sph_params pp = b->in[i].pp;
        pp.cells_per_support = cps;
        Inst J;
        sph_status r = make_instance(&b->in[i].dd, &b->in[i].sz, &pp, b->in[i].cap, J);
        if (r != SPH_OK) return r;
        J.off = b->in[i].off;
        J.slots = b->in[i].slots;
        J.n = b->in[i].n;
        next[i] = J;
    }
    b->in = next;
    sph_status r = relayout(b, -1, 0, -1);
    if (r != SPH_OK) return r;
    for (int i = 0; i < b->NI; ++i) {
        const int n = b->in[i].n;
        if (n == 0) continue;
        r = set_state_impl<T, D>(b, i, n, sn.x[i].data(), sn.g[i].data(), sn.v[i].data(), sn.h[i].data(), true,
                                 &sn.ctrl[i]);
        if (r != SPH_OK) return r;
    }
    return SPH_OK;
}

// Times `steps` steps (after two untimed ones that also capture the graph) on the batch's
// stream; the state is reloaded from the snapshot afterwards by the caller.
template <typename T, int D> sph_status time_steps(sph_batch* b, int steps, float* ms) {
    sph_status r = step_impl<T, D>(b, 2);
    if (r != SPH_OK) return r;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, b->stream));
    r = step_impl<T, D>(b, steps);
    CK(cudaEventRecord(e1, b->stream));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return r;
}

// Tries 1, 2 and 4 cells per support on the loaded state, keeps the fastest, and leaves the
// batch holding the state it had (re-represented on the chosen grid).
template <typename T, int D> sph_status autotune_impl(sph_batch* b, int steps, int32_t* chosen, float* ms_out) {
    Snapshot sn;
    sph_status r = snapshot<T, D>(b, sn);
    if (r != SPH_OK) return r;
    const int start = 1 << b->in[0].grid.sm;
    int best = start;
    float best_ms = INFINITY;
    for (int cps : {1, 2, 4}) {
        float ms = INFINITY;
        if (regrid<T, D>(b, cps, sn) == SPH_OK && time_steps<T, D>(b, steps, &ms) == SPH_OK) {
            if (ms_out) ms_out[cps == 1 ? 0 : (cps == 2 ? 1 : 2)] = ms;
            if (ms < best_ms) {
                best_ms = ms;
                best = cps;
            }
        } else if (ms_out) {
            ms_out[cps == 1 ? 0 : (cps == 2 ? 1 : 2)] = -1.0f;
        }
    }
    r = regrid<T, D>(b, best, sn);
    if (r != SPH_OK) {
        // the best grid worked a moment ago; fall back to the starting one
        r = regrid<T, D>(b, start, sn);
        if (r != SPH_OK) return r;
        best = start;
    }
    for (Inst& I : b->in) I.pp.cells_per_support = best;
    if (chosen) *chosen = best;
    return SPH_OK;
}

sph_status status_of(const Ctrl& c, int inst, bool named) {
    const char* who = named ? "instance " : "";
    char tag[32] = "";
    if (named) std::snprintf(tag, sizeof tag, "%d: ", inst);
    if (c.status & ST_NONFINITE)
        return fail(SPH_E_DIVERGED, "%s%snon-finite acceleration or position at step %lld", who, tag, c.n);
    if (c.status & ST_OUTSIDE_GRID)
        return fail(SPH_E_OVERFLOW, "%s%sa particle left the cell grid (step %lld)", who, tag, c.n);
    return SPH_OK;
}

sph_status check_status(sph_batch* b) {
    std::vector<Ctrl> c;
    sph_status r = read_ctrls(b, c);
    if (r != SPH_OK) return r;
    for (int i = 0; i < b->NI; ++i) {
        r = status_of(c[i], i, !b->mesh);
        if (r != SPH_OK) return r;
    }
    return SPH_OK;
}

void fill_report(const sph_batch* b, int inst, const Ctrl& c, sph_report* out) {
    std::memset(out, 0, sizeof *out);
    const int G = b->in[inst].params.G;
    out->phase = c.phase;
    out->n_groups = G;
    out->iteration = c.n;
    out->ramp_start = c.ramp_start;
    out->escapes = (int64_t)c.escapes;
    out->status = c.status;
    out->E_t = c.E_t;
    out->E_avg = c.E_avg;
    out->E_sys = c.E_sys;
    for (int g = 0; g < G; ++g) {
        out->vbar[g] = c.Vbar[g];
        out->dt[g] = c.dt[g];
        out->reset[g] = c.reset[g];
        const bool per_group = b->in[inst].params.group_conv != 0;
        out->group_phase[g] = per_group ? c.gphase[g] : c.phase;
        out->group_E[g] = per_group ? c.gE[g] : 0.0;
    }
}

// Steps until every instance's controller is DONE or has run max_iters steps, checking every
// `every` steps.
sph_status run_impl(sph_batch* b, int64_t max_iters, int64_t* iters_out) {
    int every = 1 << 30;
    for (const Inst& I : b->in) every = std::min(every, I.params.sample_every);
    std::vector<Ctrl> c;
    sph_status r = read_ctrls(b, c);
    if (r != SPH_OK) return r;
    auto pending = [&](int64_t& nmin) {
        bool any = false;
        nmin = INT64_MAX;
        for (int i = 0; i < b->NI; ++i)
            if (c[i].phase != PH_DONE && c[i].n < max_iters && !(c[i].status & ST_NONFINITE) && b->in[i].n > 0) {
                any = true;
                nmin = std::min<int64_t>(nmin, c[i].n);
            }
        return any;
    };
    int64_t nmin = 0;
    while (pending(nmin)) {
        const int64_t chunk = std::min<int64_t>(every, max_iters - nmin);
        r = DISPATCH(b, step_impl, b, (int32_t)chunk);
        if (r != SPH_OK) return r;
        r = read_ctrls(b, c);
        if (r != SPH_OK) return r;
    }
    int64_t it = 0;
    for (const Ctrl& x : c) it = std::max<int64_t>(it, x.n);
    if (iters_out) *iters_out = it;
    r = check_status(b);
    if (r != SPH_OK) return r;
    for (int i = 0; i < b->NI; ++i)
        if (c[i].phase != PH_DONE) {
            if (b->mesh) return fail(SPH_E_NOT_CONVERGED, "not converged after %lld steps", (long long)c[i].n);
            return fail(SPH_E_NOT_CONVERGED, "instance %d not converged after %lld steps", i, (long long)c[i].n);
        }
    return SPH_OK;
}

sph_status kernel_times_impl(sph_batch* b, sph_kernel_time* out, int32_t cap, int32_t* n_out) {
    sph_status r = collect_timing(b);
    if (r != SPH_OK) return r;
    int k = 0;
    for (; k < NSTAGE && k < cap; ++k) {
        std::memset(out[k].name, 0, sizeof out[k].name);
        std::snprintf(out[k].name, sizeof out[k].name, "%s", kStages[k].name);
        out[k].launches = b->stage_steps * stage_kernels(k, b->D);
        out[k].total_ms = b->stage_ms[k];
    }
    if (n_out) *n_out = k;
    return SPH_OK;
}

sph_status set_timing_impl(sph_batch* b, int32_t enable) {
    if (b->timing) {
        sph_status r = collect_timing(b);
        if (r != SPH_OK) return r;
    }
    b->timing = enable != 0;
    b->stage_steps = 0;
    for (double& t : b->stage_ms) t = 0;
    b->ev_pending = false;
    return SPH_OK;
}

// ---- initial sampling (sample.cu): validated device copies of a problem's domain and sizing ----
struct ProblemDev {
    Inst I;
    Domain* d_dom = nullptr;
    Sizing* d_siz = nullptr;
    cudaStream_t st = nullptr;
    ~ProblemDev() {
        if (d_dom) cudaFreeAsync(d_dom, st);
        if (d_siz) cudaFreeAsync(d_siz, st);
    }
};

sph_status problem_dev(const sph_domain_desc* dd, const sph_sizing_desc* sz, cudaStream_t st, ProblemDev& P) {
    sph_params pp;
    sph_params_default(&pp);
    sph_status r = make_instance(dd, sz, &pp, 0, P.I);
    if (r != SPH_OK) return r;
    P.st = st;
    CK(cudaMallocAsync((void**)&P.d_dom, sizeof(Domain), st));
    CK(cudaMallocAsync((void**)&P.d_siz, sizeof(Sizing), st));
    CK(cudaMemcpyAsync(P.d_dom, &P.I.dom, sizeof(Domain), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(P.d_siz, &P.I.siz, sizeof(Sizing), cudaMemcpyHostToDevice, st));
    return SPH_OK;
}

sph_status feature_counts_impl(const sph_domain_desc* dd, const sph_sizing_desc* sz, cudaStream_t st,
                               double* integral_out, int64_t* count_out) {
    ProblemDev P;
    sph_status r = problem_dev(dd, sz, st, P);
    if (r != SPH_OK) return r;
    std::vector<double> M(MAXF, 0.0);
    cudaError_t e = feature_integrals(P.I.dom, P.d_dom, P.d_siz, st, M.data());
    if (e != cudaSuccess) return fail(SPH_E_CUDA, "feature_counts: %s", cudaGetErrorString(e));
    for (int k = 0; k < dd->n_features; ++k) {
        if (integral_out) integral_out[k] = M[k];
        if (count_out) count_out[k] = (int64_t)std::llround(M[k]);
    }
    return SPH_OK;
}

sph_status sample_impl(const sph_domain_desc* dd, const sph_sizing_desc* sz, uint64_t seed, const int64_t* counts,
                       cudaStream_t st, double* x_out, int32_t* group_out) {
    ProblemDev P;
    sph_status r = problem_dev(dd, sz, st, P);
    if (r != SPH_OK) return r;
    int64_t n = 0;
    for (int k = 0; k < dd->n_features; ++k) {
        if (counts[k] < 0) return fail(SPH_E_INVALID, "sample: negative count for feature %d", k);
        if (dd->features[k].kind == SPH_FEAT_POINT && counts[k] > 1)
            return fail(SPH_E_INVALID, "sample: a point feature holds one particle");
        n += counts[k];
    }
    if (n > ((int64_t)1 << 30)) return fail(SPH_E_INVALID, "sample: %lld particles is too many", (long long)n);
    double* d_x = nullptr;
    CK(cudaMallocAsync((void**)&d_x, sizeof(double) * 3 * (size_t)std::max<int64_t>(n, 1), st));
    cudaError_t e = sample_features(P.I.dom, P.I.siz, P.d_dom, P.d_siz, seed, counts, st, d_x);
    if (e == cudaSuccess) e = cudaMemcpyAsync(x_out, d_x, sizeof(double) * 3 * (size_t)n, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(d_x, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaErrorInvalidValue) return fail(SPH_E_INVALID, "sample: acceptance too low to reach a feature's count");
    if (e != cudaSuccess) return fail(SPH_E_CUDA, "sample: %s", cudaGetErrorString(e));
    int64_t o = 0;
    for (int k = 0; k < dd->n_features; ++k)
        for (int64_t i = 0; i < counts[k]; ++i) group_out[o++] = k;
    return SPH_OK;
}

}  // namespace

// ------------------------------------------------------------------------------------------
#pragma GCC visibility push(default)
extern "C" {

const char* sph_last_error(void) { return g_err.c_str(); }

sph_status sph_params_default(sph_params* p) {
    if (!p) return fail(SPH_E_INVALID, "params: NULL");
    std::memset(p, 0, sizeof *p);
    p->kappa = 2.6;
    p->p0 = 1.0;
    p->visc = 0.1;
    p->cfl_a = 0.25;
    p->cfl_v = 1.0 / 40.0;
    p->eps1 = 0.0;
    p->dt_cap = 1e30;
    p->dt_collapse = 0.1;
    p->threshold = 5e-6;
    p->reset_period = 100;
    p->sample_every = 20;
    p->window = 10;
    p->ramp_len = 200;
    p->boundary_rho = 1;
    p->precision = 32;
    p->boundary_correction = 1;
    return SPH_OK;
}

sph_status sph_params_preset(sph_params* p, int32_t method) {
    if (!p) return fail(SPH_E_INVALID, "params: NULL");
    switch (method) {
        case SPH_METHOD_IMPROVED: p->reset_period = 100; p->boundary_correction = 1; return SPH_OK;
        case SPH_METHOD_FU2019: p->reset_period = 1; p->boundary_correction = 0; return SPH_OK;
        case SPH_METHOD_FU2019_V2: p->reset_period = 100; p->boundary_correction = 0; return SPH_OK;
        default: return fail(SPH_E_INVALID, "params: unknown method preset %d", (int)method);
    }
}

sph_status sph_grid_spec(int32_t dim, const double* lo, const double* hi, double h_lo, double h_hi, double kappa,
                         int32_t cells_per_support, sph_grid_info* out) {
    if (!lo || !hi || !out) return fail(SPH_E_INVALID, "grid: NULL argument");
    return grid_spec(dim, lo, hi, h_lo, h_hi, kappa, cells_per_support, out);
}

// ---- single instance ----

sph_status sph_mesh_create(const sph_domain_desc* dd, const sph_sizing_desc* sz, const sph_params* pp,
                           int64_t max_particles, void* stream, sph_mesh** out) {
    if (!dd || !sz || !pp || !out) return fail(SPH_E_INVALID, "create: NULL argument");
    *out = nullptr;
    Inst I;
    sph_status r = make_instance(dd, sz, pp, max_particles, I);
    if (r != SPH_OK) return r;
    sph_mesh* m = new sph_mesh();
    m->mesh = true;
    m->D = dd->dim;
    m->prec = pp->precision;
    m->in.push_back(I);
    r = batch_init(m, stream);
    if (r != SPH_OK) {
        batch_free(m);
        delete m;
        return r;
    }
    *out = m;
    return SPH_OK;
}

sph_status sph_mesh_set_state(sph_mesh* m, int64_t n, const double* x, const int32_t* group, const double* v,
                              const double* h) {
    if (!m) return fail(SPH_E_INVALID, "set_state: NULL handle");
    sph_status r = check_args(m, 0, n, x, group, v, h);
    if (r != SPH_OK) return r;
    return DISPATCH(m, set_state_impl, m, 0, n, x, group, v, h, false);
}

sph_status sph_mesh_step(sph_mesh* m, int32_t n_steps) {
    if (!m) return fail(SPH_E_INVALID, "step: NULL handle");
    if (n_steps < 0) return fail(SPH_E_INVALID, "step: n_steps < 0");
    if (m->in[0].n == 0) return SPH_OK;
    return DISPATCH(m, step_impl, m, n_steps);
}

sph_status sph_mesh_sync(sph_mesh* m) {
    if (!m) return fail(SPH_E_INVALID, "sync: NULL handle");
    CK(cudaStreamSynchronize(m->stream));
    return check_status(m);
}

sph_status sph_mesh_run_until_converged(sph_mesh* m, int64_t max_iters, int64_t* iters_out) {
    if (!m) return fail(SPH_E_INVALID, "run: NULL handle");
    if (max_iters < 0) return fail(SPH_E_INVALID, "run: max_iters < 0");
    return run_impl(m, max_iters, iters_out);
}

sph_status sph_mesh_positions(sph_mesh* m, double* x_out, int32_t* group_out, double* v_out, double* h_out,
                              int64_t capacity, int64_t* n_out) {
    if (!m) return fail(SPH_E_INVALID, "positions: NULL handle");
    const int n = m->in[0].n;
    if (n_out) *n_out = n;
    if (capacity < n) return fail(SPH_E_INVALID, "positions: capacity %lld < n %d", (long long)capacity, n);
    if (n == 0) return SPH_OK;
    return DISPATCH(m, positions_impl, m, 0, x_out, group_out, v_out, h_out);
}

sph_status sph_mesh_snapshot(sph_mesh* m, void* buf, size_t cap, size_t* used) {
    if (!m) return fail(SPH_E_INVALID, "snapshot: NULL handle");
    if (!buf && !used) return fail(SPH_E_INVALID, "snapshot: NULL buffer and size");
    return DISPATCH(m, snapshot_impl, m, 0, buf, cap, used);
}

sph_status sph_mesh_restore(sph_mesh* m, const void* buf, size_t len) {
    if (!m || !buf) return fail(SPH_E_INVALID, "restore: NULL argument");
    return DISPATCH(m, restore_impl, m, 0, buf, len);
}

sph_status sph_mesh_report(sph_mesh* m, sph_report* out) {
    if (!m || !out) return fail(SPH_E_INVALID, "report: NULL argument");
    std::vector<Ctrl> c;
    sph_status r = read_ctrls(m, c);
    if (r != SPH_OK) return r;
    fill_report(m, 0, c[0], out);
    return SPH_OK;
}

void sph_mesh_destroy(sph_mesh* m) {
    if (!m) return;
    batch_free(m);
    delete m;
}

sph_status sph_mesh_grid(const sph_mesh* m, sph_grid_info* out) {
    if (!m || !out) return fail(SPH_E_INVALID, "grid: NULL argument");
    const Inst& I = m->in[0];
    return grid_spec(m->D, I.dom.lo, I.dom.hi, I.h_lo, I.h_hi, I.params.kappa, 1 << I.grid.sm, out);
}

sph_status sph_debug_rebuild(sph_mesh* m, int64_t* key_out, int64_t* cs_out, int64_t* perm_out) {
    if (!m) return fail(SPH_E_INVALID, "debug_rebuild: NULL handle");
    if (m->in[0].n == 0) return SPH_OK;
    return DISPATCH(m, dbg_rebuild_impl, m, key_out, cs_out, perm_out);
}

sph_status sph_debug_neighbors(sph_mesh* m, int32_t mode, int64_t* counts_out, int32_t* lists_out,
                               int64_t list_capacity, int64_t* total_out) {
    if (!m) return fail(SPH_E_INVALID, "debug_neighbors: NULL handle");
    if (mode != 0 && mode != 1) return fail(SPH_E_INVALID, "debug_neighbors: mode must be 0 or 1");
    if (m->in[0].n == 0) {
        if (total_out) *total_out = 0;
        return SPH_OK;
    }
    return DISPATCH(m, dbg_neighbors_impl, m, mode, counts_out, lists_out, list_capacity, total_out);
}

sph_status sph_debug_interact(sph_mesh* m, double* a_p, double* sigma, double* gamma, double* dta, double* dtv) {
    if (!m) return fail(SPH_E_INVALID, "debug_interact: NULL handle");
    if (m->in[0].n == 0) return SPH_OK;
    return DISPATCH(m, dbg_interact_impl, m, a_p, sigma, gamma, dta, dtv);
}

sph_status sph_debug_update(sph_mesh* m, const double* dt, const int32_t* reset, double eps, double f, double* x_out,
                            double* v_out, double* h_out, double* a_v) {
    if (!m || !dt || !reset) return fail(SPH_E_INVALID, "debug_update: NULL argument");
    if (m->in[0].n == 0) return SPH_OK;
    return DISPATCH(m, dbg_update_impl, m, dt, reset, eps, f, x_out, v_out, h_out, a_v);
}

sph_status sph_debug_pair_counts(sph_mesh* m, int64_t* candidates, int64_t* accepted) {
    if (!m) return fail(SPH_E_INVALID, "pair_counts: NULL handle");
    if (m->in[0].n == 0) {
        if (candidates) *candidates = 0;
        if (accepted) *accepted = 0;
        return SPH_OK;
    }
    return DISPATCH(m, pair_counts_impl, m, candidates, accepted);
}

sph_status sph_mesh_set_timing(sph_mesh* m, int32_t enable) {
    if (!m) return fail(SPH_E_INVALID, "set_timing: NULL handle");
    return set_timing_impl(m, enable);
}

sph_status sph_mesh_kernel_times(sph_mesh* m, sph_kernel_time* out, int32_t cap, int32_t* n_out) {
    if (!m) return fail(SPH_E_INVALID, "kernel_times: NULL handle");
    if (cap > 0 && !out) return fail(SPH_E_INVALID, "kernel_times: NULL output");
    return kernel_times_impl(m, out, cap, n_out);
}

// ---- batch ----

sph_status sph_batch_create(int32_t n_inst, const sph_domain_desc* domains, const sph_sizing_desc* sizings,
                            const sph_params* params, const int64_t* max_particles, void* stream, sph_batch** out) {
    if (!domains || !sizings || !params || !max_particles || !out) return fail(SPH_E_INVALID, "batch_create: NULL argument");
    *out = nullptr;
    if (n_inst < 1 || n_inst > SPH_MAX_INSTANCES)
        return fail(SPH_E_INVALID, "batch_create: n_inst must be in [1, %d]", SPH_MAX_INSTANCES);
    std::vector<Inst> in(n_inst);
    for (int i = 0; i < n_inst; ++i) {
        sph_status r = make_instance(domains + i, sizings + i, params + i, max_particles[i], in[i]);
        if (r != SPH_OK) return fail(r, "instance %d: %s", i, g_err.c_str());
        if (domains[i].dim != domains[0].dim || params[i].precision != params[0].precision)
            return fail(SPH_E_INVALID, "instance %d: every instance needs the same dim and precision", i);
    }
    sph_batch* b = new sph_batch();
    b->D = domains[0].dim;
    b->prec = params[0].precision;
    b->in = in;
    sph_status r = batch_init(b, stream);
    if (r != SPH_OK) {
        batch_free(b);
        delete b;
        return r;
    }
    // every instance starts idle (no particles, controller DONE)
    std::vector<Ctrl> c(b->NI);
    for (Ctrl& x : c) {
        host_ctrl_init(&x);
        ctrl_inf_bits(b->prec, &x);
        host_ctrl_phase(&x, PH_DONE, 0.0, 0.0);
        x.sample_now = 0;
    }
    if (cudaMemcpyAsync(b->d_ctrl, c.data(), sizeof(Ctrl) * b->NI, cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess) {
        batch_free(b);
        delete b;
        return fail(SPH_E_CUDA, "device initialisation failed");
    }
    *out = b;
    return SPH_OK;
}

sph_status sph_batch_size(const sph_batch* b, int32_t* n_inst, int64_t* n_slots, int64_t* slot_capacity) {
    if (!b) return fail(SPH_E_INVALID, "batch_size: NULL handle");
    if (n_inst) *n_inst = b->NI;
    if (n_slots) *n_slots = b->nslots;
    if (slot_capacity) *slot_capacity = b->slot_cap;
    return SPH_OK;
}

sph_status sph_batch_set_problem(sph_batch* b, int32_t inst, const sph_domain_desc* dd, const sph_sizing_desc* sz,
                                 const sph_params* pp) {
    if (!b || !dd || !sz || !pp) return fail(SPH_E_INVALID, "set_problem: NULL argument");
    if (inst < 0 || inst >= b->NI) return fail(SPH_E_INVALID, "set_problem: instance %d out of range", inst);
    if (dd->dim != b->D || pp->precision != b->prec)
        return fail(SPH_E_INVALID, "set_problem: dim and precision must match the batch");
    Inst I;
    sph_status r = make_instance(dd, sz, pp, b->in[inst].cap, I);
    if (r != SPH_OK) return r;
    CK(cudaSetDevice(b->device));
    CK(cudaStreamSynchronize(b->stream));
    const Inst old = b->in[inst];
    I.off = old.off;
    I.slots = old.slots;
    I.n = old.n;
    b->in[inst] = I;
    r = DISPATCH(b, set_state_impl, b, inst, 0, nullptr, nullptr, nullptr, nullptr, true);
    if (r != SPH_OK) b->in[inst] = old;
    return r;
}

sph_status sph_batch_set_state(sph_batch* b, int32_t inst, int64_t n, const double* x, const int32_t* group,
                               const double* v, const double* h) {
    if (!b) return fail(SPH_E_INVALID, "set_state: NULL handle");
    if (inst < 0 || inst >= b->NI) return fail(SPH_E_INVALID, "set_state: instance %d out of range", inst);
    sph_status r = check_args(b, inst, n, x, group, v, h);
    if (r != SPH_OK) return r;
    return DISPATCH(b, set_state_impl, b, inst, n, x, group, v, h, true);
}

sph_status sph_batch_step(sph_batch* b, int32_t n_steps) {
    if (!b) return fail(SPH_E_INVALID, "step: NULL handle");
    if (n_steps < 0) return fail(SPH_E_INVALID, "step: n_steps < 0");
    return DISPATCH(b, step_impl, b, n_steps);
}

sph_status sph_batch_sync(sph_batch* b) {
    if (!b) return fail(SPH_E_INVALID, "sync: NULL handle");
    CK(cudaStreamSynchronize(b->stream));
    return check_status(b);
}

sph_status sph_batch_run_until_converged(sph_batch* b, int64_t max_iters, int64_t* iters_out) {
    if (!b) return fail(SPH_E_INVALID, "run: NULL handle");
    if (max_iters < 0) return fail(SPH_E_INVALID, "run: max_iters < 0");
    return run_impl(b, max_iters, iters_out);
}

sph_status sph_batch_positions(sph_batch* b, int32_t inst, double* x_out, int32_t* group_out, double* v_out,
                               double* h_out, int64_t capacity, int64_t* n_out) {
    if (!b) return fail(SPH_E_INVALID, "positions: NULL handle");
    if (inst < 0 || inst >= b->NI) return fail(SPH_E_INVALID, "positions: instance %d out of range", inst);
    const int n = b->in[inst].n;
    if (n_out) *n_out = n;
    if (capacity < n) return fail(SPH_E_INVALID, "positions: capacity %lld < n %d", (long long)capacity, n);
    if (n == 0) return SPH_OK;
    return DISPATCH(b, positions_impl, b, inst, x_out, group_out, v_out, h_out);
}

sph_status sph_batch_reports(sph_batch* b, sph_report* out, int32_t cap) {
    if (!b || !out) return fail(SPH_E_INVALID, "reports: NULL argument");
    if (cap < b->NI) return fail(SPH_E_INVALID, "reports: capacity %d < %d instances", cap, b->NI);
    std::vector<Ctrl> c;
    sph_status r = read_ctrls(b, c);
    if (r != SPH_OK) return r;
    for (int i = 0; i < b->NI; ++i) fill_report(b, i, c[i], out + i);
    return SPH_OK;
}

sph_status sph_batch_set_timing(sph_batch* b, int32_t enable) {
    if (!b) return fail(SPH_E_INVALID, "set_timing: NULL handle");
    return set_timing_impl(b, enable);
}

sph_status sph_batch_kernel_times(sph_batch* b, sph_kernel_time* out, int32_t cap, int32_t* n_out) {
    if (!b) return fail(SPH_E_INVALID, "kernel_times: NULL handle");
    if (cap > 0 && !out) return fail(SPH_E_INVALID, "kernel_times: NULL output");
    return kernel_times_impl(b, out, cap, n_out);
}

sph_status sph_batch_slot_bytes(int32_t dim, int32_t precision, int64_t* bytes_per_slot) {
    if (!bytes_per_slot) return fail(SPH_E_INVALID, "slot_bytes: NULL argument");
    if (dim != 2 && dim != 3) return fail(SPH_E_INVALID, "slot_bytes: dim must be 2 or 3");
    if (precision != 32 && precision != 64) return fail(SPH_E_INVALID, "slot_bytes: precision must be 32 or 64");
    sph_batch b;
    b.D = dim;
    b.prec = precision;
    b.slot_cap = 1 << 20;
    const size_t bytes = precision == 32 ? slot_layout<float>(&b, nullptr, false) : slot_layout<double>(&b, nullptr, false);
    // plus the chunk table
    *bytes_per_slot = (int64_t)((bytes + (size_t)b.slot_cap - 1) / (size_t)b.slot_cap) + 1;
    return SPH_OK;
}

sph_status sph_batch_autotune(sph_batch* b, int32_t trial_steps, int32_t* cells_per_support, float* trial_ms) {
    if (!b) return fail(SPH_E_INVALID, "autotune: NULL handle");
    if (trial_steps < 1) return fail(SPH_E_INVALID, "autotune: trial_steps must be positive");
    if (b->nslots == 0) return fail(SPH_E_INVALID, "autotune: no instance is loaded");
    CK(cudaSetDevice(b->device));
    return DISPATCH(b, autotune_impl, b, trial_steps, cells_per_support, trial_ms);
}

sph_status sph_batch_snapshot(sph_batch* b, int32_t inst, void* buf, size_t cap, size_t* used) {
    if (!b) return fail(SPH_E_INVALID, "snapshot: NULL handle");
    if (inst < 0 || inst >= b->NI) return fail(SPH_E_INVALID, "snapshot: instance %d out of range", inst);
    if (!buf && !used) return fail(SPH_E_INVALID, "snapshot: NULL buffer and size");
    return DISPATCH(b, snapshot_impl, b, inst, buf, cap, used);
}

sph_status sph_batch_restore(sph_batch* b, int32_t inst, const void* buf, size_t len) {
    if (!b || !buf) return fail(SPH_E_INVALID, "restore: NULL argument");
    if (inst < 0 || inst >= b->NI) return fail(SPH_E_INVALID, "restore: instance %d out of range", inst);
    return DISPATCH(b, restore_impl, b, inst, buf, len);
}

void sph_batch_destroy(sph_batch* b) {
    if (!b) return;
    batch_free(b);
    delete b;
}

sph_status sph_feature_counts(const sph_domain_desc* domain, const sph_sizing_desc* sizing, void* stream,
                              double* integral_out, int64_t* count_out) {
    if (!count_out && !integral_out) return fail(SPH_E_INVALID, "feature_counts: no output");
    return feature_counts_impl(domain, sizing, (cudaStream_t)stream, integral_out, count_out);
}

sph_status sph_sample_particles(const sph_domain_desc* domain, const sph_sizing_desc* sizing, uint64_t seed,
                                const int64_t* counts, void* stream, double* x_out, int32_t* group_out) {
    if (!counts || !x_out || !group_out) return fail(SPH_E_INVALID, "sample_particles: NULL argument");
    return sample_impl(domain, sizing, seed, counts, (cudaStream_t)stream, x_out, group_out);
}

sph_status sph_mesh_sample(sph_mesh* m, uint64_t seed, int64_t* n_out) {
    if (!m) return fail(SPH_E_INVALID, "mesh_sample: NULL handle");
    const Inst& I = m->in[0];
    std::vector<int64_t> cnt(I.dd.n_features);
    sph_status r = feature_counts_impl(&I.dd, &I.sz, m->stream, nullptr, cnt.data());
    if (r != SPH_OK) return r;
    int64_t n = 0;
    for (int64_t c : cnt) n += c;
    if (n > I.cap)
        return fail(SPH_E_NOMEM, "mesh_sample: %lld particles for a mesh created for %lld", (long long)n, (long long)I.cap);
    std::vector<double> x((size_t)std::max<int64_t>(n, 1) * 3);
    std::vector<int32_t> g((size_t)std::max<int64_t>(n, 1));
    r = sample_impl(&I.dd, &I.sz, seed, cnt.data(), m->stream, x.data(), g.data());
    if (r != SPH_OK) return r;
    r = sph_mesh_set_state(m, n, x.data(), g.data(), nullptr, nullptr);
    if (r == SPH_OK && n_out) *n_out = n;
    return r;
}

}  // extern "C"
#pragma GCC visibility pop
