// capi.cu -- host side of libsphmesh.so: descriptor validation, the cell-grid specification,
// device memory, the per-step launch sequence (captured once into a CUDA graph), and the
// inspection entry points.  See include/sphmesh.h for the contract of every function.
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
sph_status grid_spec(int D, const double* lo, const double* hi, double h_lo, double h_hi, double kappa,
                     sph_grid_info* out) {
    if (D != 2 && D != 3) return fail(SPH_E_INVALID, "grid: dim must be 2 or 3");
    if (!(h_lo > 0) || !(h_hi >= h_lo) || !(kappa > 0)) return fail(SPH_E_INVALID, "grid: need 0 < h_lo <= h_hi, kappa > 0");
    for (int a = 0; a < D; ++a)
        if (!(hi[a] > lo[a])) return fail(SPH_E_INVALID, "grid: empty bounding box on axis %d", a);
    const double m = 1.0 + std::ldexp(1.0, -10);
    sph_grid_info g;
    std::memset(&g, 0, sizeof g);
    g.dim = D;
    g.c0 = round_up_f(kappa * h_lo * m);
    int L = 1;
    while (std::ldexp((double)g.c0, L - 1) < kappa * h_hi * m) {
        if (L == SPH_MAX_LEVELS) return fail(SPH_E_INVALID, "grid: h_hi/h_lo too large for %d levels", SPH_MAX_LEVELS);
        ++L;
    }
    g.levels = L;
    for (int l = 0; l < SPH_MAX_LEVELS; ++l)
        g.thr[l] = l < L - 1 ? round_down_f(std::ldexp((double)g.c0, l) / (kappa * m)) : INFINITY;
    const double top = std::ldexp((double)g.c0, L - 1);
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
const KTime kStages[4] = {{"rebuild", 6}, {"interact", 1}, {"control", 1}, {"integrate", 1}};

}  // namespace

struct sph_mesh {
    int D = 2, prec = 32;
    int64_t cap = 0;
    int n = 0;
    Grid grid;
    Params params;
    Domain hdom;
    Sizing hsiz;
    double h_lo = 0, h_hi = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    void* pool = nullptr;
    State<float> sf;
    State<double> sd;
    Domain* d_dom = nullptr;
    Sizing* d_siz = nullptr;
    Ctrl* d_ctrl = nullptr;
    Ctrl* d_ctrl_dbg = nullptr;
    // CUDA graph of one step
    cudaGraphExec_t gexec = nullptr;
    int graph_n = -1;
    bool graph_timed = false;
    // stage timing
    bool timing = false;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    bool ev_pending = false;
    double stage_ms[4] = {0, 0, 0, 0};
    int64_t stage_steps = 0;
};

namespace {

template <typename T> State<T>& st(sph_mesh* m);
template <> State<float>& st<float>(sph_mesh* m) { return m->sf; }
template <> State<double>& st<double>(sph_mesh* m) { return m->sd; }

// carve every device array out of one allocation (256-byte aligned pieces)
template <typename T> size_t layout(sph_mesh* m, char* base, bool assign) {
    const size_t cap = (size_t)std::max<int64_t>(m->cap, 1);
    const size_t ncell = (size_t)m->grid.ncell;
    const size_t nblk = (size_t)div_up((long long)cap * LPP_MAX, BLOCK);
    const int t = m->grid.L - 1;
    const size_t nocc = (size_t)m->grid.dims[t][0] * m->grid.dims[t][1] * m->grid.dims[t][2];
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
        s.Vs[a] = (T*)take(cap * sizeof(T));
    }
    s.H = (T*)take(cap * sizeof(T));
    s.G = (unsigned*)take(cap * 4);
    s.ID = (int*)take(cap * 4);
    s.K = (int*)take(cap * 4);
    s.Hs = (T*)take(cap * sizeof(T));
    s.Ms = (unsigned*)take(cap * 4);
    s.IDs = (int*)take(cap * 4);
    s.Ks = (int*)take(cap * 4);
    s.P = (Vec4<T>*)take(cap * sizeof(Vec4<T>));
    s.A = (Vec4<T>*)take(cap * sizeof(Vec4<T>));
    s.count = (int*)take(ncell * 4);
    s.cell_start = (int*)take((ncell + 1) * 4);
    s.bsum = (int*)take((size_t)SCAN_TILE * 4);
    s.perm = (int*)take(cap * 4);
    s.sperm = (int*)take(cap * 4);
    s.partials = (double*)take(nblk * MAXF * sizeof(double));
    s.occ = (unsigned*)take(nocc * 4);
    const size_t nlanes = cap * LPP_MAX;
    s.vj = (int*)take(nlanes * VCAP_MAX * 4);
    s.vr = (T*)take(nlanes * VCAP_MAX * sizeof(T));
    s.vcnt = (int*)take(nlanes * 4);
    if (assign) {
        s.n = 0;
        s.nblk = 0;
        s.nocc = (int)nocc;
        s.ctrl = m->d_ctrl;
        s.dom = m->d_dom;
        s.siz = m->d_siz;
        st<T>(m) = s;
    }
    return off + 256;
}

void host_ctrl_init(Ctrl* c) {
    std::memset(c, 0, sizeof *c);
    c->phase = PH1;
    c->sample_now = 1;
    c->f = 1.0;
    c->f_f = 1.0f;
}

template <typename T> void ctrl_inf_bits(Ctrl* c) {
    for (int g = 0; g < MAXF; ++g) {
        c->dta_bits[g] = inf_bits<T>();
        c->dtv_bits[g] = inf_bits<T>();
    }
}

template <typename T, int D> void enqueue_rebuild(sph_mesh* m, const State<T>& s, cudaStream_t stream) {
    launch_hash<T, D>(m->grid, s, stream);
    launch_scan(m->grid.ncell, s.count, s.cell_start, s.bsum, stream, s.occ, s.nocc, true);
    launch_scatter<T>(s, stream);
    launch_gather<T, D>(m->grid, s, stream);
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
    return o;
}

template <typename T, int D> void enqueue_step(sph_mesh* m, bool timed) {
    const State<T>& s = st<T>(m);
    cudaStream_t stream = m->stream;
    if (timed) cudaEventRecordWithFlags(m->ev[0], stream, cudaEventRecordExternal);
    enqueue_rebuild<T, D>(m, s, stream);
    if (timed) cudaEventRecordWithFlags(m->ev[1], stream, cudaEventRecordExternal);
    launch_interact<T, D>(m->grid, m->params, s, nullptr, nullptr, stream);
    if (timed) cudaEventRecordWithFlags(m->ev[2], stream, cudaEventRecordExternal);
    launch_control<T>(m->params, s, stream);
    if (timed) cudaEventRecordWithFlags(m->ev[3], stream, cudaEventRecordExternal);
    launch_integrate<T, D>(m->grid, m->params, s, s.ctrl, out_stored<T>(s), stream);
    if (timed) cudaEventRecordWithFlags(m->ev[4], stream, cudaEventRecordExternal);
}

sph_status collect_timing(sph_mesh* m) {
    if (!m->ev_pending) return SPH_OK;
    CK(cudaEventSynchronize(m->ev[4]));
    for (int k = 0; k < 4; ++k) {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, m->ev[k], m->ev[k + 1]));
        m->stage_ms[k] += ms;
    }
    m->stage_steps += 1;
    m->ev_pending = false;
    return SPH_OK;
}

template <typename T, int D> sph_status build_graph(sph_mesh* m) {
    if (m->gexec) {
        cudaGraphExecDestroy(m->gexec);
        m->gexec = nullptr;
    }
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal));
    enqueue_step<T, D>(m, m->timing);
    cudaError_t e = cudaStreamEndCapture(m->stream, &graph);
    if (e != cudaSuccess) return fail(SPH_E_CUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&m->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(SPH_E_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    m->graph_n = m->n;
    m->graph_timed = m->timing;
    return SPH_OK;
}

template <typename T, int D> sph_status step_impl(sph_mesh* m, int32_t n_steps) {
    if (m->n == 0) return SPH_OK;
    CK(cudaSetDevice(m->device));
    if (!m->gexec || m->graph_n != m->n || m->graph_timed != m->timing) {
        sph_status r = build_graph<T, D>(m);
        if (r != SPH_OK) return r;
    }
    for (int i = 0; i < n_steps; ++i) {
        if (m->timing) {
            sph_status r = collect_timing(m);
            if (r != SPH_OK) return r;
        }
        CK(cudaGraphLaunch(m->gexec, m->stream));
        if (m->timing) m->ev_pending = true;
    }
    return SPH_OK;
}

#define DISPATCH(m, fn, ...)                                              \
    ((m)->prec == 32 ? ((m)->D == 2 ? fn<float, 2>(__VA_ARGS__) : fn<float, 3>(__VA_ARGS__)) \
                     : ((m)->D == 2 ? fn<double, 2>(__VA_ARGS__) : fn<double, 3>(__VA_ARGS__)))

// state in device memory -> host arrays in original order (from an Out-like set of arrays)
template <typename T>
sph_status download(sph_mesh* m, int* const Cd[3], T* const Od[3], T* const V[3], T* H, unsigned* G, int* ID,
                    double* x_out, int32_t* group_out, double* v_out, double* h_out) {
    const int n = m->n, D = m->D;
    std::vector<int> id(n);
    CK(cudaMemcpyAsync(id.data(), ID, sizeof(int) * n, cudaMemcpyDeviceToHost, m->stream));
    std::vector<int> cs(x_out ? (size_t)n * 3 : 0);
    std::vector<T> os(x_out ? (size_t)n * 3 : 0);
    std::vector<T> vs(v_out ? (size_t)n * 3 : 0), hs(h_out ? n : 0);
    std::vector<unsigned> gs(group_out ? n : 0);
    for (int a = 0; a < D; ++a) {
        if (x_out) {
            CK(cudaMemcpyAsync(cs.data() + (size_t)a * n, Cd[a], sizeof(int) * n, cudaMemcpyDeviceToHost, m->stream));
            CK(cudaMemcpyAsync(os.data() + (size_t)a * n, Od[a], sizeof(T) * n, cudaMemcpyDeviceToHost, m->stream));
        }
        if (v_out) CK(cudaMemcpyAsync(vs.data() + (size_t)a * n, V[a], sizeof(T) * n, cudaMemcpyDeviceToHost, m->stream));
    }
    // FP64 position = origin + cell * c0 + offset
    std::vector<double> xs(x_out ? (size_t)n * 3 : 0);
    for (int a = 0; x_out && a < D; ++a)
        for (int k = 0; k < n; ++k)
            xs[(size_t)a * n + k] = ((double)m->grid.origin[a] + (double)cs[(size_t)a * n + k] * m->grid.c[0]) +
                                    (double)os[(size_t)a * n + k];
    if (h_out) CK(cudaMemcpyAsync(hs.data(), H, sizeof(T) * n, cudaMemcpyDeviceToHost, m->stream));
    if (group_out) CK(cudaMemcpyAsync(gs.data(), G, sizeof(unsigned) * n, cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    for (int k = 0; k < n; ++k) {
        const int i = id[k];
        if (i < 0 || i >= n) return fail(SPH_E_CUDA, "corrupt particle index on the device");
        for (int a = 0; a < 3; ++a) {
            if (x_out) x_out[(size_t)i * 3 + a] = a < D ? xs[(size_t)a * n + k] : 0.0;
            if (v_out) v_out[(size_t)i * 3 + a] = a < D ? (double)vs[(size_t)a * n + k] : 0.0;
        }
        if (h_out) h_out[i] = (double)hs[k];
        if (group_out) group_out[i] = (int32_t)(gs[k] & 63u);
    }
    return SPH_OK;
}

template <typename T, int D> sph_status set_state_impl(sph_mesh* m, int64_t n, const double* x, const int32_t* group,
                                                       const double* v, const double* h) {
    State<T>& s = st<T>(m);
    const int nn = (int)n;
    std::vector<int> cs((size_t)std::max(nn, 1) * 3);
    std::vector<T> os((size_t)std::max(nn, 1) * 3), vs((size_t)std::max(nn, 1) * 3, T(0)), hs(std::max(nn, 1));
    std::vector<unsigned> gs(std::max(nn, 1));
    std::vector<int> ids(std::max(nn, 1));
    const double c0 = m->grid.c[0], inv_c0 = m->grid.inv_c[0];
    for (int i = 0; i < nn; ++i) {
        const int gi = group[i];
        for (int a = 0; a < D; ++a) {
            // finest cell and offset: c = floor((x - origin) * (1/c0)), o = (x - origin) - c*c0
            const double rel = x[(size_t)i * 3 + a] - (double)m->grid.origin[a];
            double t = std::floor(rel * inv_c0);
            int ca = (int)std::fmax(std::fmin(t, 2.0e9), -2.0e9);
            ca = std::min(std::max(ca, 0), m->grid.dims[0][a] - 1);
            cs[(size_t)a * nn + i] = ca;
            os[(size_t)a * nn + i] = (T)(rel - (double)ca * c0);
            if (v) vs[(size_t)a * nn + i] = (T)v[(size_t)i * 3 + a];
        }
        if (h) hs[i] = (T)h[i];
        gs[i] = (unsigned)gi | ((unsigned)m->hdom.f[gi].dim << 6);
        ids[i] = i;
    }
    CK(cudaSetDevice(m->device));
    for (int a = 0; a < D; ++a) {
        CK(cudaMemcpyAsync(s.C[a], cs.data() + (size_t)a * nn, sizeof(int) * nn, cudaMemcpyHostToDevice, m->stream));
        CK(cudaMemcpyAsync(s.O[a], os.data() + (size_t)a * nn, sizeof(T) * nn, cudaMemcpyHostToDevice, m->stream));
        CK(cudaMemcpyAsync(s.V[a], vs.data() + (size_t)a * nn, sizeof(T) * nn, cudaMemcpyHostToDevice, m->stream));
    }
    CK(cudaMemcpyAsync(s.G, gs.data(), 4 * (size_t)nn, cudaMemcpyHostToDevice, m->stream));
    CK(cudaMemcpyAsync(s.ID, ids.data(), 4 * (size_t)nn, cudaMemcpyHostToDevice, m->stream));
    s.n = nn;
    s.nblk = div_up((long long)nn * Lpp<D>::v, BLOCK);   // blocks of the pair passes
    m->n = nn;
    if (h) CK(cudaMemcpyAsync(s.H, hs.data(), sizeof(T) * nn, cudaMemcpyHostToDevice, m->stream));
    else if (nn > 0) launch_init_h<T, D>(m->grid, s, m->stream);
    Ctrl c;
    host_ctrl_init(&c);
    ctrl_inf_bits<T>(&c);
    CK(cudaMemcpyAsync(m->d_ctrl, &c, sizeof c, cudaMemcpyHostToDevice, m->stream));
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(m->stream));
    m->stage_steps = 0;
    for (double& t : m->stage_ms) t = 0;
    m->ev_pending = false;
    return SPH_OK;
}

// a copy of the state whose controller is the scratch controller (inspection calls never
// touch the real controller)
template <typename T> sph_status dbg_state(sph_mesh* m, State<T>& out, const Ctrl* init) {
    out = st<T>(m);
    Ctrl c;
    if (init) c = *init;
    else {
        CK(cudaMemcpyAsync(&c, m->d_ctrl, sizeof c, cudaMemcpyDeviceToHost, m->stream));
        CK(cudaStreamSynchronize(m->stream));
    }
    ctrl_inf_bits<T>(&c);
    c.sample_now = 0;
    CK(cudaMemcpyAsync(m->d_ctrl_dbg, &c, sizeof c, cudaMemcpyHostToDevice, m->stream));
    out.ctrl = m->d_ctrl_dbg;
    return SPH_OK;
}

template <typename T, int D> sph_status dbg_rebuild_impl(sph_mesh* m, int64_t* key_out, int64_t* cs_out, int64_t* perm_out) {
    State<T> s;
    sph_status r = dbg_state<T>(m, s, nullptr);
    if (r != SPH_OK) return r;
    const int n = m->n, nc = m->grid.ncell;
    enqueue_rebuild<T, D>(m, s, m->stream);     // the same kernels as a step's rebuild
    CK(cudaGetLastError());
    std::vector<int> k(n), cs(nc + 1), p(n);
    CK(cudaMemcpyAsync(k.data(), s.K, 4 * (size_t)n, cudaMemcpyDeviceToHost, m->stream));
    CK(cudaMemcpyAsync(cs.data(), s.cell_start, 4 * (size_t)(nc + 1), cudaMemcpyDeviceToHost, m->stream));
    CK(cudaMemcpyAsync(p.data(), s.sperm, 4 * (size_t)n, cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    for (int i = 0; i < n; ++i) {
        if (key_out) key_out[i] = k[i];
        if (perm_out) perm_out[i] = p[i];
    }
    if (cs_out)
        for (int c = 0; c <= nc; ++c) cs_out[c] = cs[c];
    return SPH_OK;
}

template <typename T, int D> sph_status dbg_prepare(sph_mesh* m, State<T>& s, const Ctrl* init) {
    sph_status r = dbg_state<T>(m, s, init);
    if (r != SPH_OK) return r;
    enqueue_rebuild<T, D>(m, s, m->stream);
    CK(cudaGetLastError());
    return SPH_OK;
}

template <typename T, int D>
sph_status dbg_neighbors_impl(sph_mesh* m, int32_t mode, int64_t* counts_out, int32_t* lists_out, int64_t cap,
                              int64_t* total_out) {
    State<T> s;
    sph_status r = dbg_prepare<T, D>(m, s, nullptr);
    if (r != SPH_OK) return r;
    const int n = m->n;
    int* d_counts = nullptr;
    long long* d_off = nullptr;
    int* d_lists = nullptr;
    CK(cudaMalloc(&d_counts, 4 * (size_t)std::max(n, 1)));
    launch_neighbors<T, D>(m->grid, m->params, s, mode, d_counts, nullptr, nullptr, m->stream);
    std::vector<int> cnt(n), ids(n);
    CK(cudaMemcpyAsync(cnt.data(), d_counts, 4 * (size_t)n, cudaMemcpyDeviceToHost, m->stream));
    CK(cudaMemcpyAsync(ids.data(), s.IDs, 4 * (size_t)n, cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    std::vector<long long> off(n + 1, 0);
    for (int k = 0; k < n; ++k) off[k + 1] = off[k] + cnt[k];
    const long long total = off[n];
    CK(cudaMalloc(&d_off, sizeof(long long) * (size_t)(n + 1)));
    CK(cudaMalloc(&d_lists, 4 * (size_t)std::max<long long>(total, 1)));
    CK(cudaMemcpyAsync(d_off, off.data(), sizeof(long long) * (size_t)(n + 1), cudaMemcpyHostToDevice, m->stream));
    launch_neighbors<T, D>(m->grid, m->params, s, mode, d_counts, d_off, d_lists, m->stream);
    std::vector<int> lists((size_t)std::max<long long>(total, 1));
    CK(cudaMemcpyAsync(lists.data(), d_lists, 4 * (size_t)total, cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    cudaFree(d_counts);
    cudaFree(d_off);
    cudaFree(d_lists);
    // regroup by original index, map sorted slots to original indices, ascending
    std::vector<int> slot_of(n);
    for (int k = 0; k < n; ++k) slot_of[ids[k]] = k;
    long long w = 0;
    bool overflow = false;
    for (int i = 0; i < n; ++i) {
        const int k = slot_of[i];
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
sph_status dbg_interact_impl(sph_mesh* m, double* a_p, double* sigma, double* gamma, double* dta, double* dtv) {
    State<T> s;
    sph_status r = dbg_prepare<T, D>(m, s, nullptr);
    if (r != SPH_OK) return r;
    const int n = m->n, G = m->params.G;
    T *d_sig = nullptr, *d_gam = nullptr;
    CK(cudaMalloc(&d_sig, sizeof(T) * (size_t)std::max(n, 1)));
    CK(cudaMalloc(&d_gam, sizeof(T) * (size_t)std::max(n, 1)));
    launch_interact<T, D>(m->grid, m->params, s, d_sig, d_gam, m->stream);
    CK(cudaGetLastError());
    std::vector<Vec4<T>> A(n);
    std::vector<T> sg(n), gm(n);
    std::vector<int> ids(n);
    Ctrl c;
    CK(cudaMemcpyAsync(A.data(), s.A, sizeof(Vec4<T>) * (size_t)n, cudaMemcpyDeviceToHost, m->stream));
    CK(cudaMemcpyAsync(sg.data(), d_sig, sizeof(T) * (size_t)n, cudaMemcpyDeviceToHost, m->stream));
    CK(cudaMemcpyAsync(gm.data(), d_gam, sizeof(T) * (size_t)n, cudaMemcpyDeviceToHost, m->stream));
    CK(cudaMemcpyAsync(ids.data(), s.IDs, 4 * (size_t)n, cudaMemcpyDeviceToHost, m->stream));
    CK(cudaMemcpyAsync(&c, m->d_ctrl_dbg, sizeof c, cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    cudaFree(d_sig);
    cudaFree(d_gam);
    for (int k = 0; k < n; ++k) {
        const int i = ids[k];
        if (a_p) {
            a_p[(size_t)i * 3 + 0] = (double)A[k].x;
            a_p[(size_t)i * 3 + 1] = (double)A[k].y;
            a_p[(size_t)i * 3 + 2] = D == 3 ? (double)A[k].z : 0.0;
        }
        if (sigma) sigma[i] = (double)sg[k];
        if (gamma) gamma[i] = (double)gm[k];
    }
    for (int g = 0; g < G; ++g) {
        T a, b;
        if (sizeof(T) == 4) {
            unsigned ua = (unsigned)c.dta_bits[g], ub = (unsigned)c.dtv_bits[g];
            float fa, fb;
            std::memcpy(&fa, &ua, 4);
            std::memcpy(&fb, &ub, 4);
            a = (T)fa;
            b = (T)fb;
        } else {
            double fa, fb;
            std::memcpy(&fa, &c.dta_bits[g], 8);
            std::memcpy(&fb, &c.dtv_bits[g], 8);
            a = (T)fa;
            b = (T)fb;
        }
        if (dta) dta[g] = (double)a;
        if (dtv) dtv[g] = (double)b;
    }
    return SPH_OK;
}

template <typename T, int D>
sph_status dbg_update_impl(sph_mesh* m, const double* dt, const int32_t* reset, double eps, double f, double* x_out,
                           double* v_out, double* h_out, double* a_v) {
    const int n = m->n, G = m->params.G;
    Ctrl c;
    host_ctrl_init(&c);
    for (int g = 0; g < G; ++g) {
        c.dt[g] = dt[g];
        c.dt_f[g] = (float)dt[g];
        c.reset[g] = reset[g];
    }
    c.eps = eps;
    c.f = f;
    c.eps_f = (float)eps;
    c.f_f = (float)f;
    State<T> s;
    sph_status r = dbg_prepare<T, D>(m, s, &c);
    if (r != SPH_OK) return r;
    launch_interact<T, D>(m->grid, m->params, s, nullptr, nullptr, m->stream);
    // scratch output arrays
    Out<T> o;
    void* buf = nullptr;
    const size_t nn = (size_t)std::max(n, 1);
    const size_t bytes = 16 * ((nn * (3 * 4 + 9 * sizeof(T) + sizeof(T) + 8) + 4096 + 15) / 16) + 16 * 256;
    CK(cudaMalloc(&buf, bytes));
    char* p = (char*)buf;
    auto take = [&](size_t b) {
        char* q = p;
        p += (b + 255) & ~(size_t)255;
        return q;
    };
    for (int a = 0; a < 3; ++a) o.C[a] = (int*)take(nn * 4);
    for (int a = 0; a < 3; ++a) o.O[a] = (T*)take(nn * sizeof(T));
    for (int a = 0; a < 3; ++a) o.V[a] = (T*)take(nn * sizeof(T));
    for (int a = 0; a < 3; ++a) o.av[a] = (T*)take(nn * sizeof(T));
    o.H = (T*)take(nn * sizeof(T));
    o.G = (unsigned*)take(nn * 4);
    o.ID = (int*)take(nn * 4);
    launch_integrate<T, D>(m->grid, m->params, s, m->d_ctrl_dbg, o, m->stream);
    CK(cudaGetLastError());
    r = download<T>(m, o.C, o.O, o.V, o.H, o.G, o.ID, x_out, nullptr, v_out, h_out);
    if (r == SPH_OK && a_v) {
        T* const avs[3] = {o.av[0], o.av[1], o.av[2]};
        r = download<T>(m, o.C, o.O, avs, o.H, o.G, o.ID, nullptr, nullptr, a_v, nullptr);
    }
    cudaFree(buf);
    return r;
}

template <typename T, int D> sph_status pair_counts_impl(sph_mesh* m, int64_t* cand, int64_t* accd) {
    State<T> s;
    sph_status r = dbg_prepare<T, D>(m, s, nullptr);
    if (r != SPH_OK) return r;
    unsigned long long* d = nullptr;
    CK(cudaMalloc(&d, 16));
    CK(cudaMemsetAsync(d, 0, 16, m->stream));
    launch_pair_counts<T, D>(m->grid, m->params, s, d, m->stream);
    unsigned long long h[2];
    CK(cudaMemcpyAsync(h, d, 16, cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    cudaFree(d);
    if (cand) *cand = (int64_t)h[0];
    if (accd) *accd = (int64_t)h[1];
    return SPH_OK;
}

template <typename T, int D>
sph_status positions_impl(sph_mesh* m, double* x_out, int32_t* group_out, double* v_out, double* h_out) {
    State<T>& s = st<T>(m);
    return download<T>(m, s.C, s.O, s.V, s.H, s.G, s.ID, x_out, group_out, v_out, h_out);
}

sph_status check_status(sph_mesh* m) {
    Ctrl c;
    CK(cudaMemcpyAsync(&c, m->d_ctrl, sizeof c, cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    if (c.status & ST_NONFINITE) return fail(SPH_E_DIVERGED, "non-finite acceleration or position at step %lld", c.n);
    if (c.status & ST_OUTSIDE_GRID) return fail(SPH_E_OVERFLOW, "a particle left the cell grid (step %lld)", c.n);
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
    p->kappa = 2.0;
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
    return SPH_OK;
}

sph_status sph_grid_spec(int32_t dim, const double* lo, const double* hi, double h_lo, double h_hi, double kappa,
                         sph_grid_info* out) {
    if (!lo || !hi || !out) return fail(SPH_E_INVALID, "grid: NULL argument");
    return grid_spec(dim, lo, hi, h_lo, h_hi, kappa, out);
}

sph_status sph_mesh_create(const sph_domain_desc* dd, const sph_sizing_desc* sz, const sph_params* pp,
                           int64_t max_particles, void* stream, sph_mesh** out) {
    if (!dd || !sz || !pp || !out) return fail(SPH_E_INVALID, "create: NULL argument");
    *out = nullptr;
    if (dd->dim != 2 && dd->dim != 3) return fail(SPH_E_INVALID, "domain: dim must be 2 or 3");
    if (dd->n_features < 1 || dd->n_features > SPH_MAX_FEATURES) return fail(SPH_E_INVALID, "domain: n_features out of range");
    if (dd->n_holes < 0 || dd->n_holes > SPH_MAX_HOLES) return fail(SPH_E_INVALID, "domain: n_holes out of range");
    if (dd->base != 0 && dd->base != 1) return fail(SPH_E_INVALID, "domain: base must be 0 (box) or 1 (ball)");
    if (pp->precision != 32 && pp->precision != 64) return fail(SPH_E_INVALID, "params: precision must be 32 or 64");
    if (!(pp->kappa > 0) || !(pp->p0 > 0) || pp->visc < 0 || !(pp->cfl_a > 0) || !(pp->cfl_v > 0) || pp->eps1 < 0 ||
        !(pp->dt_cap > 0) || pp->dt_collapse < 0 || !(pp->threshold > 0) || pp->reset_period < 1 ||
        pp->sample_every < 1 || pp->window < 1 || pp->ramp_len < 1)
        return fail(SPH_E_INVALID, "params: value out of range");
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
    }
    sph_grid_info gi;
    sph_status r = grid_spec(D, dd->bbox_lo, dd->bbox_hi, sz->lo, sz->hi, pp->kappa, &gi);
    if (r != SPH_OK) return r;
    if (gi.n_cells > (int64_t)SCAN_TILE * SCAN_TILE)
        return fail(SPH_E_INVALID, "grid: %lld cells is more than the %lld the cell scan supports", (long long)gi.n_cells,
                    (long long)SCAN_TILE * SCAN_TILE);
    for (int l = 0; l < gi.levels; ++l)
        if (gi.dims[l][0] >= ((int64_t)1 << 23) || gi.dims[l][1] >= ((int64_t)1 << 14) || gi.dims[l][2] >= ((int64_t)1 << 14))
            return fail(SPH_E_INVALID, "grid: too many cells (x < 2^23, y and z < 2^14 per level)");

    sph_mesh* m = new sph_mesh();
    m->D = D;
    m->prec = pp->precision;
    m->cap = max_particles;
    m->h_lo = sz->lo;
    m->h_hi = sz->hi;
    Grid& g = m->grid;
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
        g.base[l] = l < gi.levels ? (int)gi.base[l] : (int)gi.n_cells;
    }
    g.base[MAXL] = (int)gi.n_cells;
    g.ncell = (int)gi.n_cells;
    Params& p = m->params;
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
    p.kappa_f = (float)p.kappa;
    p.p0_f = (float)p.p0;
    p.visc_f = (float)p.visc;
    p.cfl_a_f = (float)p.cfl_a;
    p.cfl_v_f = (float)p.cfl_v;
    p.G = dd->n_features;
    for (int k = 0; k < MAXF; ++k) p.gdim[k] = k < dd->n_features ? dd->features[k].dim : 0;
    Domain& dm = m->hdom;
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
            if (!(L > 0)) {
                delete m;
                return fail(SPH_E_INVALID, "feature %d: zero-length segment", k);
            }
            for (int a = 0; a < 3; ++a) F.ftg[a] = (float)(ab[a] / L);
        } else if (f.kind == SPH_FEAT_RECT) {
            for (int a = 0; a < 3; ++a) F.ftg[a] = (float)f.normal[a];
        }
        if (f.kind == SPH_FEAT_CIRCLE || f.kind == SPH_FEAT_SPHERE)
            for (int a = 0; a < 3; ++a) F.fc[a] = (float)f.geom[a];
        if (f.kind == SPH_FEAT_CIRCLE) F.fc[2] = 0.0f;
    }
    Sizing& zs = m->hsiz;
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

    auto cleanup = [&](sph_status s) {
        sph_mesh_destroy(m);
        return s;
    };
    if (cudaGetDevice(&m->device) != cudaSuccess) return cleanup(fail(SPH_E_CUDA, "no CUDA device"));
    if (stream) m->stream = (cudaStream_t)stream;
    else {
        if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess)
            return cleanup(fail(SPH_E_CUDA, "cudaStreamCreate failed"));
        m->own_stream = true;
    }
    if (cudaMalloc(&m->d_dom, sizeof(Domain)) != cudaSuccess || cudaMalloc(&m->d_siz, sizeof(Sizing)) != cudaSuccess ||
        cudaMalloc(&m->d_ctrl, sizeof(Ctrl)) != cudaSuccess || cudaMalloc(&m->d_ctrl_dbg, sizeof(Ctrl)) != cudaSuccess)
        return cleanup(fail(SPH_E_NOMEM, "device allocation of descriptors failed"));
    size_t bytes = m->prec == 32 ? layout<float>(m, nullptr, false) : layout<double>(m, nullptr, false);
    if (cudaMalloc(&m->pool, bytes) != cudaSuccess)
        return cleanup(fail(SPH_E_NOMEM, "device allocation of %zu bytes failed", bytes));
    if (m->prec == 32) layout<float>(m, (char*)m->pool, true);
    else layout<double>(m, (char*)m->pool, true);
    if (cudaMemsetAsync(m->pool, 0, bytes, m->stream) != cudaSuccess ||
        cudaMemcpyAsync(m->d_dom, &m->hdom, sizeof(Domain), cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
        cudaMemcpyAsync(m->d_siz, &m->hsiz, sizeof(Sizing), cudaMemcpyHostToDevice, m->stream) != cudaSuccess)
        return cleanup(fail(SPH_E_CUDA, "device initialisation failed"));
    Ctrl c;
    host_ctrl_init(&c);
    if (m->prec == 32) ctrl_inf_bits<float>(&c);
    else ctrl_inf_bits<double>(&c);
    if (cudaMemcpyAsync(m->d_ctrl, &c, sizeof c, cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess)
        return cleanup(fail(SPH_E_CUDA, "device initialisation failed"));
    for (int k = 0; k < 5; ++k)
        if (cudaEventCreate(&m->ev[k]) != cudaSuccess) return cleanup(fail(SPH_E_CUDA, "cudaEventCreate failed"));
    *out = m;
    return SPH_OK;
}

sph_status sph_mesh_set_state(sph_mesh* m, int64_t n, const double* x, const int32_t* group, const double* v,
                              const double* h) {
    if (!m) return fail(SPH_E_INVALID, "set_state: NULL handle");
    if (n < 0 || n > m->cap) return fail(SPH_E_INVALID, "set_state: n=%lld outside [0, %lld]", (long long)n, (long long)m->cap);
    if (n > 0 && (!x || !group)) return fail(SPH_E_INVALID, "set_state: x and group are required");
    const int D = m->D;
    for (int64_t i = 0; i < n; ++i) {
        if (group[i] < 0 || group[i] >= m->params.G) return fail(SPH_E_INVALID, "set_state: particle %lld has group %d", (long long)i, group[i]);
        for (int a = 0; a < D; ++a) {
            double xa = x[i * 3 + a];
            if (!(xa >= m->hdom.lo[a] - 1e-9 * (1 + std::fabs(m->hdom.lo[a])) && xa <= m->hdom.hi[a] + 1e-9 * (1 + std::fabs(m->hdom.hi[a]))))
                return fail(SPH_E_INVALID, "set_state: particle %lld outside the bounding box", (long long)i);
        }
        // the grid's top level covers kappa*h_hi*(1+2^-10); allow h up to h_hi*(1+2^-11) so that
        // values rounded to the working precision are accepted
        if (h && !(h[i] > 0 && h[i] <= m->h_hi * (1 + 1.0 / 2048.0)))
            return fail(SPH_E_INVALID, "set_state: h of particle %lld outside [lo, hi]", (long long)i);
        if (v)
            for (int a = 0; a < D; ++a)
                if (!std::isfinite(v[i * 3 + a])) return fail(SPH_E_INVALID, "set_state: non-finite velocity");
    }
    return DISPATCH(m, set_state_impl, m, n, x, group, v, h);
}

sph_status sph_mesh_step(sph_mesh* m, int32_t n_steps) {
    if (!m) return fail(SPH_E_INVALID, "step: NULL handle");
    if (n_steps < 0) return fail(SPH_E_INVALID, "step: n_steps < 0");
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
    Ctrl c;
    CK(cudaMemcpyAsync(&c, m->d_ctrl, sizeof c, cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    while (c.phase != PH_DONE && c.n < max_iters) {
        int64_t chunk = std::min<int64_t>(m->params.sample_every, max_iters - c.n);
        sph_status r = sph_mesh_step(m, (int32_t)chunk);
        if (r != SPH_OK) return r;
        CK(cudaMemcpyAsync(&c, m->d_ctrl, sizeof c, cudaMemcpyDeviceToHost, m->stream));
        CK(cudaStreamSynchronize(m->stream));
        if (c.status & ST_NONFINITE) break;
        if (m->n == 0) break;
    }
    if (iters_out) *iters_out = c.n;
    sph_status r = check_status(m);
    if (r != SPH_OK) return r;
    if (c.phase != PH_DONE) return fail(SPH_E_NOT_CONVERGED, "not converged after %lld steps", (long long)c.n);
    return SPH_OK;
}

sph_status sph_mesh_positions(sph_mesh* m, double* x_out, int32_t* group_out, double* v_out, double* h_out,
                              int64_t capacity, int64_t* n_out) {
    if (!m) return fail(SPH_E_INVALID, "positions: NULL handle");
    if (n_out) *n_out = m->n;
    if (capacity < m->n) return fail(SPH_E_INVALID, "positions: capacity %lld < n %d", (long long)capacity, m->n);
    if (m->n == 0) return SPH_OK;
    return DISPATCH(m, positions_impl, m, x_out, group_out, v_out, h_out);
}

sph_status sph_mesh_report(sph_mesh* m, sph_report* out) {
    if (!m || !out) return fail(SPH_E_INVALID, "report: NULL argument");
    Ctrl c;
    CK(cudaMemcpyAsync(&c, m->d_ctrl, sizeof c, cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    std::memset(out, 0, sizeof *out);
    out->phase = c.phase;
    out->n_groups = m->params.G;
    out->iteration = c.n;
    out->ramp_start = c.ramp_start;
    out->escapes = (int64_t)c.escapes;
    out->status = c.status;
    out->E_t = c.E_t;
    out->E_avg = c.E_avg;
    out->E_sys = c.E_sys;
    for (int g = 0; g < m->params.G; ++g) {
        out->vbar[g] = c.Vbar[g];
        out->dt[g] = c.dt[g];
        out->reset[g] = c.reset[g];
    }
    return SPH_OK;
}

void sph_mesh_destroy(sph_mesh* m) {
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    if (m->gexec) cudaGraphExecDestroy(m->gexec);
    for (int k = 0; k < 5; ++k)
        if (m->ev[k]) cudaEventDestroy(m->ev[k]);
    cudaFree(m->pool);
    cudaFree(m->d_dom);
    cudaFree(m->d_siz);
    cudaFree(m->d_ctrl);
    cudaFree(m->d_ctrl_dbg);
    if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

sph_status sph_mesh_grid(const sph_mesh* m, sph_grid_info* out) {
    if (!m || !out) return fail(SPH_E_INVALID, "grid: NULL argument");
    return grid_spec(m->D, m->hdom.lo, m->hdom.hi, m->h_lo, m->h_hi, m->params.kappa, out);
}

sph_status sph_debug_rebuild(sph_mesh* m, int64_t* key_out, int64_t* cs_out, int64_t* perm_out) {
    if (!m) return fail(SPH_E_INVALID, "debug_rebuild: NULL handle");
    if (m->n == 0) return SPH_OK;
    return DISPATCH(m, dbg_rebuild_impl, m, key_out, cs_out, perm_out);
}

sph_status sph_debug_neighbors(sph_mesh* m, int32_t mode, int64_t* counts_out, int32_t* lists_out,
                               int64_t list_capacity, int64_t* total_out) {
    if (!m) return fail(SPH_E_INVALID, "debug_neighbors: NULL handle");
    if (mode != 0 && mode != 1) return fail(SPH_E_INVALID, "debug_neighbors: mode must be 0 or 1");
    if (m->n == 0) {
        if (total_out) *total_out = 0;
        return SPH_OK;
    }
    return DISPATCH(m, dbg_neighbors_impl, m, mode, counts_out, lists_out, list_capacity, total_out);
}

sph_status sph_debug_interact(sph_mesh* m, double* a_p, double* sigma, double* gamma, double* dta, double* dtv) {
    if (!m) return fail(SPH_E_INVALID, "debug_interact: NULL handle");
    if (m->n == 0) return SPH_OK;
    return DISPATCH(m, dbg_interact_impl, m, a_p, sigma, gamma, dta, dtv);
}

sph_status sph_debug_update(sph_mesh* m, const double* dt, const int32_t* reset, double eps, double f, double* x_out,
                            double* v_out, double* h_out, double* a_v) {
    if (!m || !dt || !reset) return fail(SPH_E_INVALID, "debug_update: NULL argument");
    if (m->n == 0) return SPH_OK;
    return DISPATCH(m, dbg_update_impl, m, dt, reset, eps, f, x_out, v_out, h_out, a_v);
}

sph_status sph_debug_pair_counts(sph_mesh* m, int64_t* candidates, int64_t* accepted) {
    if (!m) return fail(SPH_E_INVALID, "pair_counts: NULL handle");
    if (m->n == 0) {
        if (candidates) *candidates = 0;
        if (accepted) *accepted = 0;
        return SPH_OK;
    }
    return DISPATCH(m, pair_counts_impl, m, candidates, accepted);
}

sph_status sph_mesh_set_timing(sph_mesh* m, int32_t enable) {
    if (!m) return fail(SPH_E_INVALID, "set_timing: NULL handle");
    if (m->timing) {
        sph_status r = collect_timing(m);
        if (r != SPH_OK) return r;
    }
    m->timing = enable != 0;
    m->stage_steps = 0;
    for (double& t : m->stage_ms) t = 0;
    m->ev_pending = false;
    return SPH_OK;
}

sph_status sph_mesh_kernel_times(sph_mesh* m, sph_kernel_time* out, int32_t cap, int32_t* n_out) {
    if (!m) return fail(SPH_E_INVALID, "kernel_times: NULL handle");
    sph_status r = collect_timing(m);
    if (r != SPH_OK) return r;
    int k = 0;
    for (; k < 4 && k < cap; ++k) {
        std::memset(out[k].name, 0, sizeof out[k].name);
        std::snprintf(out[k].name, sizeof out[k].name, "%s", kStages[k].name);
        out[k].launches = m->stage_steps * kStages[k].kernels;
        out[k].total_ms = m->stage_ms[k];
    }
    if (n_out) *n_out = k;
    return SPH_OK;
}

}  // extern "C"
#pragma GCC visibility pop
