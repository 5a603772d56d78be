// sph_device.cuh -- device-side data layout and inline helpers of the relaxation kernels.
//
// Layout in HBM (a batch of instances packed into n slots; per-instance slot ranges):
//   stored state (in the order of the previous step's sort):
//     C[a][n] int32   finest-level cell of the position;  O[a][n] T  offset inside that cell
//                     (position = origin + C*c0 + O, reconstructed in FP64 where needed)
//     V[a][n] T       velocities;  H[n] T smoothing length;  G[n] uint32 meta;  ID[n] int32
//   sorted state (written by the gather of the rebuild, read by the pair passes):
//     Cs, Os, IDs as above, VH[n] T4 = (v, h), Ks[n] cell key, Ms[n] meta with the x-cell,
//     P[n] T4 = offsets inside the particle's own level cell + h (FP32 build, 2D:
//     (ox, oy, h, meta bits)), A[n] T4 = (a_p.x, a_p.y, a_p.z, V~) from the pressure pass.
//   meta bits: 0-5 group (feature index), 6-7 intrinsic dimension, 8-31 x index of the cell
//   (sorted arrays only).
// T is float (FP32 pair sums) or double (FP64 build); D is 2 or 3.
#pragma once
#include <cuda_runtime.h>
#include <math_constants.h>
#include <climits>
#include <stdint.h>

namespace sph {

constexpr int MAXF = 64;
constexpr int MAXH = 8;
constexpr int MAXL = 8;
// words per occupancy cell: per level, the largest smoothing length of its particles in the
// cell (float bits, rounded up; 0: none there)
constexpr int OCCW = MAXL;
#ifndef SPH_BLOCK
#define SPH_BLOCK 128
#endif
constexpr int BLOCK = SPH_BLOCK;   // threads per block of the per-slot and pair-pass kernels

enum { K_VOLUME = 0, K_POINT = 1, K_SEGMENT = 2, K_CIRCLE = 3, K_RECT = 4, K_SPHERE = 5 };
enum { PH1 = 1, PH_RAMP = 2, PH2 = 3, PH_DONE = 4 };
enum { ST_NONFINITE = 1u, ST_OUTSIDE_GRID = 2u, ST_H_RANGE = 4u, ST_SCAN = 8u };

struct Feat {
    int kind, dim;
    double g[12];
    double nb[3];
    double orient;
    float fnb[3];        // float copies used by the FP32 pair sums
    float ftg[3];        // SEGMENT: unit tangent; RECT: unit normal
    float fc[3];         // CIRCLE / SPHERE centre
    float forient;
};

struct Domain {
    int D, base;
    double lo[3], hi[3], bc[3], br;
    int nh;
    double hc[MAXH][3];
    double hr[MAXH];
    float flo[3], fhi[3], fbc[3], fbr;   // float copies for the FP32 level-set pre-check
    float fhc[MAXH][3], fhr[MAXH];
    int nf;
    Feat f[MAXF];
};

struct Sizing {
    int kind;
    double a, b, lo, hi;
    double q[3];
    int nref;
    double rc[MAXH][3];
    double rr[MAXH];
    float fa, fb, flo, fhi, fq[3];       // float copies for the FP32 evaluation of h_t
    float frc[MAXH][3], frr[MAXH];
};

struct Grid {
    int D, L;
    float c0;
    float origin[3];
    double c[MAXL];      // c0 * 2^l
    double inv_c[MAXL];  // 1 / c_l rounded once in FP64
    float cf[MAXL];      // c0 * 2^l as float (exact)
    float thr[MAXL];
    int dims[MAXL][3];
    int base[MAXL + 1];  // first key of each level; base[MAXL]: the instance's dummy key
    int ncell;           // cells of the instance (its keys are base[0] .. base[0]+ncell-1)
    int sm;              // log2 of the cells per support m: level l holds kappa h <= m c_l
    int osh;             // occupancy cells of 2^osh finest cells per axis
    int od[3];           // occupancy grid dimensions
    int occ_base;        // first entry of the instance's occupancy cells in the occupancy array
};

struct Params {
    double kappa, p0, visc, cfl_a, cfl_v, eps1, dt_cap, dt_collapse, threshold;
    int reset_period, sample_every, window, ramp_len, boundary_rho;
    int boundary_corr;   // 0: the boundary sum of Eq. 19 is left out (earlier method, Sec. 4.1)
    int group_conv;      // 1: every group runs its own phases (Algorithm 1's per-feature check)
    int feature_order;   // 1: Algorithm 1's feature loop in sequence: the step runs one pass per
                         // intrinsic dimension (curves, surfaces, volume), each reading the lower
                         // classes' new positions; 0: one pass for all (Jacobi)
    int G;
    int gdim[MAXF];      // intrinsic dimension of every group (feature)
    float kappa_f, p0_f, visc_f, cfl_a_f, cfl_v_f;   // float copies for the FP32 kernels
};

// controller state + per-step accumulators (one per instance, in device memory; 16-byte
// aligned so that it is copied in vectors)
struct alignas(16) Ctrl {
    int phase, wcount, nwin, sample_now;
    long long n, ramp_start;
    unsigned long long escapes;
    unsigned int status;
    int pad;
    double wsum[MAXF], A_last[MAXF], A_prev[MAXF], Vbar[MAXF], dt_prev[MAXF], dt[MAXF];
    int reset[MAXF];
    double E_t, E_avg, E_sys, eps, f;
    float dt_f[MAXF], eps_f, f_f;      // float copies of dt, eps, f for the FP32 update
    unsigned long long dta_bits[MAXF], dtv_bits[MAXF];   // per-group minima of Eq. 24 terms
    // per group, used only with group_convergence = 1 (kept last: the instance controller
    // copies the part before it): phase, damping and attenuation of the last step, window
    // counters, switch step, last error
    int gphase[MAXF];
    double geps[MAXF], gf[MAXF];
    float geps_f[MAXF], gf_f[MAXF];
    int gwcount[MAXF], gnwin[MAXF];
    long long gramp_start[MAXF];
    double gE[MAXF];
    // feature order: the step's largest errors of the groups evaluated in the earlier class passes
    double seq_et, seq_ea;
    int seq_ev, seq_pad[3];
};

template <typename T> struct alignas(4 * sizeof(T)) Vec4 { T x, y, z, w; };

// ---- rounding-explicit arithmetic (the neighbour predicate must be evaluated op by op) ----
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }

__device__ __forceinline__ unsigned long long min_bits(float v) { return (unsigned long long)__float_as_uint(v); }
__device__ __forceinline__ unsigned long long min_bits(double v) { return (unsigned long long)__double_as_longlong(v); }
// a working-precision value as a float not below it
template <typename T> __device__ __forceinline__ float float_up(T v);
template <> __device__ __forceinline__ float float_up<float>(float v) { return v; }
template <> __device__ __forceinline__ float float_up<double>(double v) { return __double2float_ru(v); }
template <typename T> __device__ __forceinline__ T from_bits(unsigned long long b);
template <> __device__ __forceinline__ float from_bits<float>(unsigned long long b) { return __uint_as_float((unsigned)b); }
template <> __device__ __forceinline__ double from_bits<double>(unsigned long long b) { return __longlong_as_double((long long)b); }
template <typename T> __host__ __device__ __forceinline__ unsigned long long inf_bits();
template <> __host__ __device__ __forceinline__ unsigned long long inf_bits<float>() { return 0x7f800000ull; }
template <> __host__ __device__ __forceinline__ unsigned long long inf_bits<double>() { return 0x7ff0000000000000ull; }

template <typename T> __device__ __forceinline__ T t_sqrt(T v);
template <> __device__ __forceinline__ float t_sqrt<float>(float v) { return sqrtf(v); }
template <> __device__ __forceinline__ double t_sqrt<double>(double v) { return sqrt(v); }
template <typename T> __device__ __forceinline__ T t_floor(T v);
template <> __device__ __forceinline__ float t_floor<float>(float v) { return floorf(v); }
template <> __device__ __forceinline__ double t_floor<double>(double v) { return floor(v); }

// a constant in the working precision: the float copy in the FP32 build (a double-to-float
// conversion runs on the FP64 pipe, which is narrow on this GPU), the double in the FP64 build
template <typename T> __device__ __forceinline__ T wp(double d, float f);
template <> __device__ __forceinline__ float wp<float>(double, float f) { return f; }
template <> __device__ __forceinline__ double wp<double>(double d, float) { return d; }

// h^k for small non-negative integer k
template <typename T> __device__ __forceinline__ T ipow(T h, int k) {
    T r = T(1);
    for (int i = 0; i < k; ++i) r *= h;
    return r;
}

// h^d and h^(2d) for an intrinsic dimension d in {1, 2, 3}
template <typename T> __device__ __forceinline__ void hpow(T h, int d, T& hd, T& h2d) {
    const T h2 = h * h;
    hd = d == 1 ? h : (d == 2 ? h2 : h2 * h);
    h2d = hd * hd;
}

// Wendland C2 normalisation alpha_d / (its R-dependence): alpha_1 = 3/(2R), alpha_2 = 7/(pi R^2),
// alpha_3 = 21/(2 pi R^3); given invR = 1/R.
template <typename T> __device__ __forceinline__ T wendland_alpha(int d, T invR) {
    if (d == 1) return T(1.5) * invR;
    if (d == 2) return T(7.0 / CUDART_PI) * invR * invR;
    return T(21.0 / (2.0 * CUDART_PI)) * invR * invR * invR;
}

// ---- particle record access (sorted arrays) ----
template <typename T, int D> struct Rec {
    // (float, 2D): P = (ox, oy, h, meta); every other case: P = (ox, oy, oz, h) + M
    static constexpr bool packed = (sizeof(T) == 4 && D == 2);
    __device__ __forceinline__ static void load(const Vec4<T>* __restrict__ P, const unsigned* __restrict__ M, int j,
                                                T off[3], T& h, unsigned& meta) {
        Vec4<T> p = P[j];
        off[0] = p.x;
        off[1] = p.y;
        if (packed) {
            off[2] = T(0);
            h = p.z;
            meta = __float_as_uint((float)p.w);
        } else {
            off[2] = p.z;
            h = p.w;
            meta = M[j];
        }
    }
    __device__ __forceinline__ static void store(Vec4<T>* P, unsigned* M, int j, const T off[3], T h, unsigned meta) {
        Vec4<T> p;
        p.x = off[0];
        p.y = off[1];
        if (packed) {
            p.z = h;
            p.w = (T)__uint_as_float(meta);
        } else {
            p.z = off[2];
            p.w = h;
        }
        P[j] = p;
        M[j] = meta;
    }
};

__device__ __forceinline__ int meta_group(unsigned m) { return (int)(m & 63u); }
__device__ __forceinline__ int meta_dim(unsigned m) { return (int)((m >> 6) & 3u); }
__device__ __forceinline__ int meta_cx(unsigned m) { return (int)(m >> 8); }

// level of a smoothing length: first l with h <= thr[l] (the top level takes the rest)
template <typename T> __device__ __forceinline__ int level_of(const Grid& g, T h) {
    int l = 0;
    while (l < g.L - 1 && h > (T)g.thr[l]) ++l;
    return l;
}

// Positions are stored as the finest-level cell (integers) and the offset from that cell's
// origin in the working precision.  From an FP64 position:
//   c = floor((x - origin) * inv_c0) (clamped into the finest grid), o = (x - origin) - c * c0
template <typename T, int D>
__device__ __forceinline__ bool fine_of(const Grid& g, const double x[3], int c[3], T o[3]) {
    bool clamped = false;
    for (int a = 0; a < 3; ++a) {
        if (a >= D) { c[a] = 0; o[a] = T(0); continue; }
        double rel = __dsub_rn(x[a], (double)g.origin[a]);
        double t = floor(__dmul_rn(rel, g.inv_c[0]));
        int ca = (int)fmax(fmin(t, 2.0e9), -2.0e9);
        if (ca < 0) { ca = 0; clamped = true; }
        if (ca > g.dims[0][a] - 1) { ca = g.dims[0][a] - 1; clamped = true; }
        c[a] = ca;
        o[a] = (T)__dsub_rn(rel, __dmul_rn((double)ca, g.c[0]));
    }
    return clamped;
}

// the FP64 position of a stored (finest cell, offset) pair
template <typename T, int D> __device__ __forceinline__ void pos64(const Grid& g, const int c[3], const T o[3], double x[3]) {
    for (int a = 0; a < 3; ++a)
        x[a] = a < D ? __dadd_rn(__dadd_rn((double)g.origin[a], __dmul_rn((double)c[a], g.c[0])), (double)o[a]) : 0.0;
}

// the same position in the working precision (for the sizing function, the level-set
// pre-check and tangent directions; absolute error ~ the precision of |x|)
template <typename T, int D> __device__ __forceinline__ void pos_t(const Grid& g, const int c[3], const T o[3], T x[3]) {
    for (int a = 0; a < 3; ++a) x[a] = a < D ? (T)g.origin[a] + (T)c[a] * (T)g.c0 + o[a] : T(0);
}

// level-l representation derived from the stored one, each operation rounded in T:
//   cell = c >> l, off = o + (c - (cell << l)) * c0
template <typename T, int D>
__device__ __forceinline__ void level_repr(const Grid& g, int l, const int c[3], const T o[3], int cell[3], T off[3]) {
    for (int a = 0; a < 3; ++a) {
        if (a >= D) { cell[a] = 0; off[a] = T(0); continue; }
        cell[a] = c[a] >> l;
        off[a] = rn_add(o[a], rn_mul((T)(c[a] - (cell[a] << l)), (T)g.c0));
    }
}

__device__ __forceinline__ int key_of(const Grid& g, int l, const int cell[3]) {
    return g.base[l] + (cell[2] * g.dims[l][1] + cell[1]) * g.dims[l][0] + cell[0];
}

// decode a key into level and cell coordinates
__device__ __forceinline__ void decode_key(const Grid& g, int key, int& l, int cell[3]) {
    l = 0;
    while (l < g.L - 1 && key >= g.base[l + 1]) ++l;
    int r = key - g.base[l];
    cell[0] = r % g.dims[l][0];
    r /= g.dims[l][0];
    cell[1] = r % g.dims[l][1];
    cell[2] = r / g.dims[l][1];
}

// ---- analytic geometry (FP64) ----
__device__ __forceinline__ double dnorm3(const double v[3]) { return sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }

__device__ inline double sizing_h(const Sizing& s, const double x[3]) {
    if (s.kind == 0) return s.a;
    double h;
    if (s.kind == 1) {
        double dmin = 1e300;
        for (int k = 0; k < s.nref; ++k) {
            double d[3] = {x[0] - s.rc[k][0], x[1] - s.rc[k][1], x[2] - s.rc[k][2]};
            double dk = fabs(dnorm3(d) - s.rr[k]);
            dmin = fmin(dmin, dk);
        }
        h = s.a + s.b * dmin;
    } else {
        double d[3] = {x[0] - s.q[0], x[1] - s.q[1], x[2] - s.q[2]};
        h = s.a + s.b * dnorm3(d);
    }
    return fmin(fmax(h, s.lo), s.hi);
}

// level set of the domain and its gradient (positive inside)
__device__ inline double domain_phi(const Domain& dom, const double x[3], double grad[3]) {
    double phi = 1e300;
    grad[0] = grad[1] = grad[2] = 0.0;
    if (dom.base == 0) {
        for (int a = 0; a < dom.D; ++a) {
            double dlo = x[a] - dom.lo[a], dhi = dom.hi[a] - x[a];
            if (dlo < phi) { phi = dlo; grad[0] = grad[1] = grad[2] = 0.0; grad[a] = 1.0; }
            if (dhi < phi) { phi = dhi; grad[0] = grad[1] = grad[2] = 0.0; grad[a] = -1.0; }
        }
    } else {
        double d[3] = {x[0] - dom.bc[0], x[1] - dom.bc[1], dom.D == 3 ? x[2] - dom.bc[2] : 0.0};
        double r = dnorm3(d);
        phi = dom.br - r;
        for (int a = 0; a < 3; ++a) grad[a] = r > 0 ? -d[a] / r : (a == 0 ? -1.0 : 0.0);
    }
    for (int k = 0; k < dom.nh; ++k) {
        double d[3] = {x[0] - dom.hc[k][0], x[1] - dom.hc[k][1], dom.D == 3 ? x[2] - dom.hc[k][2] : 0.0};
        double r = dnorm3(d);
        double pk = r - dom.hr[k];
        if (pk < phi) {
            phi = pk;
            for (int a = 0; a < 3; ++a) grad[a] = r > 0 ? d[a] / r : (a == 0 ? 1.0 : 0.0);
        }
    }
    return phi;
}

// closest point on a curve / surface / point feature (FP64)
__device__ inline void project_feature(const Feat& f, int D, double x[3]) {
    if (f.kind == K_POINT) {
        for (int a = 0; a < 3; ++a) x[a] = a < D ? f.g[a] : 0.0;
    } else if (f.kind == K_SEGMENT) {
        double ab[3], ax[3];
        for (int a = 0; a < 3; ++a) { ab[a] = f.g[3 + a] - f.g[a]; ax[a] = x[a] - f.g[a]; }
        double t = (ax[0] * ab[0] + ax[1] * ab[1] + ax[2] * ab[2]) / (ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2]);
        t = fmin(fmax(t, 0.0), 1.0);
        for (int a = 0; a < 3; ++a) x[a] = f.g[a] + t * ab[a];
    } else if (f.kind == K_CIRCLE || f.kind == K_SPHERE) {
        double c[3] = {f.g[0], f.g[1], f.kind == K_SPHERE ? f.g[2] : 0.0};
        double R = f.kind == K_SPHERE ? f.g[3] : f.g[2];
        double d[3] = {0, 0, 0};
        for (int a = 0; a < D; ++a) d[a] = x[a] - c[a];
        double r = dnorm3(d);
        for (int a = 0; a < 3; ++a) {
            double u = r > 0 ? d[a] / r : (a == 0 ? 1.0 : 0.0);
            x[a] = a < D ? c[a] + R * u : 0.0;
        }
    } else if (f.kind == K_RECT) {
        double ox[3];
        for (int a = 0; a < 3; ++a) ox[a] = x[a] - f.g[a];
        double s = ox[0] * f.g[3] + ox[1] * f.g[4] + ox[2] * f.g[5];
        double t = ox[0] * f.g[6] + ox[1] * f.g[7] + ox[2] * f.g[8];
        s = fmin(fmax(s, 0.0), f.g[9]);
        t = fmin(fmax(t, 0.0), f.g[10]);
        for (int a = 0; a < 3; ++a) x[a] = f.g[a] + s * f.g[3 + a] + t * f.g[6 + a];
    }
}

// the tangent-space descriptor of a particle of feature f at position x: unit tangent for
// curves (SEGMENT, CIRCLE), unit normal for surfaces (RECT, SPHERE)
template <typename T> __device__ inline void feature_tangent(const Feat& f, const T x[3], T tg[3]) {
    tg[0] = tg[1] = tg[2] = T(0);
    if (f.kind == K_SEGMENT || f.kind == K_RECT) {
        for (int a = 0; a < 3; ++a) tg[a] = (T)f.ftg[a];
        if (sizeof(T) == 8) {   // FP64 build: exact descriptor
            if (f.kind == K_RECT) { for (int a = 0; a < 3; ++a) tg[a] = (T)f.nb[a]; }
            else {
                double ab[3] = {f.g[3] - f.g[0], f.g[4] - f.g[1], f.g[5] - f.g[2]};
                double L = dnorm3(ab);
                for (int a = 0; a < 3; ++a) tg[a] = (T)(ab[a] / L);
            }
        }
    } else if (f.kind == K_CIRCLE) {
        T d0 = x[0] - (T)f.g[0], d1 = x[1] - (T)f.g[1];
        T r = t_sqrt(d0 * d0 + d1 * d1);
        T u0 = r > T(0) ? d0 / r : T(1), u1 = r > T(0) ? d1 / r : T(0);
        tg[0] = -u1;
        tg[1] = u0;
    } else if (f.kind == K_SPHERE) {
        T d[3] = {x[0] - (T)f.g[0], x[1] - (T)f.g[1], x[2] - (T)f.g[2]};
        T r = t_sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int a = 0; a < 3; ++a) tg[a] = r > T(0) ? d[a] / r : (a == 0 ? T(1) : T(0));
    }
}

// v <- Pi v : identity (volume), t t^T (curves), I - n n^T (surfaces), 0 (points)
template <typename T> __device__ __forceinline__ void tangent_map(int dim, int D, const T tg[3], T v[3]) {
    if (dim == D) return;
    if (dim == 0) { v[0] = v[1] = v[2] = T(0); return; }
    T s = v[0] * tg[0] + v[1] * tg[1] + v[2] * tg[2];
    if (dim == 1) { for (int a = 0; a < 3; ++a) v[a] = s * tg[a]; }
    else { for (int a = 0; a < 3; ++a) v[a] = v[a] - s * tg[a]; }
}

// outward normal n_b of a boundary particle of feature f at (absolute) position x
template <typename T> __device__ __forceinline__ void boundary_normal(const Feat& f, const T x[3], T nb[3]) {
    if (f.kind == K_CIRCLE || f.kind == K_SPHERE) {
        T d[3] = {x[0] - (T)f.fc[0], x[1] - (T)f.fc[1], f.kind == K_SPHERE ? x[2] - (T)f.fc[2] : T(0)};
        if (sizeof(T) == 8) {
            d[0] = x[0] - (T)f.g[0];
            d[1] = x[1] - (T)f.g[1];
            if (f.kind == K_SPHERE) d[2] = x[2] - (T)f.g[2];
        }
        T r = t_sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        T s = (T)f.forient / (r > T(0) ? r : T(1));
        for (int a = 0; a < 3; ++a) nb[a] = s * d[a];
    } else {
        for (int a = 0; a < 3; ++a) nb[a] = sizeof(T) == 8 ? (T)f.nb[a] : (T)f.fnb[a];
    }
}

// the two predicates of the pair sums, evaluated op by op:
//   pair: r2 < ((h_i + h_j) * kappa/2)^2   (j != i);   self: r2 < (kappa h_i)^2
template <typename T> __device__ __forceinline__ T pair_rc2(T hi, T hj, T half_kappa) {
    T rc = rn_mul(rn_add(hi, hj), half_kappa);
    return rn_mul(rc, rc);
}
template <typename T> __device__ __forceinline__ T self_rc2(T hi, T kappa) {
    T rc = rn_mul(hi, kappa);
    return rn_mul(rc, rc);
}

// ---- reciprocal / reciprocal square root for the pair arithmetic (not the predicate) ----
__device__ __forceinline__ float fast_rcp(float v) { return __fdividef(1.0f, v); }   // 2-ulp intrinsic division
__device__ __forceinline__ double fast_rcp(double v) { return 1.0 / v; }
__device__ __forceinline__ float fast_rsqrt(float v) { return rsqrtf(v); }
__device__ __forceinline__ double fast_rsqrt(double v) { return 1.0 / sqrt(v); }

// ---- sub-warp stencil walk ----
// For query particle i at level li with cell coordinates ci (at li) and offsets offi, the walk
// visits every particle j stored in the cells that can hold a j with
// |x_i - x_j| < max(kappa (h_i + h_j)/2, kappa h_i).  At level l all particles have
// kappa h_j <= c_l, and those in the occupancy cells around i have h_j <= H_l (the largest h of
// the level there, recorded by the gather; a level with none there is skipped), so the radius
// R_l = max((kappa h_i + min(c_l, kappa H_l))/2, kappa h_i) (widened by 2^-10) bounds every
// candidate.  dx = x_i - x_j is computed as (off_i - off_j) + m c0 with m = ci 2^li - cj 2^l
// (exact integers), r2 = |dx|^2, both op by op.
// LPP consecutive lanes handle one particle.  In 2D they split the candidates of every stencil
// row between them (lane r takes s+r, s+r+LPP, ...); in 3D (the flat walk) each lane first cuts
// one row to the cells that reach the ball of radius R_l, and the lanes then step through the
// concatenated candidates of LPP rows.  A candidate j for which accept(j, dx, r2, h_j, meta_j)
// holds is kept in the lane's slice of `buf` (CAP entries of (j, level | row), stride BLOCK, in
// shared memory); the kept candidates are handed to fn(j, dx, r2, h_j, meta_j, off_j, l, cx_j,
// cy, cz) when the buffer is full and at the end, so the per-pair work runs with the lanes
// mostly converged.  Every lane count computes dx and r2 identically, so a candidate is
// accepted or rejected the same way whatever LPP; the flat walk's only warp-synchronous
// operations (the row-length scan and its shared-memory hand-off) name the particle's own
// lanes, which all reach them.  (Measured and not kept: sharing the occupancy loads among the
// lanes, loading the next row's range ahead of the current row's scan, deriving a 3D
// candidate's x cell from the row's cell starts instead of its meta word, and a
// warp-cooperative walk over the union of the warp's stencils with candidates staged in
// shared memory -- the first three cost more registers or instructions than they saved, the
// last tests about twice the candidates, since a warp's particles span several cells.)
template <typename T, int D>
__device__ __forceinline__ int candidate_dx(const Vec4<T>* __restrict__ P, const unsigned* __restrict__ M, int j,
                                            const int Pi[3], const T offi[3], T c0, int l, int cy, int cz, T offj[3],
                                            T& hj, unsigned& mj, T dx[3], T& r2) {
    Rec<T, D>::load(P, M, j, offj, hj, mj);
    const int cxj = meta_cx(mj);
    dx[0] = rn_add(rn_sub(offi[0], offj[0]), rn_mul((T)(Pi[0] - (cxj << l)), c0));
    dx[1] = rn_add(rn_sub(offi[1], offj[1]), rn_mul((T)(Pi[1] - (cy << l)), c0));
    if (D == 3) dx[2] = rn_add(rn_sub(offi[2], offj[2]), rn_mul((T)(Pi[2] - (cz << l)), c0));
    else dx[2] = T(0);
    r2 = rn_add(rn_mul(dx[0], dx[0]), rn_mul(dx[1], dx[1]));
    if (D == 3) r2 = rn_add(r2, rn_mul(dx[2], dx[2]));
    return cxj;
}

// the largest smoothing length of the level-l particles in the occupancy cells that cover the
// level-l cell box lo..hb (recorded by the gather; 0: the level has none there, infinite: not
// known)
template <int D>
__device__ __forceinline__ float level_hmax(const Grid& g, const unsigned* __restrict__ occ, int l, const int lo[3],
                                            const int hb[3]) {
    if (!occ) return CUDART_INF_F;
    const int sh = g.osh;
    int o0[3] = {0, 0, 0}, o1[3] = {0, 0, 0};
    for (int a = 0; a < D; ++a) {   // a particle past the last occupancy cell is counted in it
        o0[a] = min((lo[a] << l) >> sh, g.od[a] - 1);
        o1[a] = min((hb[a] << l) >> sh, g.od[a] - 1);
    }
    // a box of many occupancy cells is searched without the bound (it would cost more loads
    // than it can save)
    if ((o1[0] - o0[0] + 1) * (o1[1] - o0[1] + 1) * (o1[2] - o0[2] + 1) > 64) return CUDART_INF_F;
    unsigned m = 0;   // positive floats order as their bits
    for (int z = o0[2]; z <= o1[2]; ++z)
        for (int y = o0[1]; y <= o1[1]; ++y)
            for (int x = o0[0]; x <= o1[0]; ++x) {
                const unsigned v = __ldg(occ + (size_t)(g.occ_base + (z * g.od[1] + y) * g.od[0] + x) * OCCW + l);
                m = v > m ? v : m;
            }
    return __uint_as_float(m);
}

// Flat walk of the stencil rows (below) per dimension; off, each row is walked on its own,
// whole.  Measured on the 1.2M cube with 2 cells per support, 8 lanes per particle: the flat
// walk visits 29 % fewer candidates (439 against 620 per particle) in 37 % fewer warp-level
// loop bodies; with the local support bound the pressure pass takes 3.42 ms against 3.57 ms
// for the row walk.  In 2D (4 lanes, ~7 rows per particle) it is 8 % slower, and with 4
// cells per support in 3D the rows' set-up outweighs the tighter cut (3.91 ms).
#ifndef SPH_FLAT_WALK_2D
#define SPH_FLAT_WALK_2D 0
#endif
#ifndef SPH_FLAT_WALK_3D
#define SPH_FLAT_WALK_3D 1
#endif
template <int D> struct FlatWalk {
    static constexpr bool on = D == 2 ? SPH_FLAT_WALK_2D != 0 : SPH_FLAT_WALK_3D != 0;
};

template <typename T, int D, int LPP, int CAP, typename A, typename F>
__device__ __forceinline__ void walk_sub(const Grid& g, const int* __restrict__ cell_start,
                                         const unsigned* __restrict__ occ, int n, const Vec4<T>* __restrict__ P,
                                         const unsigned* __restrict__ M, int2* __restrict__ buf, bool active, int li,
                                         const int ci[3], const T offi[3], T hi, T kappa, A&& accept, F&& fn) {
    if (!active) return;
    const int sub = (int)(threadIdx.x % LPP);
    const T c0 = (T)g.c0;
    const T inv_c0 = T(1) / c0;
    int Pi[3];
    T fi[3];
    for (int a = 0; a < 3; ++a) {
        Pi[a] = ci[a] << li;
        fi[a] = offi[a] * inv_c0;
    }
    const T rhi = kappa * hi;
    int cnt = 0;
    auto flush = [&]() {
        for (int t = 0; t < cnt; ++t) {
            const int2 e = buf[t * BLOCK];
            const int l = e.y >> 28, cz = (e.y >> 14) & 0x3fff, cy = e.y & 0x3fff;
            T offj[3], hj, dx[3], r2;
            unsigned mj;
            const int cxj = candidate_dx<T, D>(P, M, e.x, Pi, offi, c0, l, cy, cz, offj, hj, mj, dx, r2);
            fn(e.x, dx, r2, hj, mj, offj, l, cxj, cy, cz);
        }
        cnt = 0;
    };
    for (int l = 0; l < g.L; ++l) {
        // every particle of level l has kappa h_j <= m c_l
        const T cl = wp<T>(g.c[l], g.cf[l]) * (T)(1 << g.sm);
        T R = T(0.5) * (rhi + cl);
        R = (R > rhi ? R : rhi) * T(1.0 + 1.0 / 1024.0);
        const T Rb = R * inv_c0;
        int lo[3] = {0, 0, 0}, hb[3] = {0, 0, 0};
        bool empty = false;
        for (int a = 0; a < D; ++a) {
            const int a0 = (Pi[a] + (int)t_floor(fi[a] - Rb)) >> l;
            const int a1 = (Pi[a] + (int)t_floor(fi[a] + Rb)) >> l;
            lo[a] = a0 < 0 ? 0 : a0;
            hb[a] = a1 > g.dims[l][a] - 1 ? g.dims[l][a] - 1 : a1;
            empty = empty || lo[a] > hb[a];
        }
        if (empty) continue;
        {
            // the level's particles near this one: none, or R from their largest support when
            // that is below the level's bound (a box of fewer cells, fewer candidates inside R).
            // Measured against one test of the 3^D occupancy cells around the particle for all
            // levels: 9 % faster per 3D step before the bound, and with it 2 % faster in 2D.
            const float hm = level_hmax<D>(g, occ, l, lo, hb);
            if (hm == 0.0f) continue;
            const T cm = kappa * (T)hm;
            if (cm < cl) {
                R = T(0.5) * (rhi + cm);
                R = (R > rhi ? R : rhi) * T(1.0 + 1.0 / 1024.0);
                const T Rt = R * inv_c0;
                for (int a = 0; a < D; ++a) {
                    const int a0 = (Pi[a] + (int)t_floor(fi[a] - Rt)) >> l;
                    const int a1 = (Pi[a] + (int)t_floor(fi[a] + Rt)) >> l;
                    lo[a] = a0 < 0 ? 0 : a0;
                    hb[a] = a1 > g.dims[l][a] - 1 ? g.dims[l][a] - 1 : a1;
                    empty = empty || lo[a] > hb[a];
                }
                if (empty) continue;
            }
        }
        const T Rc = R * inv_c0;
        // every radius the callers test at this level is below R: candidates beyond it are
        // rejected on the distance alone
        const T R2 = R * R;
        const int dxl = g.dims[l][0], dyl = g.dims[l][1];
        auto test = [&](int j, T mcy, T mcz, int tag) {
            T offj[3], hj, dx[3];
            unsigned mj;
            Rec<T, D>::load(P, M, j, offj, hj, mj);
            dx[0] = rn_add(rn_sub(offi[0], offj[0]), rn_mul((T)(Pi[0] - (meta_cx(mj) << l)), c0));
            dx[1] = rn_add(rn_sub(offi[1], offj[1]), mcy);
            dx[2] = D == 3 ? rn_add(rn_sub(offi[2], offj[2]), mcz) : T(0);
            T r2 = rn_add(rn_mul(dx[0], dx[0]), rn_mul(dx[1], dx[1]));
            if (D == 3) r2 = rn_add(r2, rn_mul(dx[2], dx[2]));
            if (r2 < R2 && accept(j, dx, r2, hj, mj)) {
                buf[cnt * BLOCK] = make_int2(j, tag);
                if (++cnt == CAP) flush();
            }
        };
        if constexpr (FlatWalk<D>::on) {
            // Flat walk.  The stencil rows are taken LPP at a time, one row per lane: the lane
            // cuts its row to the cells that reach the ball of radius R (the row's nearest
            // point in the other axes fixes the chord), the lengths are scanned across the
            // particle's lanes, and the lanes then step through the concatenated candidates,
            // so that no lane idles at the end of a short row.  The cut only drops candidates
            // at distance >= R, which the test below rejects anyway: the accepted pairs are
            // those of the full box.
            __shared__ int4 s_row[BLOCK];   // (end of the row's span, first index - span start, tag, -)
            __shared__ T s_mc[2 * BLOCK];   // the row's cell offsets in y and z, times c0
            const unsigned pmask =
                LPP == 32 ? 0xffffffffu
                          : ((1u << (LPP & 31)) - 1u) << ((threadIdx.x & 31u) & ~(unsigned)(LPP - 1));
            const int gb = (int)(threadIdx.x & ~(unsigned)(LPP - 1));
            const T Rc2 = Rc * Rc;
            const int wl = 1 << l;
            const int ny = hb[1] - lo[1] + 1, nrows = ny * (hb[2] - lo[2] + 1);
            for (int r0 = 0; r0 < nrows; r0 += LPP) {
                const int r = r0 + sub;
                int len = 0, first = 0, tag = 0;
                T mcy = T(0), mcz = T(0);
                if (r < nrows) {
                    const int rz = r / ny, cz = lo[2] + rz, cy = lo[1] + (r - rz * ny);
                    // the row's cells span [oy, oy + 2^l) and [oz, oz + 2^l) in finest cells,
                    // counted from the particle's cell corner
                    const int oy = (cy << l) - Pi[1], oz = (cz << l) - Pi[2];
                    T dy = (T)oy - fi[1], ey = fi[1] - (T)(oy + wl);
                    dy = dy > ey ? dy : ey;
                    dy = dy > T(0) ? dy : T(0);
                    T dz = T(0);
                    if (D == 3) {
                        T ez = fi[2] - (T)(oz + wl);
                        dz = (T)oz - fi[2];
                        dz = dz > ez ? dz : ez;
                        dz = dz > T(0) ? dz : T(0);
                    }
                    const T d2 = dy * dy + dz * dz;
                    if (d2 < Rc2) {
                        const T w = t_sqrt(Rc2 - d2);
                        const int a0 = max((Pi[0] + (int)t_floor(fi[0] - w)) >> l, lo[0]);
                        const int a1 = min((Pi[0] + (int)t_floor(fi[0] + w)) >> l, hb[0]);
                        if (a0 <= a1) {
                            const int row = g.base[l] + (cz * dyl + cy) * dxl;
                            first = max(__ldg(cell_start + row + a0), 0);
                            len = max(min(__ldg(cell_start + row + a1 + 1), n) - first, 0);
                        }
                    }
                    mcy = rn_mul((T)(Pi[1] - (cy << l)), c0);
                    if (D == 3) mcz = rn_mul((T)(Pi[2] - (cz << l)), c0);
                    tag = (l << 28) | (cz << 14) | cy;
                }
                int incl = len;
#pragma unroll
                for (int o = 1; o < LPP; o <<= 1) {
                    const int v = __shfl_up_sync(pmask, incl, o, LPP);
                    if (sub >= o) incl += v;
                }
                const int total = __shfl_sync(pmask, incl, LPP - 1, LPP);
                __syncwarp(pmask);   // the lanes are done with the previous rows
                s_row[threadIdx.x] = make_int4(incl, first - (incl - len), tag, 0);
                s_mc[2 * threadIdx.x] = mcy;
                s_mc[2 * threadIdx.x + 1] = mcz;
                __syncwarp(pmask);
                int cur = gb - 1, cend = 0, delta = 0, rtag = 0;
                T my = T(0), mz = T(0);
                for (int k = sub; k < total; k += LPP) {
                    while (k >= cend) {   // ends rise to total: stops at a lane of this group
                        ++cur;
                        const int4 q = s_row[cur];
                        cend = q.x;
                        delta = q.y;
                        rtag = q.z;
                        my = s_mc[2 * cur];
                        mz = s_mc[2 * cur + 1];
                    }
                    test(k + delta, my, mz, rtag);
                }
            }
            continue;
        }
        for (int cz = lo[2]; cz <= hb[2]; ++cz) {
            const T mcz = D == 3 ? rn_mul((T)(Pi[2] - (cz << l)), c0) : T(0);
            for (int cy = lo[1]; cy <= hb[1]; ++cy) {
                const T mcy = rn_mul((T)(Pi[1] - (cy << l)), c0);
                const int rid = cz * dyl + cy;
                const int row = g.base[l] + rid * dxl;
                const int s = max(__ldg(cell_start + row + lo[0]), 0);
                const int e = min(__ldg(cell_start + row + hb[0] + 1), n);
                for (int j = s + sub; j < e; j += LPP) test(j, mcy, mcz, (l << 28) | (cz << 14) | cy);
            }
        }
    }
    flush();
}

// sum over the LPP lanes of one particle (xor butterfly: every lane gets the same bits).  The
// lanes of a particle are consecutive and aligned, and the mask names only them: a caller may
// branch per particle (all lanes of a particle take the same branch).
template <int LPP, typename T> __device__ __forceinline__ T sub_sum(T v) {
    static_assert(LPP >= 1 && LPP <= 32 && (LPP & (LPP - 1)) == 0, "lanes per particle: a power of two");
    const unsigned mask =
        LPP == 32 ? 0xffffffffu : ((1u << (LPP & 31)) - 1u) << ((threadIdx.x & 31u) & ~(unsigned)(LPP - 1));
#pragma unroll
    for (int o = 1; o < LPP; o <<= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

}  // namespace sph
