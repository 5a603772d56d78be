// sample.cu -- the initial particle set on the device (Sec. 3.6; Algorithm 1: "calculate the
// target information (Eqs. 10, 11)" and "allocate particles ... initial particle sampling").
//
// Target counts: N_k = integral over feature k of rho_t = h_t^-d (Eqs. 10, 11), by the midpoint
// rule on a fixed grid of the feature's parameter space (volume: the bounding box, cells whose
// centre has phi > 0); per-block FP64 partial sums added on the host in block order.
//
// Sampling: particles of feature k are drawn with probability proportional to rho_t by
// rejection.  Candidate c of feature k takes the four 32-bit outputs of Philox4x32-10 (Salmon,
// Moraes, Dror, Shaw, SC 2011) for counter (c, c >> 32, k, 0) under the key (seed, seed >> 32),
// as uniforms u = (x + 1/2) 2^-32; it is accepted with probability (h_min/h_t(x))^d (h_min the
// sizing's lower bound), volume candidates only where phi(x) > h_t(x)/4, face candidates only
// h_t/4 inside the face's edges, and feature k keeps its first N_k accepted candidates in
// candidate order.  Every FP64 operation that decides acceptance is rounded one by one, so a
// candidate is accepted or rejected exactly as by any other correctly rounded evaluation of
// the same expressions.
#include "sph_internal.cuh"

#include <algorithm>
#include <vector>

namespace sph {

namespace {

constexpr int SB = 256;   // threads per block of the sampling kernels

__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }

// |x - c| over the first n components, summed in component order
__device__ double dist_n(const double x[3], const double* c, int n) {
    double s = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double d = a < n ? dsub(x[a], c[a]) : 0.0;
        s = dadd(s, dmul(d, d));
    }
    return __dsqrt_rn(s);
}

// h_t(x) (Eq. 2, the analytic sizing) in FP64
__device__ double samp_h(const Sizing& z, const double x[3]) {
    if (z.kind == 0) return z.a;
    double h;
    if (z.kind == 1) {
        double dmin = 1.7976931348623157e308;
        for (int k = 0; k < z.nref; ++k) {
            const double dk = fabs(dsub(dist_n(x, z.rc[k], 3), z.rr[k]));
            if (dk < dmin) dmin = dk;
        }
        h = dadd(z.a, dmul(z.b, dmin));
    } else {
        h = dadd(z.a, dmul(z.b, dist_n(x, z.q, 3)));
    }
    if (h < z.lo) h = z.lo;
    if (h > z.hi) h = z.hi;
    return h;
}

// the level set phi(x) (Eq. 1): box or ball minus the holes, in FP64
__device__ double samp_phi(const Domain& dm, const double x[3]) {
    double phi = 1.7976931348623157e308;
    if (dm.base == 0) {
        for (int a = 0; a < dm.D; ++a) {
            const double dlo = dsub(x[a], dm.lo[a]), dhi = dsub(dm.hi[a], x[a]);
            if (dlo < phi) phi = dlo;
            if (dhi < phi) phi = dhi;
        }
    } else {
        phi = dsub(dm.br, dist_n(x, dm.bc, dm.D));
    }
    for (int k = 0; k < dm.nh; ++k) {
        const double pk = dsub(dist_n(x, dm.hc[k], dm.D), dm.hr[k]);
        if (pk < phi) phi = pk;
    }
    return phi;
}

// Philox4x32-10: ten rounds of the Philox S-box, the key advanced by the Weyl constants between
// rounds (Salmon et al., SC 2011)
__device__ __forceinline__ void philox(unsigned c[4], unsigned k0, unsigned k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const unsigned lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        const unsigned lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const unsigned n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

__device__ __forceinline__ void uniforms(unsigned long long seed, int k, long long c, double u[4]) {
    unsigned w[4] = {(unsigned)c, (unsigned)((unsigned long long)c >> 32), (unsigned)k, 0u};
    philox(w, (unsigned)seed, (unsigned)(seed >> 32));
#pragma unroll
    for (int a = 0; a < 4; ++a) u[a] = ((double)w[a] + 0.5) * (1.0 / 4294967296.0);
}

// acceptance of candidate u of feature f, and its position
__device__ bool accept(const Domain& dm, const Sizing& z, const Feat& f, const double u[4], double x[3]) {
    x[0] = x[1] = x[2] = 0.0;
    const int D = dm.D;
    switch (f.kind) {
        case SPH_FEAT_VOLUME: {
            for (int a = 0; a < D; ++a) x[a] = dadd(dm.lo[a], dmul(u[a], dsub(dm.hi[a], dm.lo[a])));
            const double h = samp_h(z, x);
            if (!(samp_phi(dm, x) > dmul(0.25, h))) return false;
            const double r = ddiv(z.lo, h);
            double rd = dmul(r, r);
            if (D == 3) rd = dmul(rd, r);
            return u[3] < rd;
        }
        case SPH_FEAT_SEGMENT:
            for (int a = 0; a < 3; ++a) x[a] = dadd(f.g[a], dmul(u[0], dsub(f.g[3 + a], f.g[a])));
            return u[1] < ddiv(z.lo, samp_h(z, x));
        case SPH_FEAT_CIRCLE: {
            const double p0 = dsub(dmul(2.0, u[0]), 1.0), p1 = dsub(dmul(2.0, u[1]), 1.0);
            const double q = dadd(dmul(p0, p0), dmul(p1, p1));
            if (!(q > 0.0 && q <= 1.0)) return false;
            const double r = __dsqrt_rn(q);
            x[0] = dadd(f.g[0], dmul(f.g[2], ddiv(p0, r)));
            x[1] = dadd(f.g[1], dmul(f.g[2], ddiv(p1, r)));
            return u[2] < ddiv(z.lo, samp_h(z, x));
        }
        case SPH_FEAT_SPHERE: {
            const double p0 = dsub(dmul(2.0, u[0]), 1.0), p1 = dsub(dmul(2.0, u[1]), 1.0),
                         p2 = dsub(dmul(2.0, u[2]), 1.0);
            const double q = dadd(dadd(dmul(p0, p0), dmul(p1, p1)), dmul(p2, p2));
            if (!(q > 0.0 && q <= 1.0)) return false;
            const double r = __dsqrt_rn(q);
            x[0] = dadd(f.g[0], dmul(f.g[3], ddiv(p0, r)));
            x[1] = dadd(f.g[1], dmul(f.g[3], ddiv(p1, r)));
            x[2] = dadd(f.g[2], dmul(f.g[3], ddiv(p2, r)));
            const double acc = ddiv(z.lo, samp_h(z, x));
            return u[3] < dmul(acc, acc);
        }
        case SPH_FEAT_RECT: {
            const double sv = dmul(u[0], f.g[9]), tv = dmul(u[1], f.g[10]);
            for (int a = 0; a < 3; ++a) x[a] = dadd(dadd(f.g[a], dmul(sv, f.g[3 + a])), dmul(tv, f.g[6 + a]));
            const double h = samp_h(z, x);
            const double m = dmul(0.25, h);
            if (!(sv > m && sv < dsub(f.g[9], m) && tv > m && tv < dsub(f.g[10], m))) return false;
            const double acc = ddiv(z.lo, h);
            return u[2] < dmul(acc, acc);
        }
        default:
            for (int a = 0; a < D; ++a) x[a] = f.g[a];
            return true;
    }
}

// pass 1: accepted candidates per block
__global__ void __launch_bounds__(SB) k_sample_count(const Domain* dmp, const Sizing* zp, int k,
                                                     unsigned long long seed, long long c0, long long nc,
                                                     int* block_count) {
    const Domain& dm = *dmp;
    const long long c = c0 + (long long)blockIdx.x * SB + threadIdx.x;
    bool ok = false;
    if (c < c0 + nc) {
        double u[4], x[3];
        uniforms(seed, k, c, u);
        ok = accept(dm, *zp, dm.f[k], u, x);
    }
    const int n = __syncthreads_count(ok ? 1 : 0);
    if (threadIdx.x == 0) block_count[blockIdx.x] = n;
}

// pass 2: accepted candidates written in candidate order, the first `want` of them
__global__ void __launch_bounds__(SB) k_sample_emit(const Domain* dmp, const Sizing* zp, int k,
                                                    unsigned long long seed, long long c0, long long nc,
                                                    const long long* block_off, long long want, double* out) {
    __shared__ int wsum[SB / 32];
    const Domain& dm = *dmp;
    const long long c = c0 + (long long)blockIdx.x * SB + threadIdx.x;
    bool ok = false;
    double x[3] = {0.0, 0.0, 0.0};
    if (c < c0 + nc) {
        double u[4];
        uniforms(seed, k, c, u);
        ok = accept(dm, *zp, dm.f[k], u, x);
    }
    const unsigned bal = __ballot_sync(0xffffffffu, ok);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) wsum[wid] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int w = 0; w < wid; ++w) before += wsum[w];
    const long long rank = block_off[blockIdx.x] + before + __popc(bal & ((1u << lane) - 1u));
    if (ok && rank < want)
        for (int a = 0; a < 3; ++a) out[3 * rank + a] = x[a];
}

// midpoint-rule integral of rho_t over feature k (Eqs. 10, 11), per-block partial sums
__global__ void __launch_bounds__(SB) k_feature_integral(const Domain* dmp, const Sizing* zp, int k, long long npts,
                                                         int nq, double* partial) {
    __shared__ double ws[SB / 32];
    const Domain& dm = *dmp;
    const Sizing& z = *zp;
    const Feat& f = dm.f[k];
    const int D = dm.D;
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * SB + threadIdx.x; i < npts; i += (long long)gridDim.x * SB) {
        double x[3] = {0.0, 0.0, 0.0};
        switch (f.kind) {
            case SPH_FEAT_VOLUME: {
                long long r = i;
                double cellv = 1.0;
                for (int a = 0; a < D; ++a) {
                    const long long ia = r % nq;
                    r /= nq;
                    const double dx = (dm.hi[a] - dm.lo[a]) / nq;
                    cellv *= dx;
                    x[a] = dm.lo[a] + (ia + 0.5) * dx;
                }
                if (samp_phi(dm, x) > 0.0) {
                    const double h = samp_h(z, x);
                    acc += cellv / (D == 3 ? h * h * h : h * h);
                }
                break;
            }
            case SPH_FEAT_SEGMENT: {
                double ab[3], L2 = 0.0;
                for (int a = 0; a < 3; ++a) {
                    ab[a] = f.g[3 + a] - f.g[a];
                    L2 += ab[a] * ab[a];
                }
                const double t = (i + 0.5) / nq;
                for (int a = 0; a < 3; ++a) x[a] = f.g[a] + t * ab[a];
                acc += (sqrt(L2) / nq) / samp_h(z, x);
                break;
            }
            case SPH_FEAT_CIRCLE: {
                const double th = 2.0 * CUDART_PI * (i + 0.5) / nq;
                x[0] = f.g[0] + f.g[2] * cos(th);
                x[1] = f.g[1] + f.g[2] * sin(th);
                acc += (2.0 * CUDART_PI * f.g[2] / nq) / samp_h(z, x);
                break;
            }
            case SPH_FEAT_RECT: {
                const long long ii = i % nq, jj = i / nq;
                const double si = (ii + 0.5) / nq * f.g[9], tj = (jj + 0.5) / nq * f.g[10];
                for (int a = 0; a < 3; ++a) x[a] = f.g[a] + si * f.g[3 + a] + tj * f.g[6 + a];
                const double h = samp_h(z, x);
                acc += (f.g[9] / nq) * (f.g[10] / nq) / (h * h);
                break;
            }
            case SPH_FEAT_SPHERE: {
                const long long ii = i / (2 * nq), jj = i % (2 * nq);
                const double th = CUDART_PI * (ii + 0.5) / nq, ph = CUDART_PI * (jj + 0.5) / nq;
                const double R = f.g[3];
                x[0] = f.g[0] + R * sin(th) * cos(ph);
                x[1] = f.g[1] + R * sin(th) * sin(ph);
                x[2] = f.g[2] + R * cos(th);
                const double h = samp_h(z, x);
                acc += R * R * sin(th) * (CUDART_PI / nq) * (CUDART_PI / nq) / (h * h);
                break;
            }
            default:
                break;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < SB / 32; ++w) s += ws[w];
        partial[blockIdx.x] = s;
    }
}

}  // namespace

int quad_points(int kind, int D, long long* npts) {
    int nq = 0;
    switch (kind) {
        case SPH_FEAT_VOLUME:
            nq = D == 2 ? SPH_QUAD_AREA : SPH_QUAD_VOLUME;
            *npts = D == 2 ? (long long)nq * nq : (long long)nq * nq * nq;
            break;
        case SPH_FEAT_SEGMENT:
        case SPH_FEAT_CIRCLE:
            nq = SPH_QUAD_CURVE;
            *npts = nq;
            break;
        case SPH_FEAT_RECT:
            nq = SPH_QUAD_FACE;
            *npts = (long long)nq * nq;
            break;
        case SPH_FEAT_SPHERE:
            nq = SPH_QUAD_SPHERE;
            *npts = 2LL * nq * nq;
            break;
        default:
            *npts = 0;
    }
    return nq;
}

cudaError_t feature_integrals(const Domain& dm, const Domain* d_dom, const Sizing* d_siz, cudaStream_t st,
                              double* integral) {
    // every feature's partial sums in one buffer, one copy back and one wait for all of them
    constexpr int NB = 4 * 152;
    double* d_part = nullptr;
    const size_t np = (size_t)NB * std::max(dm.nf, 1);
    cudaError_t e = cudaMallocAsync(&d_part, sizeof(double) * np, st);
    if (e != cudaSuccess) return e;
    std::vector<double> part(np, 0.0);
    e = cudaMemsetAsync(d_part, 0, sizeof(double) * np, st);
    for (int k = 0; k < dm.nf && e == cudaSuccess; ++k) {
        if (dm.f[k].kind == SPH_FEAT_POINT) continue;
        long long npts = 0;
        const int nq = quad_points(dm.f[k].kind, dm.D, &npts);
        k_feature_integral<<<NB, SB, 0, st>>>(d_dom, d_siz, k, npts, nq, d_part + (size_t)k * NB);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(part.data(), d_part, sizeof(double) * np, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (int k = 0; k < dm.nf; ++k) {
        if (dm.f[k].kind == SPH_FEAT_POINT) {
            integral[k] = 1.0;
            continue;
        }
        double sum = 0.0;
        for (int b = 0; b < NB; ++b) sum += part[(size_t)k * NB + b];
        integral[k] = sum;
    }
    cudaError_t f = cudaFreeAsync(d_part, st);
    if (e == cudaSuccess) e = f;
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

// Expected fraction of accepted candidates of feature k when it holds n particles (n is close to
// the integral of rho_t, so the acceptance (h_min/h)^d averages to n h_min^d / measure), times
// the fraction its geometry keeps (the disc in its square, the ball in its cube)
double acceptance_estimate(const Domain& dm, const Sizing& z, int k, long long n) {
    const Feat& f = dm.f[k];
    const int d = f.dim;
    double meas = 1.0, geo = 1.0;
    switch (f.kind) {
        case SPH_FEAT_VOLUME:
            for (int a = 0; a < dm.D; ++a) meas *= dm.hi[a] - dm.lo[a];
            break;
        case SPH_FEAT_SEGMENT: {
            double L2 = 0.0;
            for (int a = 0; a < 3; ++a) L2 += (f.g[3 + a] - f.g[a]) * (f.g[3 + a] - f.g[a]);
            meas = std::sqrt(L2);
            break;
        }
        case SPH_FEAT_CIRCLE:
            meas = 2.0 * CUDART_PI * f.g[2];
            geo = CUDART_PI / 4.0;
            break;
        case SPH_FEAT_RECT:
            meas = f.g[9] * f.g[10];
            break;
        case SPH_FEAT_SPHERE:
            meas = 4.0 * CUDART_PI * f.g[3] * f.g[3];
            geo = CUDART_PI / 6.0;
            break;
        default:
            return 1.0;
    }
    const double p = geo * (double)n * std::pow(z.lo, d) / meas;
    return std::min(1.0, std::max(p, 1e-9));
}

cudaError_t sample_features(const Domain& dm, const Sizing& z, const Domain* d_dom, const Sizing* d_siz,
                            unsigned long long seed, const int64_t* counts, cudaStream_t st, double* d_out) {
    // candidates per pass: enough for the remaining count at the expected acceptance, so that
    // one pass (one host round trip) usually suffices; a short pass is followed by another one
    // sized by the acceptance seen so far.  The result does not depend on the pass sizes: it is
    // always the first accepted candidates in candidate order.
    constexpr long long MAXB = 1LL << 26;
    int* d_cnt = nullptr;
    long long* d_off = nullptr;
    cudaError_t e = cudaMallocAsync(&d_cnt, sizeof(int) * (MAXB / SB), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_off, sizeof(long long) * (MAXB / SB), st);
    std::vector<int> cnt(MAXB / SB);
    std::vector<long long> off(MAXB / SB);
    long long base = 0;
    for (int k = 0; k < dm.nf && e == cudaSuccess; ++k) {
        const long long want = counts[k];
        if (want > 0 && dm.f[k].kind == SPH_FEAT_POINT) {   // the point itself
            double x[3] = {0.0, 0.0, 0.0};
            for (int a = 0; a < dm.D; ++a) x[a] = dm.f[k].g[a];
            e = cudaMemcpyAsync(d_out + 3 * base, x, sizeof x, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            base += want;
            continue;
        }
        double p = acceptance_estimate(dm, z, k, want);
        long long got = 0, c0 = 0, seen = 0, taken = 0;
        while (got < want && e == cudaSuccess) {
            const double need = (double)(want - got) / p;
            long long nc = (long long)(1.05 * need + 6.0 * std::sqrt(need)) + 4096;
            nc = std::min(MAXB, (nc + SB - 1) / SB * SB);
            const int nblk = (int)(nc / SB);
            k_sample_count<<<nblk, SB, 0, st>>>(d_dom, d_siz, k, seed, c0, nc, d_cnt);
            e = cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int) * nblk, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) break;
            long long run = got;
            for (int b = 0; b < nblk; ++b) {
                off[b] = run;
                run += cnt[b];
            }
            e = cudaMemcpyAsync(d_off, off.data(), sizeof(long long) * nblk, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) break;
            k_sample_emit<<<nblk, SB, 0, st>>>(d_dom, d_siz, k, seed, c0, nc, d_off, want, d_out + 3 * base);
            e = cudaStreamSynchronize(st);   // off is reused by the next pass
            seen += nc;
            taken += run - got;
            got = std::min(run, want);
            c0 += nc;
            p = std::max(1e-9, (double)std::max<long long>(taken, 1) / (double)seen);
            if (got < want && c0 >= (1LL << 36)) e = cudaErrorInvalidValue;   // acceptance too small
        }
        base += want;
    }
    if (d_cnt) cudaFreeAsync(d_cnt, st);
    if (d_off) cudaFreeAsync(d_off, st);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

}  // namespace sph
