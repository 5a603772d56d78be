// Loading a particle set into an instance's slots and reading it back, on the device: the
// caller's FP64 arrays are copied as they are into a staging buffer, checked and converted
// there (finest cell + working-precision offset, meta word, input index), and read back in the
// caller's order with FP64 positions rebuilt as origin + cell c0 + offset.  The arithmetic is
// the host reference's operation by operation (each FP64 product and sum rounded on its own,
// no fused multiply-add), so the stored state does not depend on where it was converted.
#include "sph_internal.cuh"

namespace sph {

namespace {

// first offending particle: key (index << 2) | check, checks in the order group (0), position
// (1), h (2), velocity (3); the smallest key is the first failure of a host loop over the
// particles taking the checks in that order
__global__ void __launch_bounds__(BLOCK) k_check_state(IoCheck c, int n, const double* __restrict__ x,
                                                       const int* __restrict__ group, const double* __restrict__ v,
                                                       const double* __restrict__ h,
                                                       unsigned long long* __restrict__ first) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int bad = -1;
    const int gi = group[i];
    if (gi < 0 || gi >= c.G) bad = 0;
    for (int a = 0; a < c.D && bad < 0; ++a) {
        const double xa = x[(size_t)i * 3 + a];
        if (!(xa >= c.lo[a] && xa <= c.hi[a])) bad = 1;
    }
    if (bad < 0 && h && !(h[i] > 0.0 && h[i] <= c.hmax)) bad = 2;
    if (bad < 0 && v)
        for (int a = 0; a < c.D; ++a)
            if (!isfinite(v[(size_t)i * 3 + a])) bad = 3;
    if (bad >= 0) atomicMin(first, ((unsigned long long)i << 2) | (unsigned long long)bad);
}

template <typename T, int D>
__global__ void __launch_bounds__(BLOCK) k_load_state(SlotArrays<T> s, IoGrid g, int ns, int n,
                                                      const double* __restrict__ x, const int* __restrict__ group,
                                                      const double* __restrict__ v, const double* __restrict__ h) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ns) return;
    if (k >= n) {   // padding: zero state, no input index
        for (int a = 0; a < D; ++a) {
            s.C[a][k] = 0;
            s.O[a][k] = T(0);
            s.V[a][k] = T(0);
        }
        s.H[k] = T(0);
        s.G[k] = 0u;
        s.ID[k] = -1;
        return;
    }
    for (int a = 0; a < D; ++a) {
        // finest cell and offset: c = floor((x - origin) (1/c0)), o = (x - origin) - c c0
        const double rel = __dsub_rn(x[(size_t)k * 3 + a], g.origin[a]);
        const double t = floor(__dmul_rn(rel, g.inv_c0));
        int ca = (int)fmax(fmin(t, 2.0e9), -2.0e9);
        ca = min(max(ca, 0), g.dims0[a] - 1);
        s.C[a][k] = ca;
        s.O[a][k] = (T)__dsub_rn(rel, __dmul_rn((double)ca, g.c0));
        s.V[a][k] = v ? (T)v[(size_t)k * 3 + a] : T(0);
    }
    s.H[k] = h ? (T)h[k] : T(0);
    const int gi = group[k];
    s.G[k] = (unsigned)gi | ((unsigned)g.fdim[gi] << 6);
    s.ID[k] = k;
}

template <typename T, int D>
__global__ void __launch_bounds__(BLOCK) k_store_state(ConstSlotArrays<T> s, IoGrid g, int ns, int n,
                                                       double* __restrict__ x, int* __restrict__ group,
                                                       double* __restrict__ v, double* __restrict__ h,
                                                       int* __restrict__ cnt) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ns) return;
    const int i = s.ID[k];
    if (i < 0) return;   // padding
    if (i >= n) {
        atomicOr(cnt + 1, 1);
        return;
    }
    atomicAdd(cnt, 1);
    for (int a = 0; a < 3; ++a) {
        if (x)
            x[(size_t)i * 3 + a] =
                a < D ? __dadd_rn(__dadd_rn(g.origin[a], __dmul_rn((double)s.C[a][k], g.c0)), (double)s.O[a][k]) : 0.0;
        if (v) v[(size_t)i * 3 + a] = a < D ? (double)s.V[a][k] : 0.0;
    }
    if (h) h[i] = (double)s.H[k];
    if (group) group[i] = (int)(s.G[k] & 63u);
}

}  // namespace

void launch_check_state(const IoCheck& c, int n, const double* x, const int* group, const double* v, const double* h,
                        unsigned long long* first, cudaStream_t st) {
    if (n > 0) k_check_state<<<div_up(n, BLOCK), BLOCK, 0, st>>>(c, n, x, group, v, h, first);
}

template <typename T, int D>
void launch_load_state(const SlotArrays<T>& s, const IoGrid& g, int ns, int n, const double* x, const int* group,
                       const double* v, const double* h, cudaStream_t st) {
    if (ns > 0) k_load_state<T, D><<<div_up(ns, BLOCK), BLOCK, 0, st>>>(s, g, ns, n, x, group, v, h);
}

template <typename T, int D>
void launch_store_state(const ConstSlotArrays<T>& s, const IoGrid& g, int ns, int n, double* x, int* group, double* v,
                        double* h, int* cnt, cudaStream_t st) {
    if (ns > 0) k_store_state<T, D><<<div_up(ns, BLOCK), BLOCK, 0, st>>>(s, g, ns, n, x, group, v, h, cnt);
}

#define SPH_INST(T, D)                                                                                            \
    template void launch_load_state<T, D>(const SlotArrays<T>&, const IoGrid&, int, int, const double*, const int*, \
                                          const double*, const double*, cudaStream_t);                              \
    template void launch_store_state<T, D>(const ConstSlotArrays<T>&, const IoGrid&, int, int, double*, int*,       \
                                           double*, double*, int*, cudaStream_t);
SPH_INST(float, 2)
SPH_INST(float, 3)
SPH_INST(double, 2)
SPH_INST(double, 3)
#undef SPH_INST

}  // namespace sph
