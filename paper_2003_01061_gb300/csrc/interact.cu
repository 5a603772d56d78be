// interact.cu -- the fused pressure pass of one relaxation step (Algorithm 1: renormalisation
// gamma_i, pressure force with the feature-boundary correction, map onto the feature, step-size
// candidates).  LPP consecutive lanes handle one particle (sorted order) and split its
// neighbour candidates; their partial sums are combined with a fixed shuffle butterfly.
//
// For particle i of group g (intrinsic dimension d, kernel W_d, rho = h^-d, P = p0 h^(2d)):
//   sigma_i = sum_{j in g, r < kappa h_i} W_d(r_ij, h_i)             (Eq. 20 denominator, j = i included)
//   gamma_i = sum_{j in g, r < kappa h_i} W_d(r_ij, h_i) h_j^d         (Eq. 18)
//   F_i     = sum_{j in g, j != i, r < kappa h_ij} (P_i + P_j) W_d'(r_ij, h_ij) e_ij          (Eq. 19, 1st sum)
//           + sum_{b: d_b < d, r < kappa h_ib} rho_b (P_i + P_b) W_d(r_ib, h_ib) n_b|i A_b  (Eq. 19, 2nd sum;
//             left out with boundary_correction = 0, the earlier method compared in Sec. 4.1)
//   a_p,i   = Pi_i(-F_i / gamma_i),  V~_i = 1 / sigma_i
// and the Eq. 24 candidates 0.25 sqrt(r_c/|a_p|), r_c/(40 |v|), reduced to per-group minima.
// On sampling steps each block also writes its per-group sums of V~ (Eq. 22) in a fixed order.
//
// A block serves BLOCK/LPP consecutive slots, which lie in one chunk and so in one instance:
// the instance's grid and parameters are copied into shared memory once per block (a batch of
// one passes them as kernel parameters instead).
#include "sph_internal.cuh"

namespace sph {

template <typename T, int D, bool ONE>
__global__ void __launch_bounds__(BLOCK, sizeof(T) == 4 ? (D == 2 ? SPH_INTERACT_MINB : SPH_INTERACT_MINB_3D) : 4)
    k_interact(State<T> s, One one, T* dbg_sigma, T* dbg_gamma, int cls) {
    dep_launch();
    dep_wait();
    constexpr int LPP = Lpp<D>::v;
    // the block's Eq. 24 minima and V~ partial sums live after the walk in the memory of its
    // candidate buffers (which the walk alone uses), leaving more of the SM's memory to L1
    constexpr bool ALIAS = (D == 2 ? SPH_ALIAS_TAIL_2D : SPH_ALIAS_TAIL_3D) != 0;
    constexpr size_t TAIL = 2 * MAXF * sizeof(unsigned long long) + (BLOCK / 32) * MAXF * sizeof(double);
    static_assert(!ALIAS || TAIL <= sizeof(int2) * BUF_CAP * BLOCK, "the tail fits in the candidate buffers");
    __shared__ __align__(16) int2 sbuf[BUF_CAP * BLOCK];
    __shared__ __align__(16) unsigned char sh_tail[ALIAS ? 16 : TAIL];
    unsigned char* const tail = ALIAS ? reinterpret_cast<unsigned char*>(sbuf) : sh_tail;
    unsigned long long* const sh_dta = reinterpret_cast<unsigned long long*>(tail);
    unsigned long long* const sh_dtv = sh_dta + MAXF;
    double (*const sh_part)[MAXF] = reinterpret_cast<double (*)[MAXF]>(sh_dtv + MAXF);
    __shared__ Grid gsh;
    __shared__ Params psh;
    const int inst = ONE ? 0 : __ldg(s.chunk_inst + (blockIdx.x * (BLOCK / LPP)) / CHUNK);
    Ctrl* const ctrl = s.ctrls + inst;
    const Domain& dom = s.doms[inst];
    if (!ONE) {
        block_copy(&gsh, s.grids + inst);
        block_copy(&psh, s.params + inst);
    }
    const Grid& g = ONE ? one.g : gsh;
    const Params& p = ONE ? one.p : psh;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const bool sample = ctrl->sample_now != 0;
    auto init_tail = [&]() {
        for (int t = threadIdx.x; t < MAXF; t += blockDim.x) {
            sh_dta[t] = inf_bits<T>();
            sh_dtv[t] = inf_bits<T>();
        }
        if (sample)
            for (int t = threadIdx.x; t < (BLOCK / 32) * MAXF; t += blockDim.x) (&sh_part[0][0])[t] = 0.0;
    };
    if (!ALIAS) init_tail();
    __syncthreads();
    const int G = p.G;

    const int k = (blockIdx.x * blockDim.x + threadIdx.x) / LPP;
    const bool lead = (threadIdx.x % LPP) == 0;
    const bool inrange = k < s.n && live(s, inst, k);
    T offi[3] = {T(0), T(0), T(0)}, hi = T(1);
    unsigned mi = 0;
    int li = 0, ci[3] = {0, 0, 0};
    if (inrange) {
        Rec<T, D>::load(s.P, s.Ms, k, offi, hi, mi);
        own_cell<T, D>(g, s, k, hi, li, ci);
    }
    const int gi = inrange ? meta_group(mi) : -1;
    const int di = inrange ? meta_dim(mi) : 0;
    // a converged (DONE) instance is frozen: no pair work
    bool active = inrange && di > 0 && ctrl->phase != PH_DONE && in_pass(p, cls, di, D);
    if (p.group_conv && active) active = ctrl->gphase[gi] != PH_DONE;   // the group itself converged
    T tg[3] = {T(0), T(0), T(0)};
    if (active && di < D) {
        T xi[3] = {T(0), T(0), T(0)};
        for (int a = 0; a < D; ++a) xi[a] = (T)g.origin[a] + (T)(ci[a] << li) * (T)g.c0 + offi[a];
        feature_tangent<T>(dom.f[gi], xi, tg);
    }
    const T kappa = wp<T>(p.kappa, p.kappa_f), hk = T(0.5) * kappa, p0 = wp<T>(p.p0, p.p0_f);
    const T rci2 = self_rc2(hi, kappa);
    const T invRi = fast_rcp(kappa * hi);
    const T alpha_i = wendland_alpha<T>(di > 0 ? di : 1, invRi);
    const T Pi = p0 * ipow(hi, 2 * di);
    T hid, hi2d;   // as the viscous pass computes them
    hpow(hi, di > 0 ? di : 1, hid, hi2d);
    const bool brho = p.boundary_rho != 0;
    const T c0 = (T)g.c0;
    const T org[3] = {(T)g.origin[0], (T)g.origin[1], (T)g.origin[2]};
    T F[3] = {T(0), T(0), T(0)};
    T sig = T(0), gam = T(0);
    constexpr int VCAP = Vcap<D>::v;
    const int NL = s.n * LPP;                              // lanes of the hand-over list
    const int lg = blockIdx.x * blockDim.x + threadIdx.x;  // this lane's column in it
    int vc = 0;

    walk_sub<T, D, LPP, BUF_CAP>(
        g, s.cell_start, s.occ, s.n, s.P, s.Ms, sbuf + threadIdx.x, active, li, ci, offi, hi, kappa,
        [&](int j, const T*, T r2, T hj, unsigned mj) -> bool {
            if (meta_group(mj) == gi) return r2 < rci2 || (j != k && r2 < pair_rc2(hi, hj, hk));
            return p.boundary_corr != 0 && meta_dim(mj) < di && r2 < pair_rc2(hi, hj, hk);
        },
        [&](int j, const T dx[3], T r2, T hj, unsigned mj, const T offj[3], int l, int cxj, int cy, int cz) {
            const T invr = r2 > T(0) ? fast_rsqrt(r2) : T(0);
            const T r = r2 * invr;
            T hjd, hj2d;
            hpow(hj, di, hjd, hj2d);
            if (meta_group(mj) == gi) {
                if (r2 < rci2) {
                    const T q = r * invRi;
                    const T t = T(1) - q;
                    const T w = alpha_i * (t * t) * (t * t) * (T(1) + T(4) * q);
                    sig += w;
                    gam += w * hjd;
                }
                if (j != k && r2 < pair_rc2(hi, hj, hk) && r2 > T(0)) {
                    const T invR = fast_rcp(hk * (hi + hj));
                    const T q = r * invR;
                    const T t = T(1) - q;
                    const T dW = wendland_alpha<T>(di, invR) * (T(-20) * q * t * t * t) * invR;
                    const T c1 = (Pi + p0 * hj2d) * dW * invr;
                    F[0] += c1 * dx[0];
                    F[1] += c1 * dx[1];
                    if (D == 3) F[2] += c1 * dx[2];
                    if (vc < VCAP) {   // the pair again in the viscous sum (Eq. 7, second term)
                        s.vj[(size_t)vc * NL + lg] = j;
                        // the viscous pass's kernel factor of the pair (Eq. 7): the same W' as here
                        s.vr[(size_t)vc * NL + lg] = (hi2d + hj2d) * dW * invr;
                    }
                    ++vc;
                }
            } else {
                const T invR = fast_rcp(hk * (hi + hj));
                const T q = r * invR;
                const T t = T(1) - q;
                const T w = wendland_alpha<T>(di, invR) * (t * t) * (t * t) * (T(1) + T(4) * q);
                const int cj[3] = {cxj, cy, cz};
                T xb[3] = {T(0), T(0), T(0)};
                for (int a = 0; a < D; ++a) xb[a] = org[a] + (T)(cj[a] << l) * c0 + offj[a];
                T nb[3];
                boundary_normal<T>(dom.f[meta_group(mj)], xb, nb);
                tangent_map<T>(di, D, tg, nb);
                const T nn2 = nb[0] * nb[0] + nb[1] * nb[1] + nb[2] * nb[2];
                if (nn2 > T(1e-12)) {
                    const T Ab = brho ? fast_rcp(hj) : hjd * fast_rcp(hj);
                    const T c2 = Ab * (Pi + p0 * hj2d) * w * fast_rsqrt(nn2);
                    F[0] += c2 * nb[0];
                    F[1] += c2 * nb[1];
                    if (D == 3) F[2] += c2 * nb[2];
                }
            }
        });
    if (inrange) s.vcnt[lg] = vc;
    if (ALIAS) {   // every walk of the block is done before its buffers become the tail
        __syncthreads();
        init_tail();
        __syncthreads();
    }
    for (int a = 0; a < D; ++a) F[a] = sub_sum<LPP>(F[a]);
    sig = sub_sum<LPP>(sig);
    gam = sub_sum<LPP>(gam);

    T ap[3] = {T(0), T(0), T(0)};
    T vtil = T(0);
    if (active && lead) {
        const T ig = T(1) / gam;
        for (int a = 0; a < 3; ++a) ap[a] = -F[a] * ig;
        tangent_map<T>(di, D, tg, ap);
        vtil = T(1) / sig;
        const T rc = kappa * hi;
        const T an = t_sqrt(ap[0] * ap[0] + ap[1] * ap[1] + ap[2] * ap[2]);
        const Vec4<T> vh = s.VH[k];
        const T v0 = vh.x, v1 = vh.y, v2 = vh.z;
        const T vn = t_sqrt(v0 * v0 + v1 * v1 + v2 * v2);
        const T dta = an > T(0) ? wp<T>(p.cfl_a, p.cfl_a_f) * t_sqrt(rc / an) : T(CUDART_INF_F);
        const T dtv = vn > T(0) ? wp<T>(p.cfl_v, p.cfl_v_f) * rc / vn : T(CUDART_INF_F);
        if (!(an == an) || !isfinite(an)) atomicOr(&ctrl->status, ST_NONFINITE);
        atomicMin(&sh_dta[gi], min_bits(dta));
        atomicMin(&sh_dtv[gi], min_bits(dtv));
    }
    if (inrange && lead) {
        Vec4<T> a4;
        a4.x = ap[0];
        a4.y = ap[1];
        a4.z = ap[2];
        a4.w = vtil;
        s.A[k] = a4;
        if (dbg_sigma) dbg_sigma[k] = sig;
        if (dbg_gamma) dbg_gamma[k] = gam;
    }
    if (sample) {
        // deterministic per-warp, per-group sums of V~: one fixed shuffle tree per group present
        const unsigned full = 0xffffffffu;
        const int gk = (active && lead) ? gi : -1;
        unsigned pending = __ballot_sync(full, gk >= 0);
        while (pending) {
            int leader = __ffs(pending) - 1;
            int gg = __shfl_sync(full, gk, leader);
            double v = (gk == gg) ? (double)vtil : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(full, v, o);
            if (lane == 0) sh_part[wid][gg] = v;
            pending &= ~__ballot_sync(full, gk == gg);
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < G; t += blockDim.x) {
        if (sh_dta[t] != inf_bits<T>()) atomicMin(&ctrl->dta_bits[t], sh_dta[t]);
        if (sh_dtv[t] != inf_bits<T>()) atomicMin(&ctrl->dtv_bits[t], sh_dtv[t]);
        if (sample) {
            double acc = 0.0;
            for (int w = 0; w < BLOCK / 32; ++w) acc += sh_part[w][t];
            s.partials[(size_t)blockIdx.x * MAXF + t] = acc;
        }
    }
    if (sample) {
        // the last block of this chunk of slots to finish adds the chunk's block rows, in block
        // order, into one row (a chunk lies in one instance; the controller then reads one row
        // per chunk instead of one per block)
        constexpr int BPC = CHUNK * LPP / BLOCK;
        __shared__ int sh_last;
        const int c = blockIdx.x / BPC;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) sh_last = atomicAdd(s.pticket + c, 1) == BPC - 1;
        __syncthreads();
        if (sh_last) {
            __threadfence();
            for (int t = threadIdx.x; t < G; t += blockDim.x) {
                double acc = 0.0;
                for (int b = 0; b < BPC; ++b) acc += __ldcg(s.partials + (size_t)(c * BPC + b) * MAXF + t);
                s.partials2[(size_t)c * MAXF + t] = acc;
            }
            if (threadIdx.x == 0) s.pticket[c] = 0;
        }
    }
}

// neighbour sets for inspection, through the same walk as the pair passes (one lane per
// particle): mode 0 pair predicate (j != i), mode 1 self predicate (j = i included), over all
// groups.  lists == nullptr: count only.  (A block spans several chunks: the instance is
// looked up per slot.)
template <typename T, int D>
__global__ void __launch_bounds__(BLOCK) k_neighbors(State<T> s, int mode, int* counts, const long long* offsets,
                                                     int* lists) {
    __shared__ int2 sbuf[BUF_CAP * BLOCK];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int inst = k < s.n ? inst_of(s, k) : 0;
    const Grid& g = s.grids[inst];
    const Params& p = s.params[inst];
    const bool active = k < s.n && live(s, inst, k);
    T offi[3] = {T(0), T(0), T(0)}, hi = T(1);
    unsigned mi = 0;
    int li = 0, ci[3] = {0, 0, 0};
    if (active) {
        Rec<T, D>::load(s.P, s.Ms, k, offi, hi, mi);
        own_cell<T, D>(g, s, k, hi, li, ci);
    }
    const T kappa = wp<T>(p.kappa, p.kappa_f), hk = T(0.5) * kappa;
    const T rci2 = self_rc2(hi, kappa);
    int cnt = 0;
    const long long base = (lists && active) ? offsets[k] : 0;
    walk_sub<T, D, 1, BUF_CAP>(
        g, s.cell_start, s.occ, s.n, s.P, s.Ms, sbuf + threadIdx.x, active, li, ci, offi, hi, kappa,
        [&](int j, const T*, T r2, T hj, unsigned) -> bool {
            return mode == 0 ? (j != k && r2 < pair_rc2(hi, hj, hk)) : (r2 < rci2);
        },
        [&](int j, const T*, T, T, unsigned, const T*, int, int, int, int) {
            if (lists) lists[base + cnt] = j;
            ++cnt;
        });
    if (k < s.n && !lists) counts[k] = cnt;
}

// candidate pairs examined and pairs inside the interaction support of the pressure pass,
// summed over all particles (one lane per particle)
template <typename T, int D>
__global__ void __launch_bounds__(BLOCK) k_pair_counts(State<T> s, unsigned long long* out2) {
    __shared__ int2 sbuf[BUF_CAP * BLOCK];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int inst = k < s.n ? inst_of(s, k) : 0;
    const Grid& g = s.grids[inst];
    const Params& p = s.params[inst];
    const bool inrange = k < s.n && live(s, inst, k);
    T offi[3] = {T(0), T(0), T(0)}, hi = T(1);
    unsigned mi = 0;
    int li = 0, ci[3] = {0, 0, 0};
    if (inrange) {
        Rec<T, D>::load(s.P, s.Ms, k, offi, hi, mi);
        own_cell<T, D>(g, s, k, hi, li, ci);
    }
    const int gi = inrange ? meta_group(mi) : -1, di = inrange ? meta_dim(mi) : 0;
    const bool active = inrange && di > 0;
    const T kappa = wp<T>(p.kappa, p.kappa_f), hk = T(0.5) * kappa;
    unsigned long long cand = 0, accd = 0;
    walk_sub<T, D, 1, BUF_CAP>(
        g, s.cell_start, s.occ, s.n, s.P, s.Ms, sbuf + threadIdx.x, active, li, ci, offi, hi, kappa,
        [&](int j, const T*, T r2, T hj, unsigned mj) -> bool {
            ++cand;
            return (meta_group(mj) == gi || meta_dim(mj) < di) && j != k && r2 < pair_rc2(hi, hj, hk);
        },
        [&](int, const T*, T, T, unsigned, const T*, int, int, int, int) { ++accd; });
    for (int o = 16; o > 0; o >>= 1) {
        cand += __shfl_down_sync(0xffffffffu, cand, o);
        accd += __shfl_down_sync(0xffffffffu, accd, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out2, cand);
        atomicAdd(out2 + 1, accd);
    }
}

template <typename T, int D>
void launch_interact(const State<T>& s, const One* one, T* dbg_sigma, T* dbg_gamma, cudaStream_t st, bool pdl,
                     int cls) {
    if (one) launch_k(k_interact<T, D, true>, s.nblk, BLOCK, st, pdl, s, *one, dbg_sigma, dbg_gamma, cls);
    else launch_k(k_interact<T, D, false>, s.nblk, BLOCK, st, pdl, s, One(), dbg_sigma, dbg_gamma, cls);
}
template <typename T, int D>
void launch_neighbors(const State<T>& s, int mode, int* counts, const long long* offsets, int* lists, cudaStream_t st) {
    k_neighbors<T, D><<<div_up(s.n, BLOCK), BLOCK, 0, st>>>(s, mode, counts, offsets, lists);
}
template <typename T, int D> void launch_pair_counts(const State<T>& s, unsigned long long* out2, cudaStream_t st) {
    k_pair_counts<T, D><<<div_up(s.n, BLOCK), BLOCK, 0, st>>>(s, out2);
}

#define SPH_INST(T, D)                                                                                        \
    template void launch_interact<T, D>(const State<T>&, const One*, T*, T*, cudaStream_t, bool, int);        \
    template void launch_neighbors<T, D>(const State<T>&, int, int*, const long long*, int*, cudaStream_t);   \
    template void launch_pair_counts<T, D>(const State<T>&, unsigned long long*, cudaStream_t);
SPH_INST(float, 2)
SPH_INST(float, 3)
SPH_INST(double, 2)
SPH_INST(double, 3)

}  // namespace sph
