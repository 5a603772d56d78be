// integrate.cu -- per-step controller (Sec. 3.4, Eq. 24) and the viscous pass + update +
// projection of one relaxation step (Algorithm 1: mid-point velocity, viscous force, map,
// predicted velocity, position, map).
#include "sph_internal.cuh"

namespace sph {

__device__ __forceinline__ double rel_err(double a, double b) {
    if (b != 0.0) return fabs(a - b) / fabs(b);
    return a == 0.0 ? 0.0 : CUDART_INF;
}

__device__ inline void window_reset(Ctrl* c) {
    c->wcount = 0;
    c->nwin = 0;
    for (int g = 0; g < MAXF; ++g) {
        c->wsum[g] = 0.0;
        c->A_last[g] = 0.0;
        c->A_prev[g] = 0.0;
    }
}

// One block.  Reduces the per-block V~ sums of a sampling step in a fixed order, then thread 0
// runs the controller for step n:
//  1. RAMP -> PHASE2 after ramp_len steps (windows restart);
//  2. in PHASE1 / PHASE2 on steps n % sample_every == 0: V-bar_g enters the open window; a full
//     window closes with its mean; with two closed windows E_t = max_g |V-bar - A_last|/|A_last|,
//     E_avg = max_g |A_last - A_prev|/|A_prev|, E_sys = max; E_sys < threshold moves
//     PHASE1 -> RAMP or PHASE2 -> DONE (Sec. 3.4.2);
//  3. step parameters: PHASE1 eps = eps1, f = 1, nullify when n % reset_period == 0; RAMP
//     s = (n - ramp_start)/ramp_len, eps = eps1 (1 - s), f = (1 + cos(pi s))/2; PHASE2 eps = 0,
//     nullify every step (Sec. 3.4.3, 3.4.4);
//  4. per group dt = min(dta, dtv/f), nullified (dt = dta) on the schedule or when dt falls
//     below dt_collapse times the group's previous step; dt <= dt_cap (Eq. 24).
template <typename T> __global__ void __launch_bounds__(256) k_control(Params p, State<T> s) {
    __shared__ double vs[MAXF];
    Ctrl* c = s.ctrl;
    const int G = p.G;
    const bool sample = c->sample_now != 0;
    if (sample) {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int g = wid; g < G; g += nw) {
            double acc = 0.0;
            for (int b = lane; b < s.nblk; b += 32) acc += s.partials[(size_t)b * G + g];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
            if (lane == 0) vs[g] = acc;
        }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;

    double dta[MAXF], dtv[MAXF];
    for (int g = 0; g < G; ++g) {
        dta[g] = (double)from_bits<T>(c->dta_bits[g]);
        dtv[g] = (double)from_bits<T>(c->dtv_bits[g]);
        c->dta_bits[g] = inf_bits<T>();
        c->dtv_bits[g] = inf_bits<T>();
    }
    bool done = c->phase == PH_DONE;
    if (!done && c->phase == PH_RAMP && c->n - c->ramp_start >= p.ramp_len) {
        c->phase = PH2;
        window_reset(c);
    }
    if (!done && (c->phase == PH1 || c->phase == PH2) && c->n % p.sample_every == 0) {
        for (int g = 0; g < G; ++g) {
            c->Vbar[g] = s.dom->f[g].dim > 0 ? vs[g] : 0.0;
            c->wsum[g] += c->Vbar[g];
        }
        c->wcount += 1;
        if (c->wcount == p.window) {
            for (int g = 0; g < G; ++g) {
                c->A_prev[g] = c->A_last[g];
                c->A_last[g] = c->wsum[g] / p.window;
                c->wsum[g] = 0.0;
            }
            c->wcount = 0;
            c->nwin += 1;
        }
        if (c->nwin >= 2) {
            double et = 0.0, ea = 0.0;
            for (int g = 0; g < G; ++g) {
                if (s.dom->f[g].dim < 1) continue;
                et = fmax(et, rel_err(c->Vbar[g], c->A_last[g]));
                ea = fmax(ea, rel_err(c->A_last[g], c->A_prev[g]));
            }
            c->E_t = et;
            c->E_avg = ea;
            c->E_sys = fmax(et, ea);
            if (c->E_sys < p.threshold) {
                if (c->phase == PH1) {
                    c->phase = PH_RAMP;
                    c->ramp_start = c->n;
                    window_reset(c);
                } else {
                    c->phase = PH_DONE;
                    done = true;
                }
            }
        }
    }
    if (done) {
        c->phase = PH_DONE;
        for (int g = 0; g < G; ++g) {
            c->dt[g] = 0.0;
            c->reset[g] = 1;
        }
        c->eps = 0.0;
        c->f = 0.0;
        c->sample_now = 0;
        return;
    }
    double eps = p.eps1, f = 1.0;
    bool periodic = (c->n % p.reset_period) == 0;
    if (c->phase == PH_RAMP) {
        double sr = (double)(c->n - c->ramp_start) / (double)p.ramp_len;
        eps = p.eps1 * (1.0 - sr);
        f = 0.5 * (1.0 + cos(CUDART_PI * sr));
    } else if (c->phase == PH2) {
        eps = 0.0;
        periodic = true;
    }
    for (int g = 0; g < G; ++g) {
        if (s.dom->f[g].dim < 1) {
            c->dt[g] = 0.0;
            c->reset[g] = 1;
            continue;
        }
        double dv = f > 0.0 ? dtv[g] / f : CUDART_INF;
        double cand = fmin(dta[g], dv);
        bool rs = periodic || (c->dt_prev[g] > 0.0 && cand < p.dt_collapse * c->dt_prev[g]);
        double dt = rs ? dta[g] : cand;
        dt = fmin(dt, p.dt_cap);
        c->dt_prev[g] = dt;
        c->dt[g] = dt;
        c->reset[g] = rs ? 1 : 0;
    }
    c->eps = eps;
    c->f = f;
    c->n += 1;
    c->sample_now = (c->n % p.sample_every) == 0 ? 1 : 0;
}

// Viscous pass + update, one thread per sorted particle, writing the new state in sorted order:
//   v'_i = 0 (nullified) or f v_i;  v~_i = v'_i + dt (a_p,i - eps v'_i)                       (Eq. 23)
//   a_v,i = Pi_i sum_{j in g, j != i} [2 eta_i eta_j/(eta_i+eta_j)] (rho_i^-2 + rho_j^-2)
//                 W_d'(r_ij, h_ij) (v~_i - v~_j) / r_ij,  eta = rho nu, nu = visc r_c |v~|    (Eq. 7, Eq. 8)
//   v+ = v~ + dt a_v;  x+ = x + dt v+  (FP64);  curves/surfaces: x+ onto the feature, v+ <- Pi(x+) v+;
//   volume: phi(x+) < 0 -> back to phi = 0.01 h along grad phi, v+ = 0, escape counted;  h+ = h_t(x+).
template <typename T, int D>
__global__ void __launch_bounds__(BLOCK) k_integrate(Grid g, Params p, State<T> s, const Ctrl* cu, Out<T> o) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= s.n) return;
    T offi[3], hi;
    unsigned mi;
    Rec<T, D>::load(s.P, s.Ms, k, offi, hi, mi);
    const int gi = meta_group(mi), di = meta_dim(mi);
    double x[3] = {s.Xs[0][k], s.Xs[1][k], D == 3 ? s.Xs[2][k] : 0.0};
    T v[3] = {s.Vs[0][k], s.Vs[1][k], D == 3 ? s.Vs[2][k] : T(0)};
    T av[3] = {T(0), T(0), T(0)};
    T hnew = hi;
    if (di == 0 || cu->phase == PH_DONE) {
        if (di == 0) v[0] = v[1] = v[2] = T(0);
    } else {
        const T dt = (T)cu->dt[gi];
        const bool rs = cu->reset[gi] != 0;
        const T f = (T)cu->f, eps = (T)cu->eps;
        const Vec4<T> ai = s.A[k];
        const T api[3] = {ai.x, ai.y, ai.z};
        T vt[3];
        for (int a = 0; a < 3; ++a) {
            T vp = rs ? T(0) : f * v[a];
            vt[a] = vp + dt * (api[a] - eps * vp);
        }
        const Feat& fi = s.dom->f[gi];
        T tg[3] = {T(0), T(0), T(0)};
        if (di < D) {
            T xi[3] = {(T)x[0], (T)x[1], (T)x[2]};
            feature_tangent<T>(fi, xi, tg);
        }
        if (p.visc > 0.0) {
            const T kappa = (T)p.kappa, hk = T(0.5) * kappa, visc = (T)p.visc;
            const T ri2 = ipow(hi, 2 * di);
            const T eta_i = visc * kappa * hi * t_sqrt(vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2]) / ipow(hi, di);
            int li, ci[3];
            decode_key(g, s.Ks[k], li, ci);
            walk<T, D>(g, s.cell_start, s.n, s.P, s.Ms, li, ci, offi, hi, kappa,
                       [&](int j, const T dx[3], T r2, T hj, unsigned mj, const T*, int, int, int, int) {
                           if (meta_group(mj) != gi || j == k || !(r2 < pair_rc2(hi, hj, hk))) return;
                           T r = t_sqrt(r2);
                           if (!(r > T(0))) return;
                           const Vec4<T> aj = s.A[j];
                           const T apj[3] = {aj.x, aj.y, aj.z};
                           T vtj[3];
                           for (int a = 0; a < D; ++a) {
                               T vp = rs ? T(0) : f * s.Vs[a][j];
                               vtj[a] = vp + dt * (apj[a] - eps * vp);
                           }
                           if (D == 2) vtj[2] = T(0);
                           T eta_j = visc * kappa * hj * t_sqrt(vtj[0] * vtj[0] + vtj[1] * vtj[1] + vtj[2] * vtj[2]) /
                                     ipow(hj, di);
                           T es = eta_i + eta_j;
                           if (!(es > T(0))) return;
                           T eb = T(2) * eta_i * eta_j / es;
                           T invR = T(2) / (kappa * (hi + hj));
                           T q = r * invR;
                           T t = T(1) - q;
                           T dW = wendland_alpha<T>(di, invR) * (T(-20) * q * t * t * t) * invR;
                           T coef = eb * (ri2 + ipow(hj, 2 * di)) * dW / r;
                           for (int a = 0; a < D; ++a) av[a] += coef * (vt[a] - vtj[a]);
                       });
            tangent_map<T>(di, D, tg, av);
        }
        for (int a = 0; a < 3; ++a) {
            v[a] = vt[a] + dt * av[a];
            if (a < D) x[a] = x[a] + (double)dt * (double)v[a];
        }
        if (fi.kind == K_VOLUME) {
            double gph[3];
            double ph = domain_phi(*s.dom, x, gph);
            if (ph < 0.0) {
                const double target = 0.01 * (double)hi;
                for (int it = 0; it < 3 && ph < 0.5 * target; ++it) {
                    double g2 = gph[0] * gph[0] + gph[1] * gph[1] + gph[2] * gph[2];
                    for (int a = 0; a < D; ++a) x[a] += (target - ph) * gph[a] / g2;
                    ph = domain_phi(*s.dom, x, gph);
                }
                v[0] = v[1] = v[2] = T(0);
                atomicAdd(&s.ctrl->escapes, 1ull);
            }
        } else {
            project_feature(fi, D, x);
            double t64[3], v64[3] = {(double)v[0], (double)v[1], (double)v[2]};
            feature_tangent<double>(fi, x, t64);
            tangent_map<double>(di, D, t64, v64);
            for (int a = 0; a < 3; ++a) v[a] = (T)v64[a];
        }
        hnew = (T)sizing_h(*s.siz, x);
        bool fin = true;
        for (int a = 0; a < D; ++a) fin = fin && isfinite(x[a]) && isfinite((double)v[a]);
        if (!fin) atomicOr(&s.ctrl->status, ST_NONFINITE);
    }
    for (int a = 0; a < D; ++a) {
        o.X[a][k] = x[a];
        o.V[a][k] = v[a];
        if (o.av[a]) o.av[a][k] = av[a];
    }
    o.H[k] = hnew;
    o.G[k] = mi & 255u;
    o.ID[k] = s.IDs[k];
}

template <typename T> void launch_control(const Params& p, const State<T>& s, cudaStream_t st) {
    k_control<T><<<1, 256, 0, st>>>(p, s);
}
template <typename T, int D>
void launch_integrate(const Grid& g, const Params& p, const State<T>& s, const Ctrl* use, const Out<T>& o,
                      cudaStream_t st) {
    k_integrate<T, D><<<div_up(s.n, BLOCK), BLOCK, 0, st>>>(g, p, s, use, o);
}

template void launch_control<float>(const Params&, const State<float>&, cudaStream_t);
template void launch_control<double>(const Params&, const State<double>&, cudaStream_t);
#define SPH_INST(T, D)                                                                                          \
    template void launch_integrate<T, D>(const Grid&, const Params&, const State<T>&, const Ctrl*, const Out<T>&, \
                                         cudaStream_t);
SPH_INST(float, 2)
SPH_INST(float, 3)
SPH_INST(double, 2)
SPH_INST(double, 3)

}  // namespace sph
