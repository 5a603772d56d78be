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

constexpr int CTL_THREADS = 512;   // threads of the controller's block
constexpr int CTL_GP = 8;          // groups summed per pass of the sampling reduction

__device__ inline void group_window_reset(Ctrl& c, int g) {
    c.gwcount[g] = 0;
    c.gnwin[g] = 0;
    c.wsum[g] = 0.0;
    c.A_last[g] = 0.0;
    c.A_prev[g] = 0.0;
}

// The controller run by every group on its own (group_convergence = 1; Algorithm 1 skips a
// feature whose V-bar_k has converged), one thread per group, on the block's copy of the
// controller: RAMP -> PHASE2 after ramp_len steps since the group's switch; on sampling steps
// V-bar_g enters the group's window and, with two closed windows, E_g = max(E_t,g, E_avg,g)
// below the threshold moves the group PHASE1 -> RAMP or PHASE2 -> DONE; the group's eps, f,
// nullification schedule and step size follow its phase; a DONE group does not move.  Thread
// 0 then sets the instance's phase to that of its least advanced moving group (DONE when all
// are), E_sys to the largest E_g and ramp_start to the step the last group left PHASE1.  With
// Algorithm 1's feature loop in sequence (feature_order), the pass for dimension class cls runs
// the groups of that class only, the step's errors are gathered over its passes, and the
// summary (and the step counter) closes the last pass.
template <typename T>
__device__ void control_groups(Ctrl& sc, const Params& p, const double* vs, int t, int cls, int D) {
    __shared__ int gl[MAXF], gev[MAXF];
    __shared__ double ge1[MAXF], ge2[MAXF];
    const int G = p.G;
    const bool inst_done = sc.phase == PH_DONE;
    const bool sampling = sc.n % p.sample_every == 0;
    // with the feature loop in sequence this pass serves the groups of dimension class cls only
    const bool seq = cls != 0 && p.feature_order;
    if (t < MAXF) {
        gl[t] = t < G ? sc.gphase[t] : PH_DONE;
        gev[t] = 0;
        ge1[t] = 0.0;
        ge2[t] = 0.0;
    }
    if (t < G && (!seq || p.gdim[t] == cls)) {
        const int g = t;
        int ph = inst_done ? PH_DONE : sc.gphase[g];
        if (p.gdim[g] >= 1 && ph != PH_DONE) {
            if (ph == PH_RAMP && sc.n - sc.gramp_start[g] >= p.ramp_len) {
                ph = PH2;
                group_window_reset(sc, g);
            }
            if ((ph == PH1 || ph == PH2) && sampling) {
                sc.Vbar[g] = vs[g];
                sc.wsum[g] += sc.Vbar[g];
                sc.gwcount[g] += 1;
                if (sc.gwcount[g] == p.window) {
                    sc.A_prev[g] = sc.A_last[g];
                    sc.A_last[g] = sc.wsum[g] / p.window;
                    sc.wsum[g] = 0.0;
                    sc.gwcount[g] = 0;
                    sc.gnwin[g] += 1;
                }
                if (sc.gnwin[g] >= 2) {
                    const double e1 = rel_err(sc.Vbar[g], sc.A_last[g]);
                    const double e2 = rel_err(sc.A_last[g], sc.A_prev[g]);
                    sc.gE[g] = fmax(e1, e2);
                    ge1[g] = e1;
                    ge2[g] = e2;
                    gev[g] = 1;
                    if (sc.gE[g] < p.threshold) {
                        if (ph == PH1) {
                            ph = PH_RAMP;
                            sc.gramp_start[g] = sc.n;
                            group_window_reset(sc, g);
                        } else {
                            ph = PH_DONE;
                        }
                    }
                }
            }
            gl[g] = ph;
        }
        if (p.gdim[g] >= 1) sc.gphase[g] = ph;
        double eps = 0.0, f = 0.0;
        if (p.gdim[g] < 1 || ph == PH_DONE) {
            sc.dt[g] = 0.0;
            sc.dt_f[g] = 0.0f;
            sc.reset[g] = 1;
        } else {
            eps = p.eps1;
            f = 1.0;
            bool periodic = (sc.n % p.reset_period) == 0;
            if (ph == PH_RAMP) {
                const double sr = (double)(sc.n - sc.gramp_start[g]) / (double)p.ramp_len;
                eps = p.eps1 * (1.0 - sr);
                f = 0.5 * (1.0 + cos(CUDART_PI * sr));
            } else if (ph == PH2) {
                eps = 0.0;
                periodic = true;
            }
            const double dta = (double)from_bits<T>(sc.dta_bits[g]);
            const double dtv = (double)from_bits<T>(sc.dtv_bits[g]);
            const double dv = f > 0.0 ? dtv / f : CUDART_INF;
            const double cand = fmin(dta, dv);
            const bool rs = periodic || (sc.dt_prev[g] > 0.0 && cand < p.dt_collapse * sc.dt_prev[g]);
            double dt = rs ? dta : cand;
            dt = fmin(dt, p.dt_cap);
            sc.dt_prev[g] = dt;
            sc.dt[g] = dt;
            sc.dt_f[g] = (float)dt;
            sc.reset[g] = rs ? 1 : 0;
        }
        sc.geps[g] = eps;
        sc.gf[g] = f;
        sc.geps_f[g] = (float)eps;
        sc.gf_f[g] = (float)f;
    }
    if (t < MAXF) {
        sc.dta_bits[t] = inf_bits<T>();
        sc.dtv_bits[t] = inf_bits<T>();
    }
    __syncthreads();
    if (t == 0 && !inst_done && seq) {   // the errors of the step's passes so far
        int any = 0;
        double et = 0.0, ea = 0.0;
        for (int g = 0; g < G; ++g)
            if (p.gdim[g] >= 1 && gev[g]) {
                any = 1;
                et = fmax(et, ge1[g]);
                ea = fmax(ea, ge2[g]);
            }
        if (cls == 1) {
            sc.seq_et = 0.0;
            sc.seq_ea = 0.0;
            sc.seq_ev = 0;
        }
        sc.seq_et = fmax(sc.seq_et, et);
        sc.seq_ea = fmax(sc.seq_ea, ea);
        sc.seq_ev |= any;
    }
    if (t == 0 && !inst_done && (!seq || cls == D)) {
        int lowest = PH_DONE;
        double es = 0.0, et = 0.0, ea = 0.0;
        int any = 0;
        for (int g = 0; g < G; ++g) {
            if (p.gdim[g] < 1) continue;
            lowest = min(lowest, gl[g]);
            es = fmax(es, sc.gE[g]);
            if (!seq && gev[g]) {
                any = 1;
                et = fmax(et, ge1[g]);
                ea = fmax(ea, ge2[g]);
            }
        }
        if (seq) {
            et = sc.seq_et;
            ea = sc.seq_ea;
            any = sc.seq_ev;
        }
        if (any) {
            sc.E_t = et;
            sc.E_avg = ea;
        }
        sc.E_sys = es;
        if (sc.phase == PH1 && lowest > PH1) sc.ramp_start = sc.n;
        sc.phase = lowest;
        if (lowest == PH_DONE) {
            sc.sample_now = 0;
        } else {
            sc.n += 1;
            sc.sample_now = (sc.n % p.sample_every) == 0 ? 1 : 0;
        }
    }
}

// One block of CTL_THREADS threads per instance.  The controller state is copied into shared memory at once, the
// per-block V~ sums of a sampling step are reduced in a fixed order, and the controller for
// step n runs with one thread per group (thread 0 keeps the scalar state):
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
// DONE freezes the state (dt = 0, the step counter stops).
template <typename T, int D, bool ONE>
__global__ void __launch_bounds__(CTL_THREADS) k_control(State<T> s, One one, int cls) {
    dep_launch();
    dep_wait();
    __shared__ double vs[MAXF], et[MAXF], ea[MAXF];
    __shared__ Ctrl sc;
    __shared__ Params psh;
    __shared__ int fl[4];          // 0: done, 1: sampling step, 2: window closes, 3: reset windows
    __shared__ double par[3];      // eps, f, periodic
    const int inst = blockIdx.x;
    static_assert(sizeof(Ctrl) % sizeof(int4) == 0, "the controller is copied in 16-byte vectors");
    constexpr int NWALL = (int)(sizeof(Ctrl) / sizeof(int4));
    static_assert(offsetof(Ctrl, gphase) % sizeof(int4) == 0, "the per-group tail starts on a 16-byte boundary");
    const int NW = one.p.group_conv || !ONE ? NWALL : (int)(offsetof(Ctrl, gphase) / sizeof(int4));
    int4* scw = reinterpret_cast<int4*>(&sc);
    int4* gw = reinterpret_cast<int4*>(s.ctrls + inst);
    const int t = threadIdx.x;
    for (int k = t; k < NW; k += blockDim.x) scw[k] = gw[k];
    if (!ONE) block_copy(&psh, s.params + inst);
    const Params& p = ONE ? one.p : psh;
    __syncthreads();
    // an instance stepping all its groups at once runs its controller in the last class pass
    if (cls != 0 && !p.feature_order && cls != D) return;
    const int G = p.G;
    if (sc.sample_now != 0) {
        // the chunk rows of this instance (CHUNK slots each, added up by the pressure pass),
        // CTL_GP groups at a time: every thread sums a fixed stride of chunks (many loads in
        // flight), then a fixed shuffle tree per warp and the warps in order
        constexpr int NWC = CTL_THREADS / 32;
        __shared__ double wpart[CTL_GP][NWC];
        const int b0 = __ldg(s.inst_off + inst) / CHUNK, b1 = __ldg(s.inst_off + inst + 1) / CHUNK;
        const int lane = t & 31, wid = t >> 5;
        for (int g0 = 0; g0 < G; g0 += CTL_GP) {
            double acc[CTL_GP];
#pragma unroll
            for (int q = 0; q < CTL_GP; ++q) acc[q] = 0.0;
            // four rows' loads in flight before their sums (rows added in increasing order, as
            // one at a time)
            int b = b0 + t;
            for (; b + 3 * CTL_THREADS < b1; b += 4 * CTL_THREADS) {
                double v[4][CTL_GP];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const double* row = s.partials2 + (size_t)(b + u * CTL_THREADS) * MAXF + g0;
#pragma unroll
                    for (int q = 0; q < CTL_GP; ++q) v[u][q] = g0 + q < G ? row[q] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int q = 0; q < CTL_GP; ++q)
                        if (g0 + q < G) acc[q] += v[u][q];
            }
            for (; b < b1; b += CTL_THREADS) {
                const double* row = s.partials2 + (size_t)b * MAXF + g0;
#pragma unroll
                for (int q = 0; q < CTL_GP; ++q)
                    if (g0 + q < G) acc[q] += row[q];
            }
#pragma unroll
            for (int q = 0; q < CTL_GP; ++q) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_down_sync(0xffffffffu, acc[q], o);
                if (lane == 0) wpart[q][wid] = acc[q];
            }
            __syncthreads();
            if (t < CTL_GP && g0 + t < G) {
                double v = 0.0;
                for (int w = 0; w < NWC; ++w) v += wpart[t][w];
                vs[g0 + t] = v;
            }
            __syncthreads();
        }
    }
    if (p.group_conv) {
        __syncthreads();
        control_groups<T>(sc, p, vs, t, cls, D);
        __syncthreads();
        for (int k = t; k < NW; k += blockDim.x) gw[k] = scw[k];
        return;
    }
    if (t == 0) {
        const bool done = sc.phase == PH_DONE;
        bool reset = false;
        if (!done && sc.phase == PH_RAMP && sc.n - sc.ramp_start >= p.ramp_len) {
            sc.phase = PH2;
            sc.wcount = 0;
            sc.nwin = 0;
            reset = true;
        }
        const bool smp = !done && (sc.phase == PH1 || sc.phase == PH2) && sc.n % p.sample_every == 0;
        fl[0] = done;
        fl[1] = smp;
        fl[2] = smp && sc.wcount + 1 == p.window;
        fl[3] = reset;
    }
    __syncthreads();
    if (fl[3] && t < MAXF) {
        sc.wsum[t] = 0.0;
        sc.A_last[t] = 0.0;
        sc.A_prev[t] = 0.0;
    }
    __syncthreads();
    if (fl[1] && t < G) {
        sc.Vbar[t] = p.gdim[t] > 0 ? vs[t] : 0.0;
        sc.wsum[t] += sc.Vbar[t];
        if (fl[2]) {
            sc.A_prev[t] = sc.A_last[t];
            sc.A_last[t] = sc.wsum[t] / p.window;
            sc.wsum[t] = 0.0;
        }
    }
    if (t == 0 && fl[1]) {
        sc.wcount += 1;
        if (fl[2]) {
            sc.wcount = 0;
            sc.nwin += 1;
        }
    }
    __syncthreads();
    const bool evaluate = fl[1] && sc.nwin >= 2;
    if (evaluate && t < MAXF) {
        const bool use = t < G && p.gdim[t] >= 1;
        et[t] = use ? rel_err(sc.Vbar[t], sc.A_last[t]) : 0.0;
        ea[t] = use ? rel_err(sc.A_last[t], sc.A_prev[t]) : 0.0;
    }
    __syncthreads();
    if (t == 0) {
        bool reset = false;
        if (evaluate) {
            double e1 = 0.0, e2 = 0.0;
            for (int g = 0; g < G; ++g) {
                e1 = fmax(e1, et[g]);
                e2 = fmax(e2, ea[g]);
            }
            sc.E_t = e1;
            sc.E_avg = e2;
            sc.E_sys = fmax(e1, e2);
            if (sc.E_sys < p.threshold) {
                if (sc.phase == PH1) {
                    sc.phase = PH_RAMP;
                    sc.ramp_start = sc.n;
                    sc.wcount = 0;
                    sc.nwin = 0;
                    reset = true;
                } else {
                    sc.phase = PH_DONE;
                    fl[0] = 1;
                }
            }
        }
        fl[3] = reset;
        double eps = p.eps1, f = 1.0;
        bool periodic = (sc.n % p.reset_period) == 0;
        if (sc.phase == PH_RAMP) {
            const double sr = (double)(sc.n - sc.ramp_start) / (double)p.ramp_len;
            eps = p.eps1 * (1.0 - sr);
            f = 0.5 * (1.0 + cos(CUDART_PI * sr));
        } else if (sc.phase == PH2) {
            eps = 0.0;
            periodic = true;
        }
        par[0] = eps;
        par[1] = f;
        par[2] = periodic ? 1.0 : 0.0;
    }
    __syncthreads();
    if (fl[3] && t < MAXF) {
        sc.wsum[t] = 0.0;
        sc.A_last[t] = 0.0;
        sc.A_prev[t] = 0.0;
    }
    if (t < G) {
        const double dta = (double)from_bits<T>(sc.dta_bits[t]);
        const double dtv = (double)from_bits<T>(sc.dtv_bits[t]);
        if (fl[0] || p.gdim[t] < 1) {
            sc.dt[t] = 0.0;
            sc.dt_f[t] = 0.0f;
            sc.reset[t] = 1;
        } else {
            const double f = par[1];
            const double dv = f > 0.0 ? dtv / f : CUDART_INF;
            const double cand = fmin(dta, dv);
            const bool rs = par[2] != 0.0 || (sc.dt_prev[t] > 0.0 && cand < p.dt_collapse * sc.dt_prev[t]);
            double dt = rs ? dta : cand;
            dt = fmin(dt, p.dt_cap);
            sc.dt_prev[t] = dt;
            sc.dt[t] = dt;
            sc.dt_f[t] = (float)dt;
            sc.reset[t] = rs ? 1 : 0;
        }
    }
    if (t < MAXF) {
        sc.dta_bits[t] = inf_bits<T>();
        sc.dtv_bits[t] = inf_bits<T>();
    }
    if (t == 0) {
        if (fl[0]) {
            sc.phase = PH_DONE;
            sc.eps = 0.0;
            sc.f = 0.0;
            sc.sample_now = 0;
        } else {
            sc.eps = par[0];
            sc.f = par[1];
            sc.n += 1;
            sc.sample_now = (sc.n % p.sample_every) == 0 ? 1 : 0;
        }
        sc.eps_f = (float)sc.eps;
        sc.f_f = (float)sc.f;
    }
    __syncthreads();
    for (int k = t; k < NW; k += blockDim.x) gw[k] = scw[k];
}

// h_t(x) and the level set in the working precision, from the position in that precision and
// constants stored in it (no FP64 instruction in the FP32 build): the FP32 build stores h as a
// float, and the level set only decides whether a particle is clearly inside.

template <typename T> __device__ __forceinline__ T sizing_h_t(const Sizing& s, const T x[3]) {
    if (s.kind == 0) return wp<T>(s.a, s.fa);
    T h;
    if (s.kind == 1) {
        T dmin = T(1e30);
        for (int k = 0; k < s.nref; ++k) {
            const T d0 = x[0] - wp<T>(s.rc[k][0], s.frc[k][0]), d1 = x[1] - wp<T>(s.rc[k][1], s.frc[k][1]),
                    d2 = x[2] - wp<T>(s.rc[k][2], s.frc[k][2]);
            const T dk = fabs(t_sqrt(d0 * d0 + d1 * d1 + d2 * d2) - wp<T>(s.rr[k], s.frr[k]));
            dmin = dk < dmin ? dk : dmin;
        }
        h = wp<T>(s.a, s.fa) + wp<T>(s.b, s.fb) * dmin;
    } else {
        const T d0 = x[0] - wp<T>(s.q[0], s.fq[0]), d1 = x[1] - wp<T>(s.q[1], s.fq[1]),
                d2 = x[2] - wp<T>(s.q[2], s.fq[2]);
        h = wp<T>(s.a, s.fa) + wp<T>(s.b, s.fb) * t_sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    }
    const T lo = wp<T>(s.lo, s.flo), hi = wp<T>(s.hi, s.fhi);
    h = h < lo ? lo : h;
    return h > hi ? hi : h;
}

template <typename T> __device__ __forceinline__ T domain_phi_t(const Domain& dom, const T x[3]) {
    T phi;
    if (dom.base == 0) {
        phi = T(1e30);
        for (int a = 0; a < dom.D; ++a) {
            const T dlo = x[a] - wp<T>(dom.lo[a], dom.flo[a]), dhi = wp<T>(dom.hi[a], dom.fhi[a]) - x[a];
            phi = dlo < phi ? dlo : phi;
            phi = dhi < phi ? dhi : phi;
        }
    } else {
        const T d0 = x[0] - wp<T>(dom.bc[0], dom.fbc[0]), d1 = x[1] - wp<T>(dom.bc[1], dom.fbc[1]);
        const T d2 = dom.D == 3 ? x[2] - wp<T>(dom.bc[2], dom.fbc[2]) : T(0);
        phi = wp<T>(dom.br, dom.fbr) - t_sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    }
    for (int k = 0; k < dom.nh; ++k) {
        const T d0 = x[0] - wp<T>(dom.hc[k][0], dom.fhc[k][0]), d1 = x[1] - wp<T>(dom.hc[k][1], dom.fhc[k][1]);
        const T d2 = dom.D == 3 ? x[2] - wp<T>(dom.hc[k][2], dom.fhc[k][2]) : T(0);
        const T pk = t_sqrt(d0 * d0 + d1 * d1 + d2 * d2) - wp<T>(dom.hr[k], dom.fhr[k]);
        phi = pk < phi ? pk : phi;
    }
    return phi;
}

// Viscous pass + update, one thread per sorted particle, writing the new state in sorted order:
//   v'_i = 0 (nullified) or f v_i;  v~_i = v'_i + dt (a_p,i - eps v'_i)                       (Eq. 23)
//   a_v,i = Pi_i sum_{j in g, j != i} [2 eta_i eta_j/(eta_i+eta_j)] (rho_i^-2 + rho_j^-2)
//                 W_d'(r_ij, h_ij) (v~_i - v~_j) / r_ij,  eta = rho nu, nu = visc r_c |v~|    (Eq. 7, Eq. 8)
//   v+ = v~ + dt a_v;  x+ = x + dt v+  (FP64);  curves/surfaces: x+ onto the feature in FP64,
//   v+ <- Pi(x+) v+;  volume: phi(x+) < 0 -> back to phi = 0.01 h along grad phi (FP64),
//   v+ = 0, escape counted;  h+ = h_t(x+).
// The neighbour sum runs over the same-group pairs the pressure pass handed over (its LPI
// list columns per particle, LPI/LPP of them per lane of this pass), or, where a column
// overflowed, over the walk of the pressure pass (same pairs, same predicate) with LPP lanes;
// the lead lane does the update.  As in the pressure pass, a block lies in one instance.
// Padding slots are copied through unchanged.
// MODE 0 runs both parts; MODE 1 only the viscous sum, leaving the projected a_v of each moving
// particle in o.V (the stored velocities, which nothing reads during a step once the rebuild
// has gathered them); MODE 2 (one lane per particle) only the update, taking a_v from o.V.
template <typename T, int D, int MODE> constexpr int integrate_minb() {
    if (sizeof(T) != 4) return 4;
    if (MODE == 1) return D == 2 ? SPH_VISC_MINB_2D : SPH_VISC_MINB_3D;
    if (MODE == 2) return SPH_UPDATE_MINB;
    return D == 2 ? SPH_INTEGRATE_MINB_2D : SPH_INTEGRATE_MINB_3D;
}
template <typename T, int D, bool ONE, int MODE>
__global__ void __launch_bounds__(BLOCK, (integrate_minb<T, D, MODE>()))
    k_integrate(State<T> s, One one, const Ctrl* use, Out<T> o, int cls) {
    dep_launch();
    dep_wait();
    constexpr int LPP = MODE == 2 ? 1 : ILpp<D>::v, LPI = Lpp<D>::v, NCOL = LPI / LPP;
    __shared__ int2 sbuf[BUF_CAP * BLOCK];
    __shared__ Grid gsh;
    __shared__ Params psh;
    const int inst = ONE ? 0 : __ldg(s.chunk_inst + (blockIdx.x * (BLOCK / LPP)) / CHUNK);
    const Ctrl* const cu = use + inst;
    Ctrl* const ctrl = s.ctrls + inst;
    const Domain& dom = s.doms[inst];
    if (!ONE) {
        block_copy(&gsh, s.grids + inst);
        block_copy(&psh, s.params + inst);
        __syncthreads();
    }
    const Grid& g = ONE ? one.g : gsh;
    const Params& p = ONE ? one.p : psh;
    if (MODE != 1 && o.K) reset_scan_state(s);   // this kernel produces the next scan's histogram
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) / LPP;
    const bool lead = (threadIdx.x % LPP) == 0;
    if (MODE != 1 && k < s.n && !live(s, inst, k)) {   // padding: keep the slot as it is
        if (lead) {
            const Vec4<T> vh = s.VH[k];
            const T vv[3] = {vh.x, vh.y, vh.z};
            for (int a = 0; a < D; ++a) {
                o.C[a][k] = s.Cs[a][k];
                o.O[a][k] = s.Os[a][k];
                o.V[a][k] = vv[a];
                if (o.av[a]) o.av[a][k] = T(0);
            }
            o.H[k] = vh.w;
            o.G[k] = 0u;
            o.ID[k] = s.IDs[k];
            if (o.K) {   // the next rebuild's key: the instance's dummy cell
                o.K[k] = g.base[MAXL];
                atomicAdd(o.count + g.base[MAXL], 1);
            }
        }
    }
    const bool inrange = k < s.n && live(s, inst, k);
    T offi[3] = {T(0), T(0), T(0)}, hi = T(1);
    unsigned mi = 0;
    int c[3] = {0, 0, 0};            // stored position: finest cell + offset
    T o3[3] = {T(0), T(0), T(0)};
    T v[3] = {T(0), T(0), T(0)};
    if (inrange) {
        Rec<T, D>::load(s.P, s.Ms, k, offi, hi, mi);
        const Vec4<T> vh = s.VH[k];
        const T vv[3] = {vh.x, vh.y, vh.z};
        for (int a = 0; a < D; ++a) {
            c[a] = s.Cs[a][k];
            o3[a] = s.Os[a][k];
            v[a] = vv[a];
        }
    }
    const int gi = inrange ? meta_group(mi) : -1, di = inrange ? meta_dim(mi) : 0;
    // a converged instance (or, with group_convergence, group) stays put; the instance's
    // scalars need no load that waits for the particle's group
    bool done = cu->phase == PH_DONE;
    if (p.group_conv && !done && inrange && di > 0) done = cu->gphase[gi] == PH_DONE;
    const bool moving = inrange && di > 0 && !done && in_pass(p, cls, di, D);
    T av[3] = {T(0), T(0), T(0)};
    T hnew = hi;
    T dt = T(0), f = T(1), eps = T(0);
    bool rs = true;
    T vt[3] = {T(0), T(0), T(0)};
    T tg[3] = {T(0), T(0), T(0)};
    if (moving) {
        dt = wp<T>(cu->dt[gi], cu->dt_f[gi]);
        rs = cu->reset[gi] != 0;
        f = wp<T>(cu->f, cu->f_f);
        eps = wp<T>(cu->eps, cu->eps_f);
        if (p.group_conv) {
            f = wp<T>(cu->gf[gi], cu->gf_f[gi]);
            eps = wp<T>(cu->geps[gi], cu->geps_f[gi]);
        }
        const Vec4<T> ai = s.A[k];
        const T api[3] = {ai.x, ai.y, ai.z};
        for (int a = 0; a < 3; ++a) {
            const T vp = rs ? T(0) : f * v[a];
            vt[a] = vp + dt * (api[a] - eps * vp);
        }
        if (MODE != 2 && di < D) {
            T xi[3];
            pos_t<T, D>(g, c, o3, xi);
            feature_tangent<T>(dom.f[gi], xi, tg);
        }
    }
    if (MODE != 2 && p.visc > 0.0 && !done) {
        const T kappa = wp<T>(p.kappa, p.kappa_f), hk = T(0.5) * kappa, visc = wp<T>(p.visc, p.visc_f);
        T hid, hi2d;
        hpow(hi, di > 0 ? di : 1, hid, hi2d);
        const T eta_i = visc * kappa * hi * t_sqrt(vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2]) * fast_rcp(hid);
        // the pair's kernel factor of Eq. 7, (rho_i^-2 + rho_j^-2) W'(r, h_ij) / r (the pressure
        // pass hands it over with the pair; computed here for the pairs of an overflowed list)
        auto kfac = [&](T hj, T r) {
            T hjd, hj2d;
            hpow(hj, di, hjd, hj2d);
            const T invR = fast_rcp(hk * (hi + hj));
            const T q = r * invR;
            const T t = T(1) - q;
            const T dW = wendland_alpha<T>(di, invR) * (T(-20) * q * t * t * t) * invR;
            return (hi2d + hj2d) * dW * fast_rcp(r);
        };
        // one same-group pair (its kernel factor kv, its a_p and (v, h) loaded): the viscous term
        // of Eq. 7
        auto pair = [&](const Vec4<T>& aj, const Vec4<T>& vhj, T kv) {
            const T hj = vhj.w;
            const T apj[3] = {aj.x, aj.y, aj.z};
            const T vj3[3] = {vhj.x, vhj.y, vhj.z};
            T vtj[3] = {T(0), T(0), T(0)};
            for (int a = 0; a < D; ++a) {
                const T vp = rs ? T(0) : f * vj3[a];
                vtj[a] = vp + dt * (apj[a] - eps * vp);
            }
            T hjd, hj2d;
            hpow(hj, di, hjd, hj2d);
            const T eta_j = visc * kappa * hj * t_sqrt(vtj[0] * vtj[0] + vtj[1] * vtj[1] + vtj[2] * vtj[2]) *
                            fast_rcp(hjd);
            const T es = eta_i + eta_j;
            if (!(es > T(0))) return;
            const T eb = T(2) * eta_i * eta_j / es;
            const T coef = eb * kv;
            for (int a = 0; a < D; ++a) av[a] += coef * (vt[a] - vtj[a]);
        };
        // the pairs the pressure pass found (list), or the cell walk where the list overflowed
        constexpr int VCAP = Vcap<D>::v;
        // this lane's columns of the hand-over list: pressure-pass lanes sub + t LPP, t < NCOL
        const int NL = s.n * LPI, lg0 = k * LPI + (int)(threadIdx.x % LPP);
        int vc[NCOL];
        int over = 0;
#pragma unroll
        for (int t = 0; t < NCOL; ++t) {
            vc[t] = moving ? s.vcnt[lg0 + t * LPP] : 0;
            over |= vc[t] > VCAP ? 1 : 0;
        }
        const bool ov = sub_sum<LPP>(over) != 0;   // overflow in any column of the particle
        if (moving && !ov)
#pragma unroll
            for (int t = 0; t < NCOL; ++t) {
                const int lg = lg0 + t * LPP;
                // SPH_VISC_BATCH entries at a time: their loads are all issued before the first use
                for (int e0 = 0; e0 < vc[t]; e0 += SPH_VISC_BATCH) {
                    constexpr int U = SPH_VISC_BATCH;
                    int jj[U];
                    T rr[U];
                    Vec4<T> aj[U], vhj[U];
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (e0 + u < vc[t]) {
                            jj[u] = s.vj[(size_t)(e0 + u) * NL + lg];
                            rr[u] = s.vr[(size_t)(e0 + u) * NL + lg];
                        }
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (e0 + u < vc[t]) {
                            aj[u] = s.A[jj[u]];
                            vhj[u] = s.VH[jj[u]];
                        }
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (e0 + u < vc[t]) pair(aj[u], vhj[u], rr[u]);
                }
            }
        int li = 0, ci[3] = {0, 0, 0};
        if (moving && ov) own_cell<T, D>(g, s, k, hi, li, ci);
        walk_sub<T, D, LPP, BUF_CAP>(
            g, s.cell_start, s.occ, s.n, s.P, s.Ms, sbuf + threadIdx.x, moving && ov, li, ci, offi, hi, kappa,
            [&](int j, const T*, T r2, T hj, unsigned mj) -> bool {
                return meta_group(mj) == gi && j != k && r2 < pair_rc2(hi, hj, hk) && r2 > T(0);
            },
            [&](int j, const T*, T r2, T hj, unsigned, const T*, int, int, int, int) {
                pair(s.A[j], s.VH[j], kfac(hj, r2 * fast_rsqrt(r2)));
            });
        for (int a = 0; a < D; ++a) av[a] = sub_sum<LPP>(av[a]);
        if (moving) tangent_map<T>(di, D, tg, av);
    }
    if constexpr (MODE == 1) {
        if (lead && moving)
            for (int a = 0; a < D; ++a) o.V[a][k] = av[a];
        return;
    }
    if (MODE == 2 && moving)
        for (int a = 0; a < D; ++a) av[a] = o.V[a][k];
    if (!lead) return;
    if (moving) {
        const Feat& fi = dom.f[gi];
        // x+ = x + dt v+, advanced on the offset and re-normalised into the finest cell
        const T c0 = (T)g.c0, inv_c0 = T(1) / c0;
        bool clamped = false;
        for (int a = 0; a < 3; ++a) {
            v[a] = vt[a] + dt * av[a];
            if (a >= D) continue;
            T oa = o3[a] + dt * v[a];
            const T q = t_floor(oa * inv_c0);
            if (q != T(0)) {
                c[a] += (int)q;
                oa -= q * c0;
            }
            if (c[a] < 0 || c[a] > g.dims[0][a] - 1) {
                clamped = true;
                c[a] = min(max(c[a], 0), g.dims[0][a] - 1);
            }
            o3[a] = oa;
        }
        if (clamped) atomicOr(&ctrl->status, ST_OUTSIDE_GRID);
        T xt[3];
        pos_t<T, D>(g, c, o3, xt);
        if (fi.kind == K_VOLUME) {
            // working-precision pre-check; the FP64 level set only close to or outside the boundary
            if (!(domain_phi_t<T>(dom, xt) > T(1e-3) * hi)) {
                double x[3], gph[3];
                pos64<T, D>(g, c, o3, x);
                double ph = domain_phi(dom, x, gph);
                if (ph < 0.0) {
                    const double target = 0.01 * (double)hi;
                    for (int it = 0; it < 3 && ph < 0.5 * target; ++it) {
                        double g2 = gph[0] * gph[0] + gph[1] * gph[1] + gph[2] * gph[2];
                        for (int a = 0; a < D; ++a) x[a] += (target - ph) * gph[a] / g2;
                        ph = domain_phi(dom, x, gph);
                    }
                    v[0] = v[1] = v[2] = T(0);
                    atomicAdd(&ctrl->escapes, 1ull);
                    fine_of<T, D>(g, x, c, o3);
                    pos_t<T, D>(g, c, o3, xt);
                }
            }
        } else {
            // projection onto the feature in FP64 (Algorithm 1: map r_{n+1} onto feature k)
            double x[3];
            pos64<T, D>(g, c, o3, x);
            project_feature(fi, D, x);
            double t64[3], v64[3] = {(double)v[0], (double)v[1], (double)v[2]};
            feature_tangent<double>(fi, x, t64);
            tangent_map<double>(di, D, t64, v64);
            for (int a = 0; a < 3; ++a) v[a] = (T)v64[a];
            fine_of<T, D>(g, x, c, o3);
            pos_t<T, D>(g, c, o3, xt);
        }
        hnew = sizing_h_t<T>(s.sizs[inst], xt);
        bool fin = true;
        for (int a = 0; a < D; ++a) fin = fin && isfinite(o3[a]) && isfinite(v[a]);
        if (!fin) atomicOr(&ctrl->status, ST_NONFINITE);
    }
    if (!inrange) return;
    if (di == 0) v[0] = v[1] = v[2] = T(0);
    for (int a = 0; a < D; ++a) {
        o.C[a][k] = c[a];
        o.O[a][k] = o3[a];
        o.V[a][k] = v[a];
        if (o.av[a]) o.av[a][k] = av[a];
    }
    o.H[k] = hnew;
    o.G[k] = mi & 255u;
    o.ID[k] = s.IDs[k];
    if (o.K) {   // the next rebuild's key and histogram (what the hash pass would compute)
        const int l = level_of(g, hnew);
        int cell[3] = {c[0] >> l, c[1] >> l, D == 3 ? c[2] >> l : 0};
        const int key = key_of(g, l, cell);
        o.K[k] = key;
        const unsigned peers = __match_any_sync(__activemask(), key);   // one atomic per cell in the warp
        if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(o.count + key, __popc(peers));
    }
}

template <typename T, int D> void launch_control(const State<T>& s, const One* one, cudaStream_t st, bool pdl, int cls) {
    if (one) launch_k(k_control<T, D, true>, s.NI, CTL_THREADS, st, pdl, s, *one, cls);
    else launch_k(k_control<T, D, false>, s.NI, CTL_THREADS, st, pdl, s, One(), cls);
}
template <typename T, int D>
void launch_integrate(const State<T>& s, const One* one, const Ctrl* use, const Out<T>& o, cudaStream_t st,
                      bool pdl, int cls) {
    const int nb = div_up((long long)s.n * ILpp<D>::v, BLOCK);
    if (D == 2 ? SPH_SPLIT_INTEGRATE_2D : SPH_SPLIT_INTEGRATE_3D) {   // viscous sum, then update
        const int nu = div_up((long long)s.n, BLOCK);
        if (one) {
            launch_k(k_integrate<T, D, true, 1>, nb, BLOCK, st, pdl, s, *one, use, o, cls);
            launch_k(k_integrate<T, D, true, 2>, nu, BLOCK, st, pdl, s, *one, use, o, cls);
        } else {
            launch_k(k_integrate<T, D, false, 1>, nb, BLOCK, st, pdl, s, One(), use, o, cls);
            launch_k(k_integrate<T, D, false, 2>, nu, BLOCK, st, pdl, s, One(), use, o, cls);
        }
    } else if (one) launch_k(k_integrate<T, D, true, 0>, nb, BLOCK, st, pdl, s, *one, use, o, cls);
    else launch_k(k_integrate<T, D, false, 0>, nb, BLOCK, st, pdl, s, One(), use, o, cls);
}

#define SPH_INST(T, D)                                                      \
    template void launch_control<T, D>(const State<T>&, const One*, cudaStream_t, bool, int);      \
    template void launch_integrate<T, D>(const State<T>&, const One*, const Ctrl*, const Out<T>&, cudaStream_t, bool, int);
SPH_INST(float, 2)
SPH_INST(float, 3)
SPH_INST(double, 2)
SPH_INST(double, 3)

}  // namespace sph
