// control.cuh -- the per-step controller of one instance (Sec. 3.4, Eq. 24), run inside the
// pressure pass by the last of the instance's blocks to finish.
#pragma once
#include "sph_internal.cuh"

namespace sph {

// shared-memory working set of the controller (it reuses the pressure pass's candidate buffer)
struct CtrlShared {
    double vs[MAXF], et[MAXF], ea[MAXF];
    Ctrl sc;
    int fl[4];          // 0: done, 1: sampling step, 2: window closes, 3: reset windows
    double par[3];      // eps, f, periodic
};
static_assert(sizeof(CtrlShared) <= sizeof(int2) * BUF_CAP * BLOCK, "the controller must fit the candidate buffer");

__device__ __forceinline__ double rel_err(double a, double b) {
    if (b != 0.0) return fabs(a - b) / fabs(b);
    return a == 0.0 ? 0.0 : CUDART_INF;
}

// Run by the last block of an instance's pressure pass (all its threads; at least MAXF of
// them).  The controller state is copied into shared memory at once, the
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
template <typename T, int D>
__device__ __noinline__ void controller_step(const State<T>& s, int inst, const Params& p, CtrlShared& sm) {
    double* const vs = sm.vs;
    double* const et = sm.et;
    double* const ea = sm.ea;
    Ctrl& sc = sm.sc;
    int* const fl = sm.fl;
    double* const par = sm.par;
    constexpr int NW = (int)(sizeof(Ctrl) / sizeof(unsigned));
    unsigned* scw = reinterpret_cast<unsigned*>(&sc);
    unsigned* gw = reinterpret_cast<unsigned*>(s.ctrls + inst);
    const int t = threadIdx.x;
    for (int k = t; k < NW; k += blockDim.x) scw[k] = gw[k];
    __syncthreads();
    const int G = p.G;
    if (sc.sample_now != 0) {
        // the pair-pass blocks of this instance (BLOCK/LPP slots each)
        constexpr int PB = BLOCK / Lpp<D>::v;
        const int b0 = __ldg(s.inst_off + inst) / PB, b1 = __ldg(s.inst_off + inst + 1) / PB;
        const int lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
        for (int g = wid; g < G; g += nw) {
            double acc = 0.0;
            for (int b = b0 + lane; b < b1; b += 32) acc += s.partials[(size_t)b * MAXF + g];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
            if (lane == 0) vs[g] = acc;
        }
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
        sc.blocks_done = 0;   // the pressure pass of the next step counts again
    }
    __syncthreads();
    for (int k = t; k < NW; k += blockDim.x) gw[k] = scw[k];
}


}  // namespace sph
