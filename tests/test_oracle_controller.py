"""Pins of the two-phase controller (Sec. 3.4) on hand-computed traces (no GPU)."""
import math

import numpy as np

from oracle import oracle as O
from paper_2003_01061_gb300 import workloads as WL


def make(params_over=None, G=3, gdim=(2, 1, 0)):
    w = WL.square2d(h=0.1)
    p = dict(w["params"])
    p.update(params_over or {})
    o = O.Oracle(w, params=p)
    o.G = G
    o.gdim = np.array(gdim, np.int32)
    return o, p


def drive(o, values, dta=None, dtv=None, nsteps=None):
    """Calls the controller once per step with V-bar sequence values(n) and returns a trace."""
    trace = []
    n_steps = nsteps or 10_000
    for n in range(n_steps):
        V = np.array([values(n, g) for g in range(o.G)])
        a = np.array([dta(n, g) if dta else 1.0 for g in range(o.G)])
        v = np.array([dtv(n, g) if dtv else np.inf for g in range(o.G)])
        o.control(V, a, v)
        trace.append((o.ctrl.n, o.ctrl.phase, o.ctrl.dt[0], o.ctrl.reset[0], o.ctrl.ramp_f, o.ctrl.eps))
        if o.ctrl.phase == O.DONE:
            break
        o.ctrl.n += 1
    return trace


def test_constant_volume_switches_after_two_windows():
    S, W, R = 20, 10, 200
    o, p = make(dict(sample_every=S, window=W, ramp_len=R))
    tr = drive(o, lambda n, g: 1.0 + g)
    phases = {t[0]: t[1] for t in tr}
    switch = (2 * W - 1) * S                      # second window closes at sample 2W-1
    assert phases[switch - 1] == O.PHASE1 and phases[switch] == O.RAMP
    assert phases[switch + R - 1] == O.RAMP and phases[switch + R] == O.PHASE2
    done = switch + R + (2 * W - 1) * S
    assert tr[-1][0] == done and tr[-1][1] == O.DONE


def test_decaying_volume_switch_step_by_hand():
    # V-bar_s = 1 + 0.01 * 0.5^s at sample s.  Window means of samples [10k, 10k+9].
    S, W = 5, 10
    o, p = make(dict(sample_every=S, window=W, ramp_len=50))
    seq = lambda s: 1.0 + 0.01 * 0.5 ** s
    tr = drive(o, lambda n, g: seq(n // S) if g == 0 else 2.0)
    # by hand: at sample s >= 19 the last two closed windows are k-1, k with k = (s+1)//10 - 1
    expect = None
    for s in range(19, 200):
        k = (s + 1) // 10 - 1
        A_last = np.mean([seq(10 * k + i) for i in range(10)])
        A_prev = np.mean([seq(10 * (k - 1) + i) for i in range(10)])
        E = max(abs(seq(s) - A_last) / A_last, abs(A_last - A_prev) / A_prev)
        if E < 5e-6:
            expect = s * S
            break
    first_ramp = next(t[0] for t in tr if t[1] == O.RAMP)
    assert first_ramp == expect


def test_ramp_attenuation_and_damping():
    S, W, R = 2, 2, 8
    o, p = make(dict(sample_every=S, window=W, ramp_len=R, eps1=0.2))
    tr = drive(o, lambda n, g: 1.0, nsteps=40)
    ramp = [t for t in tr if t[1] == O.RAMP]
    n0 = ramp[0][0]
    for n, ph, dt, rs, f, eps in ramp:
        s = (n - n0) / R
        assert abs(f - 0.5 * (1 + math.cos(math.pi * s))) < 1e-15
        assert abs(eps - 0.2 * (1 - s)) < 1e-15
    ph1 = [t for t in tr if t[1] == O.PHASE1]
    assert all(t[5] == 0.2 and t[4] == 1.0 for t in ph1)
    ph2 = [t for t in tr if t[1] == O.PHASE2]
    assert ph2 and all(t[5] == 0.0 and t[3] == 1 for t in ph2)


def test_reset_period_and_dt_collapse():
    o, p = make(dict(reset_period=100, sample_every=10 ** 6, window=10))
    # dta = 1, dtv shrinks 20x at step 150, then recovers
    tr = drive(o, lambda n, g: 1.0, dta=lambda n, g: 1.0,
               dtv=lambda n, g: (0.04 if n == 150 else 0.5), nsteps=260)
    resets = [t[0] for t in tr if t[3] == 1]
    assert resets == [0, 100, 150, 200]
    by_n = {t[0]: t for t in tr}
    assert by_n[150][2] == 1.0 and by_n[149][2] == 0.5 and by_n[100][2] == 1.0


def drive_groups(o, values, nsteps):
    """Per-step (n, instance phase, per-group phases, dt, f) under group_convergence = 1."""
    tr = []
    for n in range(nsteps):
        V = np.array([values(n, g) for g in range(o.G)])
        o.control(V, np.ones(o.G), np.full(o.G, np.inf))
        tr.append((o.ctrl.n, o.ctrl.phase, [o.ctrl.gphase[g] for g in range(o.G)],
                   [o.ctrl.dt[g] for g in range(o.G)], [o.ctrl.gf[g] for g in range(o.G)]))
        if o.ctrl.phase == O.DONE:
            break
        o.ctrl.n += 1
    return tr


def test_per_group_convergence_switches_each_group_on_its_own():
    # Algorithm 1 checks convergence feature by feature.  Group 0 has a constant V-bar and
    # switches after its second window; group 1's V-bar decays as 1 + 0.01*0.85^s and switches
    # when its own error first falls below the threshold (found by hand, as in the
    # single-controller test); group 2 is singular and never counts.
    S, W, R = 5, 10, 50
    o, p = make(dict(sample_every=S, window=W, ramp_len=R, group_convergence=1))
    seq = lambda s: 1.0 + 0.01 * 0.85 ** s
    tr = drive_groups(o, lambda n, g: 2.0 if g == 0 else seq(n // S), 20_000)
    by_n = {t[0]: t for t in tr}
    sw0 = (2 * W - 1) * S
    expect1 = None
    for s in range(19, 400):
        k = (s + 1) // 10 - 1
        A_last = np.mean([seq(10 * k + i) for i in range(10)])
        A_prev = np.mean([seq(10 * (k - 1) + i) for i in range(10)])
        if max(abs(seq(s) - A_last) / A_last, abs(A_last - A_prev) / A_prev) < 5e-6:
            expect1 = s * S
            break
    assert expect1 > sw0 + R + sw0          # group 0 is done before group 1 leaves Phase One
    assert by_n[sw0 - 1][2][0] == O.PHASE1 and by_n[sw0][2][0] == O.RAMP
    assert by_n[sw0 + R][2][0] == O.PHASE2
    done0 = sw0 + R + (2 * W - 1) * S
    assert by_n[done0 - 1][2][0] == O.PHASE2 and by_n[done0][2][0] == O.DONE
    assert by_n[done0][3][0] == 0.0 and by_n[done0][3][1] == 1.0      # group 0 frozen, 1 moving
    assert by_n[expect1 - 1][2][1] == O.PHASE1 and by_n[expect1][2][1] == O.RAMP
    # the instance reports its least advanced group and leaves Phase One with the last group
    assert all(t[1] == min(t[2][0], t[2][1]) for t in tr)
    assert o.ctrl.ramp_start == expect1
    # the ramp of group 1 runs on its own clock
    for n in range(expect1, expect1 + R):
        assert abs(by_n[n][4][1] - 0.5 * (1 + math.cos(math.pi * (n - expect1) / R))) < 1e-15
    assert tr[-1][1] == O.DONE and tr[-1][0] == expect1 + R + (2 * W - 1) * S


def test_per_group_convergence_with_one_group_is_the_instance_controller():
    # with a single moving group both readings are the same controller, step for step
    S, W, R = 4, 5, 30
    seq = lambda s: 1.0 + 0.05 * 0.7 ** s + 1e-4 * math.sin(s)
    traces = []
    for gc in (0, 1):
        o, p = make(dict(sample_every=S, window=W, ramp_len=R, eps1=0.1, group_convergence=gc), G=2, gdim=(2, 0))
        tr = []
        for n in range(3000):
            o.control(np.full(2, seq(n // S)), np.array([1.0 + 0.001 * n] * 2), np.array([3.0 + math.cos(n)] * 2))
            c = o.ctrl
            tr.append((c.n, c.phase, c.gphase[0], c.dt[0], c.reset[0], c.gf[0], c.geps[0], c.E_sys, c.ramp_start))
            if c.phase == O.DONE:
                break
            c.n += 1
        traces.append(tr)
    assert traces[0][-1][1] == O.DONE
    assert traces[0] == traces[1]
