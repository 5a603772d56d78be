"""Multi-step GPU runs against the oracle (needs a GB300).

Trajectories of a particle relaxation drift apart from rounding differences, so after K steps
the comparison is statistical (the acceptance bounds stated for the method): the histogram of
nearest-neighbour spacing / h_t (50 bins on [0.5, 1.5]) within 1 % (L1), the minimum angle of
the Delaunay mesh within 0.5 degrees and its radius ratio (minimum and mean; 2 r_in / r_circ
in 2D, 3 r_in / r_circ in 3D) within 0.01; in 3D also the minimum dihedral angle within 0.5
degrees.  Two cases need a wider histogram bound, each set from the oracle against itself:
  * the FP32 square: the FP32 path computes each step's forces with a relative error up to the
    per-step tolerance 1e-5; the oracle whose accelerations carry a random relative error of
    1e-5 in every step drifts from the unperturbed oracle by 1.5-1.9 % L1 in 200 steps (1e-6:
    0.4-1.2 %), so the bound is 2 %;
  * the disk (6,000 particles, 150 steps): the same per-step noise makes the oracle drift from
    itself by 3.2-6.6 % L1 (1e-6: 3.9-5.5 %), about the sampling noise of a 50-bin histogram of
    6,000 values once trajectories decorrelate, so its bound is 8 %.
The minimum angle and the radius ratio move far less under the same perturbations (square:
<= 0.03 degrees and <= 0.005; disk: <= 0.24 degrees and <= 0.0004).  The FP64 build is also compared position by position
over a shorter horizon.
"""
import math

import numpy as np
import pytest
from scipy.spatial import Delaunay, cKDTree

from oracle import oracle as O
from paper_2003_01061_gb300 import build as B
from paper_2003_01061_gb300 import sphmesh as S
from paper_2003_01061_gb300 import workloads as WL

import bench

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def spacing_hist(w, x, h_of):
    groups = w["group"]
    dims = np.array([f["dim"] for f in w["domain"]["features"]])
    vals = []
    for g in np.unique(groups):
        if dims[g] < 1:
            continue
        sel = np.where(groups == g)[0]
        if len(sel) < 3:
            continue
        tr = cKDTree(x[sel])
        d, _ = tr.query(x[sel], k=2)
        vals.append(d[:, 1] / h_of[sel])
    v = np.concatenate(vals)
    hist, _ = np.histogram(v, bins=50, range=(0.5, 1.5))
    return hist / len(v)


def quality_2d(w, x):
    """(mean minimum angle, mean G, minimum angle, minimum radius ratio, mean radius ratio)."""
    q = bench.mesh_quality_2d(w, x)
    return q["theta_min_avg"], q["G_avg"], q["theta_min"], q["rr_min"], q["rr_avg"]


def run_both(w, prec, steps):
    o = O.Oracle(w)
    h0 = o.h.copy()
    if prec == 32:
        h0 = h0.astype(np.float32).astype(np.float64)
        o = O.Oracle(w, h=h0)
    m = S.Mesh(w, precision=prec)
    m.set_state(h=h0)
    m.step(steps)
    m.sync()
    got = m.positions()
    rep = m.report()
    o.step(steps, use_grid=True)
    m.close()
    return o, got, rep


@pytest.mark.parametrize("prec", [64, 32])
def test_square_200_steps_statistics(prec):
    w = WL.square2d()
    w["params"] = WL.scaled_controller(w["params"])
    o, got, rep = run_both(w, prec, 200)
    assert rep.status == 0
    assert rep.iteration == o.iteration
    hx = np.full(len(o.x), 0.02)
    hg, ho = spacing_hist(w, got["x"], hx), spacing_hist(w, o.x, hx)
    # FP64: 1 % L1; FP32: 2 %, the drift of the oracle whose forces carry the FP32 path's
    # per-step tolerance as noise (module docstring)
    assert np.abs(hg - ho).sum() <= (0.01 if prec == 64 else 0.02)
    qg, qo = quality_2d(w, got["x"]), quality_2d(w, o.x)
    assert abs(qg[2] - qo[2]) <= 0.5, (qg[2], qo[2])          # minimum angle
    assert abs(qg[3] - qo[3]) <= 0.01 and abs(qg[4] - qo[4]) <= 0.01   # radius ratio
    assert abs(qg[0] - qo[0]) <= 0.5 and abs(qg[1] - qo[1]) <= 0.01
    # a relaxed lattice is at least as regular as the jittered start
    q0 = quality_2d(w, w["x"])
    assert qg[0] >= q0[0] - 0.5


def test_fp64_trajectory_follows_oracle():
    w = WL.square2d(h=0.04, seed=5, jitter=0.2)
    w["params"] = WL.scaled_controller(w["params"], sample_every=2, window=5, ramp_len=10, reset_period=25)
    o, got, rep = run_both(w, 64, 60)
    assert rep.iteration == o.iteration and rep.phase == o.phase
    err = np.abs(got["x"] - o.x).max()
    assert err <= 1e-9 * 0.04, err
    for g in range(o.G):
        assert abs(rep.dt[g] - o.ctrl.dt[g]) <= 1e-8 * max(o.ctrl.dt[g], 1e-300)
    assert abs(rep.E_sys - o.ctrl.E_sys) <= 1e-6 * max(o.ctrl.E_sys, 1e-12) + 1e-12


@pytest.mark.parametrize("steps", [57, 120])
def test_group_convergence_fp64_follows_oracle(steps):
    # Algorithm 1's per-feature check (group_convergence = 1): on this case the edges switch
    # and converge first and stay put while the volume group is still relaxing; after 57 steps
    # some groups are DONE and others are not, after 120 the instance is DONE.  The FP64 path
    # follows the oracle group by group.
    w = WL.square2d(h=0.04, seed=5, jitter=0.2)
    w["params"] = WL.scaled_controller(w["params"], sample_every=2, window=5, ramp_len=10, reset_period=25)
    # step counts found for a 2h support: the edges are done by step 56, the volume at 80
    w["params"].update(threshold=1e-2, group_convergence=1, kappa=2.0)
    o, got, rep = run_both(w, 64, steps)
    gph = [rep.group_phase[g] for g in range(o.G)]
    assert gph[:5] == [o.ctrl.gphase[g] for g in range(5)]
    assert rep.iteration == o.iteration and rep.phase == o.phase
    if steps == 57:
        assert S.DONE in gph[:5] and gph[0] != S.DONE      # mixed: some groups frozen
    else:
        assert rep.phase == S.DONE
    err = np.abs(got["x"] - o.x).max()
    assert err <= 1e-9 * 0.04, err
    assert np.abs(got["v"] - o.v).max() <= 1e-6 * max(np.abs(o.v).max(), 1e-300)
    for g in range(5):
        assert abs(rep.group_E[g] - o.ctrl.gE[g]) <= 1e-6 * max(o.ctrl.gE[g], 1e-12) + 1e-12


def test_disk_statistics_fp32():
    w = WL.disk_holes(n_target=6000, seed=2)
    w["params"] = WL.scaled_controller(w["params"], sample_every=5, window=10, ramp_len=50)
    o, got, rep = run_both(w, 32, 150)
    assert rep.status == 0 and rep.iteration == o.iteration
    siz = w["sizing"]
    hg = spacing_hist(w, got["x"], WL.sizing_eval(siz, got["x"]))
    ho = spacing_hist(w, o.x, WL.sizing_eval(siz, o.x))
    assert np.abs(hg - ho).sum() <= 0.08, np.abs(hg - ho).sum()
    qg, qo = quality_2d(w, got["x"]), quality_2d(w, o.x)
    assert abs(qg[2] - qo[2]) <= 0.5, (qg[2], qo[2])
    assert abs(qg[3] - qo[3]) <= 0.01 and abs(qg[4] - qo[4]) <= 0.01
    assert abs(qg[0] - qo[0]) <= 0.5 and abs(qg[1] - qo[1]) <= 0.01
    # every curve particle stays on its circle (to the precision of the stored FP32 offset)
    for k, f in enumerate(w["domain"]["features"]):
        if f["kind"] == "circle":
            sel = got["group"] == k
            r = np.linalg.norm(got["x"][sel, :2] - np.asarray(f["c"][:2]), axis=1)
            assert np.abs(r - f["r"]).max() < 1e-6 * w["h_lo"]


def test_cube_sphere_statistics_fp32():
    # the 3D workload's family (cube minus a sphere: edges, faces, sphere surface, volume,
    # fixed corners) at ~8,000 particles for 100 steps; 3D trajectories drift little (the
    # oracle with per-step force noise of 1e-5 stays within 0.05 % L1 of itself), so the
    # 1 % histogram bound holds as stated
    w = WL.cube_sphere(n_target=8000, seed=3, mc_samples=200_000)
    w["params"] = WL.scaled_controller(w["params"], sample_every=5, window=10, ramp_len=50)
    o, got, rep = run_both(w, 32, 100)
    assert rep.status == 0 and rep.iteration == o.iteration
    siz = w["sizing"]
    hg = spacing_hist(w, got["x"], WL.sizing_eval(siz, got["x"]))
    ho = spacing_hist(w, o.x, WL.sizing_eval(siz, o.x))
    assert np.abs(hg - ho).sum() <= 0.01, np.abs(hg - ho).sum()
    qg, qo = bench.mesh_quality_3d(w, got["x"]), bench.mesh_quality_3d(w, o.x)
    assert abs(qg["theta_min"] - qo["theta_min"]) <= 0.5, (qg["theta_min"], qo["theta_min"])   # minimum dihedral
    assert abs(qg["theta_min_avg"] - qo["theta_min_avg"]) <= 0.5
    assert abs(qg["gamma_min"] - qo["gamma_min"]) <= 0.01 and abs(qg["gamma_avg"] - qo["gamma_avg"]) <= 0.01
    # curve and surface particles stay on their features
    for k, f in enumerate(w["domain"]["features"]):
        sel = got["group"] == k
        if f["kind"] == "sphere":
            r = np.linalg.norm(got["x"][sel] - np.asarray(f["c"]), axis=1)
            assert np.abs(r - f["r"]).max() < 1e-6 * w["h_lo"]


def test_run_until_converged_reaches_done():
    # With Eq. 24 as stated, Phase One keeps a CFL-limited oscillation and E_sys levels off
    # near 1e-2 on this small case, so the threshold is raised to a level both sides reach.
    w = WL.square2d(h=0.05, seed=3, jitter=0.1)
    w["params"] = WL.scaled_controller(w["params"], sample_every=2, window=10, ramp_len=20)
    w["params"]["threshold"] = 2e-2
    m = S.Mesh(w, precision=64)
    m.set_state()
    ok, iters = S.sph_mesh_run_until_converged(m.h, 5000)
    rep = m.report()
    o = O.Oracle(w)
    o.step(5000, use_grid=True)
    assert ok and rep.phase == S.DONE and rep.ramp_start > 0
    assert o.phase == O.DONE
    assert iters == rep.iteration
    # the switch steps agree up to a couple of sampling windows (trajectories diverge slowly)
    assert abs(iters - o.iteration) <= 2 * 10 * 2
    ok2, iters2 = S.sph_mesh_run_until_converged(m.h, 5000)
    assert ok2 and iters2 == iters                   # DONE freezes the state
    m.set_state()
    ok3, iters3 = S.sph_mesh_run_until_converged(m.h, 10)
    assert not ok3 and iters3 == 10                  # max_iters reached: not converged, state valid
    m.close()


def test_square_eq25_both_phases_fp32():
    # The Square of Sec. 4.1 (Eq. 25 sizing) through Phase One, the ramp and Phase Two to DONE,
    # with the paper's controller at the threshold this build's readings reach (1e-2; the paper's
    # 5e-6 is not reached).  The oracle whose forces carry per-step relative noise of 1e-5 (the
    # FP32 tolerance) switches at the same step and is DONE at the same step as without noise;
    # its final mean minimum angle, mean radius ratio and mean G move by <= 0.27 degrees, 0.002
    # and 0.0034, its histogram by 5-8.5 % L1, while the extreme angle and radius ratio of
    # 1,160-step trajectories move by up to 3.9 degrees and 0.08 and are not compared.
    w = WL.square_radial(seed=6)
    w["params"] = dict(w["params"], threshold=1e-2)
    o = O.Oracle(w)
    h0 = o.h.astype(np.float32).astype(np.float64)
    o = O.Oracle(w, h=h0)
    m = S.Mesh(w, precision=32)
    m.set_state(h=h0)
    ok, iters = S.sph_mesh_run_until_converged(m.h, 4000)
    rep = m.report()
    got = m.positions()
    m.close()
    o.step(4000, use_grid=True)
    assert ok and rep.phase == S.DONE and o.phase == O.DONE
    window = w["params"]["sample_every"] * w["params"]["window"]
    assert abs(rep.ramp_start - o.ctrl.ramp_start) <= window, (rep.ramp_start, o.ctrl.ramp_start)
    assert abs(iters - o.iteration) <= window, (iters, o.iteration)
    hof = lambda x: WL.sizing_eval(w["sizing"], x)
    hg, ho = spacing_hist(w, got["x"], hof(got["x"])), spacing_hist(w, o.x, hof(o.x))
    assert np.abs(hg - ho).sum() <= 0.10, np.abs(hg - ho).sum()
    qg, qo = bench.mesh_quality_2d(w, got["x"]), bench.mesh_quality_2d(w, o.x)
    assert abs(qg["theta_min_avg"] - qo["theta_min_avg"]) <= 0.5
    assert abs(qg["rr_avg"] - qo["rr_avg"]) <= 0.01 and abs(qg["G_avg"] - qo["G_avg"]) <= 0.01
    # context: the paper's table prints G_avg 0.95 for its own initial particles
    assert qg["G_avg"] > 0.85
