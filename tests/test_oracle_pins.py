"""Pins of the oracle's relaxation step against what the paper and the mathematics fix (no GPU).

Each test is chosen so that a plausible slip in the oracle (a dropped term, a wrong sign or
exponent, a swapped index) fails it:
  * momentum conservation of the symmetric pair sums (Eq. 7 / Eq. 19, first sum),
  * zero force on a uniform lattice (constant pressure has no gradient),
  * the boundary term cancels the truncated-support force at a flat feature (Eqs. 14-19),
  * exact invariance of trajectories under P0 -> 4 P0 (Eq. 6 / Eq. 9 scaling),
  * the Phase-Two step length 0.0625 r_c of the step-limiting particle (Eq. 24 + update),
  * viscous forces conserve momentum, vanish for uniform motion and dissipate energy (Eq. 7),
  * projection lands on the feature and the tangent map is idempotent,
  * the printed particle counts of two paper cases follow from rho_t = h^-d (Eqs. 2, 10, 11).
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2003_01061_gb300 import workloads as WL

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_cases.json")))


def box_workload(x, group, feats, h, lo=(-10, -10, 0), hi=(10, 10, 0), D=2, params=None, sizing=None):
    dom = dict(D=D, base="box", lo=list(lo), hi=list(hi), ball_c=[0, 0, 0], ball_r=0.0, holes=[], features=feats)
    siz = sizing or dict(kind="const", a=h, b=0.0, lo=h, hi=h, q=[0, 0, 0], refs=[])
    return dict(domain=dom, sizing=siz, params=dict(params or WL.PAPER_PARAMS), x=np.asarray(x, float),
                group=np.asarray(group, np.int32))


def lattice(n, s, D=2, jitter=0.0, rng=None, origin=0.0):
    g = np.arange(n) * s + origin
    if D == 2:
        X, Y = np.meshgrid(g, g, indexing="ij")
        x = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], 1)
    else:
        X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
        x = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    if jitter:
        x[:, :D] += rng.uniform(-jitter * s, jitter * s, (len(x), D))
    return x


def test_paper_parameters_match_printed_values():
    p, P = GOLD["parameters"], WL.PAPER_PARAMS
    assert P["visc"] == p["visc"] and P["cfl_a"] == p["cfl_a"] and P["cfl_v"] == p["cfl_v"]
    assert P["sample_every"] == p["sample_every"] and P["window"] * P["sample_every"] == p["window_steps"]
    assert P["threshold"] == p["threshold"] and P["reset_period"] == p["reset_period"]
    assert 0.0 <= P["eps1"] <= p["eps_max"]
    # the viscous limit of Eq. 24 never binds when nu = 0.1 r_c |v|: 0.125 r_c^2 / nu >= r_c/(40|v|)
    assert p["cfl_nu"] / p["visc"] > p["cfl_v"]


@pytest.mark.parametrize("D", [2, 3])
def test_pair_force_conserves_momentum(D):
    # Isolated patch, variable h, volume particles only: the un-renormalised pair force F is
    # antisymmetric pair by pair, so sum_i F_i = 0 to rounding.
    rng = np.random.default_rng(11)
    n = 300 if D == 2 else 400
    x = np.zeros((n, 3))
    x[:, :D] = rng.uniform(0, 1.0, (n, D))
    siz = dict(kind="radial", a=0.08, b=0.1, lo=0.05, hi=0.3, q=[0.2, 0.3, 0.1], refs=[])
    w = box_workload(x, np.zeros(n), [dict(kind="volume", dim=D)], 0.1, D=D, sizing=siz,
                     lo=(-5, -5, -5), hi=(5, 5, 5))
    o = O.Oracle(w)
    r = o.interact(use_grid=False)
    scale = np.sum(np.abs(r["F"]))
    assert scale > 0
    assert np.all(np.abs(r["F"].sum(axis=0)) < 1e-12 * scale)
    assert np.all(r["dta"][0] > 0)


def test_uniform_lattice_interior_has_no_force():
    n, h = 21, 0.1
    x = lattice(n, h)
    w = box_workload(x, np.zeros(len(x)), [dict(kind="volume", dim=2)], h)
    o = O.Oracle(w)
    c = (n // 2) * n + n // 2
    r = o.interact(sub=[c], use_grid=False)
    assert np.linalg.norm(r["a_p"][0]) <= 1e-12 * r["S"][0]
    assert r["S"][0] > 0
    # Shepard coefficient of the lattice with spacing h (Eq. 18): near the continuum value 1
    assert 1.0 < r["gamma"][0] < 1.08
    assert abs(r["gamma"][0] - r["sigma"][0] * h * h) < 1e-14


def _wall_setup(h, rows=12, half_width=20, boundary=True, boundary_rho=1, correction=1):
    # volume particles at cell centres ((i h, (j+1/2) h)); boundary (curve) particles on y = 0
    xs, gs = [], []
    for j in range(rows):
        for i in range(-half_width, half_width + 1):
            xs.append((i * h, (j + 0.5) * h, 0.0))
            gs.append(0)
    for i in range(-half_width - 3, half_width + 4):
        xs.append((i * h, 0.0, 0.0))
        gs.append(1)
    feats = [dict(kind="volume", dim=2),
             dict(kind="segment", dim=1 if boundary else 2, a=[-100, 0, 0], b=[100, 0, 0], nb=[0, -1, 0])]
    p = dict(WL.PAPER_PARAMS)
    p["kappa"] = 2.0        # the figures of these pins (0.2 % / 2 % residual) are for a 2h support
    p["boundary_rho"] = boundary_rho
    p["boundary_correction"] = correction
    w = box_workload(xs, gs, feats, h, lo=(-100, 0, 0), hi=(100, 100, 0), params=p)
    o = O.Oracle(w)
    col = [j * (2 * half_width + 1) + half_width for j in range(3)]
    return o.interact(sub=col, use_grid=False)


@pytest.mark.parametrize("h", [1.0, 0.02, 7.5])
def test_boundary_term_cancels_truncated_support(h):
    # Eqs. 14-19: with the boundary sum, the corrected gradient of a constant pressure vanishes
    # at a flat feature.  Without it the first row feels the full truncated-support push.
    unc = _wall_setup(h, boundary=False)["a_p"]
    cor = _wall_setup(h, boundary=True)["a_p"]
    ref = np.linalg.norm(unc[0])
    assert ref > 0
    assert abs(unc[0][1]) > 0.9 * ref                      # the push is normal to the wall
    assert unc[0][1] < 0                                    # interior neighbours push the row outward
    assert np.linalg.norm(cor[0]) <= 2e-3 * ref
    assert np.linalg.norm(cor[1]) <= 2e-2 * ref


def test_boundary_term_as_printed_is_not_scale_free():
    # The units-consistent reading (boundary sum carries rho_b) cancels at every h; the term
    # exactly as printed only cancels when h = 1.  Both readings agree at h = 1.
    a1 = _wall_setup(1.0, boundary_rho=0)["a_p"][0]
    b1 = _wall_setup(1.0, boundary_rho=1)["a_p"][0]
    assert np.allclose(a1, b1, rtol=1e-12, atol=1e-15)
    h = 0.02
    ref = np.linalg.norm(_wall_setup(h, boundary=False)["a_p"][0])
    lit = np.linalg.norm(_wall_setup(h, boundary_rho=0)["a_p"][0])
    assert lit > 0.5 * ref


@pytest.mark.parametrize("h", [1.0, 0.02])
def test_method_without_correction_ignores_the_boundary(h):
    # Sec. 4.1's earlier method has no feature-boundary sum: with the correction off, the
    # volume rows feel exactly what they feel when the wall particles belong to no lower
    # dimension (they then take no part in the volume's sums at all), i.e. the full push of
    # the truncated support; with it on, the push cancels.
    off = _wall_setup(h, boundary=True, correction=0)
    ref = _wall_setup(h, boundary=False)
    on = _wall_setup(h, boundary=True, correction=1)
    for k in ("a_p", "sigma", "gamma"):
        assert np.array_equal(off[k], ref[k]), k
    assert np.linalg.norm(on["a_p"][0]) <= 2e-3 * np.linalg.norm(off["a_p"][0])
    # the presets of the three methods differ only in these two fields
    for name, d in WL.METHOD_PRESETS.items():
        q = WL.method_preset(WL.PAPER_PARAMS, name)
        assert {k for k in q if q[k] != WL.PAPER_PARAMS[k]} <= {"reset_period", "boundary_correction"}
    assert WL.method_preset(WL.PAPER_PARAMS, "improved") == WL.PAPER_PARAMS


def test_p0_invariance_is_exact():
    # P0 -> 4 P0 scales a by 4, dt by 1/2 and v by 2 exactly (powers of two), so positions
    # after K steps are bitwise identical when epsilon = 0.
    w = WL.square2d(h=0.05, seed=3)
    w["params"] = WL.scaled_controller(w["params"], sample_every=2, window=5, ramp_len=6, reset_period=7)
    p4 = dict(w["params"]); p4["p0"] = 4.0
    a, b = O.Oracle(w), O.Oracle(w, params=p4)
    a.step(40, use_grid=False)
    b.step(40, use_grid=False)
    assert a.iteration == b.iteration == 40
    assert np.array_equal(a.x, b.x)
    assert np.array_equal(2.0 * a.v, b.v)
    assert not np.array_equal(a.x, w["x"])


def test_phase_two_step_length():
    # Phase Two nullifies velocities every step, so v~ = dt a_p and x+ - x = dt^2 a_p; with
    # dt = 0.25 sqrt(r_c/|a|) the step-limiting particle moves exactly r_c/16 (viscosity off).
    w = WL.square2d(h=0.05, seed=4, jitter=0.25)
    p = dict(w["params"]); p["visc"] = 0.0
    o = O.Oracle(w, params=p)
    o.ctrl.phase = O.PHASE2
    r = o.interact(use_grid=False)
    vol = np.where(w["group"] == 0)[0]
    an = np.linalg.norm(r["a_p"], axis=1)
    rc = p["kappa"] * o.h
    lim = vol[np.argmin(0.25 * np.sqrt(rc[vol] / an[vol]))]
    x0 = o.x.copy()
    o.step(1, use_grid=False)
    assert o.ctrl.reset[0] == 1
    assert abs(np.linalg.norm(o.x[lim] - x0[lim]) / rc[lim] - 1.0 / 16.0) < 1e-12
    moved = np.linalg.norm(o.x[vol] - x0[vol], axis=1) / rc[vol]
    assert np.all(moved <= 1.0 / 16.0 * (1 + 1e-12))


def _viscous_only(x, v, h, D=2):
    n = len(x)
    w = box_workload(x, np.zeros(n), [dict(kind="volume", dim=D)], h, lo=(-50, -50, -50), hi=(50, 50, 50), D=D)
    o = O.Oracle(w, v=v)
    o.ctrl.dt[0] = 1e-3
    o.ctrl.reset[0] = 0
    o.ctrl.ramp_f = 1.0
    o.ctrl.eps = 0.0
    return o.integrate(np.zeros((n, 3)), use_grid=False)["a_v"]


def test_viscous_force_conserves_momentum_and_dissipates():
    rng = np.random.default_rng(5)
    n, h = 250, 0.1
    x = np.zeros((n, 3)); x[:, :2] = rng.uniform(0, 0.9, (n, 2))
    v = np.zeros((n, 3)); v[:, :2] = rng.normal(0, 1, (n, 2))
    av = _viscous_only(x, v, h)
    scale = np.sum(np.abs(av))
    assert scale > 0
    assert np.all(np.abs(av.sum(axis=0)) < 1e-12 * scale)       # momentum
    assert np.sum(v * av) < 0                                     # dissipation
    u = np.zeros((n, 3)); u[:, 0] = 0.7; u[:, 1] = -0.2
    assert np.all(_viscous_only(x, u, h) == 0)                    # uniform motion: no shear


def test_projection_onto_features():
    w = WL.cube_sphere(n_target=2000, seed=9)
    dom = O.make_domain(w["domain"])
    rng = np.random.default_rng(2)
    feats = w["domain"]["features"]
    for k, f in enumerate(feats):
        for _ in range(20):
            p = rng.uniform(-0.2, 1.2, 3)
            q = O.project(dom, k, p)
            nb, tg = O.frame(dom, k, q)
            if f["kind"] == "sphere":
                assert abs(np.linalg.norm(q - np.asarray(f["c"])) - f["r"]) < 1e-12
                assert abs(O.phi_at(dom, q + 1e-6 * nb)[0]) < 2e-6 and O.phi_at(dom, q - 1e-6 * nb)[0] > 0
            elif f["kind"] == "rect":
                assert abs(np.dot(q - np.asarray(f["o"]), np.asarray(f["nb"]))) < 1e-12
            elif f["kind"] == "segment":
                a, b = np.asarray(f["a"]), np.asarray(f["b"])
                t = np.cross(q - a, b - a)
                assert np.linalg.norm(t) < 1e-12
            elif f["kind"] == "point":
                assert np.array_equal(q, np.asarray(f["p"], float))
            if f["dim"] in (1, 2):
                vv = rng.normal(size=3)
                p1 = O.tangent(dom, k, q, vv)
                p2 = O.tangent(dom, k, q, p1)
                assert np.allclose(p1, p2, rtol=0, atol=1e-14)
                if f["dim"] == 2:
                    assert abs(np.dot(p1, nb)) < 1e-14
            if f["dim"] < 3 and f["kind"] != "point":
                assert abs(np.linalg.norm(nb) - 1) < 1e-14


def test_disk_circle_normals_point_out_of_the_domain():
    w = WL.disk_holes(n_target=3000, seed=2)
    dom = O.make_domain(w["domain"])
    for k, f in enumerate(w["domain"]["features"]):
        if f["kind"] != "circle":
            continue
        th = 0.3
        q = np.array([f["c"][0] + f["r"] * math.cos(th), f["c"][1] + f["r"] * math.sin(th), 0.0])
        nb, tg = O.frame(dom, k, q)
        assert O.phi_at(dom, q - 1e-5 * nb)[0] > 0          # inside along -n
        assert abs(np.dot(nb, tg)) < 1e-15


@pytest.mark.parametrize("case,tol", [("square", 0.15), ("cube", 0.15)])
def test_paper_particle_counts_follow_rho_t(case, tol):
    # Eqs. 2, 10, 11: unit-mass particles and rho_t = h^-d give the paper's printed totals to
    # within the packing convention (about 10 %); a wrong exponent misses by orders of magnitude.
    g = GOLD[case]
    L, D = g["extent"], 2 if case == "square" else 3
    corner = [L] * D + [0.0] * (3 - D)
    siz = dict(kind="radial", a=g["h_min"], b=(g["h_max"] - g["h_min"]) / (L * math.sqrt(D)), lo=g["h_min"],
               hi=g["h_max"], q=corner, refs=[])
    dom = dict(D=D, base="box", lo=[0, 0, 0], hi=[L, L, L if D == 3 else 0], ball_c=[0, 0, 0], ball_r=0.0,
               holes=[], features=[dict(kind="volume", dim=D)])
    m = O.feature_mass(O.make_domain(dom), O.make_sizing(siz), 0, nq=600 if D == 2 else 200)
    assert abs(m - g["n_particles"]) < tol * g["n_particles"]


def test_sphere02_stand_in_follows_the_printed_sizing():
    # Sec. 4 Sphere02: h_t = 0.025 + 0.2 | |x| - 0.5 |, h_min 0.025, h_max 0.125; on the unit
    # ball both printed ends are reached (the inner shell and the centre / surface)
    w = WL.sphere02(seed=9, mc_samples=50_000)
    rng = np.random.default_rng(4)
    P = rng.uniform(-1, 1, (20_000, 3))
    P = P[np.linalg.norm(P, axis=1) <= 1.0]
    ref = 0.025 + 0.2 * np.abs(np.linalg.norm(P, axis=1) - 0.5)
    assert np.allclose(WL.sizing_eval(w["sizing"], P), ref, rtol=0, atol=1e-15)
    ends = WL.sizing_eval(w["sizing"], np.array([[0, 0, 0], [0.5, 0, 0], [0, 0, 1.0]]))
    assert np.allclose(ends, [0.125, 0.025, 0.125], rtol=0, atol=1e-15)
    siz = O.make_sizing(w["sizing"])
    assert np.allclose([O.h_at(siz, q) for q in P[:50]], ref[:50], rtol=0, atol=1e-15)
    # every particle inside the closed ball, the surface group on it
    r = np.linalg.norm(w["x"], axis=1)
    assert np.all(r <= 1.0 + 1e-12)
    assert np.abs(r[w["group"] == 1] - 1.0).max() < 1e-12
