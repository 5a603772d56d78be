"""Pins of the oracle's initial sampling (Sec. 3.6) and its generator (no GPU).

* the counter-based generator reproduces the published known-answer vectors of Philox4x32-10
  (tests/golden/philox_kat.json);
* every sample lies where its feature is (inside the volume away from the boundary, on the
  segment, circle, face or sphere);
* the samples follow rho_t = h_t^-d: E[h^d] over the samples equals measure / integral of h^-d
  over the same region, both computed here with numpy on a fine grid (a wrong exponent, a
  missing margin or a non-uniform direction moves it by many standard errors);
* the result is a function of (problem, seed, count): the first n of n + m samples are the n
  samples, another seed gives other samples.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2003_01061_gb300 import workloads as WL

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "philox_kat.json")))


def test_philox_known_answers():
    for v in GOLD["philox4x32_10"]:
        ctr = [int(c, 16) for c in v["counter"]]
        key = [int(c, 16) for c in v["key"]]
        assert O.philox4x32_10(ctr, key) == [int(c, 16) for c in v["out"]]


def _h(w, x):
    return WL.sizing_eval(w["sizing"], x)


def _mean_within(vals, expect, nsig=4.5):
    m, s = vals.mean(), vals.std(ddof=1) / math.sqrt(len(vals))
    assert abs(m - expect) <= nsig * s, (m, expect, s)


def test_volume_samples_follow_rho_t_2d():
    w = WL.square_radial(seed=6)
    x, _ = O.sample_feature(w, 0, seed=11, n=40_000)
    h = _h(w, x)
    assert np.all(WL.domain_phi(w["domain"], x) > 0.25 * h)
    assert np.all(x[:, 2] == 0)
    # E[h^2] under density proportional to h^-2 on {phi > h/4}: |region| / integral of h^-2
    m = 2000
    g = (np.arange(m) + 0.5) / m * 100.0
    X, Y = np.meshgrid(g, g, indexing="ij")
    P = np.stack([X.ravel(), Y.ravel(), np.zeros(m * m)], 1)
    hp = _h(w, P)
    keep = WL.domain_phi(w["domain"], P) > 0.25 * hp
    expect = keep.sum() / np.sum(hp[keep] ** -2.0)
    _mean_within(h ** 2, expect)


def test_volume_samples_follow_rho_t_3d_with_a_hole():
    w = WL.cube_sphere(n_target=20_000, seed=3, mc_samples=100_000)
    x, _ = O.sample_feature(w, 0, seed=12, n=30_000)
    h = _h(w, x)
    assert np.all(WL.domain_phi(w["domain"], x) > 0.25 * h)
    rng = np.random.default_rng(0)
    P = rng.random((3_000_000, 3))
    hp = _h(w, P)
    keep = WL.domain_phi(w["domain"], P) > 0.25 * hp
    expect = keep.sum() / np.sum(hp[keep] ** -3.0)
    _mean_within(h ** 3, expect, nsig=6)          # the reference is itself a Monte-Carlo mean


def test_curve_samples_follow_rho_t():
    w = WL.square_radial(seed=6)
    k = 2                                            # the edge x = 100 (h varies along it)
    f = w["domain"]["features"][k]
    a, b = np.array(f["a"]), np.array(f["b"])
    x, _ = O.sample_feature(w, k, seed=13, n=40_000)
    t = (x - a) @ (b - a) / np.dot(b - a, b - a)
    assert np.all((t > 0) & (t < 1))
    assert np.abs(a + t[:, None] * (b - a) - x).max() < 1e-12
    s = (np.arange(200_000) + 0.5) / 200_000
    hs = _h(w, a + s[:, None] * (b - a))
    expect = 1.0 / np.mean(1.0 / hs)                 # E[h] under density h^-1 along the edge
    _mean_within(_h(w, x), expect)


def test_circle_and_sphere_samples_are_on_the_feature_and_uniform_in_direction():
    w = WL.disk_holes(n_target=3000, seed=2, mc_samples=50_000)
    for k, f in enumerate(w["domain"]["features"]):
        if f["kind"] != "circle":
            continue
        x, _ = O.sample_feature(w, k, seed=14, n=5000)
        r = np.linalg.norm(x[:, :2] - np.array(f["c"][:2]), axis=1)
        assert np.abs(r - f["r"]).max() < 1e-12 * max(1.0, f["r"])
    # constant sizing: acceptance 1, so directions are uniform
    w3 = WL.cube_sphere(n_target=20_000, seed=3, mc_samples=100_000)
    w3 = dict(w3, sizing=dict(kind="const", a=0.05, b=0.0, lo=0.05, hi=0.05, q=[0, 0, 0], refs=[]))
    ks = next(k for k, f in enumerate(w3["domain"]["features"]) if f["kind"] == "sphere")
    f = w3["domain"]["features"][ks]
    x, used = O.sample_feature(w3, ks, seed=15, n=40_000)
    d = (x - np.array(f["c"])) / f["r"]
    assert np.abs(np.linalg.norm(d, axis=1) - 1).max() < 1e-12
    for a in range(3):
        _mean_within(d[:, a], 0.0)
        _mean_within(d[:, a] ** 2, 1.0 / 3.0)
    # the cube [-1,1]^3 keeps a fraction pi/6 of its candidates (the inscribed ball)
    frac = 40_000 / used
    assert abs(frac - math.pi / 6) < 5 * math.sqrt(frac * (1 - frac) / used)


def test_face_samples_follow_rho_t():
    w = WL.cube_sphere(n_target=20_000, seed=3, mc_samples=100_000)
    k = next(k for k, f in enumerate(w["domain"]["features"]) if f["kind"] == "rect")
    f = w["domain"]["features"][k]
    o, u, v = (np.array(f[q]) for q in ("o", "u", "w"))
    x, _ = O.sample_feature(w, k, seed=16, n=40_000)
    st = np.stack([(x - o) @ u, (x - o) @ v], 1)
    h = _h(w, x)
    assert np.all((st[:, 0] > 0.25 * h) & (st[:, 0] < f["lu"] - 0.25 * h))
    assert np.all((st[:, 1] > 0.25 * h) & (st[:, 1] < f["lw"] - 0.25 * h))
    assert np.abs(((x - o) @ np.cross(u, v))).max() < 1e-12
    m = 1500
    g = (np.arange(m) + 0.5) / m
    S, T = np.meshgrid(g * f["lu"], g * f["lw"], indexing="ij")
    P = o + S.ravel()[:, None] * u + T.ravel()[:, None] * v
    hp = _h(w, P)
    keep = (S.ravel() > 0.25 * hp) & (S.ravel() < f["lu"] - 0.25 * hp) & (T.ravel() > 0.25 * hp) & \
        (T.ravel() < f["lw"] - 0.25 * hp)
    expect = keep.sum() / np.sum(hp[keep] ** -2.0)
    _mean_within(h ** 2, expect)


def test_samples_depend_on_problem_seed_and_count_only():
    w = WL.square_radial(seed=6)
    a, ua = O.sample_feature(w, 0, seed=21, n=300)
    b, ub = O.sample_feature(w, 0, seed=21, n=500)
    c, _ = O.sample_feature(w, 0, seed=22, n=300)
    assert np.array_equal(a, b[:300]) and ua <= ub
    assert not np.array_equal(a, c)
    p, _ = O.sample_feature(w, 5, seed=21, n=1)       # a point feature gives its point
    assert np.array_equal(p[0], np.array(w["domain"]["features"][5]["p"]))
