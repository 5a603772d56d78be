"""Seeded synthetic workloads: domain description, target feature size and initial particles.

This module only builds INPUTS (the geometry of an analytic signed-distance domain, the
target feature-size function h_t(x) given as an analytic formula, the paper's default
parameters, and a seeded initial particle set).  It holds none of the relaxation method's
arithmetic.  The CUDA binding and the oracle both consume the plain dictionaries it returns.

Workloads (shapes and sizes follow the 2D/3D tests of Sec. 4: a square with edges and
corners, a disk with holes, a cube with edges/corners minus a sphere):

* ``square2d``   -- [0,1]^2, constant h = 0.02, jittered lattice (uniform jitter 0.1h),
                    4 edge curves + 4 fixed corners, 2,601 particles.
* ``disk_holes`` -- unit disk minus 3 seeded circular holes (radii 0.1-0.25),
                    h = clamp(a + b d, lo, hi), d = distance to the nearest hole boundary,
                    literal range 0.004-0.04; ``scale`` shrinks h to reach a particle target.
* ``cube_sphere``-- [0,1]^3 minus a centred sphere r = 0.3, h = min(0.008+0.04|d_sphere|, 0.05),
                    12 edges, 6 faces, the sphere surface, the volume, 8 fixed corners.

Initial sampling: volume and surface particles are drawn at random with probability
proportional to the target density rho_t = h^-d (Sec. 3.6); curve particles are placed by
inverting the cumulative line density with a seeded jitter; the per-feature counts are the
integrals of rho_t over each feature (Eqs. 10/11), rounded.
"""
from __future__ import annotations

import math

import numpy as np

# Paper defaults (Sec. 2.3, Sec. 3.4): Eq. 8 coefficient, Eq. 9/24 constants, reset period
# 100, sampling every 20 steps, 10 samples per averaging window, threshold 5e-6.  The paper does
# not relate the kernel's support r_c to the target size h; r_c = 2.6 h (a Wendland C2 kernel of
# smoothing length 1.3 h, support twice that) is the reading under which the relaxed meshes reach
# the quality the paper prints for its Square (mean G 0.92 against 0.95; 0.78 with r_c = 2 h).
PAPER_PARAMS = dict(
    kappa=2.6, p0=1.0, visc=0.1, cfl_a=0.25, cfl_v=1.0 / 40.0, eps1=0.0, dt_cap=1e30,
    dt_collapse=0.1, threshold=5e-6, reset_period=100, sample_every=20, window=10,
    ramp_len=200, boundary_rho=1, max_newton=3, boundary_correction=1, group_convergence=0,
)

# The methods compared in Sec. 4.1 (Square): velocities set to zero every reset_period steps
# in Phase One, with or without the feature-boundary sum of Eq. 19.
METHOD_PRESETS = {
    "improved": dict(reset_period=100, boundary_correction=1),
    "fu2019": dict(reset_period=1, boundary_correction=0),
    "fu2019_v2": dict(reset_period=100, boundary_correction=0),
}


def method_preset(params: dict, method: str) -> dict:
    """params with the two fields that distinguish the methods of Sec. 4.1 set for `method`."""
    return dict(params, **METHOD_PRESETS[method])


# ----------------------------------------------------------------------------------------
# analytic inputs evaluated in numpy (for sampling only)
# ----------------------------------------------------------------------------------------
def sizing_eval(siz: dict, x: np.ndarray) -> np.ndarray:
    """Target feature size h_t at points x (n,3) -- the analytic input of Eq. 2."""
    if siz["kind"] == "const":
        return np.full(len(x), siz["a"])
    if siz["kind"] == "hole_dist":
        d = np.full(len(x), np.inf)
        for c, r in siz["refs"]:
            d = np.minimum(d, np.abs(np.linalg.norm(x - np.asarray(c), axis=1) - r))
        h = siz["a"] + siz["b"] * d
    else:
        h = siz["a"] + siz["b"] * np.linalg.norm(x - np.asarray(siz["q"]), axis=1)
    return np.clip(h, siz["lo"], siz["hi"])


def domain_phi(dom: dict, x: np.ndarray) -> np.ndarray:
    """Level set of the domain (positive inside, Eq. 1)."""
    D = dom["D"]
    if dom["base"] == "box":
        lo, hi = np.asarray(dom["lo"]), np.asarray(dom["hi"])
        phi = np.min(np.concatenate([x[:, :D] - lo[:D], hi[:D] - x[:, :D]], axis=1), axis=1)
    else:
        phi = dom["ball_r"] - np.linalg.norm(x - np.asarray(dom["ball_c"]), axis=1)
    for c, r in dom["holes"]:
        phi = np.minimum(phi, np.linalg.norm(x - np.asarray(c), axis=1) - r)
    return phi


# ----------------------------------------------------------------------------------------
# samplers
# ----------------------------------------------------------------------------------------
def _sample_volume(rng, dom, siz, n, hmin):
    D = dom["D"]
    lo, hi = np.asarray(dom["lo"], float), np.asarray(dom["hi"], float)
    out = []
    got = 0
    while got < n:
        m = max(4 * (n - got), 4096) * 8
        p = np.zeros((m, 3))
        p[:, :D] = lo[:D] + rng.random((m, D)) * (hi[:D] - lo[:D])
        h = sizing_eval(siz, p)
        keep = (domain_phi(dom, p) > 0.25 * h) & (rng.random(m) < (hmin / h) ** D)
        p = p[keep]
        out.append(p[: n - got])
        got += len(out[-1])
    return np.concatenate(out)[:n]


def _line_positions(rng, n, L, point_at, siz, jitter=0.1, closed=False):
    """n points along a curve of length L, spaced by inverting the cumulative 1/h density."""
    m = 4096
    s = (np.arange(m) + 0.5) / m * L
    dens = 1.0 / sizing_eval(siz, point_at(s))
    cdf = np.concatenate([[0.0], np.cumsum(dens)])
    cdf /= cdf[-1]
    sgrid = np.concatenate([[0.0], s + 0.5 * L / m])
    sgrid[-1] = L
    if closed:
        u = (np.arange(n) + rng.uniform(-jitter, jitter, n)) / n
        u = np.mod(u, 1.0)
    else:
        u = (np.arange(n) + 1 + rng.uniform(-jitter, jitter, n)) / (n + 1)
    return point_at(np.interp(u, cdf, sgrid))


def _count_curve(L, point_at, siz):
    m = 4096
    s = (np.arange(m) + 0.5) / m * L
    return float(np.sum(1.0 / sizing_eval(siz, point_at(s))) * L / m)


def _sample_rect(rng, f, siz, n, hmin):
    o, u, w = (np.asarray(f[k], float) for k in ("o", "u", "w"))
    out, got = [], 0
    while got < n:
        m = max(4 * (n - got), 4096) * 8
        st = rng.random((m, 2)) * np.array([f["lu"], f["lw"]])
        p = o + st[:, :1] * u + st[:, 1:] * w
        h = sizing_eval(siz, p)
        margin = 0.25 * h
        inside = (st[:, 0] > margin) & (st[:, 0] < f["lu"] - margin) & (st[:, 1] > margin) & (st[:, 1] < f["lw"] - margin)
        keep = inside & (rng.random(m) < (hmin / h) ** 2)
        out.append(p[keep][: n - got])
        got += len(out[-1])
    return np.concatenate(out)[:n]


def _sample_sphere(rng, f, siz, n, hmin):
    c = np.asarray(f["c"], float)
    out, got = [], 0
    while got < n:
        m = max(4 * (n - got), 4096) * 8
        g = rng.standard_normal((m, 3))
        p = c + f["r"] * g / np.linalg.norm(g, axis=1, keepdims=True)
        h = sizing_eval(siz, p)
        keep = rng.random(m) < (hmin / h) ** 2
        out.append(p[keep][: n - got])
        got += len(out[-1])
    return np.concatenate(out)[:n]


def _mc_volume_count(rng, dom, siz, m=2_000_000):
    D = dom["D"]
    lo, hi = np.asarray(dom["lo"], float), np.asarray(dom["hi"], float)
    p = np.zeros((m, 3))
    p[:, :D] = lo[:D] + rng.random((m, D)) * (hi[:D] - lo[:D])
    inside = domain_phi(dom, p) > 0
    vol = float(np.prod(hi[:D] - lo[:D]))
    return float(np.sum(sizing_eval(siz, p[inside]) ** (-D)) / m * vol)


def _finish(name, dom, siz, feats, xs, groups, params, **extra):
    x = np.concatenate(xs).astype(np.float64)
    g = np.concatenate(groups).astype(np.int32)
    dom = dict(dom)
    dom["features"] = feats
    return dict(name=name, domain=dom, sizing=siz, params=dict(params), x=x, group=g, **extra)


# ----------------------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------------------
def square2d(h: float = 0.02, seed: int = 1, jitter: float = 0.1, params: dict | None = None):
    """[0,1]^2, constant h, jittered lattice: volume (i h, j h), edges at i h, fixed corners."""
    rng = np.random.default_rng(seed)
    n = int(round(1.0 / h)) - 1
    dom = dict(D=2, base="box", lo=[0.0, 0.0, 0.0], hi=[1.0, 1.0, 0.0], ball_c=[0, 0, 0], ball_r=0.0, holes=[])
    siz = dict(kind="const", a=h, b=0.0, lo=h, hi=h, q=[0, 0, 0], refs=[])
    s2 = 1.0 / math.sqrt(2.0)
    feats = [dict(kind="volume", dim=2)]
    # edges: bottom, right, top, left (outward normals)
    edges = [((0, 0), (1, 0), (0, -1)), ((1, 0), (1, 1), (1, 0)), ((1, 1), (0, 1), (0, 1)), ((0, 1), (0, 0), (-1, 0))]
    for a, b, nb in edges:
        feats.append(dict(kind="segment", dim=1, a=[a[0], a[1], 0.0], b=[b[0], b[1], 0.0], nb=[nb[0], nb[1], 0.0]))
    corners = [((0, 0), (-s2, -s2)), ((1, 0), (s2, -s2)), ((1, 1), (s2, s2)), ((0, 1), (-s2, s2))]
    for p, nb in corners:
        feats.append(dict(kind="point", dim=0, p=[p[0], p[1], 0.0], nb=[nb[0], nb[1], 0.0]))
    ii, jj = np.meshgrid(np.arange(1, n + 1), np.arange(1, n + 1), indexing="ij")
    vol = np.zeros((n * n, 3))
    vol[:, 0] = ii.ravel() * h + rng.uniform(-jitter * h, jitter * h, n * n)
    vol[:, 1] = jj.ravel() * h + rng.uniform(-jitter * h, jitter * h, n * n)
    xs, gs = [vol], [np.zeros(n * n)]
    t = np.arange(1, n + 1) * h
    for k, (a, b, _) in enumerate(edges):
        tt = t + rng.uniform(-jitter * h, jitter * h, n)
        a_, b_ = np.array([a[0], a[1], 0.0]), np.array([b[0], b[1], 0.0])
        xs.append(a_ + tt[:, None] * (b_ - a_))
        gs.append(np.full(n, 1 + k))
    for k, (p, _) in enumerate(corners):
        xs.append(np.array([[p[0], p[1], 0.0]]))
        gs.append(np.full(1, 5 + k))
    return _finish("square2d", dom, siz, feats, xs, gs, params or PAPER_PARAMS, h_lo=h, h_hi=h)


def square_radial(seed: int = 6, params: dict | None = None, mc_samples: int = 400_000):
    """The Square of Sec. 4.1: [0,100]^2 with h_t = (h_max - h_min)/(100 sqrt 2) |x - (100,100)|
    + h_min (Eq. 25), h_min = 0.244, h_max = 4.88.  Volume particles by rejection sampling
    proportional to h_t^-2, edge particles by inverting the cumulative 1/h_t density, 4 fixed
    corners; per-feature counts from the integrals of rho_t = h_t^-d (Eqs. 10, 11).  The paper's
    own initial distribution is not given; this is a seeded stand-in with its density."""
    rng = np.random.default_rng(seed)
    L, hmin, hmax = 100.0, 0.244, 4.88
    dom = dict(D=2, base="box", lo=[0.0, 0.0, 0.0], hi=[L, L, 0.0], ball_c=[0, 0, 0], ball_r=0.0, holes=[])
    siz = dict(kind="radial", a=hmin, b=(hmax - hmin) / (L * math.sqrt(2.0)), lo=hmin, hi=hmax,
               q=[L, L, 0.0], refs=[])
    s2 = 1.0 / math.sqrt(2.0)
    feats = [dict(kind="volume", dim=2)]
    edges = [((0, 0), (L, 0), (0, -1)), ((L, 0), (L, L), (1, 0)), ((L, L), (0, L), (0, 1)), ((0, L), (0, 0), (-1, 0))]
    for a, b, nb in edges:
        feats.append(dict(kind="segment", dim=1, a=[a[0], a[1], 0.0], b=[b[0], b[1], 0.0], nb=[nb[0], nb[1], 0.0]))
    corners = [((0, 0), (-s2, -s2)), ((L, 0), (s2, -s2)), ((L, L), (s2, s2)), ((0, L), (-s2, s2))]
    for c, nb in corners:
        feats.append(dict(kind="point", dim=0, p=[c[0], c[1], 0.0], nb=[nb[0], nb[1], 0.0]))
    nv = int(round(_mc_volume_count(np.random.default_rng(seed + 100), dom, siz, mc_samples)))
    xs, gs = [_sample_volume(rng, dom, siz, nv, hmin)], [np.zeros(nv)]
    for k, (a, b, _) in enumerate(edges):
        a_, b_ = np.array([a[0], a[1], 0.0]), np.array([b[0], b[1], 0.0])
        at = lambda t, a_=a_, b_=b_: a_ + (t / L)[:, None] * (b_ - a_)
        m = int(round(_count_curve(L, at, siz)))
        xs.append(_line_positions(rng, m, L, at, siz))
        gs.append(np.full(m, 1 + k))
    for k, (c, _) in enumerate(corners):
        xs.append(np.array([[c[0], c[1], 0.0]]))
        gs.append(np.full(1, 5 + k))
    return _finish("square_radial", dom, siz, feats, xs, gs, params or PAPER_PARAMS, h_lo=hmin, h_hi=hmax)


def cube_radial(seed: int = 7, params: dict | None = None, mc_samples: int = 400_000):
    """The Cube of Sec. 4: [0,100]^3 with h_t = (h_max - h_min)/(100 sqrt 3) |x - (100,100,100)|
    + h_min (Eq. 28), h_min = 0.488, h_max = 4.88; 6 faces, 12 edges, 8 fixed corners, the volume.
    Particles by rejection sampling proportional to rho_t = h_t^-d per feature, counts from the
    integrals of rho_t (Eqs. 10, 11).  The paper's own initial distribution is not given."""
    rng = np.random.default_rng(seed)
    L, hmin, hmax = 100.0, 0.488, 4.88
    dom = dict(D=3, base="box", lo=[0.0, 0.0, 0.0], hi=[L, L, L], ball_c=[0, 0, 0], ball_r=0.0, holes=[])
    siz = dict(kind="radial", a=hmin, b=(hmax - hmin) / (L * math.sqrt(3.0)), lo=hmin, hi=hmax, q=[L, L, L], refs=[])
    s2, s3 = 1.0 / math.sqrt(2.0), 1.0 / math.sqrt(3.0)
    faces, edges, corners = [], [], []
    for ax in range(3):
        for side in (0.0, L):
            o = np.zeros(3); o[ax] = side
            u = np.zeros(3); u[(ax + 1) % 3] = 1.0
            w = np.zeros(3); w[(ax + 2) % 3] = 1.0
            nb = np.zeros(3); nb[ax] = 1.0 if side == L else -1.0
            faces.append(dict(kind="rect", dim=2, o=o.tolist(), u=u.tolist(), w=w.tolist(), lu=L, lw=L, nb=nb.tolist()))
    for ax in range(3):
        for s1 in (0.0, L):
            for s2_ in (0.0, L):
                a = np.zeros(3); b = np.zeros(3)
                a[(ax + 1) % 3] = b[(ax + 1) % 3] = s1
                a[(ax + 2) % 3] = b[(ax + 2) % 3] = s2_
                b[ax] = L
                nb = np.zeros(3)
                nb[(ax + 1) % 3] = s2 if s1 == L else -s2
                nb[(ax + 2) % 3] = s2 if s2_ == L else -s2
                edges.append(dict(kind="segment", dim=1, a=a.tolist(), b=b.tolist(), nb=nb.tolist()))
    for cx in (0.0, L):
        for cy in (0.0, L):
            for cz in (0.0, L):
                corners.append(dict(kind="point", dim=0, p=[cx, cy, cz], nb=[s3 if c == L else -s3 for c in (cx, cy, cz)]))
    nv = int(round(_mc_volume_count(np.random.default_rng(seed + 100), dom, siz, mc_samples)))
    xs, gs = [_sample_volume(rng, dom, siz, nv, hmin)], [np.zeros(nv)]
    for k, f in enumerate(faces):
        m = 256
        st = (np.arange(m) + 0.5) / m * L
        S, T = np.meshgrid(st, st, indexing="ij")
        P = np.asarray(f["o"]) + S.ravel()[:, None] * np.asarray(f["u"]) + T.ravel()[:, None] * np.asarray(f["w"])
        cnt = int(round(float(np.sum(sizing_eval(siz, P) ** -2.0)) * (L / m) ** 2))
        xs.append(_sample_rect(rng, f, siz, cnt, hmin))
        gs.append(np.full(cnt, 1 + k))
    for k, e in enumerate(edges):
        a_, b_ = np.asarray(e["a"]), np.asarray(e["b"])
        at = lambda t, a_=a_, b_=b_: a_ + (t / L)[:, None] * (b_ - a_)
        cnt = int(round(_count_curve(L, at, siz)))
        xs.append(_line_positions(rng, cnt, L, at, siz))
        gs.append(np.full(cnt, 7 + k))
    for k, c in enumerate(corners):
        xs.append(np.array([c["p"]], float))
        gs.append(np.full(1, 19 + k))
    feats = [dict(kind="volume", dim=3)] + faces + edges + corners
    return _finish("cube_radial", dom, siz, feats, xs, gs, params or PAPER_PARAMS, h_lo=hmin, h_hi=hmax)


def sphere01(seed: int = 8, params: dict | None = None, mc_samples: int = 400_000):
    """The Sphere01 case of Sec. 4: a ball of radius R = 45 with h_t = (h_max - h_min)/(2R)
    |x - x_1| + h_min, x_1 a point of the sphere (here (R, 0, 0)), h_min = 0.375, h_max = 7.5;
    the volume and the sphere surface.  Particles by rejection sampling proportional to rho_t
    per feature, counts from the integrals of rho_t (Eqs. 10, 11).  The paper's own initial
    distribution is not given."""
    R, hmin, hmax = 45.0, 0.375, 7.5
    siz = dict(kind="radial", a=hmin, b=(hmax - hmin) / (2 * R), lo=hmin, hi=hmax, q=[R, 0.0, 0.0], refs=[])
    return _ball_case("sphere01", R, siz, hmin, hmax, seed, params, mc_samples)


def sphere02(seed: int = 9, params: dict | None = None, mc_samples: int = 400_000):
    """The Sphere02 case of Sec. 4: h_t = 0.025 + 0.2 | |x| - 0.5 | (h_min = 0.025 on the inner
    shell |x| = 0.5, h_max = 0.125 at the centre and on the surface), on the unit ball: the
    paper does not print the radius, and R = 1 is the one at which both ends of its h range
    are reached.  The sizing is the distance form to a sphere of radius 0.5 (the shell is a
    refinement only, not a feature); volume and surface features as for Sphere01."""
    siz = dict(kind="hole_dist", a=0.025, b=0.2, lo=0.025, hi=0.125, q=[0, 0, 0], refs=[([0.0, 0.0, 0.0], 0.5)])
    return _ball_case("sphere02", 1.0, siz, 0.025, 0.125, seed, params, mc_samples)


def _ball_case(name, R, siz, hmin, hmax, seed, params, mc_samples):
    rng = np.random.default_rng(seed)
    dom = dict(D=3, base="ball", lo=[-R, -R, -R], hi=[R, R, R], ball_c=[0.0, 0.0, 0.0], ball_r=R, holes=[])
    sphere = dict(kind="sphere", dim=2, c=[0.0, 0.0, 0.0], r=R, orient=1.0)
    nv = int(round(_mc_volume_count(np.random.default_rng(seed + 100), dom, siz, mc_samples)))
    m = 512
    th = (np.arange(m) + 0.5) / m * math.pi
    ph = (np.arange(2 * m) + 0.5) / m * math.pi
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    P = R * np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1).reshape(-1, 3)
    ns = int(round(float(np.sum(np.sin(TH).ravel() * sizing_eval(siz, P) ** -2.0)) * R * R * (math.pi / m) ** 2))
    xs = [_sample_volume(rng, dom, siz, nv, hmin), _sample_sphere(rng, sphere, siz, ns, hmin)]
    gs = [np.zeros(nv), np.full(ns, 1)]
    return _finish(name, dom, siz, [dict(kind="volume", dim=3), sphere], xs, gs, params or PAPER_PARAMS,
                   h_lo=hmin, h_hi=hmax)


def _disk_holes_geometry(rng, n_holes=3):
    holes = []
    while len(holes) < n_holes:
        r = rng.uniform(0.1, 0.25)
        rho = math.sqrt(rng.random()) * (1.0 - 0.1 - r)
        th = rng.uniform(0, 2 * math.pi)
        c = np.array([rho * math.cos(th), rho * math.sin(th), 0.0])
        if np.linalg.norm(c[:2]) + r > 0.9:
            continue
        if all(np.linalg.norm(c - hc) > r + hr + 0.05 for hc, hr in holes):
            holes.append((c, r))
    return holes


def disk_holes(n_target: int | None = 120_000, seed: int = 2, params: dict | None = None,
               mc_samples: int = 2_000_000, sample: bool = True):
    """Unit disk minus 3 seeded holes; h linear in the distance to the nearest hole (0.004-0.04).

    ``n_target=None`` keeps the literal sizing; otherwise every length of h is scaled by one
    factor c chosen so that the integral of rho_t over all features is about n_target
    (volume part by Monte Carlo with ``mc_samples`` points).  ``sample=False`` returns the
    problem alone (no particles; for jobs whose particles are drawn on the device).
    """
    rng = np.random.default_rng(seed)
    holes = _disk_holes_geometry(rng)
    dom = dict(D=2, base="ball", lo=[-1.0, -1.0, 0.0], hi=[1.0, 1.0, 0.0], ball_c=[0.0, 0.0, 0.0], ball_r=1.0,
               holes=[(c.tolist(), float(r)) for c, r in holes])
    # d_max: the largest distance to the nearest hole boundary over the domain (grid estimate)
    g = np.linspace(-1, 1, 801)
    P = np.zeros((g.size ** 2, 3))
    P[:, 0], P[:, 1] = (a.ravel() for a in np.meshgrid(g, g, indexing="ij"))
    inside = domain_phi(dom, P) > 0
    dist = np.full(len(P), np.inf)
    for c, r in holes:
        dist = np.minimum(dist, np.abs(np.linalg.norm(P - c, axis=1) - r))
    dmax = float(dist[inside].max())
    refs = [(c.tolist(), float(r)) for c, r in holes]

    def make_siz(c):
        return dict(kind="hole_dist", a=0.004 * c, b=0.036 / dmax * c, lo=0.004 * c, hi=0.04 * c, q=[0, 0, 0], refs=refs)

    circles = [((0.0, 0.0), 1.0, +1.0)] + [((float(c[0]), float(c[1])), float(r), -1.0) for c, r in holes]

    def circ_at(cc, R):
        return lambda s: np.stack([cc[0] + R * np.cos(s / R), cc[1] + R * np.sin(s / R), np.zeros_like(s)], axis=1)

    def counts(siz):
        nv = _mc_volume_count(np.random.default_rng(seed + 100), dom, siz, mc_samples)
        nc = [_count_curve(2 * math.pi * R, circ_at(cc, R), siz) for cc, R, _ in circles]
        return nv, nc

    scale = 1.0
    if n_target is not None:
        for _ in range(4):
            nv, nc = counts(make_siz(scale))
            tot = nv + sum(nc)
            scale *= math.sqrt(tot / n_target) if tot > 0 else 1.0
    siz = make_siz(scale)
    nv, nc = counts(siz)
    feats = [dict(kind="volume", dim=2)]
    if not sample:
        feats += [dict(kind="circle", dim=1, c=[cc[0], cc[1], 0.0], r=R, orient=o) for cc, R, o in circles]
        return _finish("disk_holes", dom, siz, feats, [np.zeros((0, 3))], [np.zeros(0)], params or PAPER_PARAMS,
                       scale=scale, h_lo=siz["lo"], h_hi=siz["hi"], n_expected=int(round(nv + sum(nc))))
    xs, gs = [], []
    xs.append(_sample_volume(rng, dom, siz, int(round(nv)), siz["lo"]))
    gs.append(np.zeros(len(xs[-1])))
    for k, ((cc, R, orient), ncount) in enumerate(zip(circles, nc)):
        feats.append(dict(kind="circle", dim=1, c=[cc[0], cc[1], 0.0], r=R, orient=orient))
        m = int(round(ncount))
        xs.append(_line_positions(rng, m, 2 * math.pi * R, circ_at(cc, R), siz, closed=True))
        gs.append(np.full(m, 1 + k))
    return _finish("disk_holes", dom, siz, feats, xs, gs, params or PAPER_PARAMS, scale=scale, h_lo=siz["lo"], h_hi=siz["hi"])


def cube_sphere(n_target: int | None = 1_200_000, seed: int = 3, params: dict | None = None, sphere_r: float = 0.3,
                mc_samples: int = 2_000_000, sample: bool = True):
    """[0,1]^3 minus a centred sphere; h = min(0.008 + 0.04 |d_sphere|, 0.05), optionally scaled."""
    rng = np.random.default_rng(seed)
    cs = np.array([0.5, 0.5, 0.5])
    dom = dict(D=3, base="box", lo=[0.0, 0.0, 0.0], hi=[1.0, 1.0, 1.0], ball_c=[0, 0, 0], ball_r=0.0,
               holes=[(cs.tolist(), sphere_r)])
    refs = [(cs.tolist(), sphere_r)]

    def make_siz(c):
        return dict(kind="hole_dist", a=0.008 * c, b=0.04 * c, lo=0.008 * c, hi=0.05 * c, q=[0, 0, 0], refs=refs)

    s2, s3 = 1.0 / math.sqrt(2.0), 1.0 / math.sqrt(3.0)
    faces = []
    for ax in range(3):
        for side in (0.0, 1.0):
            o = np.zeros(3); o[ax] = side
            u = np.zeros(3); u[(ax + 1) % 3] = 1.0
            w = np.zeros(3); w[(ax + 2) % 3] = 1.0
            nb = np.zeros(3); nb[ax] = 1.0 if side == 1.0 else -1.0
            faces.append(dict(kind="rect", dim=2, o=o.tolist(), u=u.tolist(), w=w.tolist(), lu=1.0, lw=1.0, nb=nb.tolist()))
    edges = []
    for ax in range(3):
        for s1 in (0.0, 1.0):
            for s2_ in (0.0, 1.0):
                a = np.zeros(3); b = np.zeros(3)
                a[(ax + 1) % 3] = b[(ax + 1) % 3] = s1
                a[(ax + 2) % 3] = b[(ax + 2) % 3] = s2_
                b[ax] = 1.0
                nb = np.zeros(3)
                nb[(ax + 1) % 3] = s2 if s1 == 1.0 else -s2
                nb[(ax + 2) % 3] = s2 if s2_ == 1.0 else -s2
                edges.append(dict(kind="segment", dim=1, a=a.tolist(), b=b.tolist(), nb=nb.tolist()))
    corners = []
    for cx in (0.0, 1.0):
        for cy in (0.0, 1.0):
            for cz in (0.0, 1.0):
                nb = [s3 if c == 1.0 else -s3 for c in (cx, cy, cz)]
                corners.append(dict(kind="point", dim=0, p=[cx, cy, cz], nb=nb))
    sphere = dict(kind="sphere", dim=2, c=cs.tolist(), r=sphere_r, orient=-1.0)

    def seg_at(e):
        a, b = np.asarray(e["a"]), np.asarray(e["b"])
        return lambda s: a + s[:, None] * (b - a)

    def face_count(f, siz, m=256):
        st = (np.arange(m) + 0.5) / m
        S, T = np.meshgrid(st, st, indexing="ij")
        p = np.asarray(f["o"]) + S.ravel()[:, None] * np.asarray(f["u"]) + T.ravel()[:, None] * np.asarray(f["w"])
        return float(np.sum(sizing_eval(siz, p) ** -2.0) / m / m)

    def counts(siz):
        nv = _mc_volume_count(np.random.default_rng(seed + 100), dom, siz, mc_samples)
        nf = [face_count(f, siz) for f in faces]
        ns = 4 * math.pi * sphere_r ** 2 / siz["lo"] ** 2 if siz["hi"] > 0 else 0
        ne = [_count_curve(1.0, seg_at(e), siz) for e in edges]
        return nv, nf, ns, ne

    scale = 1.0
    if n_target is not None:
        for _ in range(4):
            nv, nf, ns, ne = counts(make_siz(scale))
            tot = nv + sum(nf) + ns + sum(ne)
            scale *= (tot / n_target) ** (1.0 / 3.0)
    siz = make_siz(scale)
    nv, nf, ns, ne = counts(siz)
    feats = [dict(kind="volume", dim=3)] + faces + [sphere] + edges + corners
    if not sample:   # the problem alone (particles drawn on the device)
        return _finish("cube_sphere", dom, siz, feats, [np.zeros((0, 3))], [np.zeros(0)], params or PAPER_PARAMS,
                       scale=scale, h_lo=siz["lo"], h_hi=siz["hi"],
                       n_expected=int(round(nv + sum(nf) + ns + sum(ne) + len(corners))))
    xs = [_sample_volume(rng, dom, siz, int(round(nv)), siz["lo"])]
    gs = [np.zeros(len(xs[0]))]
    for k, f in enumerate(faces):
        m = int(round(nf[k]))
        xs.append(_sample_rect(rng, f, siz, m, siz["lo"]))
        gs.append(np.full(m, 1 + k))
    m = int(round(ns))
    xs.append(_sample_sphere(rng, sphere, siz, m, siz["lo"]))
    gs.append(np.full(m, 7))
    for k, e in enumerate(edges):
        m = int(round(ne[k]))
        xs.append(_line_positions(rng, m, 1.0, seg_at(e), siz))
        gs.append(np.full(m, 8 + k))
    for k, c in enumerate(corners):
        xs.append(np.array([c["p"]], float))
        gs.append(np.full(1, 20 + k))
    return _finish("cube_sphere", dom, siz, feats, xs, gs, params or PAPER_PARAMS, scale=scale, h_lo=siz["lo"], h_hi=siz["hi"])


def scaled_controller(params: dict, sample_every=2, window=10, ramp_len=20, reset_period=100) -> dict:
    """Controller cadence shrunk so that a 200-iteration run can pass through both phases."""
    p = dict(params)
    p.update(sample_every=sample_every, window=window, ramp_len=ramp_len, reset_period=reset_period)
    return p


def subset(w: dict, keep: np.ndarray) -> dict:
    """A workload restricted to the particles selected by the boolean mask / index array keep."""
    out = dict(w)
    out["x"] = w["x"][keep].copy()
    out["group"] = w["group"][keep].copy()
    return out


def _log_uniform(rng, lo, hi):
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


def batch_mix(n_inst: int = 64, seed: int = 4, n_lo: int = 1_000, n_hi: int = 200_000, mc_samples: int = 100_000):
    """Independent instances for a batch: half 2D disks with holes (seeded hole layouts), half
    3D cubes minus a sphere (seeded radius 0.2-0.35), particle counts log-uniform over
    [n_lo, n_hi].  Returns (2D workloads, 3D workloads)."""
    rng = np.random.default_rng(seed)
    w2, w3 = [], []
    for k in range(n_inst):
        n = _log_uniform(rng, n_lo, n_hi)
        s = int(rng.integers(1 << 30))
        if k % 2 == 0:
            w2.append(disk_holes(n_target=n, seed=s, mc_samples=mc_samples))
        else:
            w3.append(cube_sphere(n_target=n, seed=s, sphere_r=float(rng.uniform(0.2, 0.35)), mc_samples=mc_samples))
    return w2, w3


def request_stream(n_jobs: int = 48, rate: float = 50.0, seed: int = 5, n_lo: int = 1_000, n_hi: int = 200_000,
                   frac_3d: float = 0.5, mc_samples: int = 100_000):
    """A Poisson stream of meshing jobs: arrival times (seconds, exponential gaps of mean
    1/rate), each job a 2D disk with holes or a 3D cube minus a sphere (probability frac_3d)
    with a log-uniform particle count over [n_lo, n_hi].  Returns a list of (t_arrival, w)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    for _ in range(n_jobs):
        t += float(rng.exponential(1.0 / rate))
        n = _log_uniform(rng, n_lo, n_hi)
        s = int(rng.integers(1 << 30))
        if rng.random() < frac_3d:
            w = cube_sphere(n_target=n, seed=s, sphere_r=float(rng.uniform(0.2, 0.35)), mc_samples=mc_samples)
        else:
            w = disk_holes(n_target=n, seed=s, mc_samples=mc_samples)
        out.append((t, w))
    return out
