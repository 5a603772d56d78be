"""ctypes front-end of the FP64 CPU oracle (sph_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the benchmark's
CPU-baseline leg.  It never imports the CUDA package, and the CUDA package never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sph_oracle.c")
LIB = os.path.join(HERE, "_build", "libsph_oracle.so")

MAX_FEAT, MAX_HOLES, MAX_LEVELS = 64, 8, 8
KIND = {"volume": 0, "point": 1, "segment": 2, "circle": 3, "rect": 4, "sphere": 5}
SIZING = {"const": 0, "hole_dist": 1, "radial": 2}
PHASE1, RAMP, PHASE2, DONE = 1, 2, 3, 4


class Feature(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dim", C.c_int32), ("p", C.c_double * 12), ("nb", C.c_double * 3),
                ("orient", C.c_double)]


class Domain(C.Structure):
    _fields_ = [("D", C.c_int32), ("base", C.c_int32), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("bc", C.c_double * 3), ("br", C.c_double), ("n_holes", C.c_int32),
                ("hc", (C.c_double * 3) * MAX_HOLES), ("hr", C.c_double * MAX_HOLES), ("n_feat", C.c_int32),
                ("feat", Feature * MAX_FEAT)]


class Sizing(C.Structure):
    _fields_ = [("kind", C.c_int32), ("a", C.c_double), ("b", C.c_double), ("lo", C.c_double), ("hi", C.c_double),
                ("q", C.c_double * 3), ("n_ref", C.c_int32), ("rc", (C.c_double * 3) * MAX_HOLES),
                ("rr", C.c_double * MAX_HOLES)]


class Params(C.Structure):
    _fields_ = [("kappa", C.c_double), ("p0", C.c_double), ("visc", C.c_double), ("cfl_a", C.c_double),
                ("cfl_v", C.c_double), ("eps1", C.c_double), ("dt_cap", C.c_double), ("dt_collapse", C.c_double),
                ("threshold", C.c_double), ("reset_period", C.c_int32), ("sample_every", C.c_int32),
                ("window", C.c_int32), ("ramp_len", C.c_int32), ("boundary_rho", C.c_int32),
                ("max_newton", C.c_int32), ("boundary_correction", C.c_int32), ("group_convergence", C.c_int32),
                ("feature_order", C.c_int32)]


class Ctrl(C.Structure):
    _fields_ = [("phase", C.c_int32), ("wcount", C.c_int32), ("nwin", C.c_int32), ("pad", C.c_int32),
                ("n", C.c_int64), ("ramp_start", C.c_int64), ("escapes", C.c_int64),
                ("wsum", C.c_double * MAX_FEAT), ("A_last", C.c_double * MAX_FEAT), ("A_prev", C.c_double * MAX_FEAT),
                ("Vbar", C.c_double * MAX_FEAT), ("dt_prev", C.c_double * MAX_FEAT), ("dt", C.c_double * MAX_FEAT),
                ("reset", C.c_int32 * MAX_FEAT), ("E_t", C.c_double), ("E_avg", C.c_double), ("E_sys", C.c_double),
                ("eps", C.c_double), ("ramp_f", C.c_double),
                ("gphase", C.c_int32 * MAX_FEAT), ("gwcount", C.c_int32 * MAX_FEAT), ("gnwin", C.c_int32 * MAX_FEAT),
                ("gramp_start", C.c_int64 * MAX_FEAT), ("gE", C.c_double * MAX_FEAT), ("geps", C.c_double * MAX_FEAT),
                ("gf", C.c_double * MAX_FEAT)]


class Grid(C.Structure):
    _fields_ = [("D", C.c_int32), ("L", C.c_int32), ("cps", C.c_int32), ("c0", C.c_float), ("origin", C.c_float * 3),
                ("thr", C.c_float * MAX_LEVELS), ("dims", (C.c_int64 * 3) * MAX_LEVELS),
                ("base", C.c_int64 * MAX_LEVELS), ("ncell", C.c_int64)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP across particles)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "sph_oracle.h"))):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        d, i32, i64, vp = C.c_double, C.c_int32, C.c_int64, C.c_void_p
        L.orc_W.restype = d; L.orc_W.argtypes = [C.c_int, d, d, d]
        L.orc_dW.restype = d; L.orc_dW.argtypes = [C.c_int, d, d, d]
        L.orc_h.restype = d; L.orc_h.argtypes = [vp, vp]
        L.orc_phi.restype = d; L.orc_phi.argtypes = [vp, vp, vp]
        L.orc_project.argtypes = [vp, C.c_int, vp]
        L.orc_frame.argtypes = [vp, C.c_int, vp, vp, vp]
        L.orc_tangent.argtypes = [vp, C.c_int, vp, vp]
        L.orc_feature_measure_density.restype = d
        L.orc_feature_measure_density.argtypes = [vp, vp, C.c_int, C.c_int]
        L.orc_neighbors_brute.restype = i64
        L.orc_neighbors_brute.argtypes = [i64, C.c_int, vp, vp, d, i64, vp, i64]
        L.orc_grid_spec.argtypes = [C.c_int, vp, vp, d, d, d, C.c_int, vp]
        L.orc_grid_repr.argtypes = [vp, i64, vp, vp, i32, vp, vp, vp, vp, vp]
        L.orc_neighbors_repr.restype = i64
        L.orc_neighbors_repr.argtypes = [vp, i64, vp, vp, i32, d, i32, i64, vp, i64]
        L.orc_counting_sort.argtypes = [i64, vp, i64, vp, vp]
        L.orc_interact.argtypes = [i64, vp, vp, vp, vp, vp, vp, i64, vp, i32, vp, vp, vp, vp, vp, vp, vp]
        L.orc_control.argtypes = [vp, C.c_int, vp, vp, vp, vp, vp]
        L.orc_integrate.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, i64, vp, i32, vp, vp, vp, vp, vp]
        L.orc_ctrl_init.argtypes = [vp]
        L.orc_step.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, vp, i32, i32]
        L.orc_philox4x32_10.argtypes = [vp, vp, vp]
        L.orc_sample_feature.restype = i64
        L.orc_sample_feature.argtypes = [vp, vp, C.c_int, C.c_uint64, i64, vp]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data if a is not None else None


def _ref(s):
    return C.addressof(s)


# ----------------------------------------------------------------------------------------
# descriptors
# ----------------------------------------------------------------------------------------
def make_domain(dom: dict) -> Domain:
    d = Domain()
    d.D = dom["D"]
    d.base = 0 if dom["base"] == "box" else 1
    for a in range(3):
        d.lo[a], d.hi[a] = dom["lo"][a], dom["hi"][a]
        d.bc[a] = dom.get("ball_c", [0, 0, 0])[a]
    d.br = dom.get("ball_r", 0.0)
    d.n_holes = len(dom["holes"])
    for k, (c, r) in enumerate(dom["holes"]):
        for a in range(3):
            d.hc[k][a] = c[a]
        d.hr[k] = r
    feats = dom["features"]
    d.n_feat = len(feats)
    for k, f in enumerate(feats):
        F = d.feat[k]
        F.kind, F.dim = KIND[f["kind"]], f["dim"]
        p = [0.0] * 12
        if f["kind"] == "point":
            p[0:3] = f["p"]
        elif f["kind"] == "segment":
            p[0:3], p[3:6] = f["a"], f["b"]
        elif f["kind"] == "circle":
            p[0], p[1], p[2] = f["c"][0], f["c"][1], f["r"]
        elif f["kind"] == "sphere":
            p[0:3], p[3] = f["c"], f["r"]
        elif f["kind"] == "rect":
            p[0:3], p[3:6], p[6:9], p[9], p[10] = f["o"], f["u"], f["w"], f["lu"], f["lw"]
        for a in range(12):
            F.p[a] = p[a]
        for a in range(3):
            F.nb[a] = f.get("nb", [0, 0, 0])[a]
        F.orient = f.get("orient", 0.0)
    return d


def make_sizing(s: dict) -> Sizing:
    z = Sizing()
    z.kind = SIZING[s["kind"]]
    z.a, z.b, z.lo, z.hi = s["a"], s["b"], s["lo"], s["hi"]
    for a in range(3):
        z.q[a] = s.get("q", [0, 0, 0])[a]
    refs = s.get("refs", [])
    z.n_ref = len(refs)
    for k, (c, r) in enumerate(refs):
        for a in range(3):
            z.rc[k][a] = c[a]
        z.rr[k] = r
    return z


# fields that parameter dictionaries may leave out (their value when absent)
PARAM_DEFAULTS = {"feature_order": 0}


def make_params(p: dict) -> Params:
    q = Params()
    for name, _ in Params._fields_:
        setattr(q, name, p[name] if name in p else PARAM_DEFAULTS[name])
    return q


# ----------------------------------------------------------------------------------------
# thin wrappers
# ----------------------------------------------------------------------------------------
def W(d, r, h, kappa=2.0):
    return lib().orc_W(d, r, h, kappa)


def dW(d, r, h, kappa=2.0):
    return lib().orc_dW(d, r, h, kappa)


def h_at(siz: Sizing, x) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().orc_h(_ref(siz), _p(x))


def phi_at(dom: Domain, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    g = np.zeros(3)
    v = lib().orc_phi(_ref(dom), _p(x), _p(g))
    return v, g


def project(dom: Domain, k: int, x):
    x = np.array(x, dtype=np.float64)
    lib().orc_project(_ref(dom), k, _p(x))
    return x


def frame(dom: Domain, k: int, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    nb, tg = np.zeros(3), np.zeros(3)
    lib().orc_frame(_ref(dom), k, _p(x), _p(nb), _p(tg))
    return nb, tg


def tangent(dom: Domain, k: int, x, v):
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    lib().orc_tangent(_ref(dom), k, _p(x), _p(v))
    return v


def feature_mass(dom: Domain, siz: Sizing, k: int, nq: int = 400) -> float:
    return lib().orc_feature_measure_density(_ref(dom), _ref(siz), k, nq)


def philox4x32_10(ctr, key):
    """Philox4x32-10 of the 4-word counter under the 2-word key (Sec. 3.6 sampling)."""
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(C.addressof(c), C.addressof(k), C.addressof(o))
    return [int(v) for v in o]


def sample_feature(w: dict, k: int, seed: int, n: int):
    """The first n accepted candidates of feature k (Sec. 3.6); returns (positions, candidates)."""
    dom, siz = make_domain(w["domain"]), make_sizing(w["sizing"])
    out = np.zeros((max(n, 1), 3))
    used = lib().orc_sample_feature(_ref(dom), _ref(siz), k, seed, n, _p(out))
    return out[:n], int(used)


def sample(w: dict, seed: int, counts):
    """All features' samples in feature order (positions, groups)."""
    xs, gs = [], []
    for k, n in enumerate(counts):
        x, _ = sample_feature(w, k, seed, int(n))
        xs.append(x)
        gs.append(np.full(int(n), k, np.int32))
    return np.concatenate(xs), np.concatenate(gs)


def neighbors_brute(x, h, i, D, kappa=2.0):
    x = np.ascontiguousarray(x, dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    out = np.zeros(len(x), np.int32)
    c = lib().orc_neighbors_brute(len(x), D, _p(x), _p(h), kappa, i, _p(out), len(out))
    return out[:c].copy()


def grid_spec(D, lo, hi, h_lo, h_hi, kappa=2.0, cells_per_support=1) -> Grid:
    g = Grid()
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    lib().orc_grid_spec(D, _p(lo), _p(hi), h_lo, h_hi, kappa, int(cells_per_support), _ref(g))
    return g


def grid_repr(g: Grid, x, h, prec=32):
    x = np.ascontiguousarray(x, dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    n = len(x)
    level = np.zeros(n, np.int32)
    cell = np.zeros((n, 3), np.int64)
    off = np.zeros((n, 3), np.float64)
    key = np.zeros(n, np.int64)
    clamped = np.zeros(n, np.int32)
    lib().orc_grid_repr(_ref(g), n, _p(x), _p(h), prec, _p(level), _p(cell), _p(off), _p(key), _p(clamped))
    return dict(level=level, cell=cell, off=off, key=key, clamped=clamped)


def neighbors_repr(g: Grid, x, h, i, prec=32, kappa=2.0, self_radius=False):
    x = np.ascontiguousarray(x, dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    out = np.zeros(len(x), np.int32)
    c = lib().orc_neighbors_repr(_ref(g), len(x), _p(x), _p(h), prec, kappa, int(self_radius), i, _p(out), len(out))
    return out[:c].copy()


def counting_sort(key, ncell):
    key = np.ascontiguousarray(key, dtype=np.int64)
    cs = np.zeros(ncell + 1, np.int64)
    perm = np.zeros(len(key), np.int64)
    lib().orc_counting_sort(len(key), _p(key), ncell, _p(cs), _p(perm))
    return cs, perm


class Oracle:
    """One relaxation instance held in FP64 on the host."""

    def __init__(self, w: dict, x=None, v=None, h=None, params: dict | None = None):
        self.w = w
        self.dom = make_domain(w["domain"])
        self.siz = make_sizing(w["sizing"])
        self.params_dict = dict(params or w["params"])
        self.prm = make_params(self.params_dict)
        self.x = np.ascontiguousarray(w["x"] if x is None else x, dtype=np.float64).copy()
        self.n = len(self.x)
        self.grp = np.ascontiguousarray(w["group"], dtype=np.int32).copy()
        self.v = np.zeros((self.n, 3)) if v is None else np.ascontiguousarray(v, dtype=np.float64).copy()
        if h is None:
            h = np.array([h_at(self.siz, self.x[i]) for i in range(self.n)])
        self.h = np.ascontiguousarray(h, dtype=np.float64).copy()
        self.ctrl = Ctrl()
        lib().orc_ctrl_init(_ref(self.ctrl))
        self.G = self.dom.n_feat
        self.gdim = np.array([self.dom.feat[k].dim for k in range(self.G)], np.int32)

    # one pressure pass (Algorithm 1: gamma, F_p, map, dt) over all or a subset of particles
    def interact(self, sub=None, use_grid=True):
        L = lib()
        m = self.n if sub is None else len(sub)
        sub_a = None if sub is None else np.ascontiguousarray(sub, dtype=np.int64)
        out = dict(sigma=np.zeros(m), gamma=np.zeros(m), F=np.zeros((m, 3)), a_p=np.zeros((m, 3)), S=np.zeros(m),
                   dta=np.zeros(self.G), dtv=np.zeros(self.G))
        L.orc_interact(self.n, _ref(self.dom), _ref(self.prm), _p(self.x), _p(self.h), _p(self.grp), _p(self.v),
                       m, _p(sub_a), int(use_grid), _p(out["sigma"]), _p(out["gamma"]), _p(out["F"]),
                       _p(out["a_p"]), _p(out["S"]), _p(out["dta"]), _p(out["dtv"]))
        return out

    def set_step_params(self, dt, reset, eps, f):
        """The per-group step parameters the controller would hand to the update (Eq. 23)."""
        for g in range(self.G):
            self.ctrl.dt[g] = dt[g]
            self.ctrl.reset[g] = int(reset[g])
            self.ctrl.geps[g] = eps
            self.ctrl.gf[g] = f
        self.ctrl.eps, self.ctrl.ramp_f = eps, f

    def control(self, Vsum, dta, dtv):
        Vsum = np.ascontiguousarray(Vsum, dtype=np.float64)
        lib().orc_control(_ref(self.prm), self.G, _p(self.gdim), _p(Vsum), _p(np.ascontiguousarray(dta)),
                          _p(np.ascontiguousarray(dtv)), _ref(self.ctrl))

    def integrate(self, a_p, sub=None, use_grid=True):
        m = self.n if sub is None else len(sub)
        sub_a = None if sub is None else np.ascontiguousarray(sub, dtype=np.int64)
        a_p = np.ascontiguousarray(a_p, dtype=np.float64)
        out = dict(x=np.zeros((m, 3)), v=np.zeros((m, 3)), h=np.zeros(m), a_v=np.zeros((m, 3)))
        esc = C.c_int64(0)
        lib().orc_integrate(self.n, _ref(self.dom), _ref(self.siz), _ref(self.prm), _ref(self.ctrl), _p(self.x),
                            _p(self.h), _p(self.grp), _p(self.v), _p(a_p), m, _p(sub_a), int(use_grid),
                            _p(out["x"]), _p(out["v"]), _p(out["h"]), _p(out["a_v"]), C.addressof(esc))
        out["escapes"] = esc.value
        return out

    def step(self, n_steps=1, use_grid=True):
        lib().orc_step(self.n, _ref(self.dom), _ref(self.siz), _ref(self.prm), _ref(self.ctrl), _p(self.x),
                       _p(self.v), _p(self.h), _p(self.grp), int(use_grid), n_steps)

    @property
    def phase(self):
        return self.ctrl.phase

    @property
    def iteration(self):
        return self.ctrl.n
