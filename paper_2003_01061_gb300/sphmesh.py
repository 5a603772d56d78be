"""Thin ctypes binding of libsphmesh.so (include/sphmesh.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  All numerical work runs in
the library's CUDA kernels; if the compiled library is missing this module raises on load
instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsphmesh.so")

MAX_FEATURES, MAX_HOLES, MAX_LEVELS = 64, 8, 8
SLOT_CHUNK = 128   # SPH_SLOT_CHUNK: an instance's slots are its particle count rounded up to this
FEATURE_KIND = {"volume": 0, "point": 1, "segment": 2, "circle": 3, "rect": 4, "sphere": 5}
SIZING_KIND = {"const": 0, "hole_dist": 1, "radial": 2}
SPH_OK, SPH_E_INVALID, SPH_E_NOMEM, SPH_E_CUDA, SPH_E_DIVERGED, SPH_E_NOT_CONVERGED, SPH_E_OVERFLOW = range(7)
PHASE1, RAMP, PHASE2, DONE = 1, 2, 3, 4


class SphError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"sph status {status}: {msg}")
        self.status = status


class sph_feature(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dim", C.c_int32), ("geom", C.c_double * 12), ("normal", C.c_double * 3),
                ("orient", C.c_double)]


class sph_domain_desc(C.Structure):
    _fields_ = [("dim", C.c_int32), ("base", C.c_int32), ("bbox_lo", C.c_double * 3), ("bbox_hi", C.c_double * 3),
                ("ball_center", C.c_double * 3), ("ball_radius", C.c_double), ("n_holes", C.c_int32),
                ("hole_center", (C.c_double * 3) * MAX_HOLES), ("hole_radius", C.c_double * MAX_HOLES),
                ("n_features", C.c_int32), ("features", sph_feature * MAX_FEATURES)]


class sph_sizing_desc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("a", C.c_double), ("b", C.c_double), ("lo", C.c_double), ("hi", C.c_double),
                ("center", C.c_double * 3), ("n_ref", C.c_int32), ("ref_center", (C.c_double * 3) * MAX_HOLES),
                ("ref_radius", C.c_double * MAX_HOLES)]


class sph_params(C.Structure):
    _fields_ = [("kappa", C.c_double), ("p0", C.c_double), ("visc", C.c_double), ("cfl_a", C.c_double),
                ("cfl_v", C.c_double), ("eps1", C.c_double), ("dt_cap", C.c_double), ("dt_collapse", C.c_double),
                ("threshold", C.c_double), ("reset_period", C.c_int32), ("sample_every", C.c_int32),
                ("window", C.c_int32), ("ramp_len", C.c_int32), ("boundary_rho", C.c_int32),
                ("precision", C.c_int32), ("cells_per_support", C.c_int32), ("boundary_correction", C.c_int32),
                ("group_convergence", C.c_int32), ("feature_order", C.c_int32)]


class sph_report(C.Structure):
    _fields_ = [("phase", C.c_int32), ("n_groups", C.c_int32), ("iteration", C.c_int64), ("ramp_start", C.c_int64),
                ("escapes", C.c_int64), ("status", C.c_uint32), ("pad", C.c_uint32), ("E_t", C.c_double),
                ("E_avg", C.c_double), ("E_sys", C.c_double), ("vbar", C.c_double * MAX_FEATURES),
                ("dt", C.c_double * MAX_FEATURES), ("reset", C.c_int32 * MAX_FEATURES),
                ("group_phase", C.c_int32 * MAX_FEATURES), ("group_E", C.c_double * MAX_FEATURES)]


class sph_grid_info(C.Structure):
    _fields_ = [("dim", C.c_int32), ("levels", C.c_int32), ("cells_per_support", C.c_int32), ("c0", C.c_float),
                ("origin", C.c_float * 3),
                ("thr", C.c_float * MAX_LEVELS), ("dims", (C.c_int64 * 3) * MAX_LEVELS),
                ("base", C.c_int64 * MAX_LEVELS), ("n_cells", C.c_int64)]


class sph_kernel_time(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("total_ms", C.c_double)]


class sph_server_config(C.Structure):
    _fields_ = [("precision", C.c_int32), ("max_jobs", C.c_int32), ("slot_capacity", C.c_int64 * 2),
                ("hbm_fraction", C.c_double), ("steps_per_poll", C.c_int32)]


class sph_job_info(C.Structure):
    _fields_ = [("state", C.c_int32), ("dim", C.c_int32), ("n", C.c_int64), ("iterations", C.c_int64),
                ("phase", C.c_int32), ("status_word", C.c_uint32), ("escapes", C.c_int64), ("E_sys", C.c_double),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_finish", C.c_double)]


class sph_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("finished", C.c_int64), ("running", C.c_int64), ("queued", C.c_int64),
                ("rounds", C.c_int64), ("particle_steps", C.c_double)]


JOB_QUEUED, JOB_RUNNING, JOB_DONE, JOB_NOT_CONVERGED, JOB_FAILED = 1, 2, 3, 4, 5
METHOD_IMPROVED, METHOD_FU2019, METHOD_FU2019_V2 = 0, 1, 2


EXPORTS = ["sph_params_default", "sph_params_preset", "sph_feature_counts", "sph_sample_particles", "sph_mesh_sample",
           "sph_mesh_create", "sph_mesh_set_state", "sph_mesh_step", "sph_mesh_sync",
           "sph_mesh_run_until_converged", "sph_mesh_positions", "sph_mesh_report", "sph_mesh_destroy",
           "sph_last_error", "sph_grid_spec", "sph_mesh_grid", "sph_debug_rebuild", "sph_debug_neighbors",
           "sph_debug_interact", "sph_debug_update", "sph_mesh_set_timing", "sph_mesh_kernel_times",
           "sph_debug_pair_counts", "sph_cell_sort_noalloc", "sph_batch_create", "sph_batch_size",
           "sph_batch_set_problem", "sph_batch_set_state", "sph_batch_step", "sph_batch_sync",
           "sph_batch_run_until_converged", "sph_batch_positions", "sph_batch_reports", "sph_batch_set_timing",
           "sph_batch_kernel_times", "sph_batch_destroy", "sph_batch_slot_bytes", "sph_batch_autotune",
           "sph_mesh_snapshot", "sph_mesh_restore", "sph_batch_snapshot", "sph_batch_restore", "sph_server_create",
           "sph_server_submit", "sph_server_submit_sampled", "sph_server_poll", "sph_server_drain", "sph_server_job", "sph_server_release",
           "sph_server_destroy"]

_lib = None


def lib():
    """Loads libsphmesh.so; raises if it has not been built (there is no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2003_01061_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        sig = {
            "sph_params_default": [vp],
            "sph_params_preset": [vp, i32],
            "sph_feature_counts": [vp, vp, vp, vp, vp],
            "sph_sample_particles": [vp, vp, C.c_uint64, vp, vp, vp, vp],
            "sph_mesh_sample": [vp, C.c_uint64, vp],
            "sph_mesh_create": [vp, vp, vp, i64, vp, vp],
            "sph_mesh_set_state": [vp, i64, vp, vp, vp, vp],
            "sph_mesh_step": [vp, i32],
            "sph_mesh_sync": [vp],
            "sph_mesh_run_until_converged": [vp, i64, vp],
            "sph_mesh_positions": [vp, vp, vp, vp, vp, i64, vp],
            "sph_mesh_report": [vp, vp],
            "sph_grid_spec": [i32, vp, vp, d, d, d, i32, vp],
            "sph_mesh_grid": [vp, vp],
            "sph_debug_rebuild": [vp, vp, vp, vp],
            "sph_debug_neighbors": [vp, i32, vp, vp, i64, vp],
            "sph_debug_interact": [vp, vp, vp, vp, vp, vp],
            "sph_debug_update": [vp, vp, vp, d, d, vp, vp, vp, vp],
            "sph_mesh_set_timing": [vp, i32],
            "sph_mesh_kernel_times": [vp, vp, i32, vp],
            "sph_debug_pair_counts": [vp, vp, vp],
            "sph_cell_sort_noalloc": [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp],
            "sph_batch_create": [i32, vp, vp, vp, vp, vp, vp],
            "sph_batch_size": [vp, vp, vp, vp],
            "sph_batch_set_problem": [vp, i32, vp, vp, vp],
            "sph_batch_set_state": [vp, i32, i64, vp, vp, vp, vp],
            "sph_batch_step": [vp, i32],
            "sph_batch_sync": [vp],
            "sph_batch_run_until_converged": [vp, i64, vp],
            "sph_batch_positions": [vp, i32, vp, vp, vp, vp, i64, vp],
            "sph_batch_reports": [vp, vp, i32],
            "sph_batch_set_timing": [vp, i32],
            "sph_batch_kernel_times": [vp, vp, i32, vp],
            "sph_batch_slot_bytes": [i32, i32, vp],
            "sph_batch_autotune": [vp, i32, vp, vp],
            "sph_mesh_snapshot": [vp, vp, C.c_size_t, vp],
            "sph_mesh_restore": [vp, vp, C.c_size_t],
            "sph_batch_snapshot": [vp, i32, vp, C.c_size_t, vp],
            "sph_batch_restore": [vp, i32, vp, C.c_size_t],
            "sph_server_create": [vp, vp],
            "sph_server_submit": [vp, vp, vp, vp, i64, vp, vp, vp, i64, vp],
            "sph_server_submit_sampled": [vp, vp, vp, vp, C.c_uint64, i64, vp],
            "sph_server_poll": [vp, vp],
            "sph_server_drain": [vp, i64, vp],
            "sph_server_job": [vp, i64, vp, vp, vp, vp, i64],
            "sph_server_release": [vp, i64],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        for name in ("sph_mesh_destroy", "sph_batch_destroy", "sph_server_destroy"):
            getattr(L, name).argtypes = [vp]
            getattr(L, name).restype = None
        L.sph_last_error.argtypes = []
        L.sph_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(status):
    if status != SPH_OK:
        raise SphError(status, lib().sph_last_error().decode())
    return status


def _p(a):
    return None if a is None else a.ctypes.data


# ----------------------------------------------------------------------------------------
# descriptors from the plain dictionaries of workloads.py
# ----------------------------------------------------------------------------------------
def domain_desc(dom: dict) -> sph_domain_desc:
    d = sph_domain_desc()
    d.dim = dom["D"]
    d.base = 0 if dom["base"] == "box" else 1
    for a in range(3):
        d.bbox_lo[a], d.bbox_hi[a] = dom["lo"][a], dom["hi"][a]
        d.ball_center[a] = dom.get("ball_c", [0, 0, 0])[a]
    d.ball_radius = dom.get("ball_r", 0.0)
    d.n_holes = len(dom["holes"])
    for k, (c, r) in enumerate(dom["holes"]):
        for a in range(3):
            d.hole_center[k][a] = c[a]
        d.hole_radius[k] = r
    feats = dom["features"]
    d.n_features = len(feats)
    for k, f in enumerate(feats):
        F = d.features[k]
        F.kind, F.dim = FEATURE_KIND[f["kind"]], f["dim"]
        g = [0.0] * 12
        if f["kind"] == "point":
            g[0:3] = f["p"]
        elif f["kind"] == "segment":
            g[0:3], g[3:6] = f["a"], f["b"]
        elif f["kind"] == "circle":
            g[0], g[1], g[2] = f["c"][0], f["c"][1], f["r"]
        elif f["kind"] == "sphere":
            g[0:3], g[3] = f["c"], f["r"]
        elif f["kind"] == "rect":
            g[0:3], g[3:6], g[6:9], g[9], g[10] = f["o"], f["u"], f["w"], f["lu"], f["lw"]
        for a in range(12):
            F.geom[a] = g[a]
        for a in range(3):
            F.normal[a] = f.get("nb", [0, 0, 0])[a]
        F.orient = f.get("orient", 0.0)
    return d


def sizing_desc(s: dict) -> sph_sizing_desc:
    z = sph_sizing_desc()
    z.kind = SIZING_KIND[s["kind"]]
    z.a, z.b, z.lo, z.hi = s["a"], s["b"], s["lo"], s["hi"]
    for a in range(3):
        z.center[a] = s.get("q", [0, 0, 0])[a]
    refs = s.get("refs", [])
    z.n_ref = len(refs)
    for k, (c, r) in enumerate(refs):
        for a in range(3):
            z.ref_center[k][a] = c[a]
        z.ref_radius[k] = r
    return z


def params_struct(p: dict, precision: int = 32) -> sph_params:
    q = sph_params()
    _check(lib().sph_params_default(C.addressof(q)))
    for name, _ in sph_params._fields_:
        if name in p:
            setattr(q, name, p[name])
    q.precision = precision
    return q


def sph_feature_counts(domain: sph_domain_desc, sizing: sph_sizing_desc, stream: int | None = None):
    """(integrals, counts) of every feature: N_k of Eqs. 10, 11 on the device."""
    nf = domain.n_features
    M = np.zeros(nf)
    N = np.zeros(nf, np.int64)
    _check(lib().sph_feature_counts(C.addressof(domain), C.addressof(sizing), stream, _p(M), _p(N)))
    return M, N


def sph_sample_particles(domain: sph_domain_desc, sizing: sph_sizing_desc, seed: int, counts, stream: int | None = None):
    """(x [n][3], group [n]) drawn on the device (Sec. 3.6)."""
    counts = np.ascontiguousarray(counts, dtype=np.int64)
    n = int(counts.sum())
    x = np.zeros((max(n, 1), 3))
    g = np.zeros(max(n, 1), np.int32)
    _check(lib().sph_sample_particles(C.addressof(domain), C.addressof(sizing), seed, _p(counts), stream, _p(x), _p(g)))
    return x[:n], g[:n]


def sph_mesh_sample(m, seed: int) -> int:
    n = C.c_int64(0)
    _check(lib().sph_mesh_sample(m, seed, C.addressof(n)))
    return int(n.value)


def sph_params_preset(params: sph_params, method: int) -> sph_params:
    _check(lib().sph_params_preset(C.addressof(params), method))
    return params


# ----------------------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ----------------------------------------------------------------------------------------
def sph_grid_spec(dim, lo, hi, h_lo, h_hi, kappa=2.6, cells_per_support=1) -> sph_grid_info:
    g = sph_grid_info()
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    _check(lib().sph_grid_spec(dim, _p(lo), _p(hi), h_lo, h_hi, kappa, int(cells_per_support), C.addressof(g)))
    return g


def sph_mesh_create(domain: sph_domain_desc, sizing: sph_sizing_desc, params: sph_params, max_particles: int,
                    stream: int | None = None):
    h = C.c_void_p()
    _check(lib().sph_mesh_create(C.addressof(domain), C.addressof(sizing), C.addressof(params), int(max_particles),
                                 stream, C.addressof(h)))
    return h


def sph_mesh_set_state(m, x, group, v=None, h=None):
    x = np.ascontiguousarray(x, dtype=np.float64)
    group = np.ascontiguousarray(group, dtype=np.int32)
    v = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
    h = None if h is None else np.ascontiguousarray(h, dtype=np.float64)
    _check(lib().sph_mesh_set_state(m, len(x), _p(x), _p(group), _p(v), _p(h)))


def sph_mesh_step(m, n_steps=1):
    _check(lib().sph_mesh_step(m, int(n_steps)))


def sph_mesh_sync(m):
    _check(lib().sph_mesh_sync(m))


def sph_mesh_run_until_converged(m, max_iters):
    it = C.c_int64(0)
    st = lib().sph_mesh_run_until_converged(m, int(max_iters), C.addressof(it))
    if st not in (SPH_OK, SPH_E_NOT_CONVERGED):
        _check(st)
    return st == SPH_OK, it.value


def sph_mesh_positions(m, n):
    x = np.zeros((n, 3))
    g = np.zeros(n, np.int32)
    v = np.zeros((n, 3))
    h = np.zeros(n)
    got = C.c_int64(0)
    _check(lib().sph_mesh_positions(m, _p(x), _p(g), _p(v), _p(h), n, C.addressof(got)))
    return dict(x=x, group=g, v=v, h=h)


def sph_mesh_report(m) -> sph_report:
    r = sph_report()
    _check(lib().sph_mesh_report(m, C.addressof(r)))
    return r


def sph_mesh_destroy(m):
    if m:
        lib().sph_mesh_destroy(m)


def sph_mesh_grid(m) -> sph_grid_info:
    g = sph_grid_info()
    _check(lib().sph_mesh_grid(m, C.addressof(g)))
    return g


def sph_debug_rebuild(m, n, n_cells):
    key = np.zeros(n, np.int64)
    cs = np.zeros(n_cells + 1, np.int64)
    perm = np.zeros(n, np.int64)
    _check(lib().sph_debug_rebuild(m, _p(key), _p(cs), _p(perm)))
    return key, cs, perm


def sph_debug_neighbors(m, n, mode):
    counts = np.zeros(n, np.int64)
    total = C.c_int64(0)
    _check(lib().sph_debug_neighbors(m, mode, _p(counts), None, 0, C.addressof(total)))
    lists = np.zeros(max(total.value, 1), np.int32)
    _check(lib().sph_debug_neighbors(m, mode, _p(counts), _p(lists), len(lists), C.addressof(total)))
    return counts, lists[: total.value]


def sph_debug_interact(m, n, n_groups):
    out = dict(a_p=np.zeros((n, 3)), sigma=np.zeros(n), gamma=np.zeros(n), dta=np.zeros(n_groups),
               dtv=np.zeros(n_groups))
    _check(lib().sph_debug_interact(m, _p(out["a_p"]), _p(out["sigma"]), _p(out["gamma"]), _p(out["dta"]),
                                    _p(out["dtv"])))
    return out


def sph_debug_update(m, n, dt, reset, eps, f):
    dt = np.ascontiguousarray(dt, dtype=np.float64)
    reset = np.ascontiguousarray(reset, dtype=np.int32)
    out = dict(x=np.zeros((n, 3)), v=np.zeros((n, 3)), h=np.zeros(n), a_v=np.zeros((n, 3)))
    _check(lib().sph_debug_update(m, _p(dt), _p(reset), float(eps), float(f), _p(out["x"]), _p(out["v"]),
                                  _p(out["h"]), _p(out["a_v"])))
    return out


def sph_mesh_set_timing(m, enable):
    _check(lib().sph_mesh_set_timing(m, int(bool(enable))))


def sph_mesh_kernel_times(m):
    arr = (sph_kernel_time * 16)()
    n = C.c_int32(0)
    _check(lib().sph_mesh_kernel_times(m, arr, 16, C.addressof(n)))
    return {arr[i].name.decode(): (arr[i].launches, arr[i].total_ms) for i in range(n.value)}


def sph_debug_pair_counts(m):
    a, b = C.c_int64(0), C.c_int64(0)
    _check(lib().sph_debug_pair_counts(m, C.addressof(a), C.addressof(b)))
    return a.value, b.value


def sph_cell_sort_noalloc(grid: sph_grid_info, n, x_ptr, y_ptr, z_ptr, h_ptr, key_ptr, cell_start_ptr, perm_ptr,
                          stream=None):
    """Allocation-free rebuild on caller-owned device arrays (raw device pointers as ints)."""
    _check(lib().sph_cell_sort_noalloc(C.addressof(grid), int(n), x_ptr, y_ptr, z_ptr, h_ptr, key_ptr,
                                       cell_start_ptr, perm_ptr, stream))


def sph_batch_create(domains, sizings, params, max_particles, stream: int | None = None):
    n = len(domains)
    D = (sph_domain_desc * n)(*domains)
    Z = (sph_sizing_desc * n)(*sizings)
    P = (sph_params * n)(*params)
    M = np.ascontiguousarray(max_particles, dtype=np.int64)
    h = C.c_void_p()
    _check(lib().sph_batch_create(n, D, Z, P, _p(M), stream, C.addressof(h)))
    return h


def sph_batch_size(b):
    ni, ns, cap = C.c_int32(0), C.c_int64(0), C.c_int64(0)
    _check(lib().sph_batch_size(b, C.addressof(ni), C.addressof(ns), C.addressof(cap)))
    return ni.value, ns.value, cap.value


def sph_batch_set_problem(b, inst, domain: sph_domain_desc, sizing: sph_sizing_desc, params: sph_params):
    _check(lib().sph_batch_set_problem(b, int(inst), C.addressof(domain), C.addressof(sizing), C.addressof(params)))


def sph_batch_set_state(b, inst, x, group, v=None, h=None):
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    group = np.ascontiguousarray(group, dtype=np.int32)
    v = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
    h = None if h is None else np.ascontiguousarray(h, dtype=np.float64)
    _check(lib().sph_batch_set_state(b, int(inst), len(x), _p(x), _p(group), _p(v), _p(h)))


def sph_batch_step(b, n_steps=1):
    _check(lib().sph_batch_step(b, int(n_steps)))


def sph_batch_sync(b):
    _check(lib().sph_batch_sync(b))


def sph_batch_run_until_converged(b, max_iters):
    it = C.c_int64(0)
    st = lib().sph_batch_run_until_converged(b, int(max_iters), C.addressof(it))
    if st not in (SPH_OK, SPH_E_NOT_CONVERGED):
        _check(st)
    return st == SPH_OK, it.value


def sph_batch_positions(b, inst, n):
    x = np.zeros((n, 3))
    g = np.zeros(n, np.int32)
    v = np.zeros((n, 3))
    h = np.zeros(n)
    got = C.c_int64(0)
    _check(lib().sph_batch_positions(b, int(inst), _p(x), _p(g), _p(v), _p(h), n, C.addressof(got)))
    return dict(x=x, group=g, v=v, h=h)


def sph_batch_reports(b, n_inst):
    arr = (sph_report * n_inst)()
    _check(lib().sph_batch_reports(b, arr, n_inst))
    return list(arr)


def sph_batch_set_timing(b, enable):
    _check(lib().sph_batch_set_timing(b, int(bool(enable))))


def sph_batch_kernel_times(b):
    arr = (sph_kernel_time * 16)()
    n = C.c_int32(0)
    _check(lib().sph_batch_kernel_times(b, arr, 16, C.addressof(n)))
    return {arr[i].name.decode(): (arr[i].launches, arr[i].total_ms) for i in range(n.value)}


def sph_batch_destroy(b):
    if b:
        lib().sph_batch_destroy(b)


def sph_mesh_snapshot(m) -> bytes:
    need = C.c_size_t(0)
    _check(lib().sph_mesh_snapshot(m, None, 0, C.addressof(need)))
    buf = (C.c_char * need.value)()
    _check(lib().sph_mesh_snapshot(m, buf, need.value, C.addressof(need)))
    return bytes(buf)


def sph_mesh_restore(m, snap: bytes):
    _check(lib().sph_mesh_restore(m, snap, len(snap)))


def sph_batch_snapshot(b, inst) -> bytes:
    need = C.c_size_t(0)
    _check(lib().sph_batch_snapshot(b, int(inst), None, 0, C.addressof(need)))
    buf = (C.c_char * need.value)()
    _check(lib().sph_batch_snapshot(b, int(inst), buf, need.value, C.addressof(need)))
    return bytes(buf)


def sph_batch_restore(b, inst, snap: bytes):
    _check(lib().sph_batch_restore(b, int(inst), snap, len(snap)))


def sph_batch_autotune(b, trial_steps=10):
    """Returns (chosen cells per support, trial times in ms for 1, 2, 4; -1 = not possible)."""
    c = C.c_int32(0)
    t = (C.c_float * 3)()
    _check(lib().sph_batch_autotune(b, int(trial_steps), C.addressof(c), t))
    return c.value, list(t)


def sph_batch_slot_bytes(dim, precision=32):
    v = C.c_int64(0)
    _check(lib().sph_batch_slot_bytes(int(dim), int(precision), C.addressof(v)))
    return v.value


def sph_server_create(precision=32, max_jobs=64, slot_capacity=(-1, -1), hbm_fraction=0.5, steps_per_poll=20):
    cfg = sph_server_config()
    cfg.precision, cfg.max_jobs, cfg.hbm_fraction, cfg.steps_per_poll = precision, max_jobs, hbm_fraction, steps_per_poll
    cfg.slot_capacity[0], cfg.slot_capacity[1] = int(slot_capacity[0]), int(slot_capacity[1])
    h = C.c_void_p()
    _check(lib().sph_server_create(C.addressof(cfg), C.addressof(h)))
    return h


def sph_server_submit(s, domain: sph_domain_desc, sizing: sph_sizing_desc, params: sph_params, x, group, h=None,
                      max_iters=1000):
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    group = np.ascontiguousarray(group, dtype=np.int32)
    h = None if h is None else np.ascontiguousarray(h, dtype=np.float64)
    jid = C.c_int64(0)
    _check(lib().sph_server_submit(s, C.addressof(domain), C.addressof(sizing), C.addressof(params), len(x), _p(x),
                                   _p(group), _p(h), int(max_iters), C.addressof(jid)))
    return jid.value


def sph_server_submit_sampled(s, domain: sph_domain_desc, sizing: sph_sizing_desc, params: sph_params, seed: int,
                              max_iters=1000):
    jid = C.c_int64(0)
    _check(lib().sph_server_submit_sampled(s, C.addressof(domain), C.addressof(sizing), C.addressof(params), seed,
                                           int(max_iters), C.addressof(jid)))
    return jid.value


def sph_server_poll(s) -> sph_server_stats:
    st = sph_server_stats()
    _check(lib().sph_server_poll(s, C.addressof(st)))
    return st


def sph_server_drain(s, max_rounds=100000) -> sph_server_stats:
    st = sph_server_stats()
    _check(lib().sph_server_drain(s, int(max_rounds), C.addressof(st)))
    return st


def sph_server_job(s, job_id, n=0):
    info = sph_job_info()
    if n > 0:
        x, g, h = np.zeros((n, 3)), np.zeros(n, np.int32), np.zeros(n)
        _check(lib().sph_server_job(s, int(job_id), C.addressof(info), _p(x), _p(g), _p(h), n))
        return info, dict(x=x, group=g, h=h)
    _check(lib().sph_server_job(s, int(job_id), C.addressof(info), None, None, None, 0))
    return info, None


def sph_server_release(s, job_id):
    _check(lib().sph_server_release(s, int(job_id)))


def sph_server_destroy(s):
    if s:
        lib().sph_server_destroy(s)


class Mesh:
    """Owning handle: create from a workload dictionary, destroy on close / garbage collection."""

    def __init__(self, w: dict, precision: int = 32, max_particles: int | None = None, stream: int | None = None,
                 params: dict | None = None):
        self.w = w
        self.n_groups = len(w["domain"]["features"])
        self._dom = domain_desc(w["domain"])
        self._siz = sizing_desc(w["sizing"])
        self._prm = params_struct(params or w["params"], precision)
        self.h = sph_mesh_create(self._dom, self._siz, self._prm, max_particles or len(w["x"]), stream)
        self.n = 0

    def set_state(self, x=None, group=None, v=None, h=None):
        x = self.w["x"] if x is None else x
        group = self.w["group"] if group is None else group
        sph_mesh_set_state(self.h, x, group, v, h)
        self.n = len(x)

    def sample(self, seed: int) -> int:
        """Initial particles drawn on the device (Sec. 3.6) instead of the workload's own."""
        self.n = sph_mesh_sample(self.h, seed)
        return self.n

    def step(self, k=1):
        sph_mesh_step(self.h, k)

    def sync(self):
        sph_mesh_sync(self.h)

    def positions(self):
        return sph_mesh_positions(self.h, self.n)

    def report(self):
        return sph_mesh_report(self.h)

    def close(self):
        if self.h:
            sph_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owning batch handle over a list of workload dictionaries (one instance each)."""

    def __init__(self, ws: list, precision: int = 32, max_particles: list | None = None,
                 stream: int | None = None, params: list | None = None):
        self.ws = list(ws)
        self.precision = precision
        doms = [domain_desc(w["domain"]) for w in ws]
        sizs = [sizing_desc(w["sizing"]) for w in ws]
        prms = [params_struct((params[i] if params else None) or w["params"], precision) for i, w in enumerate(ws)]
        caps = max_particles or [len(w["x"]) for w in ws]
        self.caps = list(caps)
        self.h = sph_batch_create(doms, sizs, prms, caps, stream)
        self.n_inst = len(ws)
        self.n = [0] * self.n_inst

    def set_problem(self, inst, w, params: dict | None = None):
        sph_batch_set_problem(self.h, inst, domain_desc(w["domain"]), sizing_desc(w["sizing"]),
                              params_struct(params or w["params"], self.precision))
        self.ws[inst] = w
        self.n[inst] = 0

    def set_state(self, inst, x=None, group=None, v=None, h=None):
        w = self.ws[inst]
        x = w["x"] if x is None else x
        group = w["group"] if group is None else group
        sph_batch_set_state(self.h, inst, x, group, v, h)
        self.n[inst] = len(x)

    def step(self, k=1):
        sph_batch_step(self.h, k)

    def sync(self):
        sph_batch_sync(self.h)

    def positions(self, inst):
        return sph_batch_positions(self.h, inst, self.n[inst])

    def reports(self):
        return sph_batch_reports(self.h, self.n_inst)

    def close(self):
        if self.h:
            sph_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Owning server handle; jobs are workload dictionaries."""

    def __init__(self, precision=32, max_jobs=64, slot_capacity=(-1, -1), hbm_fraction=0.5, steps_per_poll=20):
        self.precision = precision
        self.h = sph_server_create(precision, max_jobs, slot_capacity, hbm_fraction, steps_per_poll)
        self.n_of = {}

    def submit(self, w, max_iters, params: dict | None = None, h=None):
        jid = sph_server_submit(self.h, domain_desc(w["domain"]), sizing_desc(w["sizing"]),
                                params_struct(params or w["params"], self.precision), w["x"], w["group"], h,
                                max_iters)
        self.n_of[jid] = len(w["x"])
        return jid

    def submit_sampled(self, w, max_iters, seed, params: dict | None = None):
        """A job given by its problem alone; its particles are drawn on the device at admission."""
        jid = sph_server_submit_sampled(self.h, domain_desc(w["domain"]), sizing_desc(w["sizing"]),
                                        params_struct(params or w["params"], self.precision), seed, max_iters)
        self.n_of[jid] = int(sph_server_job(self.h, jid, 0)[0].n)   # the count the server fixed
        return jid

    def poll(self):
        return sph_server_poll(self.h)

    def drain(self, max_rounds=100000):
        return sph_server_drain(self.h, max_rounds)

    def job(self, jid, with_result=True):
        return sph_server_job(self.h, jid, self.n_of[jid] if with_result else 0)

    def release(self, jid):
        sph_server_release(self.h, jid)
        self.n_of.pop(jid, None)

    def close(self):
        if self.h:
            sph_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
