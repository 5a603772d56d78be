"""Host-side checks of libsphmesh.so that need no GPU: it builds for sm_103a, loads, exports
every entry point declared in include/sphmesh.h, its cell-grid specification matches the
oracle's independent implementation bit for bit, and invalid descriptors are rejected before
any device work."""
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_2003_01061_gb300 import build as B
from paper_2003_01061_gb300 import sphmesh as S
from paper_2003_01061_gb300 import workloads as WL

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def header_functions():
    src = open(os.path.join(ROOT, "include", "sphmesh.h")).read()
    return sorted(set(re.findall(r"^(?:sph_status|void|const char\*)\s+(sph_\w+)\s*\(", src, re.M)))


def test_library_exports_every_declared_function():
    names = header_functions()
    assert len(names) >= 15
    L = S.lib()
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(S.EXPORTS)


def test_binding_constants_match_header():
    src = open(os.path.join(ROOT, "include", "sphmesh.h")).read()
    defs = dict(re.findall(r"^#define\s+(SPH_\w+)\s+(\d+)", src, re.M))
    assert int(defs["SPH_SLOT_CHUNK"]) == S.SLOT_CHUNK
    assert int(defs["SPH_MAX_FEATURES"]) == S.MAX_FEATURES
    assert int(defs["SPH_MAX_HOLES"]) == S.MAX_HOLES
    assert int(defs["SPH_MAX_LEVELS"]) == S.MAX_LEVELS


@pytest.mark.parametrize("cps", [1, 2, 4])
@pytest.mark.parametrize("D,lo,hi,hlo,hhi", [
    (2, [0, 0, 0], [1, 1, 0], 0.02, 0.02),
    (2, [-1, -1, 0], [1, 1, 0], 0.0018, 0.018),
    (3, [0, 0, 0], [1, 1, 1], 0.0053, 0.033),
    (3, [-0.3, 0.1, 2.0], [0.7, 0.4, 2.5], 0.001, 0.05),
])
def test_grid_spec_matches_oracle(D, lo, hi, hlo, hhi, cps):
    a = S.sph_grid_spec(D, lo, hi, hlo, hhi, 2.0, cps)
    b = O.grid_spec(D, lo, hi, hlo, hhi, 2.0, cps)
    assert a.cells_per_support == b.cps == cps
    assert a.levels == b.L and a.c0 == b.c0 and a.n_cells == b.ncell
    for l in range(8):
        assert a.thr[l] == b.thr[l]
    for k in range(3):
        assert a.origin[k] == b.origin[k]
    for l in range(a.levels):
        assert a.base[l] == b.base[l]
        for k in range(3):
            assert a.dims[l][k] == b.dims[l][k]


def _descs(w):
    return S.domain_desc(w["domain"]), S.sizing_desc(w["sizing"]), S.params_struct(w["params"])


def test_invalid_descriptors_are_rejected():
    w = WL.square2d(h=0.1)
    d, z, p = _descs(w)
    d.dim = 4
    with pytest.raises(S.SphError) as e:
        S.sph_mesh_create(d, z, p, 10)
    assert e.value.status == S.SPH_E_INVALID
    d, z, p = _descs(w)
    d.features[1].dim = 2            # a segment must be a curve
    with pytest.raises(S.SphError) as e:
        S.sph_mesh_create(d, z, p, 10)
    assert e.value.status == S.SPH_E_INVALID
    d, z, p = _descs(w)
    z.lo = 0.0
    with pytest.raises(S.SphError) as e:
        S.sph_mesh_create(d, z, p, 10)
    assert e.value.status == S.SPH_E_INVALID
    d, z, p = _descs(w)
    p.precision = 16
    with pytest.raises(S.SphError) as e:
        S.sph_mesh_create(d, z, p, 10)
    assert e.value.status == S.SPH_E_INVALID
    with pytest.raises(S.SphError):
        S.sph_grid_spec(2, [0, 0, 0], [1, 1, 0], 1e-6, 1.0)     # needs more than 8 levels
    for bad in (3, -1, 8):
        with pytest.raises(S.SphError):
            S.sph_grid_spec(2, [0, 0, 0], [1, 1, 0], 0.01, 0.02, 2.0, bad)
        d, z, p = _descs(w)
        p.cells_per_support = bad
        with pytest.raises(S.SphError):
            S.sph_mesh_create(d, z, p, 10)


def test_feature_order_needs_group_convergence():
    # Algorithm 1's feature loop in sequence goes with its per-feature convergence check
    w = WL.square2d(h=0.1)
    for fo, gc, ok in ((1, 0, False), (2, 1, False), (1, 1, True), (0, 0, True)):
        d, z, p = _descs(w)
        p.feature_order, p.group_convergence = fo, gc
        if ok:
            continue          # creating a mesh needs a GPU; the rejections happen before any
        with pytest.raises(S.SphError) as e:
            S.sph_mesh_create(d, z, p, 10)
        assert e.value.status == S.SPH_E_INVALID


def test_params_default_are_the_papers():
    q = S.params_struct({})
    for k in ("kappa", "p0", "visc", "cfl_a", "cfl_v", "threshold", "reset_period", "sample_every", "window",
              "boundary_correction"):
        assert getattr(q, k) == WL.PAPER_PARAMS[k], k


def test_method_presets_match_the_workload_table():
    names = {S.METHOD_IMPROVED: "improved", S.METHOD_FU2019: "fu2019", S.METHOD_FU2019_V2: "fu2019_v2"}
    for method, name in names.items():
        q = S.params_struct({"visc": 0.3, "reset_period": 7, "boundary_correction": 1})
        S.sph_params_preset(q, method)
        want = WL.method_preset({"visc": 0.3}, name)
        assert q.reset_period == want["reset_period"] and q.boundary_correction == want["boundary_correction"]
        assert q.visc == 0.3                       # other fields untouched
    with pytest.raises(S.SphError):
        S.sph_params_preset(S.params_struct({}), 3)
    w = WL.square2d(h=0.05)
    d, z, p = _descs(w)
    p.boundary_correction = 2
    with pytest.raises(S.SphError):
        S.sph_mesh_create(d, z, p, 10)


def test_noalloc_rejects_grid_with_undersized_coarse_level():
    """A caller-built grid whose coarser level does not cover the finest grid shifted down to
    that level would give keys past the level (and past the fixed scratch array at the top
    level); the allocation-free rebuild must refuse it before any device work."""
    g = S.sph_grid_spec(2, [0, 0, 0], [1, 1, 0], 0.01, 0.04, 2.0, 1)
    assert g.levels >= 2 and g.n_cells <= (1 << 20)
    need = ((g.dims[0][0] - 1) >> 1) + 1
    assert g.dims[1][0] >= need
    cells_l1 = lambda: g.dims[1][0] * g.dims[1][1] * g.dims[1][2]
    old = cells_l1()
    g.dims[1][0] = need - 1                 # one column short of the finest grid
    shrink = old - cells_l1()
    for l in range(2, g.levels):
        g.base[l] -= shrink
    g.n_cells -= shrink
    with pytest.raises(S.SphError) as e:
        S.sph_cell_sort_noalloc(g, 0, None, None, None, None, None, 1, None, None)
    assert e.value.status == S.SPH_E_INVALID and "does not cover" in str(e.value)
