"""The allocation-free rebuild entry point (sph_cell_sort_noalloc), for callers that may not
allocate device memory: an application that owns a fixed device-memory budget through its own
pool, or a latency-critical loop where an allocation could synchronise the device.

Its keys, cell starts and permutation must equal those of the handle-based rebuild
(sph_debug_rebuild) exactly -- the tolerance of every rebuild check is bit equality -- on two
calls in a row, since all calls share one scratch array.  This file is collected last on
purpose.  Needs a GB300."""
import numpy as np
import pytest

from paper_2003_01061_gb300 import build as B
from paper_2003_01061_gb300 import sphmesh as S
from paper_2003_01061_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["disk", "cube"])
def test_noalloc_rebuild_matches_handle_rebuild(name):
    import torch

    B.build()
    w = WL.disk_holes(n_target=6000, seed=2) if name == "disk" else WL.cube_sphere(n_target=12000, seed=3)
    D = w["domain"]["D"]
    h = WL.sizing_eval(w["sizing"], w["x"]).astype(np.float32)
    m = S.Mesh(w, precision=32, params=dict(w["params"], cells_per_support=1))
    m.set_state(h=h.astype(np.float64))
    grid = S.sph_mesh_grid(m.h)
    key_ref, cs_ref, perm_ref = S.sph_debug_rebuild(m.h, m.n, grid.n_cells)
    m.close()
    assert grid.n_cells <= (1 << 20)

    dev = torch.device("cuda", 0)
    n = len(w["x"])
    xs = [torch.tensor(np.ascontiguousarray(w["x"][:, a]), dtype=torch.float64, device=dev) for a in range(3)]
    hd = torch.tensor(h, dtype=torch.float32, device=dev)
    key = torch.full((n,), -7, dtype=torch.int32, device=dev)
    cs = torch.full((grid.n_cells + 1,), -7, dtype=torch.int32, device=dev)
    perm = torch.full((n,), -7, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for call in range(2):
        S.sph_cell_sort_noalloc(grid, n, xs[0].data_ptr(), xs[1].data_ptr(), xs[2].data_ptr() if D == 3 else None,
                                hd.data_ptr(), key.data_ptr(), cs.data_ptr(), perm.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize(dev)
        assert np.array_equal(key.cpu().numpy().astype(np.int64), key_ref), call
        assert np.array_equal(cs.cpu().numpy().astype(np.int64), cs_ref), call
        assert np.array_equal(perm.cpu().numpy().astype(np.int64), perm_ref), call
        key.fill_(-1)
        cs.fill_(-1)
        perm.fill_(-1)


def test_noalloc_rejects_oversized_grid():
    B.build()
    g = S.sph_grid_spec(2, [0, 0, 0], [1, 1, 0], 0.0004, 0.0004, 2.0)
    assert g.n_cells > (1 << 20)
    with pytest.raises(S.SphError) as e:
        S.sph_cell_sort_noalloc(g, 0, None, None, None, None, None, 1, None, None)
    assert e.value.status == S.SPH_E_INVALID and "at most" in str(e.value)
