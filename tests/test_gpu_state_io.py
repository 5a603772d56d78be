"""Loading a particle set and reading it back through the C ABI (needs a GB300): the caller's
arrays are checked and converted on the device.  Checked here: every rejection of
sph_mesh_set_state names the first offending particle in input order, with the checks of a
particle taken in the order group, position, h, velocity; a rejected call leaves the loaded
state as it was; and the round trip set_state -> positions returns the input, exactly for what
is stored in the working precision and to the offset's rounding for positions."""
import numpy as np
import pytest

from paper_2003_01061_gb300 import build as B
from paper_2003_01061_gb300 import sphmesh as S
from paper_2003_01061_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


@pytest.fixture(scope="module")
def square():
    return WL.square2d(h=0.05, seed=7, jitter=0.3)


def _reject(m, n, x, g, v=None, h=None):
    with pytest.raises(S.SphError) as e:
        S.sph_mesh_set_state(m.h, x[:n], g[:n], v, h)
    assert e.value.status == S.SPH_E_INVALID
    return str(e.value)


def test_set_state_rejections(square):
    w = square
    m = S.Mesh(w, precision=32)
    m.set_state()
    before = m.positions()
    n = len(w["x"])
    x, g = np.array(w["x"]), np.array(w["group"], np.int32)
    G = len(w["domain"]["features"])

    gb = g.copy(); gb[7] = G
    assert "particle 7 has group %d" % G in _reject(m, n, x, gb)
    gb = g.copy(); gb[7] = -1
    assert "particle 7 has group -1" in _reject(m, n, x, gb)
    xb = x.copy(); xb[3, 1] = w["domain"]["hi"][1] + 1e-3
    assert "particle 3 outside the bounding box" in _reject(m, n, xb, g)
    xb = x.copy(); xb[4, 0] = np.nan
    assert "particle 4 outside the bounding box" in _reject(m, n, xb, g)
    h = WL.sizing_eval(w["sizing"], x)
    hb = h.copy(); hb[11] = 0.0
    assert "h of particle 11" in _reject(m, n, x, g, h=hb)
    hb = h.copy(); hb[12] = w["h_hi"] * 1.01
    assert "h of particle 12" in _reject(m, n, x, g, h=hb)
    v = np.zeros((n, 3)); v[9, 1] = np.inf
    assert "non-finite velocity" in _reject(m, n, x, g, v=v)
    # the first offending particle wins, whatever its check; within a particle, group first
    gb = g.copy(); gb[10] = G
    xb = x.copy(); xb[5, 0] = -1.0
    assert "particle 5 outside" in _reject(m, n, xb, gb)
    xb[10, 0] = -1.0; xb[5, 0] = x[5, 0]
    assert "particle 10 has group" in _reject(m, n, xb, gb)
    # nothing changed
    after = m.positions()
    for k in ("x", "group", "v", "h"):
        assert np.array_equal(before[k], after[k]), k
    m.close()


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("name", ["square", "cube"])
def test_round_trip(square, prec, name):
    w = square if name == "square" else WL.cube_sphere(n_target=6000, seed=3, mc_samples=200_000)
    n = len(w["x"])
    rng = np.random.default_rng(4)
    D = w["domain"]["D"]
    v = rng.normal(size=(n, 3)) * 1e-3
    v[:, D:] = 0.0
    h = WL.sizing_eval(w["sizing"], w["x"]) * rng.uniform(0.9, 1.0, n)
    m = S.Mesh(w, precision=prec)
    m.set_state(v=v, h=h)
    p = m.positions()
    cast = (lambda a: np.asarray(a, np.float32).astype(np.float64)) if prec == 32 else (lambda a: np.asarray(a))
    assert np.array_equal(p["group"], w["group"])
    assert np.array_equal(p["v"], cast(v))
    assert np.array_equal(p["h"], cast(h))
    # position = origin + cell c0 + offset, the offset rounded to the working precision
    c0 = float(S.sph_mesh_grid(m.h).c0)
    scale = max(1.0, float(np.abs(w["x"]).max()))
    tol = (2.0 ** -24 * c0 if prec == 32 else 0.0) + 8 * np.finfo(float).eps * scale
    assert np.abs(p["x"] - w["x"]).max() <= tol, np.abs(p["x"] - w["x"]).max()
    m.close()
