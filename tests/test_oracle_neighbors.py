"""Pins of the oracle's neighbour search and cell-list representation (no GPU).

* The FP64/FP32 representation predicate agrees with the plain definition r_ij < kappa h_ij
  (Eq. 7) on every pair except those whose distance lies within rounding of the cut-off.
* The multi-level grid specification puts every particle in cells at least as wide as its
  support, so the 3^D-cell search of each level is exhaustive.
* The counting sort equals a library stable sort by key.
"""
import numpy as np
import pytest

from oracle import oracle as O


def random_cloud(n, D, seed, hlo=0.01, hhi=0.08):
    rng = np.random.default_rng(seed)
    x = np.zeros((n, 3))
    x[:, :D] = rng.uniform(0, 0.5, (n, D))
    h = np.exp(rng.uniform(np.log(hlo), np.log(hhi), n))
    return x, h


@pytest.mark.parametrize("D", [2, 3])
def test_grid_spec_levels_cover_supports(D):
    g = O.grid_spec(D, [0, 0, 0], [0.5, 0.5, 0.5], 0.01, 0.08)
    assert 1 <= g.L <= 8
    c = [float(g.c0) * 2 ** l for l in range(g.L)]
    assert c[0] >= 2 * 0.01 and c[-1] >= 2 * 0.08
    x, h = random_cloud(3000, D, 1)
    rep = O.grid_repr(g, x, h, prec=32)
    for l in range(g.L):
        sel = rep["level"] == l
        if sel.any():
            hf = h[sel].astype(np.float32).astype(np.float64)
            assert np.all(2.0 * hf <= c[l] * (1 - 2 ** -11))          # support inside one cell
            if l > 0:
                assert np.all(2.0 * hf > c[l - 1] / (1 + 2 ** -9))      # and not in a finer level
    assert not rep["clamped"].any()
    # offsets inside [0, c_l) and the representation reproduces x
    for i in range(0, 3000, 97):
        l = rep["level"][i]
        assert np.all(rep["off"][i, :D] >= -1e-12 * c[l]) and np.all(rep["off"][i, :D] < c[l] * (1 + 1e-12))
        xr = np.asarray(g.origin)[:D] + rep["cell"][i, :D] * c[l] + rep["off"][i, :D]
        assert np.all(np.abs(xr - x[i, :D]) < 1e-7 * c[l])


@pytest.mark.parametrize("D,prec,rel", [(2, 64, 1e-12), (2, 32, 2e-6), (3, 64, 1e-12), (3, 32, 2e-6)])
def test_repr_predicate_matches_definition(D, prec, rel):
    n = 700
    x, h = random_cloud(n, D, 7 + D)
    g = O.grid_spec(D, [0, 0, 0], [0.5, 0.5, 0.5], 0.01, 0.08)
    checked = 0
    for i in range(0, n, 7):
        a = set(O.neighbors_brute(x, h, i, D).tolist())
        b = set(O.neighbors_repr(g, x, h, i, prec=prec).tolist())
        for j in a.symmetric_difference(b):
            r = np.linalg.norm(x[i, :D] - x[j, :D])
            rc = (h[i] + h[j])
            assert abs(r - rc) <= rel * rc, (i, j, r, rc)
        checked += len(a)
    assert checked > 500


def test_repr_predicate_is_symmetric_and_self_radius():
    n, D = 500, 2
    x, h = random_cloud(n, D, 3)
    g = O.grid_spec(D, [0, 0, 0], [0.5, 0.5, 0.5], 0.01, 0.08)
    nb = [set(O.neighbors_repr(g, x, h, i, prec=32).tolist()) for i in range(n)]
    for i in range(n):
        for j in nb[i]:
            assert i in nb[j]
        s = set(O.neighbors_repr(g, x, h, i, prec=32, self_radius=True).tolist())
        assert i in s
        d = np.linalg.norm(x[:, :D] - x[i, :D], axis=1)
        far = set(np.where(d > 2 * h[i] * (1 + 1e-5))[0].tolist())
        assert not (s & far)


def test_counting_sort_equals_stable_sort():
    rng = np.random.default_rng(4)
    key = rng.integers(0, 300, 5000)
    cs, perm = O.counting_sort(key, 300)
    assert np.array_equal(perm, np.argsort(key, kind="stable"))
    assert np.array_equal(np.diff(cs), np.bincount(key, minlength=300))
    assert cs[0] == 0 and cs[-1] == 5000
