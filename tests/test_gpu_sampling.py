"""Initial particles on the device (Sec. 3.6) against the oracle (needs a GB300).

* target counts (Eqs. 10, 11): the device's midpoint-rule integrals equal the oracle's on the
  same quadrature points to 1e-9 (summation order differs), and the rounded counts are equal;
* samples: with the same counts and seed the device draws exactly the oracle's positions, bit
  for bit (the same Philox4x32-10 words, the acceptance decided by the same correctly rounded
  FP64 operations), feature by feature;
* a mesh loaded by sph_mesh_sample holds those particles (up to the rounding of its stored
  representation) and steps; a mesh too small for the counts is refused.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2003_01061_gb300 import build as B
from paper_2003_01061_gb300 import sphmesh as S
from paper_2003_01061_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

NQ = {"volume2": 2048, "volume3": 256, "segment": 65536, "circle": 65536, "rect": 1024, "sphere": 512}


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def problems():
    return {
        "square_radial": WL.square_radial(seed=6),
        "disk": WL.disk_holes(n_target=8000, seed=2, mc_samples=100_000),
        "cube": WL.cube_sphere(n_target=15_000, seed=3, mc_samples=100_000),
    }


_P = {}


def problem(name):
    if not _P:
        _P.update(problems())
    return _P[name]


def oracle_integrals(w):
    dom, siz = O.make_domain(w["domain"]), O.make_sizing(w["sizing"])
    D = w["domain"]["D"]
    out = []
    for k, f in enumerate(w["domain"]["features"]):
        kind = f["kind"]
        nq = NQ[kind + str(D)] if kind == "volume" else NQ.get(kind, 1)
        out.append(O.feature_mass(dom, siz, k, nq))
    return np.array(out)


@pytest.mark.parametrize("name", ["square_radial", "disk", "cube"])
def test_feature_counts_match_oracle(name):
    w = problem(name)
    M, N = S.sph_feature_counts(S.domain_desc(w["domain"]), S.sizing_desc(w["sizing"]))
    ref = oracle_integrals(w)
    assert np.allclose(M, ref, rtol=1e-9, atol=0), np.abs(M / ref - 1).max()
    assert np.array_equal(N, np.rint(ref).astype(np.int64))


@pytest.mark.parametrize("name,seed", [("square_radial", 1), ("disk", 7), ("cube", 3)])
def test_samples_bit_exact_against_oracle(name, seed):
    w = problem(name)
    _, N = S.sph_feature_counts(S.domain_desc(w["domain"]), S.sizing_desc(w["sizing"]))
    x, g = S.sph_sample_particles(S.domain_desc(w["domain"]), S.sizing_desc(w["sizing"]), seed, N)
    xo, go = O.sample(w, seed, N)
    assert np.array_equal(g, go)
    assert np.array_equal(x, xo), np.abs(x - xo).max()


def test_mesh_sample_loads_and_steps():
    w = problem("square_radial")
    _, N = S.sph_feature_counts(S.domain_desc(w["domain"]), S.sizing_desc(w["sizing"]))
    n = int(N.sum())
    m = S.Mesh(w, precision=32, max_particles=n)
    assert m.sample(5) == n
    xo, go = O.sample(w, 5, N)
    p = m.positions()
    assert np.array_equal(p["group"], go)
    g = S.sph_mesh_grid(m.h)
    assert np.abs(p["x"] - xo).max() <= 4 * np.float32(g.c0) * 2.0 ** -23
    assert np.all(p["v"] == 0)
    m.step(20)
    m.sync()
    assert m.report().iteration == 20
    small = S.Mesh(w, precision=32, max_particles=n - 1)
    with pytest.raises(S.SphError) as e:
        small.sample(5)
    assert e.value.status == S.SPH_E_NOMEM
    small.close()
    m.close()


def test_sample_rejects_bad_counts():
    w = problem("square_radial")
    d, z = S.domain_desc(w["domain"]), S.sizing_desc(w["sizing"])
    nf = len(w["domain"]["features"])
    bad = np.zeros(nf, np.int64)
    bad[0] = -1
    with pytest.raises(S.SphError):
        S.sph_sample_particles(d, z, 1, bad)
    two = np.zeros(nf, np.int64)
    two[5] = 2                                          # a point feature holds one particle
    with pytest.raises(S.SphError):
        S.sph_sample_particles(d, z, 1, two)
