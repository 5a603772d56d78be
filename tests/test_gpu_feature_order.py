"""Algorithm 1's feature loop in sequence (feature_order = 1) on the GPU, needs a GB300.

The step runs one pass per intrinsic dimension (curves, surfaces, volume), each re-sorting the
state the previous pass left and reading the lower classes' new positions; every group runs its
own controller (group_convergence = 1).  The FP64 path follows the oracle's sequence step by
step, and an instance keeps its results bit for bit when it shares a batch with instances that
step all their groups at once (those take their whole step in the last pass).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2003_01061_gb300 import build as B
from paper_2003_01061_gb300 import sphmesh as S
from paper_2003_01061_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def seq_params(w, **over):
    p = WL.scaled_controller(w["params"], sample_every=2, window=5, ramp_len=10, reset_period=25)
    p.update(group_convergence=1, feature_order=1, threshold=1e-2, **over)
    return p


@pytest.mark.parametrize("case,steps,tol", [("square", 60, 1e-9), ("cube", 20, 1e-8)])
def test_fp64_sequence_follows_oracle(case, steps, tol):
    if case == "square":
        w = WL.square2d(h=0.04, seed=5, jitter=0.2)
        w["params"] = seq_params(w, kappa=2.0)
        hs = 0.04
    else:
        w = WL.cube_sphere(n_target=3000, seed=3, mc_samples=200_000)
        w["params"] = seq_params(w)
        hs = w["h_lo"]
    o = O.Oracle(w)
    m = S.Mesh(w, precision=64)
    m.set_state(h=o.h)
    m.step(steps)
    m.sync()
    got, rep = m.positions(), m.report()
    m.close()
    o.step(steps, use_grid=True)
    assert rep.status == 0 and rep.iteration == o.iteration and rep.phase == o.phase
    assert [rep.group_phase[g] for g in range(o.G)] == [o.ctrl.gphase[g] for g in range(o.G)]
    err = np.abs(got["x"] - o.x).max()
    assert err <= tol * hs, err
    for g in range(o.G):
        assert abs(rep.dt[g] - o.ctrl.dt[g]) <= 1e-7 * max(o.ctrl.dt[g], 1e-300)
    # the sequence is not the Jacobi step: the volume saw the moved curves
    j = O.Oracle(w, params=dict(w["params"], feature_order=0))
    j.step(steps, use_grid=True)
    vol = o.gdim[w["group"]] == w["domain"]["D"]
    assert np.abs(j.x[vol] - o.x[vol]).max() > 100 * tol * hs


def test_sequence_and_jacobi_instances_in_one_batch_match_alone():
    wa = WL.square2d(h=0.05, seed=61, jitter=0.2)
    wa["params"] = seq_params(wa)
    wb = WL.disk_holes(n_target=3000, seed=62)       # steps all its groups at once
    b = S.Batch([wa, wb], precision=32)
    b.set_state(0)
    b.set_state(1)
    b.step(40)
    b.sync()
    reps = b.reports()
    for i, w in enumerate((wa, wb)):
        m = S.Mesh(w, precision=32)
        m.set_state()
        m.step(40)
        m.sync()
        pa, ra = m.positions(), m.report()
        m.close()
        pb = b.positions(i)
        for k in ("x", "v", "h", "group"):
            assert np.array_equal(pa[k], pb[k]), (i, k)
        assert ra.iteration == reps[i].iteration and ra.phase == reps[i].phase
    b.close()
