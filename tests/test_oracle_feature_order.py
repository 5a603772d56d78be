"""Algorithm 1's feature loop taken in sequence (feature_order = 1, Gauss-Seidel) in the oracle.

The only coupling between groups of different intrinsic dimension is one-sided: the lower
dimension acts on the higher through the boundary sum of Eq. 19 (Sec. 3.2).  So, with brute-force
neighbour sums (a fixed summation order):
  * without the boundary sum the classes do not act on each other and the two orders give
    bit-identical states;
  * the curves never see the volume: their trajectory is the same under both orders;
  * a volume particle's step in sequence equals its Jacobi step from the state in which the
    curves have already made theirs.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2003_01061_gb300 import workloads as WL


def case(**over):
    w = WL.square2d(h=0.1, seed=31, jitter=0.25)
    w["params"] = WL.scaled_controller(dict(w["params"], group_convergence=1, **over), sample_every=2, window=5,
                                       ramp_len=10, reset_period=25)
    return w


def run(w, order, steps, x=None):
    o = O.Oracle(w, x=x, params=dict(w["params"], feature_order=order))
    o.step(steps, use_grid=False)
    return o


def test_orders_agree_without_the_boundary_sum():
    w = case(boundary_correction=0)
    a, b = run(w, 0, 40), run(w, 1, 40)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.v, b.v) and np.array_equal(a.h, b.h)
    assert a.iteration == b.iteration == 40
    assert [a.ctrl.gphase[g] for g in range(a.G)] == [b.ctrl.gphase[g] for g in range(b.G)]


def test_curves_do_not_depend_on_the_order():
    w = case()
    a, b = run(w, 0, 30), run(w, 1, 30)
    curve = a.gdim[w["group"]] == 1
    vol = a.gdim[w["group"]] == 2
    assert np.array_equal(a.x[curve], b.x[curve]) and np.array_equal(a.v[curve], b.v[curve])
    assert np.abs(a.x[vol] - b.x[vol]).max() > 0           # the volume saw the moved curves


def test_volume_step_sees_the_curves_moved():
    w = case()
    one_j, one_s = run(w, 0, 1), run(w, 1, 1)
    curve = one_j.gdim[w["group"]] == 1
    vol = one_j.gdim[w["group"]] == 2
    assert np.abs(one_j.x[curve] - w["x"][curve]).max() > 0  # the curves moved in the first step
    moved = w["x"].copy()
    moved[curve] = one_j.x[curve]
    ref = run(w, 0, 1, x=moved)                               # Jacobi from the moved curves
    assert np.array_equal(one_s.x[vol], ref.x[vol]) and np.array_equal(one_s.v[vol], ref.v[vol])
    assert np.array_equal(one_s.x[curve], one_j.x[curve])


def test_singular_points_never_move():
    w = case()
    b = run(w, 1, 20)
    pts = b.gdim[w["group"]] == 0
    assert np.array_equal(b.x[pts], w["x"][pts])
