"""Checkpoint and resume (needs a GB300).

A snapshot holds an instance's particles exactly as stored, its controller and a fingerprint
of its problem; a restored instance -- in the same handle, a fresh handle, or another batch at
another place in the slot array -- must continue bit for bit like the uninterrupted run.
"""
import numpy as np
import pytest

from paper_2003_01061_gb300 import build as B
from paper_2003_01061_gb300 import sphmesh as S
from paper_2003_01061_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def same(pa, pb):
    for k in ("x", "v", "h", "group"):
        assert np.array_equal(pa[k], pb[k]), k


@pytest.mark.parametrize("prec", [32, 64])
def test_mesh_snapshot_restore_continues_bit_for_bit(prec):
    w = WL.disk_holes(n_target=5000, seed=71)
    m = S.Mesh(w, precision=prec)
    m.set_state()
    m.step(30)
    m.sync()
    snap = S.sph_mesh_snapshot(m.h)
    m.step(25)
    m.sync()
    ref, rr = m.positions(), m.report()
    assert rr.iteration == 55

    m2 = S.Mesh(w, precision=prec)
    S.sph_mesh_restore(m2.h, snap)
    m2.n = len(w["x"])
    assert m2.report().iteration == 30
    m2.step(25)
    m2.sync()
    same(ref, m2.positions())
    r2 = m2.report()
    assert r2.iteration == rr.iteration and r2.E_sys == rr.E_sys and r2.phase == rr.phase

    S.sph_mesh_restore(m.h, snap)          # back in the original handle
    m.step(25)
    m.sync()
    same(ref, m.positions())
    m.close()
    m2.close()


def test_restore_refuses_other_problems_and_bad_buffers():
    w = WL.square2d(h=0.05, seed=72)
    m = S.Mesh(w, precision=32)
    m.set_state()
    m.step(3)
    snap = S.sph_mesh_snapshot(m.h)
    other = S.Mesh(WL.square2d(h=0.04, seed=72), precision=32)
    with pytest.raises(S.SphError):
        S.sph_mesh_restore(other.h, snap)                  # another grid
    fp64 = S.Mesh(w, precision=64)
    with pytest.raises(S.SphError):
        S.sph_mesh_restore(fp64.h, snap)                   # another precision
    with pytest.raises(S.SphError):
        S.sph_mesh_restore(m.h, snap[:200])                # truncated
    bad = bytearray(snap)
    bad[0] ^= 0xFF
    with pytest.raises(S.SphError):
        S.sph_mesh_restore(m.h, bytes(bad))                # not a snapshot
    for h in (m, other, fp64):
        h.close()


def test_batch_snapshot_moves_between_batches():
    wa, wb, wc = WL.square2d(h=0.05, seed=73), WL.disk_holes(n_target=3000, seed=74), WL.square2d(h=0.04, seed=75)
    b1 = S.Batch([wa, wb], precision=32)
    b1.set_state(0)
    b1.set_state(1)
    b1.step(20)
    snap = S.sph_batch_snapshot(b1.h, 1)
    b1.step(15)
    b1.sync()
    ref = b1.positions(1)
    # another batch, where instance 2 (same problem as wb) sits after a different instance
    caps = [len(wc["x"]), len(wa["x"]), len(wb["x"])]
    b2 = S.Batch([wc, wa, wb], precision=32, max_particles=caps)
    b2.set_state(0)
    S.sph_batch_restore(b2.h, 2, snap)
    b2.n[2] = len(wb["x"])
    b2.step(15)
    b2.sync()
    same(ref, b2.positions(2))
    assert b2.reports()[2].iteration == 35
    b1.close()
    b2.close()
