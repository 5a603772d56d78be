"""The serving loop against the same jobs run alone (needs a GB300).

Jobs of both dimensions arrive while others are resident, wait when the server's slots are
full, and are retired one by one.  Every job's result must be bit-identical to the same problem
run alone through sph_mesh_run_until_converged with the same iteration limit (a multiple of the
steps per scheduling round, so that neither runs past the other), whatever else was resident.
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


def run_alone(w, max_iters, params=None):
    m = S.Mesh(w, precision=32, params=params)
    m.set_state()
    ok, it = S.sph_mesh_run_until_converged(m.h, max_iters)
    p, r = m.positions(), m.report()
    m.close()
    return p, r, ok, it


def jobs_mix():
    conv = lambda w: WL.scaled_controller(dict(w["params"], threshold=2e-2))
    js = [
        (WL.square2d(h=0.05, seed=41), 120, None),
        (WL.disk_holes(n_target=4000, seed=42), 80, None),
        (WL.cube_sphere(n_target=6000, seed=43), 40, None),
        (WL.square2d(h=0.06, seed=44), 2000, "conv"),
        (WL.square2d(h=0.04, seed=45), 60, None),
        (WL.cube_sphere(n_target=3000, seed=46, sphere_r=0.2), 60, None),
        (WL.disk_holes(n_target=2500, seed=47), 100, None),
    ]
    return [(w, it, conv(w) if p == "conv" else None) for w, it, p in js]


@pytest.mark.parametrize("cap2d", [None, 4096])
def test_served_jobs_match_alone(cap2d):
    js = jobs_mix()
    n2 = [len(w["x"]) for w, _, _ in js if w["domain"]["D"] == 2]
    n3 = [len(w["x"]) for w, _, _ in js if w["domain"]["D"] == 3]
    # cap2d: room for one or two 2D jobs at a time, so that later ones wait for retirements
    C = S.SLOT_CHUNK
    caps = (cap2d or sum(n2) + C * len(n2), sum(n3) + C * len(n3))
    srv = S.Server(precision=32, max_jobs=3, slot_capacity=caps, steps_per_poll=20)
    ids = []
    # arrivals spread over the first rounds
    for k, (w, it, prm) in enumerate(js):
        ids.append(srv.submit(w, it, params=prm))
        if k % 2 == 1:
            srv.poll()
    st = srv.drain(10000)
    assert st.finished == len(js) and st.running == 0 and st.queued == 0
    lat = []
    for jid, (w, it, prm) in zip(ids, js):
        info, res = srv.job(jid)
        p, r, ok, it_alone = run_alone(w, it, prm)
        assert info.state == (S.JOB_DONE if ok else S.JOB_NOT_CONVERGED)
        assert info.iterations == it_alone == r.iteration
        for k in ("x", "h", "group"):
            assert np.array_equal(res[k], p[k]), (jid, k)
        assert info.t_submit <= info.t_admit <= info.t_finish
        lat.append(info.t_finish - info.t_submit)
        srv.release(jid)
    assert all(v > 0 for v in lat)
    srv.close()


def test_server_rejects_and_fails_cleanly():
    w2 = WL.square2d(h=0.05, seed=51)
    srv = S.Server(precision=32, max_jobs=2, slot_capacity=(1024, 0), steps_per_poll=10)
    big = WL.square2d(h=0.02, seed=52)
    with pytest.raises(S.SphError):
        srv.submit(big, 100)                       # more particles than the server holds
    with pytest.raises(S.SphError):
        srv.submit(WL.cube_sphere(n_target=2000, seed=53), 100)   # no 3D capacity
    bad = dict(w2)
    bad["sizing"] = dict(w2["sizing"], lo=-1.0)    # invalid descriptor: fails at admission
    j_bad = srv.submit(bad, 50)
    j_ok = srv.submit(w2, 50)
    srv.drain(1000)
    assert srv.job(j_bad, with_result=False)[0].state == S.JOB_FAILED
    info, res = srv.job(j_ok)
    assert info.state == S.JOB_NOT_CONVERGED and info.iterations == 50
    p, _, _, _ = run_alone(w2, 50)
    assert np.array_equal(res["x"], p["x"])
    srv.close()


def test_sampled_jobs_match_alone():
    # jobs given by their problem alone: the server draws their particles on the device at
    # admission; each result equals the same problem sampled with the same seed and run alone
    js = [(WL.square2d(h=0.05, seed=61), 60, 3), (WL.disk_holes(n_target=3000, seed=62, mc_samples=50_000), 40, 4),
          (WL.cube_sphere(n_target=4000, seed=63, mc_samples=50_000), 20, 5)]
    srv = S.Server(precision=32, max_jobs=2, slot_capacity=(8192, 8192), steps_per_poll=20)
    ids = [srv.submit_sampled(w, it, seed) for w, it, seed in js]
    st = srv.drain(10000)
    assert st.finished == len(js)
    for jid, (w, it, seed) in zip(ids, js):
        info, res = srv.job(jid)
        m = S.Mesh(w, precision=32, max_particles=srv.n_of[jid])
        assert m.sample(seed) == srv.n_of[jid] == info.n
        ok, it_alone = S.sph_mesh_run_until_converged(m.h, it)
        p = m.positions()
        assert info.iterations == it_alone
        for k in ("x", "h", "group"):
            assert np.array_equal(res[k], p[k]), (jid, k)
        assert info.t_submit <= info.t_admit <= info.t_finish
        m.close()
        srv.release(jid)
    srv.close()
