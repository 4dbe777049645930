"""Serving loop: admission by device-memory budget (host logic, CPU) and
continuous batching on the GPU, where requests that arrive while others run
join the shared batch and every result equals the same case solved alone."""
import threading
import time

import numpy as np
import pytest

import sphcases

S = pytest.importorskip("paper_2503_16082_gb300")
from paper_2503_16082_gb300 import serve  # noqa: E402


def test_oversized_request_rejected_on_host():
    srv = serve.Server(budget_bytes=1e6)
    fut = srv.submit(sphcases.small_droplet(3, 16), n_adv=1)
    with pytest.raises(S.SphstError):
        fut.result(timeout=1)
    assert srv.idle()
    S.batch_destroy(srv.batch)


def test_particle_limit_of_one_engine_on_host():
    # an engine with neighbour lists holds at most 2^26 particles: a request
    # above the server's limit is rejected, and admission keeps the sum of
    # the residents' particles under it
    spec = sphcases.small_droplet(2, 16)
    srv = serve.Server(budget_bytes=1e12, max_particles=spec.n - 1)
    with pytest.raises(S.SphstError):
        srv.submit(spec, n_adv=1).result(timeout=1)
    assert serve.Server.__init__.__defaults__[-1] == S.MAX_LIST_ENGINE_PARTICLES == 1 << 26
    S.batch_destroy(srv.batch)


def test_loop_error_fails_every_waiting_request():
    srv = serve.Server(budget_bytes=1e12)
    futs = [srv.submit(sphcases.small_droplet(2, 12), n_adv=1) for _ in range(3)]
    err = S.SphstError(-5, "device lost")
    srv.fail_all(err)
    for f in futs:
        with pytest.raises(S.SphstError):
            f.result(timeout=1)
    with pytest.raises(S.SphstError):                 # later requests fail at once
        srv.submit(sphcases.small_droplet(2, 12), n_adv=1).result(timeout=1)
    assert not srv.queue
    S.batch_destroy(srv.batch)


def test_footprint_orders_requests():
    srv = serve.Server(budget_bytes=1e12)
    small = srv.footprint(sphcases.small_droplet(2, 12))
    big = srv.footprint(sphcases.small_droplet(3, 20))
    assert 0 < small < big
    S.batch_destroy(srv.batch)


@pytest.mark.gpu
def test_results_equal_alone_and_in_the_mix():
    specs = [sphcases.small_droplet(2, 20, R_frac=0.3, seed=1, jitter=0.1, vel_amp=0.02),
             sphcases.small_droplet(3, 10, R_frac=0.3, seed=2, jitter=0.1, vel_amp=0.02),
             sphcases.small_droplet(2, 26, R_frac=0.25, shape="square", sigma=0.5),
             sphcases.small_droplet(3, 12, R_frac=0.3, shape="mode2", amp=0.15)]
    steps = [3, 2, 4, 2]
    srv = serve.Server(budget_bytes=1e11)
    srv.start()
    futs = []
    for s, n in zip(specs, steps):          # staggered arrivals while others run
        futs.append(srv.submit(s, n_adv=n))
        time.sleep(0.01)
    results = [f.result(timeout=120) for f in futs]
    srv.stop()
    st = srv.stats()
    srv.close()
    assert st["completed"] == 4 and st["p99_s"] >= st["p50_s"] > 0
    for s, n, r in zip(specs, steps, results):
        h = S.case_from_spec(s)
        S.step(h, n)
        for f in (S.FIELD_POS, S.FIELD_VEL, S.FIELD_RHO):
            assert np.array_equal(r.fields[f], S.read_fields(h, f, s.dim))
        assert r.info["n_adv"] == n
        S.destroy(h)


@pytest.mark.gpu
def test_admission_waits_for_memory():
    a = sphcases.small_droplet(2, 20)
    srv = serve.Server(budget_bytes=1e12)
    one = srv.footprint(a)
    srv.budget = 1.5 * one                   # room for one resident case
    f1 = srv.submit(a, n_adv=2)
    f2 = srv.submit(a, n_adv=2)
    srv.step()
    assert len(srv.members) == 1 and len(srv.queue) == 1
    srv.run_until_idle(timeout=60)
    r1, r2 = f1.result(), f2.result()
    assert r2.admitted >= r1.finished
    for f in (S.FIELD_POS, S.FIELD_VEL):
        assert np.array_equal(r1.fields[f], r2.fields[f])
    srv.close()


@pytest.mark.gpu
def test_substep_stopping_rule():
    # a request that asks for n acoustic substeps retires at the first
    # advection-step boundary with at least n substeps done
    a = sphcases.small_droplet(2, 20)
    srv = serve.Server(budget_bytes=1e12)
    f = srv.submit(a, n_sub=40)
    srv.run_until_idle(timeout=60)
    r = f.result()
    assert r.info["n_sub"] >= 40
    h = S.case_from_spec(a)
    n_adv = r.info["n_adv"]
    S.step(h, n_adv - 1)
    assert S.case_info(h)["n_sub"] < 40          # one advection step fewer is not enough
    S.step(h, 1)
    assert np.array_equal(r.fields[S.FIELD_POS], S.read_fields(h, S.FIELD_POS, 2))
    S.destroy(h)
    srv.close()


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol1,tol2", [(64, 1e-12, 1e-11), (32, 2e-4, 1e-3)])
def test_served_results_equal_the_oracle(precision, tol1, tol2):
    """Seeded cases of the batched workload (seed 20250320, 2D, all three
    shapes, sigma 0.12-3.9) served with a memory budget that holds two at a
    time, so later requests are admitted while others run; every result is
    compared with the FP64 oracle's run of that case alone (fluid
    particles, each field against its maximum)."""
    import oracle

    idx = (192, 481, 89, 153, 437, 64)
    specs = [sphcases.batch_cases(512)[k].build() for k in idx]
    steps = [1, 2, 1, 2, 1, 1]
    srv = serve.Server(precision=precision, budget_bytes=1e12,
                       fields=(S.FIELD_POS, S.FIELD_VEL, S.FIELD_RHO, S.FIELD_GRADC))
    srv.budget = 2.2 * max(srv.footprint(s) for s in specs)
    srv.start()
    futs = []
    for s, n in zip(specs, steps):
        futs.append(srv.submit(s, n_adv=n))
        time.sleep(0.005)
    results = [f.result(timeout=300) for f in futs]
    srv.stop()
    srv.close()
    assert any(r.admitted > min(q.finished for q in results) for r in results)   # admitted mid-run
    for s, n, r in zip(specs, steps, results):
        assert r.info["status"] == 0 and r.info["n_adv"] == n
        pos, vel, rho, kind = s.flat()
        p1, v1, r1, oinfo, gC, _ = oracle.run(oracle.params_for_case(s), pos, vel, rho, kind, n)
        assert r.info["n_sub"] == oinfo["n_sub"]
        fl = kind < 2
        rho0 = np.asarray(s.fluid_props()[0])[kind[fl]]
        d = s.dim
        pairs = [(r.fields[S.FIELD_POS][fl] - pos[fl, :d], p1[fl, :d] - pos[fl, :d]),
                 (r.fields[S.FIELD_VEL][fl], v1[fl, :d]),
                 (r.fields[S.FIELD_RHO][fl] - rho0, r1[fl] - rho0),
                 (r.fields[S.FIELD_GRADC][fl], gC[fl, :d])]
        tol = tol1 if n == 1 else tol2
        for a, b in pairs:
            scale = np.abs(b).max()
            assert np.abs(a - b).max() <= tol * scale + 4 * np.spacing(1000.0)
