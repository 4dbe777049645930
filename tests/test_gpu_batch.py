"""Batched stepping: many independent cases in one engine (segmented cell
table, per-case time steps, one graph per advection step).  Every case must
give the same result alone and inside a batch -- bitwise, since each
particle's sums run over the same neighbours in the same order -- and a
failing case must not disturb the others."""
import numpy as np
import pytest

import sphcases

pytestmark = pytest.mark.gpu

S = pytest.importorskip("paper_2503_16082_gb300")

FIELDS = (S.FIELD_POS, S.FIELD_VEL, S.FIELD_RHO, S.FIELD_GRADC)


def specs():
    out = [sphcases.small_droplet(2, 20, R_frac=0.3, seed=1, jitter=0.1, vel_amp=0.02),
           sphcases.small_droplet(3, 10, R_frac=0.3, seed=2, jitter=0.1, vel_amp=0.02),
           sphcases.small_droplet(2, 28, R_frac=0.25, shape="square", sigma=0.5),
           sphcases.small_droplet(3, 12, R_frac=0.3, shape="mode2", amp=0.15, sigma=2.0)]
    return out


def alone(spec, n_adv, precision=32, **kw):
    h = S.case_from_spec(spec, precision=precision, **kw)
    S.step(h, n_adv)
    res = [S.read_fields(h, f, spec.dim) for f in FIELDS], S.case_info(h)
    S.destroy(h)
    return res


def fields_of(h, spec):
    return [S.read_fields(h, f, spec.dim) for f in FIELDS]


@pytest.mark.parametrize("precision,lanes,work", [(32, 1, 0), (64, 1, 0), (32, 4, 0), (32, 1, 1), (64, 4, 1)])
def test_batch_equals_alone(precision, lanes, work):
    # with L lanes per particle too: each particle's partial sums and their
    # reduction are the same alone and in the batch; and with the batch's
    # work lists (active members' tiles listed each substep), whose cases
    # here take different substep counts per advection step
    sp = specs()
    ref = [alone(s, 2, precision, lanes=lanes) for s in sp]
    b = S.batch_create(precision)
    hs = [S.case_from_spec(s, precision=precision, lanes=lanes, work_lists=work) for s in sp]
    for h in hs:
        S.batch_add(b, h)
    S.batch_step(b, 1)
    S.batch_step(b, 1)
    for h, s, (rf, ri) in zip(hs, sp, ref):
        info = S.case_info(h)
        assert info["n_adv"] == 2 and info["n_sub"] == ri["n_sub"] and info["t"] == ri["t"]
        for a, c in zip(fields_of(h, s), rf):
            assert np.array_equal(a, c)
    for h in hs:
        S.batch_remove(b, h)
        S.destroy(h)
    S.batch_destroy(b)


def test_batch_membership_changes():
    sp = specs()
    b = S.batch_create(32)
    h0 = S.case_from_spec(sp[0])
    h1 = S.case_from_spec(sp[1])
    S.batch_add(b, h0)
    S.batch_step(b, 1)                 # h0: 1 step
    S.batch_add(b, h1)                 # joins at the next step
    S.batch_step(b, 1)                 # h0: 2, h1: 1
    S.batch_remove(b, h0)
    S.step(h0, 1)                      # h0 continues alone: 3
    S.batch_step(b, 1)                 # h1: 2
    assert S.case_info(h0)["n_adv"] == 3 and S.case_info(h1)["n_adv"] == 2
    r0, _ = alone(sp[0], 3)
    r1, _ = alone(sp[1], 2)
    for a, c in zip(fields_of(h0, sp[0]), r0):
        assert np.array_equal(a, c)
    for a, c in zip(fields_of(h1, sp[1]), r1):
        assert np.array_equal(a, c)
    S.batch_remove(b, h1)
    S.batch_destroy(b)
    S.destroy(h0)
    S.destroy(h1)


def test_failing_member_does_not_disturb_others():
    sp = specs()[:2]
    # two particles at the same position: the neighbour search flags the case
    bad = sphcases.small_droplet(2, 16, R_frac=0.3)
    liq = bad.phases[0]
    liq.pos = np.concatenate([liq.pos, liq.pos[:1]])
    b = S.batch_create(32)
    hs = [S.case_from_spec(s) for s in sp]
    hb = S.case_from_spec(bad)
    for h in (hs[0], hb, hs[1]):
        S.batch_add(b, h)
    for _ in range(3):
        S.batch_step(b, 1)
    assert S.case_info(hb)["status"] == S.ERR_COINCIDENT
    for h, s in zip(hs, sp):
        ref, info = alone(s, 3)
        assert S.case_info(h)["status"] == 0 and S.case_info(h)["n_adv"] == 3
        for a, c in zip(fields_of(h, s), ref):
            assert np.array_equal(a, c)
    for h in hs + [hb]:
        S.batch_remove(b, h)
        S.destroy(h)
    S.batch_destroy(b)
