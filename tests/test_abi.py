"""CPU checks of the C ABI: the library builds and loads, exports every
function that include/sphst.h declares, and validates arguments on the host
(no call here needs a GPU)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import sphcases

S = pytest.importorskip("paper_2503_16082_gb300")

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "sphst.h")


def declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(sphst_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    lib = S.load()
    names = declared()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    # and the binding knows all of them
    assert set(names) <= set(S.EXPORTS)


def test_device_info_validates_on_the_host():
    # NULL outputs are rejected before any device call
    assert S.load().sphst_device_info(None, None, None, None) == S.ERR_INVALID_ARG


def test_struct_layout_matches_the_binding():
    sizes = [C.c_int64() for _ in range(3)]
    assert S.load().sphst_struct_sizes(*[C.byref(v) for v in sizes]) == S.OK
    assert [v.value for v in sizes] == [C.sizeof(S.CaseParams), C.sizeof(S.PhaseProps), C.sizeof(S.StepInfo)]


def test_default_params_and_validation():
    p = S.default_params(dx=0.01)
    assert p.dim == 2 and p.precision == 32 and p.h_factor == 1.3 and p.tvf_alpha == 0.2
    assert p.lanes == 1 and p.block == 128
    for bad in (dict(dx=0.0), dict(dx=0.01, c0=-1.0), dict(dx=0.01, gamma=-1.0),
                dict(dx=0.01, block=48), dict(dx=0.01, limiter=7), dict(dx=0.01, grid_pad=0),
                dict(dx=0.01, lanes=3), dict(dx=0.01, lanes=16), dict(dx=0.01, penalty_scope=2), dict(dx=0.01, block=512)):
        with pytest.raises(S.SphstError) as e:
            S.create_case(S.default_params(**bad))
        assert e.value.code == S.ERR_INVALID_ARG
    with pytest.raises(S.SphstError) as e:
        S.create_case(S.default_params(dx=0.01, dim=4))
    assert e.value.code == S.ERR_UNSUPPORTED


def test_staged_case_reads_back_and_rejects_third_fluid():
    case = sphcases.small_droplet(2, 12)
    h = S.case_from_spec(case)
    try:
        n, nf = S.num_particles(h)
        assert n == case.n and nf == case.n_fluid
        pos = S.read_fields(h, S.FIELD_POS, 2)
        assert np.array_equal(pos, case.flat()[0][:, :2])
        buf = np.full(2 * case.n + 5, np.nan)             # a caller's buffer, larger than needed
        got = S.read_fields(h, S.FIELD_POS, 2, out=buf)
        assert np.array_equal(got, pos) and np.shares_memory(got, buf) and np.isnan(buf[-1])
        with pytest.raises(ValueError):
            S.read_fields(h, S.FIELD_POS, 2, out=np.zeros(case.n))
        ph = S.read_fields(h, S.FIELD_PHASE, 2)
        assert sorted(set(ph.tolist())) == [0.0, 1.0, 2.0]
        p = S.read_fields(h, S.FIELD_PRESSURE, 2)
        assert np.all(p == 0.0)
        with pytest.raises(S.SphstError) as e:
            S.add_phase_particles(h, S.FLUID, np.zeros((1, 2)) + 0.5, rho0=2.0, eta=1.0)
        assert e.value.code == S.ERR_UNSUPPORTED
        with pytest.raises(S.SphstError) as e:
            S.add_phase_particles(h, S.WALL, np.full((1, 2), np.nan))
        assert e.value.code == S.ERR_INVALID_ARG
        out = np.zeros(3)
        rc = S.load().sphst_read_fields(h, S.FIELD_POS, out.ctypes.data, 3)
        assert rc == S.ERR_CAPACITY
    finally:
        S.destroy(h)
    assert S.load().sphst_destroy(None) == S.OK


def test_case_without_fluid_cannot_step():
    # an empty case, and one holding only walls, are rejected on the host
    for walls in (False, True):
        h = S.create_case(S.default_params(dx=0.1))
        try:
            if walls:
                S.add_phase_particles(h, S.WALL, np.array([[0.05, 0.05], [0.15, 0.05]]))
            info = S.step(h, 1, check=False)
            assert info["rc"] == S.ERR_STATE
            assert "no fluid" in S.last_error()
        finally:
            S.destroy(h)


def test_batch_bookkeeping_on_host():
    b = S.batch_create(32)
    cases = [S.case_from_spec(sphcases.small_droplet(2, 10)) for _ in range(3)]
    for h in cases:
        S.batch_add(b, h)
    assert S.batch_size(b) == 3
    with pytest.raises(S.SphstError) as e:
        S.batch_add(b, cases[0])
    assert e.value.code == S.ERR_STATE
    with pytest.raises(S.SphstError) as e:
        S.step(cases[1], 1)
    assert e.value.code == S.ERR_STATE
    with pytest.raises(S.SphstError) as e:
        S.destroy(cases[2])
    assert e.value.code == S.ERR_STATE
    h64 = S.case_from_spec(sphcases.small_droplet(2, 10), precision=64)
    with pytest.raises(S.SphstError) as e:
        S.batch_add(b, h64)
    assert e.value.code == S.ERR_UNSUPPORTED
    S.batch_remove(b, cases[2])
    assert S.batch_size(b) == 2
    S.batch_destroy(b)
    for h in cases + [h64]:
        S.destroy(h)


def test_footprint_grows_with_size():
    p = S.default_params(dx=0.01, dim=3)
    a = S.footprint_bytes(p, 10_000)
    b = S.footprint_bytes(p, 1_000_000)
    assert 100 * 10_000 < a < b
    p64 = S.default_params(dx=0.01, dim=3, precision=64)
    assert S.footprint_bytes(p64, 1_000_000) > b
