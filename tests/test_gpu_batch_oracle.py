"""Batched members against the FP64 oracle (not against the CUDA path
itself): seeded cases of the 512-case batched workload (seed 20250320),
chosen among those the oracle finishes in seconds, 2D and 3D, all three
shapes, surface tension from 0.12 to 9, stepped together in one engine
(segmented cell table, per-case time steps, one graph per advection step)
and each compared field by field with the oracle run of that case alone.

Bars (the single-case bars): FP64 <= 1e-12 of each field's maximum after one
acoustic substep and after one whole advection step; FP32 <= 1e-5 after one
substep and <= 2e-4 after a whole advection step.  One member of the seeded
batch (index 313) blows up; both sides must fail at the same advection
step."""
import numpy as np
import pytest

import oracle
import sphcases

pytestmark = pytest.mark.gpu

S = pytest.importorskip("paper_2503_16082_gb300")

# (index in batch_cases(512), dim, shape, sigma) -- the oracle's substeps per
# advection step at rest range from 49 (192) to 195 (461)
ONE_SUBSTEP = (192, 481, 89, 153, 437, 64, 264, 461, 149, 1, 16, 82)
ONE_STEP = (192, 481, 89, 153, 437, 64, 461)
FIELDS = {"pos": S.FIELD_POS, "vel": S.FIELD_VEL, "rho": S.FIELD_RHO, "gradC": S.FIELD_GRADC,
          "acc_visc": S.FIELD_ACC_VISC}


def members(indices):
    specs = sphcases.batch_cases(512)
    return [specs[k].build() for k in indices]


def oracle_fields(case, max_substeps):
    pos, vel, rho, kind = case.flat()
    P = oracle.params_for_case(case, max_substeps=max_substeps)
    p1, v1, r1, info, gC, av = oracle.run(P, pos, vel, rho, kind, 1)
    d = case.dim
    return {"pos": p1[:, :d], "vel": v1[:, :d], "rho": r1, "gradC": gC[:, :d], "acc_visc": av[:, :d]}, info


def position_resolution(case, precision):
    """A few units of the last place of a stored position: of |x| in FP64,
    of an offset inside a 2h-wide cell in FP32 (positions are kept as FP32
    offsets from their cell's origin)."""
    if precision == 64:
        return 4 * np.spacing(max(abs(v) for v in list(case.lo) + list(case.hi)))
    return 4 * float(np.spacing(np.float32(2.0 * case.h_factor * case.dx)))


def compare(case, got, ref, tol, precision):
    """Each field of the fluid particles against its maximum; displacements
    also carry the resolution of a stored position (a case at rest moves
    ~1e-6 in one substep)."""
    pos0, _, _, kind = case.flat()
    fl = kind < 2
    rho0 = np.asarray(case.fluid_props()[0])[kind[fl]]
    for key in FIELDS:
        a, b = got[key][fl], ref[key][fl]
        slack = 0.0
        if key == "pos":
            a, b = a - pos0[fl, :case.dim], b - pos0[fl, :case.dim]
            slack = position_resolution(case, precision)
        if key == "rho":
            a, b = a - rho0, b - rho0
            slack = 4 * np.spacing(1000.0)
        scale = np.abs(b).max()
        err = np.abs(a - b).max()
        if scale == 0.0:
            assert err == 0.0, (case.name, key)
            continue
        assert err <= tol * scale + slack, (case.name, key, err / scale)


def run_batch(cases, precision, lanes, max_substeps):
    kw = dict(lanes=lanes, max_substeps=max_substeps)
    hs = [S.case_from_spec(c, precision=precision, max_neighbors=192 if c.dim == 3 else 0, **kw)
          for c in cases]
    b = S.batch_create(precision)
    try:
        for h in hs:
            S.batch_add(b, h)
        S.batch_step(b, 1)
        out = []
        for h, c in zip(hs, cases):
            out.append(({k: S.read_fields(h, f, c.dim) for k, f in FIELDS.items()}, S.case_info(h)))
    finally:
        for h in hs:
            S.batch_remove(b, h)
            S.destroy(h)
        S.batch_destroy(b)
    return out


@pytest.fixture(scope="module")
def oracle_one_substep():
    cases = members(ONE_SUBSTEP)
    return cases, [oracle_fields(c, 1) for c in cases]


@pytest.fixture(scope="module")
def oracle_one_step():
    cases = members(ONE_STEP)
    return cases, [oracle_fields(c, 0) for c in cases]


def test_members_span_the_workload():
    cases = members(ONE_SUBSTEP)
    specs = [c.meta["spec"] for c in cases]
    assert {s["dim"] for s in specs} == {2, 3}
    assert {s["shape"] for s in specs} == {"square", "mode2", "mode3"}
    sig = [s["sigma"] for s in specs]
    assert min(sig) < 0.15 and max(sig) > 8.0


@pytest.mark.parametrize("precision,lanes,tol", [(64, 1, 1e-12), (32, 1, 1e-5), (32, 4, 1e-5), (64, 4, 1e-12)])
def test_batch_one_substep_equals_oracle(oracle_one_substep, precision, lanes, tol):
    cases, refs = oracle_one_substep
    got = run_batch(cases, precision, lanes, max_substeps=1)
    for c, (g, info), (o, oinfo) in zip(cases, got, refs):
        assert info["n_sub"] == oinfo["n_sub"] == 1, c.name
        compare(c, g, o, tol, precision)


@pytest.mark.parametrize("precision,lanes,tol", [(64, 1, 1e-12), (32, 1, 2e-4), (64, 4, 1e-12)])
def test_batch_one_advection_step_equals_oracle(oracle_one_step, precision, lanes, tol):
    cases, refs = oracle_one_step
    got = run_batch(cases, precision, lanes, max_substeps=0)
    for c, (g, info), (o, oinfo) in zip(cases, got, refs):
        assert info["status"] == 0 and oinfo["status"] == 0, c.name
        assert info["n_sub"] == oinfo["n_sub"] > 40, c.name
        compare(c, g, o, tol, precision)


def test_diverging_member_fails_at_the_same_step_as_the_oracle():
    """Member 313 (3D square drop, 8000 particles, sigma 6.65): at rest the
    advection criterion of Eq. 16 has only its viscous term, so its first
    advection step holds one frozen configuration for 686 acoustic
    substeps while the drop relaxes, and the second step blows up on both
    sides.  Failure: a non-zero status or a fluid speed above the sound
    speed c0 (the weakly compressible model no longer holds)."""
    case = members((313,))[0]
    pos, vel, rho, kind = case.flat()
    fl = kind < 2
    P = oracle.params_for_case(case)

    def failed(status, v):
        return status != 0 or not np.all(np.isfinite(v)) or np.abs(v).max() > case.c0

    o_fail = None
    p, v, r = pos, vel, rho
    for step in (1, 2, 3):
        p, v, r, info, _, _ = oracle.run(P, p, v, r, kind, 1)
        if failed(info["status"], v[fl]):
            o_fail = step
            break
    assert o_fail == 2
    for precision in (64, 32):
        h = S.case_from_spec(case, precision=precision, max_neighbors=192)
        g_fail = None
        try:
            for step in (1, 2, 3):
                info = S.step(h, 1, check=False)
                gv = S.read_fields(h, S.FIELD_VEL, 3)[fl]
                if failed(info["status"], gv):
                    g_fail = step
                    break
        finally:
            S.destroy(h)
        assert g_fail == o_fail, (precision, g_fail, o_fail)
