"""FP64 device diagnostics (sphst_diagnose) against the same sums computed on
the host from read-back fields: momentum, kinetic energy, phase counts, the
drop's first and second moments, Laplace sampling sums; repeated calls give
identical bits; before the first step the staged input is reduced."""
import numpy as np
import pytest

import sphcases

pytestmark = pytest.mark.gpu

S = pytest.importorskip("paper_2503_16082_gb300")
from paper_2503_16082_gb300 import observables as ob  # noqa: E402


def host_sums(h, case, center, r_in, r_out):
    dim = case.dim
    pos = S.read_fields(h, S.FIELD_POS, dim)
    vel = S.read_fields(h, S.FIELD_VEL, dim)
    p = S.read_fields(h, S.FIELD_PRESSURE, dim)
    ph = S.read_fields(h, S.FIELD_PHASE, dim).astype(int)
    rho0 = np.asarray(case.fluid_props()[0])
    fl = ph < 2
    x = np.zeros((len(pos), 3))
    x[:, :dim] = pos
    v = np.zeros((len(pos), 3))
    v[:, :dim] = vel
    m = np.where(fl, rho0[np.minimum(ph, 1)], 0.0) * case.dx ** dim
    r2 = ((x[:, :dim] - np.asarray(center)[:dim]) ** 2).sum(1)
    d0 = ph == 0
    out = {"momentum": (m[:, None] * v).sum(0), "kinetic": 0.5 * (m * (v ** 2).sum(1)).sum(),
           "count": [int(d0.sum()), int((ph == 1).sum())], "first": x[d0].sum(0),
           "second": [(x[d0, a] * x[d0, b]).sum() for a, b in ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))],
           "p_in": p[d0 & (r2 < r_in ** 2)].sum(), "n_in": int((d0 & (r2 < r_in ** 2)).sum()),
           "p_out": p[(ph == 1) & (r2 > r_out ** 2)].sum(), "n_out": int(((ph == 1) & (r2 > r_out ** 2)).sum())}
    scale = {"momentum": (m[:, None] * np.abs(v)).sum(), "kinetic": out["kinetic"],
             "first": np.abs(x[d0]).sum(), "second": (x[d0] ** 2).sum(), "p_in": np.abs(p).sum(),
             "p_out": np.abs(p).sum()}
    return out, scale


@pytest.mark.parametrize("dim,precision", [(2, 64), (3, 32), (3, 64)])
def test_diagnostics_equal_host_sums(dim, precision):
    case = sphcases.small_droplet(dim, 24 if dim == 2 else 12, R_frac=0.3, shape="mode2", amp=0.15,
                                  seed=5, jitter=0.1, vel_amp=0.05)
    h = S.case_from_spec(case, precision=precision)
    S.step(h, 2)
    center = (0.5, 0.5, 0.5)
    r_in, r_out = 0.12, 0.35
    dg = S.diagnose(h, center, r_in, r_out)
    again = S.diagnose(h, center, r_in, r_out)
    ref, scale = host_sums(h, case, center, r_in, r_out)
    S.destroy(h)
    assert dg == again                                   # fixed summation order
    assert dg["count"] == ref["count"] and dg["n_in"] == ref["n_in"] and dg["n_out"] == ref["n_out"]
    assert dg["n_nonfinite"] == 0
    assert dg["n_in"] > 0 and dg["n_out"] > 0
    for k in ("momentum", "kinetic", "first", "second", "p_in", "p_out"):
        err = np.abs(np.asarray(dg[k]) - np.asarray(ref[k])).max()
        assert err <= 1e-13 * scale[k] + 1e-300, k


def test_diagnostics_before_first_step_and_device_observables():
    case = sphcases.small_droplet(2, 30, R_frac=0.25, seed=3, jitter=0.1)
    h = S.case_from_spec(case, precision=64)
    staged = S.diagnose(h, (0.5, 0.5), 0.1, 0.3)
    ref, scale = host_sums(h, case, (0.5, 0.5, 0.5), 0.1, 0.3)
    assert staged["count"] == ref["count"] and staged["n_in"] == ref["n_in"]
    assert np.abs(np.asarray(staged["first"]) - ref["first"]).max() <= 1e-13 * scale["first"]
    S.step(h, 3)
    pos = S.read_fields(h, S.FIELD_POS, 2)
    p = S.read_fields(h, S.FIELD_PRESSURE, 2)
    ph = S.read_fields(h, S.FIELD_PHASE, 2)
    hsz = case.h_factor * case.dx
    dp_host, R_host = ob.laplace_jump(pos, p, ph, case.dx, hsz)
    dp_dev, R_dev = ob.laplace_jump_device(h, 2, case.dx, hsz)
    assert R_dev == R_host
    assert abs(dp_dev - dp_host) <= 1e-10 * max(abs(dp_host), 1e-12)
    an_host = ob.anisotropy(pos, ph)
    an_dev = ob.anisotropy_device(h, 2)
    # device moments are sum(x^2)/n - c^2: rounding of order eps * |x|^2
    x0 = pos[ph == 0]
    assert abs(an_dev - an_host) <= 1e-12 * float((x0 ** 2).mean())
    S.destroy(h)


def test_fma_peak_is_plausible():
    # 152 SMs x 128 FP32 lanes x 2 flop x ~2 GHz ~ 80 TFLOP/s; FP64 far lower
    f32 = S.fma_peak(32)["tflops"]
    f64 = S.fma_peak(64)["tflops"]
    assert 20.0 < f32 < 200.0, f32
    assert 0.05 < f64 < f32, f64
