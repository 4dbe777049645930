"""Checkpoint and resume at an advection-step boundary: the fields read back
(positions, velocities and densities in FP64, insertion order) are all the
state a case carries between advection steps, since the frozen configuration
(neighbours, correction matrices, viscous force, band) is rebuilt at the
start of every advection step.  A case re-created from them and stepped on
matches the uninterrupted run to the rounding of the position encoding (the
new case lays its own cell grid over the moved particles)."""
import dataclasses

import numpy as np
import pytest

import sphcases

pytestmark = pytest.mark.gpu

S = pytest.importorskip("paper_2503_16082_gb300")

FIELDS = (S.FIELD_POS, S.FIELD_VEL, S.FIELD_RHO)


def resumed_spec(spec, h):
    """The spec with each phase's positions, velocities and densities
    replaced by the case's current ones (insertion order: phase by phase)."""
    pos = S.read_fields(h, S.FIELD_POS, spec.dim)
    vel = S.read_fields(h, S.FIELD_VEL, spec.dim)
    rho = S.read_fields(h, S.FIELD_RHO, spec.dim)
    phases, o = [], 0
    for ph in spec.phases:
        n = len(ph.pos)
        if ph.kind == "fluid":
            phases.append(dataclasses.replace(ph, pos=pos[o:o + n].copy(), vel=vel[o:o + n].copy(),
                                              rho=rho[o:o + n].copy()))
        else:
            phases.append(dataclasses.replace(ph, pos=pos[o:o + n].copy()))
        o += n
    return dataclasses.replace(spec, phases=phases)


@pytest.mark.parametrize("precision,bar", [(64, 1e-10), (32, 2e-4)])
def test_resume_at_an_advection_boundary(precision, bar):
    spec = sphcases.small_droplet(2, 24, R_frac=0.3, seed=3, jitter=0.1, vel_amp=0.05)
    h = S.case_from_spec(spec, precision=precision)
    S.step(h, 4)
    full = [S.read_fields(h, f, spec.dim) for f in FIELDS]
    full_sub = S.case_info(h)["n_sub"]
    S.destroy(h)

    h = S.case_from_spec(spec, precision=precision)
    S.step(h, 2)
    sub_a = S.case_info(h)["n_sub"]
    again = resumed_spec(spec, h)
    S.destroy(h)
    h = S.case_from_spec(again, precision=precision)
    S.step(h, 2)
    resumed = [S.read_fields(h, f, spec.dim) for f in FIELDS]
    assert sub_a + S.case_info(h)["n_sub"] == full_sub
    S.destroy(h)
    for a, b in zip(full, resumed):
        scale = np.abs(a).max()
        assert np.abs(a - b).max() <= bar * scale, (np.abs(a - b).max(), scale)
