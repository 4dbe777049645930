"""Pins of the oracle's Wendland C2 kernel (Section 5: h = 1.3 dp, support 2h)
against its defining properties: unit integral, vanishing at the support
edge, and dW/dr being the derivative of W."""
import math

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("h", [0.0325, 1.0, 0.7])
def test_kernel_integrates_to_one(dim, h):
    # Gauss-Legendre on [0, 2h] is exact for the polynomial W(r) r^(d-1)
    x, w = np.polynomial.legendre.leggauss(12)
    r = h * (x + 1.0)
    jac = h
    shell = 2 * math.pi * r if dim == 2 else 4 * math.pi * r * r
    total = sum(wi * oracle.kernel_W(dim, h, ri) * si for wi, ri, si in zip(w, r, shell)) * jac
    assert abs(total - 1.0) < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_kernel_edges_and_signs(dim):
    h = 0.5
    assert oracle.kernel_W(dim, h, 2 * h) == 0.0
    assert oracle.kernel_dW(dim, h, 2 * h) == 0.0
    assert oracle.kernel_W(dim, h, 3 * h) == 0.0
    assert oracle.kernel_dW(dim, h, 0.0) == 0.0
    for r in np.linspace(1e-3, 2 * h - 1e-3, 50):
        assert oracle.kernel_W(dim, h, r) > 0.0
        assert oracle.kernel_dW(dim, h, r) < 0.0


@pytest.mark.parametrize("dim", [2, 3])
def test_dW_is_derivative_of_W(dim):
    h, eps = 0.8, 1e-6
    for r in np.linspace(0.01, 1.59, 40):
        fd = (oracle.kernel_W(dim, h, r + eps) - oracle.kernel_W(dim, h, r - eps)) / (2 * eps)
        an = oracle.kernel_dW(dim, h, r)
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def test_kernel_scales_with_h():
    # W(r; h) = h^-d f(r/h): doubling h and r scales W by 2^-d
    for dim in (2, 3):
        for q in (0.1, 0.7, 1.5):
            a = oracle.kernel_W(dim, 1.0, q)
            b = oracle.kernel_W(dim, 2.0, 2 * q)
            assert abs(b - a / 2 ** dim) < 1e-14
