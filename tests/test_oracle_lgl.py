"""Pins of the oracle's LGL nodes, weights and derivative matrix (not GPU)."""
import numpy as np
import pytest

from golden_io import read, values
from oracle.lgl import lgl


def test_closed_forms():
    for row in read("lgl_closed_forms.txt"):
        N, what, vals = int(row[0]), row[1], values(row[2:])
        x, w, D = lgl(N)
        ref = {"nodes": x, "weights": w, "D": D.ravel()}[what]
        np.testing.assert_allclose(ref, vals, rtol=0, atol=1e-14)


@pytest.mark.parametrize("N", range(1, 9))
def test_derivative_exact_on_polynomials(N):
    x, w, D = lgl(N)
    for p in range(N + 1):
        dp = p * x ** (p - 1) if p > 0 else np.zeros_like(x)
        np.testing.assert_allclose(D @ x ** p, dp, atol=2e-12 * N * N)


@pytest.mark.parametrize("N", range(1, 9))
def test_quadrature_exact_to_2N_minus_1(N):
    x, w, D = lgl(N)
    assert abs(w.sum() - 2.0) < 1e-14
    for p in range(2 * N):
        exact = (1.0 - (-1.0) ** (p + 1)) / (p + 1)
        assert abs(w @ x ** p - exact) < 1e-13
    # and not exact at degree 2N (LGL, not Gauss)
    exact = 2.0 / (2 * N + 1)
    assert abs(w @ x ** (2 * N) - exact) > 1e-6


@pytest.mark.parametrize("N", range(1, 9))
def test_centro_antisymmetry(N):
    x, w, D = lgl(N)
    np.testing.assert_allclose(x, -x[::-1], atol=1e-15)
    np.testing.assert_allclose(D, -D[::-1, ::-1], atol=1e-12 * N * N)
