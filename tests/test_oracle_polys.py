"""Pins for the oracle's 1D polynomial tools against library routines and closed forms."""
import numpy as np
import pytest

from oracle.polys import (gauss_legendre, jacobi, jacobi_norm, lagrange_matrix, legendre,
                          radau_left, radau_left_deriv)


@pytest.mark.parametrize("n", range(1, 9))
def test_gauss_legendre_matches_numpy(n):
    x, w = gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.allclose(x, xr, atol=1e-14, rtol=0)
    assert np.allclose(w, wr, atol=1e-14, rtol=0)


@pytest.mark.parametrize("k", range(0, 7))
def test_legendre_matches_numpy(k):
    x = np.linspace(-1, 1, 17)
    ref = np.polynomial.legendre.legval(x, [0] * k + [1])
    assert np.allclose(legendre(k, x), ref, atol=1e-14)


@pytest.mark.parametrize("a,b", [(0, 0), (1, 0), (3, 0), (5, 0), (1, 1)])
def test_jacobi_orthogonality(a, b):
    xq, wq = np.polynomial.legendre.leggauss(30)
    wt = wq * (1 - xq) ** a * (1 + xq) ** b
    G = np.array([[np.sum(wt * jacobi(m, a, b, xq) * jacobi(n, a, b, xq)) for n in range(6)]
                  for m in range(6)])
    assert np.allclose(G, np.diag([jacobi_norm(m, a, b) for m in range(6)]), atol=1e-12)


@pytest.mark.parametrize("p", range(1, 7))
def test_lagrange_cardinal_and_exact_derivative(p):
    x, _ = gauss_legendre(p + 1)
    assert np.allclose(lagrange_matrix(x, x), np.eye(p + 1), atol=1e-14)
    y = np.linspace(-1, 1, 11)
    B = lagrange_matrix(x, y)
    dB = lagrange_matrix(x, y, deriv=True)
    for k in range(p + 1):
        assert np.allclose(B @ x ** k, y ** k, atol=1e-12)
        dk = k * y ** (k - 1) if k > 0 else 0 * y
        assert np.allclose(dB @ x ** k, dk, atol=1e-11)


@pytest.mark.parametrize("p", range(1, 7))
def test_radau_closed_form(p):
    assert radau_left(p, np.array([-1.0]))[0] == pytest.approx(1.0, abs=1e-14)
    assert radau_left(p, np.array([1.0]))[0] == pytest.approx(0.0, abs=1e-14)
    # degree p+1: a (p+2)-point fit reproduces it exactly
    xs = np.linspace(-1, 1, 25)
    c = np.polynomial.polynomial.polyfit(xs, radau_left(p, xs), p + 3)
    assert np.allclose(c[p + 2:], 0, atol=1e-10)
    assert abs(c[p + 1]) > 1e-3


@pytest.mark.parametrize("p", range(1, 7))
def test_radau_derivative_is_dg_lift(p):
    """Huynh: with g_L the right Radau polynomial, FR recovers nodal DG on
    Gauss-Legendre points, whose lift is -l_i(-1)/w_i."""
    x, w = gauss_legendre(p + 1)
    lm1 = lagrange_matrix(x, np.array([-1.0]))[0]
    assert np.allclose(radau_left_deriv(p, x), -lm1 / w, atol=1e-11)
