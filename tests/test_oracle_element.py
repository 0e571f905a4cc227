"""Pins for the oracle's reference elements: bases, operators and correction lift."""
import itertools
import math

import numpy as np
import pytest

from oracle.element import ref_element, _modal_tri, _modal_tensor
from oracle.polys import gauss_legendre, lagrange_matrix, radau_left_deriv

TYPES = [("quad", p) for p in range(1, 6)] + [("tri", p) for p in range(1, 6)] + \
        [("hex", p) for p in range(1, 4)]


def _monomials(etype, p, dim):
    """Exponent tuples spanning the element's polynomial space."""
    if etype == "tri":
        return [(i, j) for i in range(p + 1) for j in range(p + 1 - i)]
    return list(itertools.product(range(p + 1), repeat=dim))


def _eval_mono(x, e):
    return np.prod([x[:, c] ** e[c] for c in range(len(e))], axis=0)


def _grad_mono(x, e, a):
    if e[a] == 0:
        return np.zeros(x.shape[0])
    out = e[a] * x[:, a] ** (e[a] - 1)
    for c in range(len(e)):
        if c != a:
            out = out * x[:, c] ** e[c]
    return out


def _tri_quadrature(n):
    """Collapsed (Duffy) Gauss rule on the reference triangle, exact for high degree."""
    g, w = np.polynomial.legendre.leggauss(n)
    A, B = np.meshgrid(g, g, indexing="ij")
    WA, WB = np.meshgrid(w, w, indexing="ij")
    r = (1 + A) * (1 - B) / 2 - 1
    s = B
    wt = WA * WB * (1 - B) / 2
    return np.stack([r.ravel(), s.ravel()], 1), wt.ravel()


def test_tri_basis_orthonormal():
    x, w = _tri_quadrature(16)
    for p in range(1, 6):
        P, _, _ = _modal_tri(p, x)
        G = P.T @ (w[:, None] * P)
        assert np.allclose(G, np.eye(P.shape[1]), atol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_tensor_basis_orthonormal(dim):
    g, w = np.polynomial.legendre.leggauss(8)
    grids = np.meshgrid(*([g] * dim), indexing="ij")
    x = np.stack([m.ravel() for m in grids], 1)
    W = np.prod(np.stack(np.meshgrid(*([w] * dim), indexing="ij"), 0), 0).ravel()
    P, _, _ = _modal_tensor(4 if dim == 2 else 3, dim, x)
    assert np.allclose(P.T @ (W[:, None] * P), np.eye(P.shape[1]), atol=1e-12)


@pytest.mark.parametrize("etype,p", TYPES)
def test_interp_and_derivative_exact(etype, p):
    el = ref_element(etype, p)
    for e in _monomials(etype, p, el.dim):
        u = _eval_mono(el.xu, e)
        assert np.allclose(el.L @ u, _eval_mono(el.xf, e), atol=1e-11)
        for a in range(el.dim):
            assert np.allclose(el.D[a] @ u, _grad_mono(el.xu, e, a), atol=1e-10)


@pytest.mark.parametrize("etype,p", TYPES)
def test_solution_point_weights_integrate_exactly(etype, p):
    el = ref_element(etype, p)
    if etype == "tri":
        x, w = _tri_quadrature(12)
    else:
        g, w1 = np.polynomial.legendre.leggauss(10)
        grids = np.meshgrid(*([g] * el.dim), indexing="ij")
        x = np.stack([m.ravel() for m in grids], 1)
        w = np.prod(np.stack(np.meshgrid(*([w1] * el.dim), indexing="ij"), 0), 0).ravel()
    for e in _monomials(etype, p, el.dim):
        assert np.dot(el.wq, _eval_mono(el.xu, e)) == pytest.approx(np.dot(w, _eval_mono(x, e)), abs=1e-12)


@pytest.mark.parametrize("etype,p", TYPES)
def test_integration_by_parts_identity(etype, p):
    """For u, v in the element space: int (d_a u) v + int u (d_a v) = sum_faces int u v n_a,
    with the nodal mass matrix M = (V V^T)^{-1}, the face rule at the flux points and
    the reference normals.  Ties D, L, the face weights and normals together."""
    el = ref_element(etype, p)
    M = np.linalg.inv(el.V @ el.V.T)
    rng = np.random.default_rng(0)
    for _ in range(3):
        u = rng.normal(size=el.nu)
        v = rng.normal(size=el.nu)
        for a in range(el.dim):
            lhs = (el.D[a] @ u) @ M @ v + u @ M @ (el.D[a] @ v)
            rhs = np.sum(el.wf * el.nref[:, a] * (el.L @ u) * (el.L @ v))
            assert lhs == pytest.approx(rhs, abs=1e-11)


@pytest.mark.parametrize("etype,p", [t for t in TYPES if t[0] != "tri"])
def test_tensor_lift_equals_radau_correction(etype, p):
    """On tensor elements the lift column of a flux point on the face xi_a = -1 is
    -g_L'(xi) along the solution-point line through it and zero elsewhere; on
    xi_a = +1 it is g_R'(xi) = -g_L'(-xi)."""
    el = ref_element(etype, p)
    g, _ = gauss_legendre(p + 1)
    gl = radau_left_deriv(p, g)
    for k in range(el.nf):
        a = int(np.argmax(np.abs(el.nref[k])))
        sgn = el.nref[k, a]
        others = [c for c in range(el.dim) if c != a]
        col = np.zeros(el.nu)
        for i in range(el.nu):
            if np.allclose(el.xu[i, others], el.xf[k, others]):
                ia = int(np.argmin(np.abs(g - el.xu[i, a])))
                col[i] = -gl[ia] if sgn < 0 else -radau_left_deriv(p, -g)[ia]
        assert np.allclose(el.LIFT[:, k], col, atol=1e-10)


@pytest.mark.parametrize("etype,p", TYPES)
def test_flux_points_on_boundary_and_normals_unit(etype, p):
    el = ref_element(etype, p)
    assert np.allclose(np.linalg.norm(el.nref, axis=1), 1.0)
    if etype == "tri":
        on = (np.isclose(el.xf[:, 1], -1) | np.isclose(el.xf[:, 0], -1)
              | np.isclose(el.xf[:, 0] + el.xf[:, 1], 0))
    else:
        on = np.isclose(np.abs(el.xf).max(1), 1.0)
    assert on.all()
    # face weights add up to the reference boundary measure
    meas = {"quad": 8.0, "hex": 24.0, "tri": 4.0 + 2.0 * math.sqrt(2.0)}[etype]
    assert el.wf.sum() == pytest.approx(meas, rel=1e-13)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_triangle_points_symmetric_interior_positive(p):
    """The triangle's solution points (Blyth-Pozrikidis map of the 1D
    Gauss-Legendre nodes; of the Chebyshev nodes of the second kind,
    cos(k pi / (p + 2)), at p = 5): the set is invariant under the vertex
    permutations, interior, and its interpolatory weights int l_i are
    positive."""
    el = ref_element("tri", p)
    x = el.xu
    lam = np.stack([-(x[:, 0] + x[:, 1]) / 2, (1 + x[:, 0]) / 2, (1 + x[:, 1]) / 2], 1)
    assert lam.min() > 0.0
    key = lambda L: sorted(tuple(np.round(r, 12)) for r in L)
    for perm in itertools.permutations(range(3)):
        assert key(lam[:, perm]) == key(lam)
    assert el.wq.min() > 0.0 and el.wq.sum() == pytest.approx(2.0, rel=1e-14)
    # the smallest barycentric coordinate is the one of lattice index (0, 0, p):
    # (1 + 2 v_0 - v_0 - v_p) / 3 with v the 1D nodes on [0, 1]
    if p == 5:
        g = np.cos(np.arange(p + 1, 0, -1) * math.pi / (p + 2))   # the roots of U_{p+1}
        t = np.arccos(g)
        assert np.allclose(np.sin((p + 2) * t) / np.sin(t), 0.0, atol=1e-12)
    else:
        g, _ = gauss_legendre(p + 1)
    v = (g + 1) / 2
    assert lam.min() == pytest.approx((1 + v[0] - v[p]) / 3, abs=1e-14)
