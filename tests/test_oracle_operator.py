"""Whole-operator pins of the oracle's residual on tiny periodic meshes.

On uniform periodic quads with a constant velocity and no sharpening
(gamma = 0), Steps 1-6 are linear and reduce to a sum of one-dimensional FR
operators along the x and y lines of solution points.  The 1D operator is
written here from its definition (Section 3.1): Gauss-Legendre points, the
Lagrange derivative, the Radau correction g_L = (-1)^(p+1)/2 (P_{p+1} - P_p)
with g_R(xi) = g_L(-xi), the central advective flux plus the penalty
tau (u_L - u_R), and LDG with beta = +1/2 seen from the L side of each face
(common solution u_R in the gradient, common viscous flux from q_L).  L is the
element with the lower index, so on the periodic wrap face it is element 0.
None of the oracle's 2D reference element, geometry or face matching is used.

Pins: the oracle's matrix-free residual equals the Kronecker sum of the 1D
operators; with tau = 0 the advection spectrum is imaginary (energy neutral),
with tau > 0 it is dissipative; the LDG diffusion operator has real
eigenvalues <= 0 whose only zero mode is the constant.
"""
import numpy as np
import numpy.polynomial.legendre as npl
import pytest
import torch

import synthetic as S
from oracle import Params, Solver


def _ref_1d(p):
    N = p + 1
    xi, _ = npl.leggauss(N)
    w = np.array([1.0 / np.prod([xi[j] - xi[k] for k in range(N) if k != j]) for j in range(N)])
    D = np.zeros((N, N))
    for i in range(N):
        for j in range(N):
            if i != j:
                D[i, j] = (w[j] / w[i]) / (xi[i] - xi[j])
        D[i, i] = -D[i].sum()
    lag = lambda x: np.array([np.prod([(x - xi[k]) / (xi[j] - xi[k]) for k in range(N) if k != j])
                              for j in range(N)])
    cL = np.zeros(p + 2)
    cL[p + 1], cL[p] = 0.5 * (-1) ** (p + 1), -0.5 * (-1) ** (p + 1)
    gLd = npl.legval(xi, npl.legder(cL))
    gRd = -npl.legval(-xi, npl.legder(cL))
    return xi, D, lag(-1.0), lag(1.0), gLd, gRd


def _fr_1d(p, n, h, a, tau, mu):
    """Matrix of du/dt on a periodic chain of n elements of size h for the
    physical flux f = a u - mu du/dx, N = p+1 Gauss-Legendre points each.
    Face k is the right face of element k; its L side is element k, except
    on the wrap face (k = n-1), where it is element 0."""
    xi, D, lL, lR, gLd, gRd = _ref_1d(p)
    N = p + 1
    J = 2.0 / h                                       # dxi/dx
    left_of = lambda k: k                             # element left of face k
    right_of = lambda k: (k + 1) % n                  # element right of face k
    L_of = lambda k: 0 if k == n - 1 else k

    def apply(u):
        u = u.reshape(n, N)
        uL, uR = u @ lL, u @ lR                       # traces at xi = -1, +1
        # common solution per face: the trace of its R side
        C = np.empty(n)
        for k in range(n):
            C[k] = uL[right_of(k)] if L_of(k) == left_of(k) else uR[left_of(k)]
        q = np.empty((n, N))
        for e in range(n):
            q[e] = J * (D @ u[e] + gLd * (C[(e - 1) % n] - uL[e]) + gRd * (C[e] - uR[e]))
        qL, qR = q @ lL, q @ lR
        f = a * u - mu * q
        fL, fR = f @ lL, f @ lR
        # common physical flux per face (positive x direction)
        Fs = np.empty(n)
        for k in range(n):
            ul, ur = uR[left_of(k)], uL[right_of(k)]
            qLside = qR[left_of(k)] if L_of(k) == left_of(k) else qL[right_of(k)]
            Fs[k] = 0.5 * a * (ul + ur) - mu * qLside + tau * (ul - ur)
        # the penalty is tau (u_self - u_other) out of each side; from the
        # right side's view the outward normal is -x, so its physical flux is
        # f* = 0.5 a (ul + ur) - mu q* - tau (ur - ul) = the same Fs[k]
        out = np.empty((n, N))
        for e in range(n):
            out[e] = -J * (D @ f[e] + gLd * (Fs[(e - 1) % n] - fL[e]) + gRd * (Fs[e] - fR[e]))
        return out.reshape(-1)

    A = np.stack([apply(c) for c in np.eye(n * N)], 1)
    return A, xi


def _oracle_matrix(n, p, a, tau, eps=0.0):
    mesh = S.quad_grid(n)
    prm = Params(gamma=0.0, eps=eps, tau=tau, tau_psi=tau, dt=1e-3)
    s = Solver(mesh, p, prm, S.Velocity("uniform", a=(a[0], a[1], 0.0)))
    s.initialize(S.Circle((0.5, 0.5), 0.25, 4.0), precondition=False)
    shape, Nd = s.phi.shape, s.phi.numel()
    A = np.zeros((Nd, Nd))
    z = torch.zeros(shape, dtype=torch.float64)
    for k in range(Nd):
        e = torch.zeros(Nd, dtype=torch.float64)
        e[k] = 1.0
        A[:, k] = s.rhs(e.reshape(shape), z, 0.0)[0].reshape(-1).numpy()
    return A, s.xu.reshape(-1, 2).numpy()


def _structured_index(x, n, p, xi):
    """Position of each oracle unknown in the x-fastest tensor ordering."""
    h, N = 1.0 / n, p + 1

    def loc(c):
        e = np.minimum((c / h + 1e-9).astype(int), n - 1)
        r = 2.0 * (c - e * h) / h - 1.0
        j = np.abs(r[:, None] - xi[None, :]).argmin(1)
        assert np.allclose(xi[j], r, atol=1e-12)
        return e * N + j
    g = loc(x[:, 1]) * (n * N) + loc(x[:, 0])
    assert sorted(g.tolist()) == list(range(len(g)))
    return g


@pytest.mark.parametrize("n,p", [(1, 1), (1, 3), (2, 1), (2, 2), (3, 3), (3, 4)])
@pytest.mark.parametrize("tau,eps", [(0.0, 0.0), (0.1, 0.0), (0.1, 0.02)])
def test_residual_equals_kronecker_sum_of_1d_operators(n, p, tau, eps):
    a = (1.0, 0.5)
    mu = eps * float(np.hypot(*a))                    # M eps with M = |v| (gamma = 0)
    A, x = _oracle_matrix(n, p, a, tau, eps)
    Ax, xi = _fr_1d(p, n, 1.0 / n, a[0], tau, mu)
    Ay, _ = _fr_1d(p, n, 1.0 / n, a[1], tau, mu)
    I = np.eye(n * (p + 1))
    ref = np.kron(I, Ax) + np.kron(Ay, I)
    g = _structured_index(x, n, p, xi)
    # scale: the operator's natural size (2/h)(p+1)^2 (1x1, p = 1 central is exactly 0)
    scale = max(np.abs(ref).max(), 2.0 * n * (p + 1) ** 2)
    assert np.abs(A - ref[np.ix_(g, g)]).max() < 1e-13 * scale


def test_central_flux_is_energy_neutral_and_penalty_dissipates():
    A0, _ = _oracle_matrix(3, 3, (1.0, 0.5), 0.0)
    ev0 = np.linalg.eigvals(A0)
    assert np.abs(ev0.real).max() < 1e-10 * np.abs(ev0).max()
    A1, _ = _oracle_matrix(3, 3, (1.0, 0.5), 0.1)
    ev1 = np.linalg.eigvals(A1)
    assert ev1.real.max() < 1e-10 * np.abs(ev1).max()
    assert ev1.real.min() < -1e-3                     # the penalty damps some modes


def test_ldg_diffusion_spectrum_is_real_and_nonpositive():
    """LDG with a per-face switch is -M^-1 B^T M^-1 B, so its eigenvalues are
    real and <= 0.  Its null space is the kernel of the discrete gradient B:
    the constants, plus, in an element whose common solution comes from its
    neighbours on every face (element 0, lower index than all neighbours),
    any u orthogonal to all derivatives of P_p, i.e. the Legendre mode P_p.
    On the periodic 3 x 3 mesh that gives 2 x 2 = 4 zero modes: 1, P_p(x) in
    the column of element 0, P_p(y) in its row, and P_p(x) P_p(y) in it."""
    n, p = 3, 3
    a, eps, tau = (1.0, 0.5), 0.05, 0.1
    A0, x = _oracle_matrix(n, p, a, tau, 0.0)
    A1, _ = _oracle_matrix(n, p, a, tau, eps)
    Ld = (A1 - A0) / (eps * float(np.hypot(*a)))      # the LDG Laplacian alone
    ev = np.linalg.eigvals(Ld)
    scale = np.abs(ev).max()
    assert np.abs(ev.imag).max() < 1e-8 * scale
    assert ev.real.max() < 1e-10 * scale
    lam = np.sort(np.abs(ev.real))
    assert lam[3] < 1e-10 * scale and lam[4] > 1.0    # exactly four zero modes
    h = 1.0 / n
    r = 2.0 * (x - h * np.floor(x / h + 1e-9)) / h - 1.0
    Pp = npl.legval(r, np.eye(p + 1)[p])
    inx, iny = x[:, 0] < h, x[:, 1] < h
    modes = [np.ones(len(x)), np.where(inx, Pp[:, 0], 0.0), np.where(iny, Pp[:, 1], 0.0),
             np.where(inx & iny, Pp[:, 0] * Pp[:, 1], 0.0)]
    for m in modes:
        assert np.abs(Ld @ m).max() < 1e-10 * scale
    # the first nonzero modes approximate -(2 pi)^2 (sin/cos in x or y)
    assert abs(lam[4] - (2 * np.pi) ** 2) < 0.02 * (2 * np.pi) ** 2


def test_ldg_1d_null_space_is_constants_and_the_wrap_mode():
    """The same count in the independent 1D operator, for several n and p."""
    for n, p in [(3, 1), (3, 3), (4, 2), (5, 4)]:
        Ld, xi = _fr_1d(p, n, 1.0 / n, 0.0, 0.0, 1.0)
        ev = np.linalg.eigvals(Ld)
        lam = np.sort(np.abs(ev))
        assert lam[1] < 1e-9 * lam[-1] and lam[2] > 1.0
        m = np.zeros(n * (p + 1))
        m[:p + 1] = npl.legval(xi, np.eye(p + 1)[p])
        assert np.abs(Ld @ m).max() < 1e-9 * lam[-1]


# ---------------------------------------------------------------- triangles
def _tri_dg_reference(mesh, p, a, tau, mu, xu):
    """Nodal matrix of du/dt for f = a u - mu grad u on a periodic triangle
    mesh, from the DG weak form with exact integration (FR with the DG
    correction reproduces it when a and mu are constant).  Physical monomial
    basis per element, Duffy-collapsed Gauss rule on the element and Gauss
    rule on the edges; neighbours found by matching edge midpoints modulo the
    period; LDG: u_hat from the face's R side, q_hat from its L side (L = lower
    element index); penalty tau (u_self - u_other) out of each side."""
    E = mesh.conn.shape[0]
    per = np.array(mesh.period, dtype=float)
    X = mesh.nodes[mesh.conn]                                  # (E, 3, 2)
    pw = [(i, j) for i in range(p + 1) for j in range(p + 1 - i)]
    Nm = len(pw)
    cen = X.mean(1)

    def basis(e, x):                                           # x (k, 2) -> (k, Nm), grads (k, Nm, 2)
        y = (x - cen[e]) * 4.0
        B = np.stack([y[:, 0] ** i * y[:, 1] ** j for i, j in pw], 1)
        dx = np.stack([i * y[:, 0] ** max(i - 1, 0) * y[:, 1] ** j * 4.0 for i, j in pw], 1)
        dy = np.stack([j * y[:, 0] ** i * y[:, 1] ** max(j - 1, 0) * 4.0 for i, j in pw], 1)
        return B, np.stack([dx, dy], -1)

    g, gw = npl.leggauss(p + 3)
    g, gw = 0.5 * (g + 1.0), 0.5 * gw
    def vol_rule(e):
        v0, v1, v2 = X[e]
        d1, d2 = v1 - v0, v2 - v0
        area2 = abs(d1[0] * d2[1] - d1[1] * d2[0])
        s_, t_ = np.meshgrid(g, g, indexing="ij")
        ws = np.outer(gw, gw) * (1.0 - t_)
        ss, tt = s_ * (1.0 - t_), t_
        pts = v0 + ss.reshape(-1, 1) * (v1 - v0) + tt.reshape(-1, 1) * (v2 - v0)
        return pts, ws.reshape(-1) * area2
    eg, egw = npl.leggauss(p + 2)
    eg = 0.5 * (eg + 1.0)

    # edges: (e, k) -> (neighbour, shift) by midpoint matching modulo the period
    edges = {}
    for e in range(E):
        for k in range(3):
            a0, a1 = X[e, k], X[e, (k + 1) % 3]
            edges[(e, k)] = (a0, a1, 0.5 * (a0 + a1))
    nbr = {}
    for (e, k), (a0, a1, m) in edges.items():
        for (e2, k2), (b0, b1, m2) in edges.items():
            if (e2, k2) == (e, k):
                continue
            d = m2 - m
            sh = per * np.round(d / per)
            if np.allclose(d, sh, atol=1e-12) and (
                    np.allclose(a0 + sh, b1) and np.allclose(a1 + sh, b0)):
                nbr[(e, k)] = (e2, sh)
    assert len(nbr) == 3 * E

    n = E * Nm
    Mb = np.zeros((n, n))
    Gx = np.zeros((2, n, n))                                   # M q = G u
    Kv = np.zeros((n, n))                                      # advective volume + face terms
    Dq = np.zeros((2, n, n))                                   # viscous terms acting on q
    sl = lambda e: slice(e * Nm, (e + 1) * Nm)
    for e in range(E):
        pts, w = vol_rule(e)
        B, dB = basis(e, pts)
        Mb[sl(e), sl(e)] = (B * w[:, None]).T @ B
        for c in range(2):
            Gx[c, sl(e), sl(e)] -= (dB[:, :, c] * w[:, None]).T @ B       # -int u d_c v
            Kv[sl(e), sl(e)] += a[c] * (dB[:, :, c] * w[:, None]).T @ B   # int a_c u d_c v
            Dq[c, sl(e), sl(e)] -= mu * (dB[:, :, c] * w[:, None]).T @ B  # -int mu q_c d_c v
        for k in range(3):
            a0, a1 = X[e, k], X[e, (k + 1) % 3]
            L = np.linalg.norm(a1 - a0)
            t = (a1 - a0) / L
            nrm = np.array([t[1], -t[0]])                      # outward for CCW vertices
            xs = a0 + eg[:, None] * (a1 - a0)
            ws = 0.5 * egw * L
            e2, sh = nbr[(e, k)]
            Bs, _ = basis(e, xs)
            Bo, _ = basis(e2, xs + sh)
            self_L = e < e2
            an = a @ nrm
            for c in range(2):
                # u_hat = trace of the R side
                Bh = Bo if self_L else Bs
                Gx[c, sl(e), sl(e2) if self_L else sl(e)] += nrm[c] * (Bs * ws[:, None]).T @ Bh
                # q_hat = q of the L side: flux out of e gets -mu q_hat . n
                Bq = Bs if self_L else Bo
                Dq[c, sl(e), sl(e) if self_L else sl(e2)] += mu * nrm[c] * (Bs * ws[:, None]).T @ Bq
            # advective common flux and penalty, out of e: -int F v
            Kv[sl(e), sl(e)] -= (0.5 * an + tau) * (Bs * ws[:, None]).T @ Bs
            Kv[sl(e), sl(e2)] -= (0.5 * an - tau) * (Bs * ws[:, None]).T @ Bo
    Mi = np.linalg.inv(Mb)
    Amod = Mi @ (Kv + sum(Dq[c] @ Mi @ Gx[c] for c in range(2)))
    V = np.zeros((n, n))
    for e in range(E):
        V[sl(e), sl(e)] = basis(e, xu[e])[0]
    return V @ Amod @ np.linalg.inv(V)


def _oracle_tri_matrix(mesh, p, a, tau, eps):
    prm = Params(gamma=0.0, eps=eps, tau=tau, tau_psi=tau, dt=1e-3)
    s = Solver(mesh, p, prm, S.Velocity("uniform", a=(a[0], a[1], 0.0)))
    s.initialize(S.Circle((0.5, 0.5), 0.25, 4.0), precondition=False)
    shape, Nd = s.phi.shape, s.phi.numel()
    A = np.zeros((Nd, Nd))
    z = torch.zeros(shape, dtype=torch.float64)
    for k in range(Nd):
        e = torch.zeros(Nd, dtype=torch.float64)
        e[k] = 1.0
        A[:, k] = s.rhs(e.reshape(shape), z, 0.0)[0].reshape(-1).numpy()
    return A, s.xu.numpy()


@pytest.mark.parametrize("nx,p", [(1, 1), (1, 2), (1, 3), (2, 2), (2, 3)])
@pytest.mark.parametrize("tau,eps", [(0.0, 0.0), (0.1, 0.0), (0.1, 0.02)])
def test_triangle_residual_equals_dg_weak_form(nx, p, tau, eps):
    a = (1.0, 0.5)
    mesh = S.tri_split(nx)
    A, xu = _oracle_tri_matrix(mesh, p, a, tau, eps)
    ref = _tri_dg_reference(mesh, p, np.array(a), tau, eps * float(np.hypot(*a)), xu)
    scale = max(np.abs(ref).max(), 2.0 * nx * (p + 1) ** 2)
    err = np.abs(A - ref).max() / scale
    assert err < 1e-13


def test_triangle_spectra():
    mesh, p, a = S.tri_split(2), 3, (1.0, 0.5)
    A0, _ = _oracle_tri_matrix(mesh, p, a, 0.0, 0.0)
    ev0 = np.linalg.eigvals(A0)
    assert np.abs(ev0.real).max() < 1e-9 * np.abs(ev0).max()
    A1, _ = _oracle_tri_matrix(mesh, p, a, 0.1, 0.0)
    ev1 = np.linalg.eigvals(A1)
    assert ev1.real.max() < 1e-10 * np.abs(ev1).max() and ev1.real.min() < -1e-3
    A2, _ = _oracle_tri_matrix(mesh, p, a, 0.1, 0.05)
    Ld = (A2 - A1) / (0.05 * float(np.hypot(*a)))
    ev = np.linalg.eigvals(Ld)
    scale = np.abs(ev).max()
    assert np.abs(ev.imag).max() < 1e-8 * scale and ev.real.max() < 1e-10 * scale
    assert np.allclose(Ld @ np.ones(Ld.shape[0]), 0.0, atol=1e-10 * scale)
