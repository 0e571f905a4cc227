"""Pin of the oracle's discrete adjoint: central finite differences of its own
forward map (the adjoint is reverse-mode differentiation of that map, so the
two must agree to the finite-difference truncation and round-off)."""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import Params
from oracle.adjoint import loss, loss_and_gradients
from oracle.solver import Solver, circle_ic


def _case(precondition):
    mesh = S.quad_grid(4, jitter=0.1, seed=3)
    p = 3
    h = 0.25
    kx, ky, A, B = S.stream_coefficients(4, seed=4, sigma=0.05)
    vel = S.Velocity("stream", T=0.0, kx=kx, ky=ky, A=A, B=B)
    prm = Params(gamma=0.09, eps=0.06 * h / p, tau=0.1, dt=0.004, pseudo_kmax=2, pseudo_fixed=True,
                 pseudo_dtau=0.1 * h / (p + 1), nu_max=0.15 * h / p)
    sol = Solver(mesh, p, prm, vel)
    phi0 = circle_ic(sol.xu, S.Circle((0.5, 0.5), 0.3, 6.0))
    phis = circle_ic(sol.xu, S.Circle((0.55, 0.45), 0.3, 6.0))
    return mesh, p, prm, vel, phi0, phis


@pytest.mark.parametrize("precondition", [False, True])
def test_oracle_adjoint_matches_central_differences(precondition):
    mesh, p, prm, vel, phi0, phis = _case(precondition)
    n = 5
    J, gphi, gA, gB = loss_and_gradients(mesh, p, prm, vel, phi0, phis, n, precondition=precondition)
    assert J == pytest.approx(loss(mesh, p, prm, vel, phi0, phis, n, precondition=precondition), rel=1e-13)
    rng = np.random.default_rng(0)
    h = 1e-6
    # random direction in phi0
    d = torch.as_tensor(rng.normal(size=phi0.shape))
    fd = (loss(mesh, p, prm, vel, phi0 + h * d, phis, n, precondition=precondition)
          - loss(mesh, p, prm, vel, phi0 - h * d, phis, n, precondition=precondition)) / (2 * h)
    assert float((gphi * d).sum()) == pytest.approx(fd, rel=1e-6)
    # each velocity coefficient
    for m in range(len(vel.A)):
        Ap, Am = vel.A.copy(), vel.A.copy()
        Ap[m] += h
        Am[m] -= h
        fd = (loss(mesh, p, prm, vel, phi0, phis, n, A=Ap, precondition=precondition)
              - loss(mesh, p, prm, vel, phi0, phis, n, A=Am, precondition=precondition)) / (2 * h)
        assert float(gA[m]) == pytest.approx(fd, rel=1e-6, abs=1e-12)


@pytest.mark.parametrize("precondition", [False, True])
def test_oracle_adjoint_dot_product_with_forward_mode_tangent(precondition):
    """Dot-product test: the reverse-mode gradient paired with a direction
    (<dJ/dphi0, dphi> + <dJ/dA, dA>) equals the tangent of J along that
    direction computed in forward mode (dual numbers through the same march),
    to round-off: the adjoint is the transpose of the linearised map."""
    import torch.autograd.forward_ad as fwAD
    from oracle.adjoint import misfit
    mesh, p, prm, vel, phi0, phis = _case(precondition)
    n = 4
    _, gphi, gA, _ = loss_and_gradients(mesh, p, prm, vel, phi0, phis, n, precondition=precondition)
    gen = torch.Generator().manual_seed(11)
    dphi = torch.randn(phi0.shape, generator=gen, dtype=torch.float64)
    dA = torch.randn(len(vel.A), generator=gen, dtype=torch.float64)
    sol = Solver(mesh, p, prm, vel)
    with fwAD.dual_level():
        ph = fwAD.make_dual(torch.as_tensor(phi0, dtype=torch.float64), dphi)
        A = fwAD.make_dual(torch.as_tensor(vel.A, dtype=torch.float64), dA)
        B = torch.as_tensor(vel.B, dtype=torch.float64)
        sol.initialize(phi=ph, precondition=precondition)
        for _ in range(n):
            sol.rk4_step(A, B)
        tangent = float(fwAD.unpack_dual(misfit(sol, sol.phi, torch.as_tensor(phis))).tangent)
    paired = float((gphi * dphi).sum() + (gA * dA).sum())
    scale = float(gphi.norm() * dphi.norm() + gA.norm() * dA.norm())
    assert abs(paired - tangent) <= 1e-12 * scale
