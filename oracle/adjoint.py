"""Discrete adjoint of the oracle by reverse-mode differentiation (test
infrastructure only).

The loss is the interface-shape misfit at the final time,
J = 1/2 int (phi_T - phi*)^2 dOmega, evaluated with the solution-point
quadrature (the exact integral of the interpolant, as in the Section 4 error
measures).  Its gradient with respect to the initial phase field phi0 (at the
solution points) and to the stream-function coefficients (A_m, B_m) of the
velocity is the exact derivative of the oracle's discrete map: torch autograd
through Steps 1-6, the RK4 march and, when requested, the psi reset and the
fixed-count preconditioning at t = 0.
"""
import torch

from .solver import Solver, circle_ic

T64 = torch.float64


def misfit(sol, phi, phi_star):
    """J = 1/2 sum_e sum_i w_i det J_ei (phi - phi*)^2."""
    d = phi - phi_star
    return 0.5 * sol.integral(d * d)


def loss_and_gradients(mesh, p, prm, vel, phi0, phi_star, n_steps, precondition=False):
    """Return J, dJ/dphi0 (E, Nu), dJ/dA (M,), dJ/dB (M,) for a stream-function velocity."""
    sol = Solver(mesh, p, prm, vel)
    phi0 = torch.as_tensor(phi0, dtype=T64).clone().requires_grad_(True)
    A = torch.as_tensor(vel.A, dtype=T64).clone().requires_grad_(True)
    B = torch.as_tensor(vel.B, dtype=T64).clone().requires_grad_(True)
    sol.initialize(phi=phi0, precondition=precondition)
    for _ in range(n_steps):
        sol.rk4_step(A, B)
    J = misfit(sol, sol.phi, torch.as_tensor(phi_star, dtype=T64))
    gphi, gA, gB = torch.autograd.grad(J, (phi0, A, B))
    return float(J.detach()), gphi.detach(), gA.detach(), gB.detach()


def loss(mesh, p, prm, vel, phi0, phi_star, n_steps, A=None, B=None, precondition=False):
    """Forward loss only (for finite differences)."""
    with torch.no_grad():
        sol = Solver(mesh, p, prm, vel)
        sol.initialize(phi=torch.as_tensor(phi0, dtype=T64), precondition=precondition)
        A = torch.as_tensor(vel.A if A is None else A, dtype=T64)
        B = torch.as_tensor(vel.B if B is None else B, dtype=T64)
        for _ in range(n_steps):
            sol.rk4_step(A, B)
        return float(misfit(sol, sol.phi, torch.as_tensor(phi_star, dtype=T64)))
