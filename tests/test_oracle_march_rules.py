"""Pins for the oracle's RK4 stage times, the pseudo-time stop rule and the
initial field.

* RK4 stage times (Section 3.1, the 4-stage Runge-Kutta march; classical
  nodes c = 0, 1/2, 1/2, 1).  A uniform velocity a g(t), g = cos(pi t / T),
  with gamma = eps = 0 and no penalty makes the semi-discrete system
  du/dt = g(t) C u with a constant matrix C, whose exact solution is
  u(t) = exp(G(t) C) u0 with G(t) = (T/pi) sin(pi t / T).  RK4 with the
  right stage times converges to it at fourth order in dt; evaluating the
  velocity at the step's start time for every stage drops the order to one.
  On a fine mesh the march also follows the exact translation of the PDE,
  u0(x - a G(t)).
* Pseudo-time stop rule (Section 3.2): stop at the first k with
  RMS((psi^k - psi^{k-1}) / dtau) <= tol over all solution points.  A
  constant psi0 = phi - 1/2 on a walled element has zero gradient, no sensor
  energy and no face flux, so the source sgn(psi0)(1 - |q|) is exactly
  sgn(psi0): every iteration moves psi by dtau sgn(psi0) and the RMS is
  exactly 1, independent of dtau and of the number of points.
* Initial field (Section 4, Eqs. initialCond, discEq):
  phi = (1 + tanh(beta (r - |x - c|))) / 2 is 1/2 on the circle, has radial
  slope -beta/2 there, and saturates to 1 inside and 0 outside.
"""
import math

import numpy as np
import pytest
import scipy.linalg
import torch

import synthetic as S
from oracle import Params, Solver, circle_ic

T64 = torch.float64


# ----------------------------------------------------------------------------
# RK4 stage times

def _modulated_solver(mesh, p, T, cls=Solver, a=(1.0, 0.5)):
    prm = Params(gamma=0.0, eps=0.0, tau=0.0, tau_psi=0.0, dt=1.0)
    return cls(mesh, p, prm, S.Velocity("uniform", a=(a[0], a[1], 0.0), T=T))


def _operator(s):
    """C with R(phi, t = 0) = C phi (g(0) = 1), assembled column by column."""
    shape = (s.E, s.Nu)
    N = s.E * s.Nu
    z = torch.zeros(shape, dtype=T64)
    C = np.zeros((N, N))
    for k in range(N):
        e = torch.zeros(N, dtype=T64)
        e[k] = 1.0
        C[:, k] = s.rhs(e.reshape(shape), z, 0.0)[0].reshape(-1).numpy()
    return C


class _StagesAtStepStart(Solver):
    """A planted mistake: the velocity of every stage taken at the step's start."""

    def rk4_step(self, A=None, B=None):
        dt, t = self.prm.dt, self.t
        phi, psi = self.phi, self.psi
        a1, b1 = self.rhs(phi, psi, t)
        a2, b2 = self.rhs(phi + 0.5 * dt * a1, psi + 0.5 * dt * b1, t)
        a3, b3 = self.rhs(phi + 0.5 * dt * a2, psi + 0.5 * dt * b2, t)
        a4, b4 = self.rhs(phi + dt * a3, psi + dt * b3, t)
        self.phi = phi + dt / 6.0 * (a1 + 2 * a2 + 2 * a3 + a4)
        self.psi = psi + dt / 6.0 * (b1 + 2 * b2 + 2 * b3 + b4)
        self.t = t + dt
        self.nstep += 1


def _stage_time_order(cls):
    """Observed order of the march against exp(G(t) C) u0 on a 2 x 2 periodic
    quad mesh, p = 2, T = 1, over t in [0, 0.7]."""
    mesh = S.quad_grid(2)
    T, t_end = 1.0, 0.7
    s = _modulated_solver(mesh, 2, T, cls)
    C = _operator(s)
    rho = np.abs(np.linalg.eigvals(C)).max()
    x = s.xu
    u0 = (torch.sin(2 * math.pi * x[..., 0]) * torch.cos(2 * math.pi * x[..., 1])
          + 0.3 * torch.cos(2 * math.pi * x[..., 0]))
    G = T / math.pi * math.sin(math.pi * t_end / T)
    exact = scipy.linalg.expm(G * C) @ u0.reshape(-1).numpy()
    errs = []
    n0 = int(math.ceil(t_end * rho / 0.5))       # dt * rho <= 1/2: the asymptotic range
    for n in (n0, 2 * n0, 4 * n0):
        s.prm.dt = t_end / n
        s.t, s.nstep = 0.0, 0
        s.phi = u0.clone()
        s.psi = torch.zeros_like(u0)
        for _ in range(n):
            s.rk4_step()
        assert s.t == pytest.approx(t_end, rel=1e-14)
        errs.append(float(np.abs(s.phi.reshape(-1).numpy() - exact).max()))
    return math.log2(errs[0] / errs[1]), math.log2(errs[1] / errs[2]), errs


def test_rk4_stage_times_give_fourth_order_under_a_time_dependent_velocity():
    o1, o2, errs = _stage_time_order(Solver)
    assert o1 > 3.7 and o2 > 3.8, (o1, o2, errs)
    assert errs[-1] < 1e-6


def test_rk4_stage_time_pin_rejects_velocity_at_the_step_start():
    o1, o2, _ = _stage_time_order(_StagesAtStepStart)
    assert o1 < 2.0 and o2 < 2.0


def test_modulated_translation_follows_the_integrated_displacement():
    """The PDE's exact solution under u = a cos(pi t / T) is the initial field
    shifted by a G(t); on 6 x 6 periodic quads at p = 5 the march tracks it."""
    mesh = S.quad_grid(6)
    T, t_end, a = 0.8, 0.6, (1.0, 0.5)
    s = _modulated_solver(mesh, 5, T, a=a)
    s.prm.tau = s.prm.tau_psi = 0.1
    x = s.xu
    f = lambda X, Y: torch.sin(2 * math.pi * X) * torch.sin(2 * math.pi * Y)
    s.phi = f(x[..., 0], x[..., 1])
    s.psi = torch.zeros_like(s.phi)
    n = 400
    s.prm.dt = t_end / n
    for _ in range(n):
        s.rk4_step()
    G = T / math.pi * math.sin(math.pi * t_end / T)
    exact = f(x[..., 0] - a[0] * G, x[..., 1] - a[1] * G)
    steady = f(x[..., 0] - a[0] * t_end, x[..., 1] - a[1] * t_end)
    err = float((s.phi - exact).abs().max())
    assert err < 2e-5
    assert float((exact - steady).abs().max()) > 0.5   # the modulation matters


# ----------------------------------------------------------------------------
# pseudo-time stop rule

class _StopWithoutDtau(Solver):
    """A planted mistake: the stop rule's residual without the division by dtau."""

    def precondition(self, fixed=None):
        return _precondition_variant(self, fixed, lambda new, psi, dtau: (new - psi),
                                     lambda R: float(torch.sqrt((R * R).sum() / R.numel())))


class _StopWithSum(Solver):
    """A planted mistake: the root of the sum of squares instead of the mean."""

    def precondition(self, fixed=None):
        return _precondition_variant(self, fixed, lambda new, psi, dtau: (new - psi) / dtau,
                                     lambda R: float(torch.sqrt((R * R).sum())))


def _precondition_variant(s, fixed, resid, norm):
    prm = s.prm
    fixed = prm.pseudo_fixed if fixed is None else fixed
    psi0 = s.phi - 0.5
    psi = psi0
    dtau = prm.pseudo_dtau
    f = lambda y: s.rhs_pseudo(y, psi0)
    it, rms = 0, float("nan")
    for it in range(1, prm.pseudo_kmax + 1):
        k1 = f(psi)
        k2 = f(psi + 0.5 * dtau * k1)
        k3 = f(psi + 0.5 * dtau * k2)
        k4 = f(psi + dtau * k3)
        new = psi + dtau / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        rms = norm(resid(new, psi, dtau))
        psi = new
        if not fixed and rms <= prm.pseudo_tol:
            break
    s.psi, s.psi0, s.pseudo_iters, s.pseudo_rms = psi, psi0, it, rms
    return it, rms


def _constant_state_stops(cls):
    """(iterations, rms) at tol 0.5 and at tol 1.5 for constant phi on one
    walled quad, p = 3 (16 points), dtau = 0.01, kmax = 7."""
    mesh = S.quad_grid(1, periodic=(False, False))
    out = []
    for phi_c in (0.8, 0.1):
        for tol in (0.5, 1.5):
            prm = Params(gamma=0.09, eps=0.01, pseudo_dtau=0.01, pseudo_kmax=7, pseudo_tol=tol,
                         nu_max=0.05, s0=-5.0, kappa=5.0)
            s = cls(mesh, 3, prm, S.Velocity("uniform", a=(0.0, 0.0)))
            s.phi = torch.full((s.E, s.Nu), phi_c, dtype=T64)
            it, rms = s.precondition()
            out.append((phi_c, tol, it, rms, s.psi))
    return out


def test_pseudo_stop_rule_on_a_constant_state_closed_form():
    for phi_c, tol, it, rms, psi in _constant_state_stops(Solver):
        sgn = 1.0 if phi_c > 0.5 else -1.0
        assert rms == pytest.approx(1.0, abs=1e-12)
        if tol < 1.0:
            assert it == 7
            assert torch.allclose(psi, torch.full_like(psi, phi_c - 0.5 + 7 * 0.01 * sgn), atol=1e-14)
        else:
            assert it == 1
            assert torch.allclose(psi, torch.full_like(psi, phi_c - 0.5 + 0.01 * sgn), atol=1e-14)


@pytest.mark.parametrize("cls", [_StopWithoutDtau, _StopWithSum])
def test_pseudo_stop_rule_pin_rejects_planted_mistakes(cls):
    ok = True
    for phi_c, tol, it, rms, psi in _constant_state_stops(cls):
        ok = ok and rms == pytest.approx(1.0, abs=1e-12) and it == (7 if tol < 1.0 else 1)
    assert not ok


def test_pseudo_stop_iteration_from_explicit_iterates():
    """On a 2 x 1 walled quad mesh with a tanh interface, the iterates are
    computed here by RK4 in pseudo time, their residual RMS by hand, and the
    tolerance is put between the RMS of iterations 2 and 3: the oracle stops
    at the first iteration whose RMS is at or below it."""
    mesh = S.quad_grid(2, 1, periodic=(False, False))
    p, dtau = 3, 0.02
    prm = Params(gamma=0.09, eps=0.01, tau_pseudo=0.1, pseudo_dtau=dtau, pseudo_kmax=6,
                 nu_max=0.05, s0=-5.0, kappa=5.0)
    s = Solver(mesh, p, prm, S.Velocity("uniform", a=(0.0, 0.0)))
    x = s.xu
    phi = 0.5 * (1 + torch.tanh(6.0 * (x[..., 0] - 0.45) + 2.0 * (x[..., 1] - 0.5)))
    psi0 = phi - 0.5
    psi = psi0.clone()
    rms = []
    for _ in range(4):
        f = lambda y: s.rhs_pseudo(y, psi0)
        k1 = f(psi)
        k2 = f(psi + 0.5 * dtau * k1)
        k3 = f(psi + 0.5 * dtau * k2)
        k4 = f(psi + dtau * k3)
        new = psi + dtau / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        d = ((new - psi) / dtau).numpy().ravel()
        rms.append(math.sqrt(np.mean(d * d)))
        psi = new
    assert rms[0] > rms[1] > rms[2] > rms[3], rms   # the iteration settles
    s.prm.pseudo_tol = 0.5 * (rms[1] + rms[2])
    s.phi = phi
    it, got = s.precondition()
    assert it == 3
    assert got == pytest.approx(rms[2], rel=1e-12)
    s.prm.pseudo_fixed = True
    it, got = s.precondition()
    assert it == 6


# ----------------------------------------------------------------------------
# initial field

@pytest.mark.parametrize("dim", [2, 3])
def test_circle_initial_field_closed_forms(dim):
    rng = np.random.default_rng(21)
    centre = (0.5, 0.75, 0.4)[:dim]
    r, beta = 0.15, 3 * 4 / (4 / 64)          # beta = 3p/(4h) at p = 4, h = 1/64
    circ = S.Circle(centre, r, beta)
    dirs = rng.normal(size=(50, dim))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    c = np.asarray(centre)
    on = torch.as_tensor(c + r * dirs, dtype=T64)
    assert torch.allclose(circle_ic(on, circ), torch.full((50,), 0.5, dtype=T64), atol=1e-14)
    # radial slope at the interface: d phi / d rho = -beta/2 (sech^2(0) = 1)
    d = 1e-6
    out = torch.as_tensor(c + (r + d) * dirs, dtype=T64)
    inn = torch.as_tensor(c + (r - d) * dirs, dtype=T64)
    slope = (circle_ic(out, circ) - circle_ic(inn, circ)) / (2 * d)
    assert torch.allclose(slope, torch.full((50,), -beta / 2, dtype=T64), rtol=1e-6)
    # saturation: 1 at the centre (beta r = 14.4), 0 far outside
    assert float(circle_ic(torch.as_tensor(c[None], dtype=T64), circ)[0]) == pytest.approx(
        0.5 * (1 + math.tanh(beta * r)), rel=1e-15)
    assert float(circle_ic(torch.as_tensor(c[None], dtype=T64), circ)[0]) > 1 - 1e-11
    far = torch.as_tensor(c + (r + 0.2) * dirs, dtype=T64)
    assert float(circle_ic(far, circ).max()) < 1e-20
    # symmetric about the interface: phi(r - s) + phi(r + s) = 1
    for sft in (0.003, 0.01, 0.05):
        a = circle_ic(torch.as_tensor(c + (r - sft) * dirs, dtype=T64), circ)
        b = circle_ic(torch.as_tensor(c + (r + sft) * dirs, dtype=T64), circ)
        assert torch.allclose(a + b, torch.ones_like(a), atol=1e-14)


# ----------------------------------------------------------------------------
# error measures (Section 4)

@pytest.mark.parametrize("et", ["quad", "tri", "hex"])
def test_error_measures_closed_forms(et):
    """phi_e = 1 + x, phi = phi_e + c x(1-x) y(1-y) (degree 2 per direction,
    total degree 4: represented exactly at p = 3 on affine tensor elements and
    at p = 4 on triangles): E_L1 = c/36,
    E_r = E_L1 / 1.5, and E_m against phi0 = phi_e is (c/36) / 1.5."""
    if et == "quad":
        mesh = S.quad_grid(3, periodic=(False, False))
    elif et == "tri":
        mesh = S.tri_split(3, periodic=(False, False))
    else:
        mesh = S.hex_grid(2)
    s = Solver(mesh, 4 if et == "tri" else 3, Params(), S.Velocity("uniform", a=(0.0, 0.0, 0.0)))
    x = s.xu
    X, Y = x[..., 0], x[..., 1]
    c = 0.7
    pe = 1 + X
    s.phi = pe + c * X * (1 - X) * Y * (1 - Y)
    el1, er = s.errors(pe)
    assert el1 == pytest.approx(c / 36, rel=1e-13)
    assert er == pytest.approx(c / 36 / 1.5, rel=1e-13)
    assert s.mass_error(pe, pe) == pytest.approx(c / 36 / 1.5, rel=1e-12)
    # below phi_e the absolute value matters: E_L1 is unchanged, E_m changes sign
    s.phi = pe - c * X * (1 - X) * Y * (1 - Y)
    assert s.errors(pe)[0] == pytest.approx(c / 36, rel=1e-13)
    assert s.mass_error(pe, pe) == pytest.approx(-c / 36 / 1.5, rel=1e-12)
