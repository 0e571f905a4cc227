"""FR-PCPF residual, RK march and preconditioning (oracle, test infrastructure only).

The state is u = [phi, psi] at the solution points (Section 3.1).  Fluxes:
  f = f_inv - f_vis,  f_inv = [phi v; psi v],
  f_vis = [max(gamma,|v|) (eps grad phi - gamma phi(1-phi) grad psi/|grad psi|); 0]
(Section 3.1, flux split; the multiplier sits inside the flux so that the
scheme stays in conservation form).  The residual follows Steps 1-6 in order
and du/dt = -J^{-1} div~ f~ is marched with the classical 4-stage RK scheme.

Readings of points the paper leaves open (each is a parameter):
  * LDG beta = +1/2 relative to the L side of each face: the common solution
    is the R trace and the viscous flux is the L side's (Steps 2 and 5).
  * The penalty enters the total common normal flux out of L as
    +tau (u_L - u_R), the dissipative sign, for both components of
    u = [phi, psi] (Eq. viscousFlux is written for the vector u); tau_psi is
    the value used for psi (default tau).  Without it psi's advection is a
    pure central flux whose weakly growing aliasing mode takes float32
    round-off to O(1) within one Rider-Kothe period.
  * The common normal flux out of R is minus the one out of L (Eq. commonFlux),
    each side scaling the physical flux by its own face metric |det J J^{-T} n~|.
  * |grad psi| is guarded as max(|grad psi|, delta) in the normal and in the
    smeared sign tanh(psi0 / |grad psi|).
  * Preconditioning source S = sgn(psi0)(1 - |q|) with the sign of
    Eq. pseudotimesystem (psi_tau = -J^{-1} div~ g~ + S), flux g = -nu_s grad psi,
    LDG common flux with penalty tau_pseudo, RK4 in pseudo time, stop when the
    RMS of (psi^k - psi^{k-1})/dtau <= tol or after kmax iterations.
  * Walls (Section 3.3): ghost states copy the interior, so the interior's
    diffusive and sharpening fluxes leave through the wall; Params.wall =
    "noflux" is an option (not the paper's) with zero common normal flux of
    the physical system at wall points.
  * Resolution indicator on psi with an orthonormal modal basis; the
    truncation drops modes of (tensor) max degree p or (triangle) total degree p;
    an element with zero energy or zero truncated energy gets nu_s = 0.

Params.normal selects the interface normal of the sharpening term: "psi"
(the preconditioned method, n = grad psi/|grad psi|, Section 2) or "phi"
(the unpreconditioned conservative phase field of Eq. altconservativephasefieldeq,
n = grad phi/|grad phi| from phi's own corrected gradient, with no psi reset
and no preconditioning; psi is still advected but feeds nothing).
"""
from dataclasses import dataclass
import math

import numpy as np
import torch

from .mesh import build_geometry

T64 = torch.float64


@dataclass
class Params:
    gamma: float = 0.09
    eps: float = 0.0
    tau: float = 0.1
    tau_psi: float = 0.1
    tau_pseudo: float = 0.1
    dt: float = 0.0
    n_precond: int = 1000
    pseudo_kmax: int = 20
    pseudo_dtau: float = 0.0
    pseudo_tol: float = 0.5
    pseudo_fixed: bool = False
    s0: float = -5.0
    kappa: float = 5.0
    nu_max: float = 0.0
    delta: float = 1e-12
    normal: str = "psi"  # "psi": preconditioned (Section 2); "phi": unpreconditioned CPF
    wall: str = "copy"   # "copy": ghost = interior (Section 3.3); "noflux": zero wall flux (an option)

    @classmethod
    def from_workload(cls, w, **kw):
        d = dict(gamma=w.gamma, eps=w.eps, tau=w.tau, tau_psi=w.tau_psi,
                 tau_pseudo=w.tau_pseudo, dt=w.dt, n_precond=w.n_precond,
                 pseudo_kmax=w.pseudo_kmax, pseudo_dtau=w.pseudo_dtau,
                 pseudo_tol=w.pseudo_tol, s0=w.s0, kappa=w.kappa, nu_max=w.nu_max,
                 delta=w.delta, normal=getattr(w, "normal", "psi"), wall=getattr(w, "wall", "copy"))
        d.update(kw)
        return cls(**d)


def velocity(vel, x, t, A=None, B=None):
    """Analytic velocity at points x (..., d) and time t (Sections 4.1-4.3)."""
    pi = math.pi
    g = math.cos(pi * t / vel.T) if vel.T > 0 else 1.0
    X = x[..., 0]
    Y = x[..., 1]
    if vel.kind == "uniform":  # a g(t): steady when T <= 0
        d = x.shape[-1]
        return (g * torch.tensor(vel.a[:d], dtype=T64)).expand(x.shape).clone()
    if vel.kind == "rider_kothe":
        u = -torch.sin(pi * X) ** 2 * torch.sin(2 * pi * Y) * g
        v = torch.sin(2 * pi * X) * torch.sin(pi * Y) ** 2 * g
        return torch.stack([u, v], -1)
    if vel.kind == "rotation":  # solid-body rotation about (a[0], a[1])
        return torch.stack([vel.a[1] - Y, X - vel.a[0]], -1)
    if vel.kind == "leveque":
        Z = x[..., 2]
        s = torch.sin
        u = 2 * s(pi * X) ** 2 * s(2 * pi * Y) * s(2 * pi * Z) * g
        v = -s(2 * pi * X) * s(pi * Y) ** 2 * s(2 * pi * Z) * g
        w = -s(2 * pi * X) * s(2 * pi * Y) * s(pi * Z) ** 2 * g
        return torch.stack([u, v, w], -1)
    if vel.kind == "stream":
        A = torch.as_tensor(vel.A, dtype=T64) if A is None else A
        B = torch.as_tensor(vel.B, dtype=T64) if B is None else B
        kx = torch.as_tensor(vel.kx, dtype=T64)
        ky = torch.as_tensor(vel.ky, dtype=T64)
        arg = 2 * pi * (X[..., None] * kx + Y[..., None] * ky)
        d = 2 * pi * (A * torch.cos(arg) - B * torch.sin(arg))
        u = (d * ky).sum(-1) * g
        v = -(d * kx).sum(-1) * g
        return torch.stack([u, v], -1)
    raise ValueError(vel.kind)


def circle_ic(x, circle):
    """phi = (1 + tanh(beta psi_d))/2, psi_d = r - |x - x0| (Eqs. initialCond, discEq)."""
    c = torch.tensor(circle.centre, dtype=T64)
    dist = torch.sqrt(((x - c) ** 2).sum(-1))
    return 0.5 * (1.0 + torch.tanh(circle.beta * (circle.radius - dist)))


class Solver:
    def __init__(self, mesh, p, prm, vel):
        self.geo = g = build_geometry(mesh, p)
        el = g.el
        self.p = p
        self.prm = prm
        self.vel = vel
        self.dim = el.dim
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=T64)
        self.L = t(el.L)
        self.D = t(el.D)
        self.LIFT = t(el.LIFT)
        self.nref = t(el.nref)
        self.wq = t(el.wq)
        self.Vinv = t(el.Vinv)
        self.high = torch.as_tensor(el.high)
        self.xu = t(g.xu)
        self.xf = t(g.xf)
        self.detJ = t(g.detJu)
        self.Jinv = t(g.Jinvu)                          # [e,i,a,b] = dxi_a/dx_b
        self.S = self.detJ[..., None, None] * self.Jinv  # det J J^{-1}
        self.pn_mag = t(g.pn_mag)
        self.nhat = t(g.nhat)
        self.pe = torch.as_tensor(g.pe)
        self.pk = torch.as_tensor(g.pk)
        self.isL = torch.as_tensor(g.isL)
        self.boundary = torch.as_tensor(g.boundary)
        self.h = g.h
        self.E = g.xu.shape[0]
        self.Nu = el.nu
        self.Nf = el.nf
        self.t = 0.0
        self.nstep = 0
        self.phi = None
        self.psi = None
        self.psi0 = None
        self.pseudo_iters = 0
        self.pseudo_rms = float("nan")

    # ---------------------------------------------------------------- helpers
    def _partner(self, Uf):
        """Value at the coinciding flux point of the neighbour (self on a boundary)."""
        return Uf[self.pe, :, self.pk].permute(0, 2, 1)

    def trace(self, U):
        """Step 1 (Eq. extrapolateSoln): u^f_k = sum_j u_j l_j(x^f_k)."""
        return torch.einsum("kj,efj->efk", self.L, U)

    def gradient(self, U, Uf):
        """Steps 2-3: common solution and corrected physical gradient.

        C = (1/2 - beta) u_self + (1/2 + beta) u_other with beta = +1/2 seen
        from the L side, i.e. C = u_R on both sides of a face.
        q~ = sum_j u_j grad~ l_j + sum_k n~_k (div g_k)(C - u^f)_k  (Eq. continuousGrad)
        q = J^{-T} q~.
        """
        Uo = self._partner(Uf)
        C = torch.where(self.isL[:, None, :], Uo, Uf)
        qt = torch.einsum("aij,efj->efia", self.D, U)
        qt = qt + torch.einsum("ik,ka,efk->efia", self.LIFT, self.nref, C - Uf)
        q = torch.einsum("eiab,efia->efib", self.Jinv, qt)
        return q, Uo

    def common_to_transformed(self, Fphys):
        """Common normal flux out of each side, transformed by the side's face metric.

        Fphys holds the flux out of L at L points; R points take minus their
        partner's value (Eq. commonFlux)."""
        Fo = self._partner(Fphys)
        Fc = torch.where(self.isL[:, None, :], Fphys, -Fo)
        return self.pn_mag[:, None, :] * Fc

    def divergence(self, ft, Ft):
        """Step 6 (Eq. continuousDivFlux) with Step 4's normal flux (Eq. normalTransFlux)."""
        fperp = torch.einsum("ka,kj,efja->efk", self.nref, self.L, ft)
        div = torch.einsum("aij,efja->efi", self.D, ft)
        div = div + torch.einsum("ik,efk->efi", self.LIFT, Ft - fperp)
        return div

    # ---------------------------------------------------------------- physical residual
    def rhs(self, phi, psi, t, A=None, B=None):
        prm = self.prm
        U = torch.stack([phi, psi], 1)
        Uf = self.trace(U)                                            # Step 1
        q, Uo = self.gradient(U, Uf)                                  # Steps 2-3
        qf = torch.einsum("kj,efjb->efkb", self.L, q)                 # Eq. extrapolateGrad
        # Step 4: flux at solution points, transformed
        v = velocity(self.vel, self.xu, t, A, B)
        M = torch.clamp(torch.sqrt((v * v).sum(-1)), min=prm.gamma)
        kn = 1 if prm.normal == "psi" else 0                          # field the normal comes from
        qpsi = q[:, kn]
        nvec = qpsi / torch.clamp(torch.sqrt((qpsi * qpsi).sum(-1)), min=prm.delta)[..., None]
        fvis = M[..., None] * (prm.eps * q[:, 0] - prm.gamma * (phi * (1 - phi))[..., None] * nvec)
        f = torch.stack([phi[..., None] * v - fvis, psi[..., None] * v], 1)
        ft = torch.einsum("eiab,efib->efia", self.S, f)
        # Step 5: common normal flux at flux points (computed on the L side)
        vf = velocity(self.vel, self.xf, t, A, B)
        vn = (vf * self.nhat).sum(-1)
        Mf = torch.clamp(torch.sqrt((vf * vf).sum(-1)), min=prm.gamma)
        qpsif = qf[:, kn]
        nvecf = qpsif / torch.clamp(torch.sqrt((qpsif * qpsif).sum(-1)), min=prm.delta)[..., None]
        phif = Uf[:, 0]
        fvisf = Mf[..., None] * (prm.eps * qf[:, 0] - prm.gamma * (phif * (1 - phif))[..., None] * nvecf)
        F_phi = (0.5 * (Uf[:, 0] + Uo[:, 0]) * vn - (self.nhat * fvisf).sum(-1)
                 + prm.tau * (Uf[:, 0] - Uo[:, 0]))
        F_psi = 0.5 * (Uf[:, 1] + Uo[:, 1]) * vn + prm.tau_psi * (Uf[:, 1] - Uo[:, 1])
        if prm.wall == "noflux":   # no normal flux through wall faces
            F_phi = torch.where(self.boundary, torch.zeros_like(F_phi), F_phi)
            F_psi = torch.where(self.boundary, torch.zeros_like(F_psi), F_psi)
        Ft = self.common_to_transformed(torch.stack([F_phi, F_psi], 1))
        div = self.divergence(ft, Ft)                                 # Step 6
        R = -div / self.detJ[:, None, :]
        return R[:, 0], R[:, 1]

    # ---------------------------------------------------------------- preconditioning
    def sensor(self, psi):
        """Resolution indicator s_e (Eq. resolutionIndicator) and nu_s (Eq. nu_s)."""
        prm = self.prm
        chi = torch.einsum("mi,ei->em", self.Vinv, psi)
        tot = (chi * chi).sum(-1)
        hi = (chi * chi * self.high.to(T64)).sum(-1)
        ok = (tot > 0) & (hi > 0)
        s = torch.log10(torch.where(ok, hi, torch.ones_like(hi)) / torch.where(ok, tot, torch.ones_like(tot)))
        lo_b, hi_b = prm.s0 - prm.kappa, prm.s0 + prm.kappa
        ramp = 0.5 * prm.nu_max * (1.0 + torch.sin(math.pi * (s - prm.s0) / (2.0 * prm.kappa)))
        nu = torch.where(s < lo_b, torch.zeros_like(s), torch.where(s > hi_b, torch.full_like(s, prm.nu_max), ramp))
        nu = torch.where(ok, nu, torch.zeros_like(nu))
        return s, nu

    def rhs_pseudo(self, psi, psi0):
        """psi_tau = -J^{-1} div~ g~ + S with g = -nu_s grad psi (Eq. pseudotimesystem)."""
        prm = self.prm
        U = psi[:, None, :]
        Uf = self.trace(U)
        q, Uo = self.gradient(U, Uf)
        qf = torch.einsum("kj,efjb->efkb", self.L, q)
        _, nu = self.sensor(psi)
        g = -nu[:, None, None, None] * q
        gt = torch.einsum("eiab,efib->efia", self.S, g)
        gf = -nu[:, None, None, None] * qf
        F = (self.nhat * gf[:, 0]).sum(-1) + prm.tau_pseudo * (Uf[:, 0] - Uo[:, 0])
        Ft = self.common_to_transformed(F[:, None, :])
        div = self.divergence(gt, Ft)
        qm = torch.sqrt((q[:, 0] * q[:, 0]).sum(-1))
        sgn = torch.tanh(psi0 / torch.clamp(qm, min=prm.delta))
        return -div[:, 0] / self.detJ + sgn * (1.0 - qm)

    def precondition(self, fixed=None):
        """psi0 = phi - 1/2, then RK4 pseudo-time iterations of the preconditioning equation."""
        prm = self.prm
        fixed = prm.pseudo_fixed if fixed is None else fixed
        psi0 = self.phi - 0.5
        psi = psi0
        dtau = prm.pseudo_dtau
        f = lambda y: self.rhs_pseudo(y, psi0)
        it, rms = 0, float("nan")
        for it in range(1, prm.pseudo_kmax + 1):
            k1 = f(psi)
            k2 = f(psi + 0.5 * dtau * k1)
            k3 = f(psi + 0.5 * dtau * k2)
            k4 = f(psi + dtau * k3)
            new = psi + dtau / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
            R = (new - psi) / dtau
            rms = float(torch.sqrt((R * R).sum() / R.numel()))
            psi = new
            if not fixed and rms <= prm.pseudo_tol:
                break
        self.psi = psi
        self.psi0 = psi0
        self.pseudo_iters = it
        self.pseudo_rms = rms
        return it, rms

    # ---------------------------------------------------------------- march
    def initialize(self, circle=None, phi=None, precondition=True):
        self.phi = circle_ic(self.xu, circle) if phi is None else torch.as_tensor(phi, dtype=T64)
        self.psi = self.phi - 0.5
        self.psi0 = self.psi.clone()
        self.t = 0.0
        self.nstep = 0
        if precondition and self.prm.normal == "psi":
            self.precondition()

    def rk4_step(self, A=None, B=None):
        dt, t = self.prm.dt, self.t
        phi, psi = self.phi, self.psi
        a1, b1 = self.rhs(phi, psi, t, A, B)
        a2, b2 = self.rhs(phi + 0.5 * dt * a1, psi + 0.5 * dt * b1, t + 0.5 * dt, A, B)
        a3, b3 = self.rhs(phi + 0.5 * dt * a2, psi + 0.5 * dt * b2, t + 0.5 * dt, A, B)
        a4, b4 = self.rhs(phi + dt * a3, psi + dt * b3, t + dt, A, B)
        self.phi = phi + dt / 6.0 * (a1 + 2 * a2 + 2 * a3 + a4)
        self.psi = psi + dt / 6.0 * (b1 + 2 * b2 + 2 * b3 + b4)
        self.t = t + dt
        self.nstep += 1

    def step(self, n=1, A=None, B=None):
        """n physical steps; psi is reset and preconditioned every n_precond steps
        (the preconditioned method only)."""
        for _ in range(n):
            if self.prm.normal == "psi" and self.nstep > 0 and self.nstep % self.prm.n_precond == 0:
                self.precondition()
            self.rk4_step(A, B)

    # ---------------------------------------------------------------- diagnostics
    def integral(self, u):
        """int u dOmega = sum_e sum_i w_i det J_ei u_ei (exact integral of the interpolant)."""
        return (self.wq[None, :] * self.detJ * u).sum()

    def errors(self, phi_exact):
        """E_L1, E_r of Section 4 against phi_exact at the solution points."""
        el1 = self.integral(torch.abs(self.phi - phi_exact))
        return float(el1), float(el1 / self.integral(phi_exact))

    def mass_error(self, phi0, phi_exact):
        """E_m of Section 4: (int phi - int phi0) / int phi_exact."""
        return float((self.integral(self.phi) - self.integral(phi0)) / self.integral(phi_exact))
