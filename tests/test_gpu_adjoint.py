"""The hand-written adjoint (fr_adjoint_record / fr_adjoint_step) against the
oracle's discrete adjoint (reverse-mode differentiation of the oracle) and
against central finite differences of the CUDA forward map.

Loss: J = 1/2 int (phi_T - phi*)^2 with the solution-point quadrature; the
gradient is taken with respect to phi0 (psi0 = phi0 - 1/2) and the
stream-function coefficients.  Both adjoints differentiate the same discrete
map, so they agree to round-off; against finite differences the bound is
1e-6 relative, the accuracy that Richardson-extrapolated central
differences of the FP64 forward map reach.
"""
import numpy as np
import pytest
import torch

import synthetic as S
from libutil import ensure_built
from oracle import Params
from oracle.adjoint import loss_and_gradients
from oracle.solver import Solver, circle_ic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    import paper_2006_10967_gb300 as G
    return G


def _wl(mesh_fn, p, h, n_modes, seed=4, sigma=0.05):
    kx, ky, A, B = S.stream_coefficients(n_modes, seed=seed, sigma=sigma)
    vel = S.Velocity("stream", T=0.0, kx=kx, ky=ky, A=A, B=B)
    w = S.Workload("adj", mesh_fn, p, vel, S.Circle((0.5, 0.5), 0.3, 6.0), t_end=1.0, h=h)
    w.eps = 0.06 * h / p
    w.nu_max = 0.15 * h / p
    w.pseudo_dtau = 0.1 * h / (p + 1)
    w.dt = 0.004
    return w


def _gpu_grad(G, w, mesh, phi0, phis, n, ck):
    M = G.Mesh.from_synthetic(mesh, w.order)
    F = G.Field(M, G.make_params(w), phi0=phi0, precondition=False)
    F.adjoint_record(n, ck)
    phiT = F.get(0)
    wq = M.quadrature()
    J = 0.5 * float((wq * (phiT - phis) ** 2).sum())
    gT = torch.from_numpy(wq * (phiT - phis)).cuda()
    nc = 2 * len(w.velocity.A) if w.velocity.kind == "stream" else 0
    du0, dc = F.adjoint_step(gT, None, nc)
    return J, (du0[0] + du0[1]).cpu().numpy(), (dc.cpu().numpy() if dc is not None else None), F


@pytest.mark.parametrize("kind", ["quad", "hex"])
def test_adjoint_matches_oracle_adjoint(G, kind):
    if kind == "quad":
        w = _wl(lambda: S.quad_grid(4, jitter=0.1, seed=3, shuffle_seed=1, rotate_seed=2), 3, 0.25, 4)
    else:
        w = _wl(lambda: S.hex_grid(2, periodic=(True, True, True), jitter=0.05, seed=3), 2, 0.5, 4)
        w.velocity = S.Velocity("leveque", T=3.0)
        w.circle = S.Circle((0.5, 0.5, 0.5), 0.3, 6.0)
    mesh = w.mesh()
    prm = Params.from_workload(w)
    sol = Solver(mesh, w.order, prm, w.velocity)
    phi0 = circle_ic(sol.xu, w.circle).numpy()
    c = (0.55, 0.45, 0.5)[: mesh.dim]
    phis = circle_ic(sol.xu, S.Circle(c, 0.3, 6.0)).numpy()
    n, ck = 5, 2
    J, gphi, gc, F = _gpu_grad(G, w, mesh, phi0, phis, n, ck)
    if kind == "quad":
        Jo, gphio, gAo, gBo = loss_and_gradients(mesh, w.order, prm, w.velocity, phi0, phis, n)
        assert J == pytest.approx(Jo, rel=1e-12)
        rel = np.abs(gphi - gphio.numpy()).max() / np.abs(gphio.numpy()).max()
        assert rel < 1e-9
        go = np.concatenate([gAo.numpy(), gBo.numpy()])
        assert np.abs(gc - go).max() / np.abs(go).max() < 1e-9
    else:
        # LeVeque field: gradient with respect to phi0 only (oracle via autograd)
        phi0t = torch.tensor(phi0, requires_grad=True)
        s2 = Solver(mesh, w.order, prm, w.velocity)
        s2.initialize(phi=phi0t, precondition=False)
        for _ in range(n):
            s2.rk4_step()
        Jt = 0.5 * s2.integral((s2.phi - torch.tensor(phis)) ** 2)
        (go,) = torch.autograd.grad(Jt, (phi0t,))
        assert J == pytest.approx(float(Jt.detach()), rel=1e-12)
        assert np.abs(gphi - go.numpy()).max() / np.abs(go.numpy()).max() < 1e-9
    # the field is left at the end of the window
    st = F.stats()
    assert st["n_steps"] == n


def _small_case(kind):
    if kind == "quad":
        w = _wl(lambda: S.quad_grid(4, jitter=0.1, seed=3, shuffle_seed=1, rotate_seed=2), 3, 0.25, 4)
    elif kind == "tri":
        w = _wl(lambda: S.tri_delaunay(5, seed=2, shuffle_seed=3), 3, 0.2, 4)
    else:
        w = _wl(lambda: S.hex_grid(2, periodic=(True, True, True), jitter=0.05, seed=3), 2, 0.5, 4)
        w.velocity = S.Velocity("leveque", T=3.0)
        w.circle = S.Circle((0.5, 0.5, 0.5), 0.3, 6.0)
    return w


@pytest.mark.parametrize("kind", ["quad", "tri", "hex"])
def test_preconditioned_adjoint_matches_oracle_adjoint(G, kind):
    """With the t = 0 preconditioning inside the window (psi0 = psi =
    phi0 - 1/2, then a fixed count of pseudo-time RK4 iterations): the
    gradient with respect to phi0 follows both paths, phi0 and psi =
    P(phi0 - 1/2), through the element viscosity's dependence on psi (the
    resolution indicator), the flux -nu_s q, the penalty and the source
    tanh(psi0 / |q|)(1 - |q|).  Against the oracle's discrete adjoint (torch
    autograd through its preconditioning and march) to round-off."""
    w = _small_case(kind)
    w.pseudo_kmax = 3
    mesh = w.mesh()
    prm = Params.from_workload(w, pseudo_fixed=True)
    sol = Solver(mesh, w.order, prm, w.velocity)
    phi0 = circle_ic(sol.xu, w.circle).numpy()
    c = (0.55, 0.45, 0.5)[: mesh.dim]
    phis = circle_ic(sol.xu, S.Circle(c, 0.3, 6.0)).numpy()
    n, ck = 5, 2
    M = G.Mesh.from_synthetic(mesh, w.order)
    F = G.Field(M, G.make_params(w, pseudo_fixed=True), phi0=phi0, precondition=False)
    F.adjoint_record(n, ck, precondition=True)
    phiT = F.get(0)
    wq = M.quadrature()
    J = 0.5 * float((wq * (phiT - phis) ** 2).sum())
    nc = 2 * len(w.velocity.A) if w.velocity.kind == "stream" else 0
    du0, dc = F.adjoint_step(torch.from_numpy(wq * (phiT - phis)).cuda(), None, nc)
    assert F.sync() == 0
    assert float(du0[1].abs().max()) == 0.0
    gphi = du0[0].cpu().numpy()
    # the preconditioning's sensor is active: some element viscosities lie on the ramp
    sol.initialize(phi=torch.tensor(phi0), precondition=False)
    _, nu = sol.sensor(sol.phi - 0.5)
    assert float(nu.max()) > 0.0
    phi0t = torch.tensor(phi0, requires_grad=True)
    s2 = Solver(mesh, w.order, prm, w.velocity)
    stream = w.velocity.kind == "stream"
    if stream:
        A = torch.as_tensor(w.velocity.A, dtype=torch.float64).clone().requires_grad_(True)
        B = torch.as_tensor(w.velocity.B, dtype=torch.float64).clone().requires_grad_(True)
    else:
        A = B = None
    s2.initialize(phi=phi0t, precondition=True)
    for _ in range(n):
        s2.rk4_step(A, B)
    Jt = 0.5 * s2.integral((s2.phi - torch.tensor(phis)) ** 2)
    assert J == pytest.approx(float(Jt.detach()), rel=1e-12)
    if stream:
        go, gA, gB = torch.autograd.grad(Jt, (phi0t, A, B))
        gco = np.concatenate([gA.numpy(), gB.numpy()])
        assert np.abs(dc.cpu().numpy() - gco).max() / np.abs(gco).max() < 1e-9
    else:
        (go,) = torch.autograd.grad(Jt, (phi0t,))
    assert np.abs(gphi - go.numpy()).max() / np.abs(go.numpy()).max() < 1e-9
    # the path through the preconditioning matters: without it the gradient differs
    F2 = G.Field(M, G.make_params(w, pseudo_fixed=True), phi0=phi0, precondition=False)
    F2.adjoint_record(n, ck)
    du2, _ = F2.adjoint_step(torch.from_numpy(wq * (F2.get(0) - phis)).cuda(), None, nc)
    assert np.abs((du2[0] + du2[1]).cpu().numpy() - gphi).max() > 1e-6 * np.abs(gphi).max()


def test_preconditioned_mixed_adjoint_against_fp64(G):
    """The same on the FP32 forward march (the preconditioning and every
    segment recomputed in FP64 for the sweep) against the FP64 adjoint."""
    w = _small_case("quad")
    w.pseudo_kmax = 3
    mesh = w.mesh()
    M = G.Mesh.from_synthetic(mesh, w.order)
    xu = M.solution_points()
    phi0 = 0.5 * (1 + np.tanh(6.0 * (0.3 - np.sqrt(((xu - 0.5) ** 2).sum(-1)))))
    phis = 0.5 * (1 + np.tanh(6.0 * (0.3 - np.sqrt(((xu - np.array([0.55, 0.45])) ** 2).sum(-1)))))
    wq = M.quadrature()
    out = {}
    for prec in ("fp64", "mixed"):
        F = G.Field(M, G.make_params(w, prec, pseudo_fixed=True), phi0=phi0, precondition=False)
        F.adjoint_record(5, 2, precondition=True)
        du0, dc = F.adjoint_step(torch.from_numpy(wq * (F.get(0) - phis)).cuda(), None, 2 * len(w.velocity.A))
        assert F.sync() == 0
        out[prec] = (du0[0].cpu().numpy(), dc.cpu().numpy())
    g64, c64 = out["fp64"]
    g32, c32 = out["mixed"]
    assert np.abs(g32 - g64).max() / np.abs(g64).max() < 1e-3
    assert np.abs(c32 - c64).max() / np.abs(c64).max() < 1e-3


@pytest.mark.parametrize("kind", ["delaunay_p3", "split_p2"])
def test_triangle_adjoint_matches_oracle_adjoint(G, kind):
    """Triangles (dense operators, one affine metric per element; the two
    sides of an edge see different reference edges, so the adjoint of the
    common flux weighs each side's lift adjoint by its own face scale):
    gradient with respect to phi0 and the stream-function coefficients
    against the oracle's reverse-mode adjoint, FP64 to round-off; the mixed
    field (FP32 march, FP64 recomputation) against the FP64 gradient."""
    if kind == "delaunay_p3":
        w = _wl(lambda: S.tri_delaunay(5, seed=2, shuffle_seed=3), 3, 0.2, 4)
    else:
        w = _wl(lambda: S.tri_split(4, shuffle_seed=1), 2, 0.25, 4)
    mesh = w.mesh()
    prm = Params.from_workload(w)
    sol = Solver(mesh, w.order, prm, w.velocity)
    phi0 = circle_ic(sol.xu, w.circle).numpy()
    phis = circle_ic(sol.xu, S.Circle((0.55, 0.45), 0.3, 6.0)).numpy()
    n, ck = 5, 2
    J, gphi, gc, F = _gpu_grad(G, w, mesh, phi0, phis, n, ck)
    assert F.sync() == 0
    Jo, gphio, gAo, gBo = loss_and_gradients(mesh, w.order, prm, w.velocity, phi0, phis, n)
    assert J == pytest.approx(Jo, rel=1e-12)
    assert np.abs(gphi - gphio.numpy()).max() / np.abs(gphio.numpy()).max() < 1e-9
    go = np.concatenate([gAo.numpy(), gBo.numpy()])
    assert np.abs(gc - go).max() / np.abs(go).max() < 1e-9
    M = G.Mesh.from_synthetic(mesh, w.order)
    Fm = G.Field(M, G.make_params(w, "mixed"), phi0=phi0, precondition=False)
    Fm.adjoint_record(n, ck)
    wq = M.quadrature()
    du0, dc = Fm.adjoint_step(torch.from_numpy(wq * (Fm.get(0) - phis)).cuda(), None, len(go))
    assert Fm.sync() == 0
    g32 = (du0[0] + du0[1]).cpu().numpy()
    assert np.abs(g32 - gphi).max() / np.abs(gphi).max() < 1e-4
    assert np.abs(dc.cpu().numpy() - gc).max() / np.abs(gc).max() < 1e-4


def test_adjoint_c5_against_central_differences(G):
    """The adjoint workload: 64^2 periodic quads, p = 4, 400 RK4 steps, velocity
    from 32 stream-function coefficients, checkpoints every 20 steps."""
    w = S.workload("c5")
    mesh = w.mesh()
    M = G.Mesh.from_synthetic(mesh, w.order)
    xu = M.solution_points()
    def circ(c):
        return 0.5 * (1 + np.tanh(c.beta * (c.radius - np.sqrt(((xu - np.array(c.centre)) ** 2).sum(-1)))))
    phi0 = circ(w.circle)
    phis = circ(w.extra["target"])
    n, ck = w.n_steps, w.extra["ckpt_every"]
    J, gphi, gc, _ = _gpu_grad(G, w, mesh, phi0, phis, n, ck)
    wq = M.quadrature()

    def loss(phi0_, A=None, B=None):
        vel = w.velocity
        if A is not None:
            vel = S.Velocity("stream", T=0.0, kx=vel.kx, ky=vel.ky, A=A, B=B)
        F = G.Field(M, G.make_params(w, velocity=vel), phi0=phi0_, precondition=False)
        F.step(n)
        return 0.5 * float((wq * (F.get(0) - phis) ** 2).sum())

    # Central differences of this strongly nonlinear 400-step map converge to
    # the adjoint only as the step shrinks (relative gap 4.5e-4 at h = 1e-6 on
    # GB300), and below 1e-7 FP64 round-off grows; Richardson extrapolation of
    # the steps 2e-7 and 1e-7 removes the O(h^2) term.
    rng = np.random.default_rng(7)
    d = rng.normal(size=phi0.shape) * (phi0 * (1 - phi0) > 0.01)   # a direction near the interface

    def fd(f, h):
        return (4.0 * (f(h / 2) - f(-h / 2)) / h - (f(h) - f(-h)) / (2 * h)) / 3.0

    g_fd = fd(lambda e: loss(phi0 + e * d), 2e-7)
    assert float((gphi * d).sum()) == pytest.approx(g_fd, rel=1e-6)
    A0, B0 = w.velocity.A, w.velocity.B
    for m in (0, 5):
        def fA(e, m=m):
            Ap = A0.copy()
            Ap[m] += e
            return loss(phi0, Ap, B0)

        def fB(e, m=m):
            Bp = B0.copy()
            Bp[m] += e
            return loss(phi0, A0, Bp)
        assert gc[m] == pytest.approx(fd(fA, 2e-7), rel=1e-6)
        assert gc[len(A0) + m] == pytest.approx(fd(fB, 2e-7), rel=1e-6)


def _grad_c5(G, precision):
    w = S.workload("c5")
    mesh = w.mesh()
    M = G.Mesh.from_synthetic(mesh, w.order)
    xu = M.solution_points()

    def circ(c):
        return 0.5 * (1 + np.tanh(c.beta * (c.radius - np.sqrt(((xu - np.array(c.centre)) ** 2).sum(-1)))))
    phi0, phis = circ(w.circle), circ(w.extra["target"])
    F = G.Field(M, G.make_params(w, precision), phi0=phi0, precondition=False)
    F.adjoint_record(w.n_steps, w.extra["ckpt_every"])
    phiT = F.get(0)
    wq = M.quadrature()
    du0, dc = F.adjoint_step(torch.from_numpy(wq * (phiT - phis)).cuda(), None, 2 * len(w.velocity.A))
    assert F.sync() == 0
    return phiT, (du0[0] + du0[1]).cpu().numpy(), dc.cpu().numpy()


def test_mixed_adjoint_c5_against_fp64_adjoint(G):
    """The adjoint workload with the FP32 (mixed-precision) forward march:
    FP32 checkpoints every 20 steps, each segment recomputed in FP64 for the
    sweep, against the FP64 adjoint (checked against central differences
    above).  The two linearise along trajectories that differ by the FP32
    march's deviation (6e-7 of max |phi| at t = T), and this 400-step map
    is strongly nonlinear (its central differences with step 1e-6 are still
    4.5e-4 away from the derivative): the gradients agree to a
    few percent in L2 (2.3 % in max norm on GB300), the coefficient
    gradient, a sum over the whole field, to 1e-3; on 20 steps of the same
    problem they agree to 3e-7."""
    phi64, g64, c64 = _grad_c5(G, "fp64")
    phi32, g32, c32 = _grad_c5(G, "mixed")
    traj = np.abs(phi32 - phi64).max() / np.abs(phi64).max()
    assert traj < 1e-5
    rel2 = np.linalg.norm(g32 - g64) / np.linalg.norm(g64)
    relc = np.abs(c32 - c64).max() / np.abs(c64).max()
    assert rel2 < 0.05, (rel2, relc)
    assert relc < 1e-3, (rel2, relc)
    cos = float((g32 * g64).sum() / (np.linalg.norm(g32) * np.linalg.norm(g64)))
    assert cos > 0.999, cos


def test_autograd_function_wraps_the_adjoint(G):
    w = _wl(lambda: S.quad_grid(3, jitter=0.1, seed=5), 2, 1 / 3, 3)
    mesh = w.mesh()
    M = G.Mesh.from_synthetic(mesh, w.order)
    kx, ky = w.velocity.kx, w.velocity.ky

    def params_fn(coef):
        m = len(kx)
        vel = S.Velocity("stream", T=0.0, kx=kx, ky=ky, A=coef[:m], B=coef[m:])
        return G.make_params(w, velocity=vel)

    flow = G.flow_function(M, params_fn, n_steps=4, ckpt_every=3)
    xu = M.solution_points()
    phi0 = torch.tensor(0.5 * (1 + np.tanh(4.0 * (0.3 - np.sqrt(((xu - 0.5) ** 2).sum(-1))))), requires_grad=True)
    coef = torch.tensor(np.concatenate([w.velocity.A, w.velocity.B]), requires_grad=True)
    wq = torch.tensor(M.quadrature())
    phiT = flow(phi0, coef)
    J = 0.5 * (wq * phiT.cpu() ** 2).sum()
    J.backward()
    assert phi0.grad is not None and coef.grad is not None
    assert torch.isfinite(phi0.grad).all() and torch.isfinite(coef.grad).all()
    # compare with Richardson-extrapolated central differences along a seeded
    # direction; the bound is relative to |grad J| |d| (the directional
    # derivative itself can nearly cancel)
    d = torch.randn(phi0.shape, generator=torch.Generator().manual_seed(7), dtype=phi0.dtype)

    def cd(h):
        with torch.no_grad():
            jp = 0.5 * (wq * flow(phi0 + h * d, coef).cpu() ** 2).sum()
            jm = 0.5 * (wq * flow(phi0 - h * d, coef).cpu() ** 2).sum()
        return float((jp - jm) / (2 * h))

    fd = (4.0 * cd(5e-7) - cd(1e-6)) / 3.0
    ad = float((phi0.grad * d).sum())
    assert abs(ad - fd) <= 1e-7 * float(phi0.grad.norm() * d.norm())
