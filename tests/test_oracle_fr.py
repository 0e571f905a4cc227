"""Pins for the oracle's FR residual, RK march, sensor and preconditioning.

Each check is fixed by mathematics rather than by the oracle itself: exactness
on polynomials, free-stream preservation, discrete conservation, the tanh
equilibrium of the diffusion/sharpening balance, convergence rates against
exact translated solutions, the temporal order of RK4, closed-form sensor
values and the sign of the reinitialisation source.
"""
import math

import numpy as np
import pytest
import torch

import synthetic as S
from oracle import Params, Solver
from oracle.element import ref_element

T64 = torch.float64


def _solver(mesh, p, vel, **kw):
    prm = Params(**{**dict(gamma=0.09, eps=0.01, tau=0.1, dt=1e-3, pseudo_dtau=1e-3,
                           nu_max=0.01), **kw})
    return Solver(mesh, p, prm, vel)


WALL_MESHES = [
    ("quad", lambda: S.quad_grid(3, periodic=(False, False), shuffle_seed=1, rotate_seed=2), [2, 3]),
    ("tri", lambda: S.tri_split(3, periodic=(False, False), shuffle_seed=1), [2, 3]),
    ("tri", lambda: S.tri_delaunay(5, jitter=0.1, seed=7), [2]),
    ("hex", lambda: S.hex_grid(2, shuffle_seed=3), [2]),
    ("hex", lambda: S.hex_grid(2, shuffle_seed=3, rotate_seed=7), [2, 3]),
]


def _cases():
    for et, mk, ps in WALL_MESHES:
        for p in ps:
            yield et, mk, p


@pytest.mark.parametrize("et,mk,p", list(_cases()))
def test_gradient_exact_for_polynomials(et, mk, p):
    """Affine meshes: a global polynomial of degree <= p has continuous traces,
    so every correction vanishes and q is its exact gradient (Steps 1-3)."""
    mesh = mk()
    s = _solver(mesh, p, S.Velocity("uniform", a=(1.0, 0.5, 0.25)))
    x = s.xu
    dim = x.shape[-1]
    u = 0.3 + x[..., 0] ** 2 - 0.7 * x[..., 0] * x[..., 1] + 0.2 * x[..., 1]
    gx = 2 * x[..., 0] - 0.7 * x[..., 1]
    gy = -0.7 * x[..., 0] + 0.2 + 0 * x[..., 0]
    if dim == 3:
        u = u + 0.4 * x[..., 2] * x[..., 1]
        gy = gy + 0.4 * x[..., 2]
        gz = 0.4 * x[..., 1]
    U = torch.stack([u, u], 1)
    q, _ = s.gradient(U, s.trace(U))
    assert torch.allclose(q[:, 0, :, 0], gx, atol=1e-11)
    assert torch.allclose(q[:, 0, :, 1], gy, atol=1e-11)
    if dim == 3:
        assert torch.allclose(q[:, 0, :, 2], gz, atol=1e-11)


def test_gradient_exact_for_linear_on_bilinear_quads():
    mesh = S.quad_grid(4, periodic=(False, False), jitter=0.15, seed=5, shuffle_seed=2, rotate_seed=3)
    for p in (1, 2, 3):
        s = _solver(mesh, p, S.Velocity("uniform", a=(1.0, 0.5)))
        x = s.xu
        u = 0.25 + 1.5 * x[..., 0] - 0.75 * x[..., 1]
        U = torch.stack([u, u], 1)
        q, _ = s.gradient(U, s.trace(U))
        assert torch.allclose(q[:, 0, :, 0], torch.full_like(u, 1.5), atol=1e-11)
        assert torch.allclose(q[:, 0, :, 1], torch.full_like(u, -0.75), atol=1e-11)


@pytest.mark.parametrize("et,mk,p", list(_cases()))
def test_residual_exact_for_quadratic_advection_diffusion(et, mk, p):
    """Uniform velocity and gamma = 0 (the multiplier is |v| and the sharpening term
    vanishes), phi quadratic: R = -v.grad phi + |v| eps lap phi exactly (Steps 1-6 on
    affine meshes, copy ghost states on the walls).  gamma = 0 also keeps the test
    away from the normal of a constant psi, which is round-off divided by delta."""
    mesh = mk()
    a = (1.0, 0.5, 0.25)
    s = _solver(mesh, p, S.Velocity("uniform", a=a), gamma=0.0, eps=0.02, tau=0.3)
    x = s.xu
    dim = x.shape[-1]
    v = torch.tensor(a[:dim], dtype=T64)
    M = float(torch.linalg.norm(v))
    phi = 0.3 + x[..., 0] ** 2 - 0.7 * x[..., 0] * x[..., 1] + 0.2 * x[..., 1]
    gx = 2 * x[..., 0] - 0.7 * x[..., 1]
    gy = -0.7 * x[..., 0] + 0.2
    lap = 2.0
    adv = v[0] * gx + v[1] * gy
    if dim == 3:
        phi = phi + 0.4 * x[..., 2] ** 2
        adv = adv + v[2] * 0.8 * x[..., 2]
        lap = 2.8
    psi = torch.full_like(phi, 0.125)
    Rphi, Rpsi = s.rhs(phi, psi, 0.0)
    assert torch.allclose(Rphi, -adv + M * 0.02 * lap, atol=1e-9)
    assert torch.allclose(Rpsi, torch.zeros_like(Rpsi), atol=1e-10)


@pytest.mark.parametrize("mk,p", [
    (lambda: S.quad_grid(4, jitter=0.15, seed=3, shuffle_seed=4, rotate_seed=5), 3),
    (lambda: S.tri_split(4, shuffle_seed=2), 3),
    (lambda: S.hex_grid(2, periodic=(True, True, True), jitter=0.1, seed=2), 2),
    (lambda: S.hex_grid(2, periodic=(True, True, True), jitter=0.1, seed=2, rotate_seed=3), 2),
])
def test_free_stream_preserved(mk, p):
    """Constant states under a uniform velocity have zero residual: with gamma = 0
    any constant phi (psi constant too), and with gamma > 0 the pure phases
    phi = 0, 1 whatever psi is (their sharpening flux phi(1-phi)n vanishes)."""
    mesh = mk()
    vel = S.Velocity("uniform", a=(1.0, 0.5, 0.25))
    s0 = _solver(mesh, p, vel, gamma=0.0)
    s1 = _solver(mesh, p, vel, gamma=0.09)
    x = s0.xu
    wavy = 0.1 * torch.sin(2 * math.pi * x[..., 0]) + 0.05 * torch.cos(2 * math.pi * x[..., 1])
    for c in (0.0, 1.0, 0.3):
        phi = torch.full((s0.E, s0.Nu), c, dtype=T64)
        Rphi, Rpsi = s0.rhs(phi, torch.full_like(phi, c - 0.5), 0.1)
        assert float(Rphi.abs().max()) < 1e-12
        assert float(Rpsi.abs().max()) < 1e-12
        if c in (0.0, 1.0):
            Rphi, _ = s1.rhs(phi, wavy, 0.1)
            assert float(Rphi.abs().max()) < 1e-12


@pytest.mark.parametrize("mk,p,vel", [
    (lambda: S.quad_grid(5, jitter=0.15, seed=3, shuffle_seed=4, rotate_seed=5), 3,
     S.Velocity("rider_kothe", T=8.0)),
    (lambda: S.tri_split(5, shuffle_seed=2), 3, S.Velocity("rider_kothe", T=8.0)),
    (lambda: S.hex_grid(3, periodic=(True, True, True), jitter=0.1, seed=2), 2,
     S.Velocity("leveque", T=3.0)),
    (lambda: S.hex_grid(3, periodic=(True, True, True), jitter=0.1, seed=2, rotate_seed=8), 2,
     S.Velocity("leveque", T=3.0)),
])
def test_discrete_conservation(mk, p, vel):
    """Periodic meshes: sum_e sum_i w_i det J_i R_i = 0 up to round-off (F_R = -F_L)."""
    mesh = mk()
    s = _solver(mesh, p, vel)
    c = (0.45, 0.55, 0.5)[: mesh.dim]
    s.initialize(S.Circle(c, 0.2, 20.0), precondition=False)
    s.psi = s.psi + 0.05 * torch.sin(7 * s.xu[..., 0])        # a non-trivial normal field
    Rphi, Rpsi = s.rhs(s.phi, s.psi, 0.7)
    scale = float(s.integral(Rphi.abs()))
    assert abs(float(s.integral(Rphi))) < 1e-13 * max(scale, 1.0)
    assert abs(float(s.integral(Rpsi))) < 1e-13 * max(float(s.integral(Rpsi.abs())), 1.0)


def _planar(s, w):
    x = s.xu[..., 0]
    return 0.5 * (1 + torch.tanh((x - 0.5) / (2 * w)))


def test_equilibrium_profile_and_sharpening_sign():
    """u = 0: the tanh profile of width eps/gamma balances diffusion against
    sharpening (Section 2), so its residual is small and falls with h; a profile
    twice as wide is steepened (phi falls left of the interface, rises right)."""
    gamma, eps = 0.09, 0.09 * 0.06
    res = []
    for n in (16, 32):
        mesh = S.quad_grid(n, periodic=(False, True))
        s = _solver(mesh, 4, S.Velocity("uniform", a=(0.0, 0.0)), gamma=gamma, eps=eps)
        phi = _planar(s, eps / gamma)
        Rphi, _ = s.rhs(phi, phi - 0.5, 0.0)
        res.append(float(Rphi.abs().max()))
        if n == 32:
            wide = _planar(s, 2 * eps / gamma)
            Rw, _ = s.rhs(wide, wide - 0.5, 0.0)
            assert float(Rw.abs().max()) > 20 * res[-1]
            x = s.xu[..., 0]
            band = (x - 0.5).abs() < 0.1
            assert float(Rw[band & (x < 0.5)].sum()) < 0
            assert float(Rw[band & (x > 0.5)].sum()) > 0
    assert res[1] < res[0] / 4


def test_unpreconditioned_normal_comes_from_phi_alone():
    """Unpreconditioned CPF (Eq. altconservativephasefieldeq, n = grad phi/|grad phi|):
    phi's residual does not depend on psi at all, while the preconditioned
    method's does; with psi = phi - 1/2 the two normals coincide."""
    mesh = S.quad_grid(6, jitter=0.1, seed=2)
    vel = S.Velocity("rider_kothe", T=8.0)
    sp = _solver(mesh, 3, vel, gamma=0.09, eps=0.09 * 0.05)
    sc = _solver(mesh, 3, vel, gamma=0.09, eps=0.09 * 0.05, normal="phi")
    x = sc.xu
    r = torch.sqrt((x[..., 0] - 0.45) ** 2 + (x[..., 1] - 0.55) ** 2)
    phi = 0.5 * (1 + torch.tanh(8.0 * (0.25 - r)))
    other = 0.3 * torch.sin(5 * x[..., 0]) * torch.cos(3 * x[..., 1]) + (x[..., 1] - 0.5)
    Rc1, _ = sc.rhs(phi, phi - 0.5, 0.3)
    Rc2, _ = sc.rhs(phi, other, 0.3)
    assert torch.equal(Rc1, Rc2)
    Rp1, _ = sp.rhs(phi, phi - 0.5, 0.3)
    Rp2, _ = sp.rhs(phi, other, 0.3)
    assert float((Rp1 - Rp2).abs().max()) > 1e-3 * float(Rp1.abs().max())
    assert float((Rc1 - Rp1).abs().max()) <= 1e-12 * float(Rp1.abs().max())


def test_unpreconditioned_equilibrium_profile():
    """u = 0, unpreconditioned CPF: the planar tanh of width eps/gamma is
    stationary up to a residual that falls with h, whatever psi holds."""
    gamma, eps = 0.09, 0.09 * 0.06
    res = []
    for n in (16, 32):
        mesh = S.quad_grid(n, periodic=(False, True))
        s = _solver(mesh, 4, S.Velocity("uniform", a=(0.0, 0.0)), gamma=gamma, eps=eps, normal="phi")
        phi = _planar(s, eps / gamma)
        junk = torch.cos(7 * s.xu[..., 1]) * s.xu[..., 0]
        Rphi, _ = s.rhs(phi, junk, 0.0)
        res.append(float(Rphi.abs().max()))
    assert res[1] < res[0] / 4


def test_unpreconditioned_march_skips_preconditioning():
    """No psi reset or pseudo-time iterations in the unpreconditioned method."""
    mesh = S.quad_grid(4)
    runs = []
    for n_precond in (2, 10 ** 6):
        s = _solver(mesh, 2, S.Velocity("uniform", a=(1.0, 0.5)), gamma=0.09, eps=0.01, dt=1e-3,
                    normal="phi", n_precond=n_precond, pseudo_kmax=3, pseudo_dtau=1e-3, nu_max=0.01)
        it0 = s.pseudo_iters
        s.initialize(S.Circle((0.5, 0.5), 0.25, 6.0), precondition=True)
        psi_before = s.psi.clone()
        s.step(5)
        assert s.pseudo_iters == it0
        assert not torch.equal(psi_before, s.psi)
        runs.append((s.phi, s.psi))
    assert torch.equal(runs[0][0], runs[1][0]) and torch.equal(runs[0][1], runs[1][1])


def test_paper_parameters_make_the_initial_profile_an_equilibrium():
    """gamma = 0.09, eps = 0.06 h/p (Section 2) and beta = 3p/(4h) (Section 4):
    the initial width 1/(2 beta) equals eps/gamma."""
    for name in ("c2q", "c2t", "c3"):
        w = S.workload(name)
        assert w.gamma == 0.09
        assert w.eps == pytest.approx(0.06 * w.h / w.order)
        assert w.circle.beta == pytest.approx(3 * w.order / (4 * w.h))
        assert w.eps / w.gamma == pytest.approx(1 / (2 * w.circle.beta), rel=1e-12)


def _advect_error(n, p, dt, t_end=0.25):
    mesh = S.quad_grid(n, jitter=0.0)
    s = _solver(mesh, p, S.Velocity("uniform", a=(1.0, 0.5)), gamma=0.0, eps=0.0, tau=0.1, dt=dt)
    x = s.xu
    f = lambda X, Y: torch.sin(2 * math.pi * X) * torch.sin(2 * math.pi * Y)
    s.phi = f(x[..., 0], x[..., 1])
    s.psi = torch.zeros_like(s.phi)
    nsteps = int(round(t_end / dt))
    for _ in range(nsteps):
        s.rk4_step()
    ex = f(x[..., 0] - 1.0 * s.t, x[..., 1] - 0.5 * s.t)
    return float(torch.sqrt(s.integral((s.phi - ex) ** 2)))


@pytest.mark.parametrize("p", [2, 3])
def test_translation_converges_at_high_order(p):
    """Smooth translation with the central inviscid flux plus a small penalty:
    the L2 error falls at least like h^p (h^{p+1} is the upwind optimum)."""
    e1 = _advect_error(8, p, 0.25 / 128)
    e2 = _advect_error(16, p, 0.25 / 256)
    rate = math.log2(e1 / e2)
    assert rate > p


def test_rk4_temporal_order():
    ref = None
    mesh = S.quad_grid(4)

    def run(dt):
        s = _solver(mesh, 3, S.Velocity("uniform", a=(1.0, 0.5)), gamma=0.0, eps=0.0, dt=dt)
        x = s.xu
        s.phi = torch.sin(2 * math.pi * x[..., 0]) * torch.cos(2 * math.pi * x[..., 1])
        s.psi = torch.zeros_like(s.phi)
        for _ in range(int(round(0.2 / dt))):
            s.rk4_step()
        return s.phi
    ref = run(0.2 / 256)
    e1 = float((run(0.2 / 8) - ref).abs().max())
    e2 = float((run(0.2 / 16) - ref).abs().max())
    assert math.log2(e1 / e2) > 3.7


def test_sensor_closed_forms():
    """s_e = log10(sum of squared truncated modes / sum of squared modes)."""
    for et, mesh in (("quad", S.quad_grid(1)), ("tri", S.tri_split(1)), ("hex", S.hex_grid(1))):
        p = 3
        s = _solver(mesh, p, S.Velocity("uniform", a=(1.0, 0.0, 0.0)), s0=-5.0, kappa=5.0, nu_max=0.3)
        el = ref_element(et, p)
        V = torch.as_tensor(el.V)
        hi = torch.as_tensor(el.high)
        E = s.E
        chi = torch.zeros(E, el.nu, dtype=T64)
        chi[:, 0] = 1.0
        # polynomial of lower degree: no truncated energy -> nu = 0
        _, nu = s.sensor(chi @ V.T)
        assert torch.all(nu == 0)
        # a single highest mode: s = 0 -> nu = nu_max
        chi2 = torch.zeros_like(chi)
        chi2[:, int(torch.nonzero(hi)[0])] = 2.0
        sv, nu = s.sensor(chi2 @ V.T)
        assert torch.allclose(sv, torch.zeros_like(sv), atol=1e-12)
        assert torch.allclose(nu, torch.full_like(nu, 0.3))
        # prescribed ratio 10^-5 -> s = s0 -> nu = nu_max/2
        a2 = 1e-5 / (1 - 1e-5)
        chi3 = chi.clone()
        chi3[:, int(torch.nonzero(hi)[0])] = math.sqrt(a2)
        sv, nu = s.sensor(chi3 @ V.T)
        assert torch.allclose(sv, torch.full_like(sv, -5.0), atol=1e-9)
        assert torch.allclose(nu, torch.full_like(nu, 0.15), atol=1e-9)
        # s = s0 - kappa/3: ramp value (1 + sin(-pi/6))/2 * nu_max
        r = 10 ** (-5 - 5 / 3)
        chi4 = chi.clone()
        chi4[:, int(torch.nonzero(hi)[0])] = math.sqrt(r / (1 - r))
        _, nu = s.sensor(chi4 @ V.T)
        assert torch.allclose(nu, torch.full_like(nu, 0.15 * (1 + math.sin(-math.pi / 6))), atol=1e-9)


def test_sensor_truncation_by_degree():
    """The truncated modes are those of max degree p (tensor) or total degree
    p (triangle): their count is (p+1)^d - p^d or p + 1; a polynomial of degree
    p - 1, sampled at the solution points, has no energy in them (nu = 0) and
    one of degree p has some."""
    import numpy as np
    for et, mesh, d in (("quad", S.quad_grid(1), 2), ("tri", S.tri_split(1), 2), ("hex", S.hex_grid(1), 3)):
        for p in (2, 3, 4):
            el = ref_element(et, p)
            assert int(el.high.sum()) == (p + 1 if et == "tri" else (p + 1) ** d - p ** d)
            s = _solver(mesh, p, S.Velocity("uniform", a=(1.0, 0.0, 0.0)), s0=-5.0, kappa=5.0, nu_max=0.3)
            x = s.xu
            low = (x[..., 0] + 0.3 * x[..., 1]) ** (p - 1) + 0.2
            top = x[..., 0] ** p + 0.2
            tot_lo, tot_hi = [], []
            for u in (low, top):
                chi = torch.einsum("mi,ei->em", torch.as_tensor(el.Vinv), u)
                tot_hi.append(float((chi[:, torch.as_tensor(el.high)] ** 2).sum()))
                tot_lo.append(float((chi ** 2).sum()))
            assert tot_hi[0] < 1e-24 * tot_lo[0]
            assert tot_hi[1] > 1e-6 * tot_lo[1]
            _, nu = s.sensor(low)
            assert torch.all(nu == 0)


def test_preconditioning_fixed_point_and_sign():
    """psi = x - 1/2 (|grad psi| = 1) is a fixed point of the preconditioning equation;
    psi = 2(x - 1/2) relaxes towards slope one (source of Eq. pseudotimesystem)."""
    mesh = S.quad_grid(6, periodic=(False, True))
    s = _solver(mesh, 3, S.Velocity("uniform", a=(0.0, 0.0)), pseudo_dtau=0.1 / 6 / 4,
                pseudo_kmax=10, pseudo_fixed=True, nu_max=0.15 / 6 / 3)
    x = s.xu[..., 0]
    psi = x - 0.5
    R = s.rhs_pseudo(psi, psi)
    assert float(R.abs().max()) < 1e-12
    psi2 = 2 * (x - 0.5)
    R2 = s.rhs_pseudo(psi2, psi2)
    assert torch.allclose(R2, -torch.tanh(psi2 / 2), atol=1e-11)
    s.phi = 0.5 + 2 * (x - 0.5)
    s.precondition(fixed=True)
    q, _ = s.gradient(s.psi[:, None], s.trace(s.psi[:, None]))
    slope = q[:, 0, :, 0]
    assert float(slope.mean()) < 2.0 and float(slope.mean()) > 1.0


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_triangle_advection_operator_is_nearly_energy_neutral(p):
    """The advection operator (gamma = eps = 0, with the LDG penalty tau = 0.1) of the
    Rider-Kothe field on split and Delaunay triangles has no mode that grows
    by more than e^0.2 over the period T = 8 (max Re lambda < 0.025): the
    triangle solution points keep the collocated flux from exciting growing
    modes."""
    import numpy as np
    for mesh in (S.tri_split(4, periodic=(False, False)), S.tri_delaunay(6, jitter=0.1, seed=2)):
        s = _solver(mesh, p, S.Velocity("rider_kothe", T=8.0), gamma=0.0, eps=0.0)
        s.initialize(S.Circle((0.5, 0.75), 0.15, 10.0), precondition=False)
        shape, N = s.phi.shape, s.phi.numel()
        A = np.zeros((N, N))
        z = torch.zeros(shape, dtype=torch.float64)
        for k in range(N):
            e = torch.zeros(N, dtype=torch.float64)
            e[k] = 1.0
            A[:, k] = s.rhs(e.reshape(shape), z, 0.0)[0].reshape(-1).numpy()
        assert np.linalg.eigvals(A).real.max() < 0.025


@pytest.mark.parametrize("et", ["quad", "tri", "hex"])
def test_integral_of_polynomial_fields_is_exact_on_mapped_meshes(et):
    """A field of degree q <= p in the physical coordinates is exactly
    represented on bilinear / affine / trilinear elements (degree q per
    reference direction), so the solution-point quadrature of its interpolant
    (the Section 4 error measures and the mass integral) gives the exact
    integral over the unit square / cube on jittered wall meshes."""
    p = 3
    if et == "quad":
        mesh = S.quad_grid(5, periodic=(False, False), jitter=0.15, seed=9)
    elif et == "tri":
        mesh = S.tri_delaunay(7, jitter=0.15, seed=4)
    else:
        mesh = S.hex_grid(3, jitter=0.15, seed=5)
    s = _solver(mesh, p, S.Velocity("uniform", a=(1.0, 0.0, 0.0)))
    x = s.xu
    X, Y = x[..., 0], x[..., 1]
    f = 1 + 2 * X - 3 * Y + 4 * X * Y + X ** 2 + Y ** 3
    exact = 1 + 1 - 1.5 + 1 + 1 / 3 + 0.25
    if et == "hex":
        Z = x[..., 2]
        f = f + 5 * Z * X - Z ** 3
        exact += 1.25 - 0.25
    assert float(s.integral(f)) == pytest.approx(exact, rel=1e-13)
    assert float(s.integral(torch.ones_like(f))) == pytest.approx(1.0, rel=1e-14)


@pytest.mark.parametrize("mk,p,vel", [
    (lambda: S.quad_grid(4, periodic=(False, False), jitter=0.12, seed=3, shuffle_seed=4, rotate_seed=5), 3,
     S.Velocity("rider_kothe", T=8.0)),
    (lambda: S.tri_delaunay(6, jitter=0.1, seed=7), 3, S.Velocity("rider_kothe", T=8.0)),
    (lambda: S.hex_grid(3, jitter=0.1, seed=2, rotate_seed=4), 2, S.Velocity("leveque", T=3.0)),
])
def test_wall_flux_copy_ghost_and_noflux_option(mk, p, vel):
    """Section 3.3 walls copy the interior, so an interface that reaches a wall
    loses mass through it (sum_e sum_i w_i det J_i R_i != 0); with the no-flux
    option the same residual sums to zero (conservation as on periodic
    meshes) and differs from the copy-ghost one only on wall elements."""
    mesh = mk()
    d = mesh.dim
    c = (0.5, 0.2, 0.5)[:d]                     # disk / sphere near the wall y = 0
    out = {}
    for wall in ("copy", "noflux"):
        s = _solver(mesh, p, vel, wall=wall)
        s.initialize(S.Circle(c, 0.15, 8.0), precondition=False)
        s.psi = s.psi + 0.05 * torch.sin(7 * s.xu[..., 0])
        out[wall] = (s, *s.rhs(s.phi, s.psi, 0.7))
    s, Rc, Rcs = out["copy"]
    _, Rn, Rns = out["noflux"]
    scale = float(s.integral(Rc.abs()))
    assert abs(float(s.integral(Rn))) < 1e-13 * scale
    assert abs(float(s.integral(Rns))) < 1e-13 * float(s.integral(Rns.abs()))
    assert abs(float(s.integral(Rc))) > 1e-4 * scale   # mass leaves through the copy-ghost wall
    wall_el = s.boundary.any(1)
    assert bool(wall_el.any()) and bool((~wall_el).any())
    assert torch.allclose(Rc[~wall_el], Rn[~wall_el], atol=1e-13 * float(Rc.abs().max()))
    assert not torch.allclose(Rc[wall_el], Rn[wall_el], atol=1e-6 * float(Rc.abs().max()))
