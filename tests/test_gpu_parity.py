"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs, element by element.

Tolerances: FP64 path 1e-12 relative (max-norm of the difference over the
max-norm of the oracle's value) per residual evaluation and per RK step; the
mixed path 1e-4 relative per residual (float32 stage values and fluxes, unit
round-off 6e-8, amplified by the FR operator norm ~ (p+1)^2 / h times the flux
scale over the residual scale).
"""
import math

import numpy as np
import pytest
import torch

import synthetic as S
from libutil import ensure_built
from oracle import Params, Solver

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-4


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    import paper_2006_10967_gb300 as G
    return G


def _workload(mesh_fn, p, vel, circle, h, **kw):
    w = S.Workload("t", mesh_fn, p, vel, circle, t_end=1.0, h=h)
    w.eps = 0.06 * h / p
    w.nu_max = 0.15 * h / p
    w.pseudo_dtau = 0.1 * h / (p + 1)
    from synthetic.workloads import _umax
    w.dt = 0.1 * h / ((p + 1) * max(1.0, _umax(vel, 3 if vel.kind == "leveque" else 2)))
    for k, v in kw.items():
        setattr(w, k, v)
    return w


def _pair(G, w, precision="fp64", precondition=False, fixed=True, vel_cache=True, variant="auto", **okw):
    mesh = w.mesh()
    prm = Params.from_workload(w, pseudo_fixed=fixed, **okw)
    sol = Solver(mesh, w.order, prm, w.velocity)
    sol.initialize(w.circle, precondition=precondition)
    M = G.Mesh.from_synthetic(mesh, w.order)
    P = G.make_params(w, precision, pseudo_fixed=fixed, vel_cache=vel_cache, variant=variant, **okw)
    F = G.Field(M, P, ic=w.circle, precondition=precondition)
    return sol, F


def _perturb(sol, F):
    """A generic psi (smooth but not aligned with phi) on both sides."""
    x = sol.xu
    pert = 0.05 * torch.sin(5.0 * x[..., 0] + 1.0) * torch.cos(3.0 * x[..., 1])
    psi = sol.phi - 0.5 + pert
    sol.psi = psi
    F.set(1, psi.numpy())


def _rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


CASES = {
    "quad_periodic_jitter_p3": lambda: _workload(
        lambda: S.quad_grid(6, jitter=0.12, seed=3, shuffle_seed=4, rotate_seed=5), 3,
        S.Velocity("rider_kothe", T=8.0), S.Circle((0.45, 0.55), 0.25, 3 * 3 / (4 / 6)), 1 / 6),
    "quad_walls_jitter_p4": lambda: _workload(
        lambda: S.quad_grid(7, 5, periodic=(False, False), jitter=0.1, seed=1, shuffle_seed=11, rotate_seed=12), 4,
        S.Velocity("rider_kothe", T=8.0), S.Circle((0.5, 0.6), 0.25, 3 * 4 / (4 / 6)), 1 / 6),
    "quad_stream_p5": lambda: _workload(
        lambda: S.quad_grid(5, jitter=0.05, seed=8), 5,
        S.Velocity("stream", T=4.0, **dict(zip(("kx", "ky", "A", "B"), S.stream_coefficients(16, seed=4)))),
        S.Circle((0.5, 0.5), 0.2, 3 * 5 / (4 / 5)), 1 / 5),
    "tri_delaunay_p3": lambda: _workload(
        lambda: S.tri_delaunay(9, seed=2, shuffle_seed=13), 3,
        S.Velocity("rider_kothe", T=8.0), S.Circle((0.5, 0.6), 0.25, 3 * 3 / (4 / 8)), 1 / 8),
    "tri_delaunay_p5": lambda: _workload(
        lambda: S.tri_delaunay(7, seed=3, shuffle_seed=5), 5,
        S.Velocity("rider_kothe", T=8.0), S.Circle((0.5, 0.6), 0.25, 3 * 5 / (4 / 6)), 1 / 6),
    "tri_split_periodic_p2": lambda: _workload(
        lambda: S.tri_split(5, shuffle_seed=1), 2,
        S.Velocity("rotation", a=(0.5, 0.5)), S.Circle((0.5, 0.6), 0.25, 3 * 2 / (4 / 5)), 1 / 5),
    "hex_walls_p3": lambda: _workload(
        lambda: S.hex_grid(3, shuffle_seed=2), 3,
        S.Velocity("leveque", T=3.0), S.Circle((0.4, 0.45, 0.5), 0.3, 3 * 3 / (4 / 3)), 1 / 3),
    "hex_periodic_jitter_p2": lambda: _workload(
        lambda: S.hex_grid(3, periodic=(True, True, True), jitter=0.1, seed=4), 2,
        S.Velocity("leveque", T=3.0), S.Circle((0.4, 0.45, 0.5), 0.3, 3 * 2 / (4 / 3)), 1 / 3),
    # every hex with one of the 24 rotations of its vertex list: shared faces
    # meet in all 8 relative orientations of their point grids
    "hex_rotated_walls_p3": lambda: _workload(
        lambda: S.hex_grid(3, shuffle_seed=2, rotate_seed=5), 3,
        S.Velocity("leveque", T=3.0), S.Circle((0.4, 0.45, 0.5), 0.3, 3 * 3 / (4 / 3)), 1 / 3),
    "hex_rotated_periodic_jitter_p2": lambda: _workload(
        lambda: S.hex_grid(3, periodic=(True, True, True), jitter=0.1, seed=4, rotate_seed=6), 2,
        S.Velocity("leveque", T=3.0), S.Circle((0.4, 0.45, 0.5), 0.3, 3 * 2 / (4 / 3)), 1 / 3),
    # 64 elements: several full tiles of the p = 3 hex kernels and a ragged one
    "hex_periodic_jitter_p3": lambda: _workload(
        lambda: S.hex_grid(4, periodic=(True, True, True), jitter=0.1, seed=5, shuffle_seed=3), 3,
        S.Velocity("leveque", T=3.0), S.Circle((0.45, 0.5, 0.4), 0.3, 3 * 3 / (4 / 4)), 1 / 4),
}


@pytest.mark.parametrize("case", list(CASES))
def test_rhs_parity_fp64(G, case):
    w = CASES[case]()
    sol, F = _pair(G, w)
    assert _rel(F.get(0), sol.phi.numpy()) < 1e-14
    _perturb(sol, F)
    for t in (0.0, 0.7):
        R = F.rhs(t).cpu().numpy()
        Ro = sol.rhs(sol.phi, sol.psi, t)
        assert _rel(R[0], Ro[0].numpy()) < TOL64, case
        assert _rel(R[1], Ro[1].numpy()) < TOL64, case


@pytest.mark.parametrize("case", ["quad_walls_jitter_p4", "quad_stream_p5", "tri_delaunay_p3", "tri_split_periodic_p2",
                                  "hex_periodic_jitter_p2", "hex_periodic_jitter_p3"])
@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("mixed", TOL32)])
def test_rhs_parity_velocity_evaluated_in_kernel(G, case, precision, tol):
    """The same residual with the velocity evaluated in the kernels instead of
    read from the per-point cache."""
    w = CASES[case]()
    sol, F = _pair(G, w, precision=precision, vel_cache=False)
    _perturb(sol, F)
    R = F.rhs(0.7).cpu().numpy()
    Ro = sol.rhs(sol.phi, sol.psi, 0.7)
    assert _rel(R[0], Ro[0].numpy()) < tol, case
    assert _rel(R[1], Ro[1].numpy()) < tol, case


@pytest.mark.parametrize("case", list(CASES))
def test_pseudo_rhs_parity_fp64(G, case):
    w = CASES[case]()
    sol, F = _pair(G, w)
    _perturb(sol, F)
    # psi0 = phi - 1/2 on both sides (set at init); the state's psi is perturbed
    R = F.rhs_pseudo().cpu().numpy()
    Ro = sol.rhs_pseudo(sol.psi, sol.phi - 0.5).numpy()
    assert _rel(R, Ro) < TOL64, case


@pytest.mark.parametrize("case", ["quad_periodic_jitter_p3", "tri_delaunay_p3", "hex_walls_p3", "hex_rotated_walls_p3"])
def test_rk_steps_and_preconditioning_parity_fp64(G, case):
    w = CASES[case]()
    w.n_precond = 2
    w.pseudo_kmax = 3
    sol, F = _pair(G, w, precondition=True)
    assert _rel(F.get(1), sol.psi.numpy()) < TOL64
    # psi0 = phi - 1/2 from each side's own tanh of the initial condition
    assert _rel(F.get(2), sol.psi0.numpy()) < 1e-13
    for nsteps in (1, 4):
        F.step(nsteps)
        sol.step(nsteps)
        assert _rel(F.get(0), sol.phi.numpy()) < TOL64, case
        assert _rel(F.get(1), sol.psi.numpy()) < TOL64, case
    st = F.stats()
    assert st["n_steps"] == 5 and st["n_preconditions"] == 3
    assert st["t"] == pytest.approx(sol.t, rel=1e-15)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_replay_matches_direct_launches(G, precision):
    """fr_step replays captured CUDA graphs (16-step chunks, single steps, the
    preconditioning sequence); with profiling on it launches every kernel
    directly.  Both must produce the same bits, preconditionings included."""
    w = CASES["quad_periodic_jitter_p3"]()
    w.n_precond = 10
    w.pseudo_kmax = 3
    _, Fg = _pair(G, w, precision=precision, precondition=True)
    _, Fd = _pair(G, w, precision=precision, precondition=True)
    Fd.profile(True)
    for n in (37, 5):
        Fg.step(n)
        Fd.step(n)
    for which in (0, 1, 2):
        assert np.array_equal(Fg.get(which), Fd.get(which)), which
    sg, sd = Fg.stats(), Fd.stats()
    assert sg["n_steps"] == sd["n_steps"] == 42
    assert sg["n_preconditions"] == sd["n_preconditions"] == 5
    assert sg["t"] == sd["t"]


def test_profile_kernel_leaves_the_state(G):
    """fr_profile_kernel replays residual launches on the current state: the
    march that follows is bit-identical to one without it."""
    w = CASES["quad_periodic_jitter_p3"]()
    _, Fa = _pair(G, w, precision="mixed")
    _, Fb = _pair(G, w, precision="mixed")
    Fa.step(3)
    Fb.step(3)
    assert Fa.profile_kernel(0, 10) > 0.0
    Fa.step(3)
    Fb.step(3)
    for which in (0, 1):
        assert np.array_equal(Fa.get(which), Fb.get(which))
    with pytest.raises(G.FRError):
        Fa.profile_kernel(1, 10)


def test_pseudo_stop_rule_matches_oracle(G):
    w = CASES["quad_periodic_jitter_p3"]()
    w.pseudo_kmax = 20
    w.pseudo_tol = 2.0
    sol, F = _pair(G, w, precondition=True, fixed=False)
    st = F.stats()
    assert st["last_pseudo_iters"] == sol.pseudo_iters
    assert st["last_pseudo_rms"] == pytest.approx(sol.pseudo_rms, rel=1e-10)
    assert _rel(F.get(1), sol.psi.numpy()) < TOL64


@pytest.mark.parametrize("case", ["quad_periodic_jitter_p3", "tri_split_periodic_p2", "hex_periodic_jitter_p2"])
def test_mass_integral_and_conservation(G, case):
    w = CASES[case]()
    sol, F = _pair(G, w)
    m0 = F.mass(0)
    assert m0 == pytest.approx(float(sol.integral(sol.phi)), rel=1e-14)
    assert F.mass(1) == pytest.approx(float(sol.integral(sol.psi)), rel=1e-12, abs=1e-15)
    F.step(10)
    assert abs(F.mass(0) - m0) < 1e-13 * abs(m0)


@pytest.mark.parametrize("case", ["quad_periodic_jitter_p3", "quad_walls_jitter_p4", "tri_delaunay_p3", "tri_delaunay_p5",
                                  "hex_walls_p3", "hex_periodic_jitter_p3", "hex_rotated_walls_p3",
                                  "hex_rotated_periodic_jitter_p2"])
def test_rhs_parity_mixed(G, case):
    w = CASES[case]()
    sol, F = _pair(G, w, precision="mixed")
    _perturb(sol, F)
    R = F.rhs(0.3).cpu().numpy()
    Ro = sol.rhs(sol.phi, sol.psi, 0.3)
    assert _rel(R[0], Ro[0].numpy()) < TOL32, case
    assert _rel(R[1], Ro[1].numpy()) < TOL32, case
    Rp = F.rhs_pseudo().cpu().numpy()
    assert _rel(Rp, sol.rhs_pseudo(sol.psi, sol.phi - 0.5).numpy()) < TOL32


@pytest.mark.parametrize("case", ["quad_periodic_jitter_p3", "quad_stream_p5", "hex_periodic_jitter_p2",
                                  "hex_periodic_jitter_p3", "hex_rotated_periodic_jitter_p2", "tri_split_periodic_p2"])
def test_mixed_mass_conserved_to_round_off(G, case):
    """Mixed path: each element's float-float solution is corrected so that its
    mass change equals the FP64 sum of its (antisymmetric) face fluxes, so the
    global mass is conserved to double round-off on periodic meshes."""
    w = CASES[case]()
    sol, F = _pair(G, w, precision="mixed")
    m0 = F.mass(0)
    F.step(60)
    assert F.sync() == 0
    assert abs(F.mass(0) - m0) < 1e-13 * abs(m0)


def test_mixed_steps_track_fp64(G):
    w = CASES["quad_periodic_jitter_p3"]()
    sol, F64 = _pair(G, w)
    _, F32 = _pair(G, w, precision="mixed")
    F64.step(20)
    F32.step(20)
    sol.step(20)
    assert _rel(F64.get(0), sol.phi.numpy()) < TOL64
    assert _rel(F32.get(0), sol.phi.numpy()) < 1e-5


def test_full_size_c2q_rhs_parity(G):
    """The benchmark's configuration (128^2 jittered quads, p = 4, Rider-Kothe)
    at full size: every residual value against the oracle."""
    w = S.workload("c2q")
    sol, F = _pair(G, w)
    for t in (0.0, 2.5):
        R = F.rhs(t).cpu().numpy()
        Ro = sol.rhs(sol.phi, sol.psi, t)
        assert _rel(R[0], Ro[0].numpy()) < TOL64
        assert _rel(R[1], Ro[1].numpy()) < TOL64


def test_nonfinite_state_is_reported(G):
    w = CASES["quad_periodic_jitter_p3"]()
    sol, F = _pair(G, w)
    phi = F.get(0)
    phi[3, 2] = np.nan
    F.set(0, phi)
    F.step(1)
    assert F.sync() == -4


# ---------------------------------------------------------------------------
# Unpreconditioned conservative phase field (normal from phi's gradient)

@pytest.mark.parametrize("case", ["quad_walls_jitter_p4", "quad_periodic_jitter_p3", "tri_delaunay_p3",
                                  "hex_walls_p3", "hex_periodic_jitter_p2"])
@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("mixed", TOL32)])
def test_unpreconditioned_rhs_parity(G, case, precision, tol):
    """Eq. altconservativephasefieldeq with n = grad phi / |grad phi|, odd and
    even orders (the residual kernel fuses Step 4 differently), with a psi
    that is not phi - 1/2 so that the choice of normal matters."""
    w = CASES[case]()
    sol, F = _pair(G, w, precision=precision, normal="phi")
    _perturb(sol, F)
    R = F.rhs(0.3).cpu().numpy()
    Ro = sol.rhs(sol.phi, sol.psi, 0.3)
    assert _rel(R[0], Ro[0].numpy()) < tol, case
    assert _rel(R[1], Ro[1].numpy()) < tol, case
    # the preconditioned residual of the same state is a different one
    Rpc = sol.__class__(w.mesh(), w.order, Params.from_workload(w), w.velocity)
    Rp = Rpc.rhs(sol.phi, sol.psi, 0.3)[0].numpy()
    gap = _rel(Ro[0].numpy(), Rp)
    assert gap > 1e-3
    assert _rel(R[0], Rp) > 0.5 * gap


def test_unpreconditioned_march_parity_without_preconditioning(G):
    w = CASES["quad_walls_jitter_p4"]()
    w.n_precond = 2
    w.pseudo_kmax = 3
    sol, F = _pair(G, w, precondition=True, normal="phi")
    for nsteps in (1, 4):
        F.step(nsteps)
        sol.step(nsteps)
        assert _rel(F.get(0), sol.phi.numpy()) < TOL64
        assert _rel(F.get(1), sol.psi.numpy()) < TOL64
    st = F.stats()
    assert st["n_steps"] == 5 and st["n_preconditions"] == 0


def test_unpreconditioned_mixed_conserves_mass_and_has_no_adjoint(G):
    w = CASES["quad_periodic_jitter_p3"]()
    _, F = _pair(G, w, precision="mixed", normal="phi")
    m0 = F.mass(0)
    F.step(20)
    assert F.sync() == 0
    assert abs(F.mass(0) - m0) < 1e-12 * abs(m0)
    _, F64 = _pair(G, w, normal="phi")
    with pytest.raises(G.FRError):
        F64.adjoint_record(4, 2)


# ---------------------------------------------------------------------------
# Slotted disk in solid-body rotation (Section 4.1), rotation about (2, 2)

@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("mixed", 1e-5)])
def test_rudman_slotted_disk_parity(G, precision, tol):
    """Rudman's problem on a coarse [0,4]^2 mesh (p = 3): the slotted disk's
    initial field (an array input), preconditioning, and RK4 steps of the
    rotation about (2, 2), against the oracle on the same phi0."""
    n, p = 8, 3
    h = 4.0 / n
    w = _workload(lambda: S.quad_grid(n, lengths=(4.0, 4.0), periodic=(False, False)), p,
                  S.Velocity("rotation", a=(2.0, 2.0, 0.0)),
                  S.SlottedDisk((2.0, 2.75), 0.5, 0.06, 2.65, 3 * p / (4 * h)), h)
    w.n_precond = 2
    w.pseudo_kmax = 3
    mesh = w.mesh()
    sol = Solver(mesh, p, Params.from_workload(w, pseudo_fixed=True), w.velocity)
    phi0 = S.initial_phi(w, sol.xu.numpy())
    sol.initialize(phi=torch.from_numpy(phi0), precondition=True)
    M = G.Mesh.from_synthetic(mesh, p)
    F = G.Field(M, G.make_params(w, precision, pseudo_fixed=True), phi0=phi0, precondition=True)
    assert _rel(F.get(1), sol.psi.numpy()) < tol
    R = F.rhs(0.0).cpu().numpy()
    Ro = sol.rhs(sol.phi, sol.psi, 0.0)
    assert _rel(R[0], Ro[0].numpy()) < (TOL64 if precision == "fp64" else TOL32)
    F.step(3)
    sol.step(3)
    assert _rel(F.get(0), sol.phi.numpy()) < tol
    assert F.stats()["n_preconditions"] == sol_preconditions(3, w.n_precond)


def sol_preconditions(n_steps, n_precond):
    """Preconditionings in n_steps steps from set-up (one at set-up, then one
    before every step whose index is a positive multiple of n_precond)."""
    return 1 + sum(1 for k in range(1, n_steps) if k % n_precond == 0)


# ---------------------------------------------------------------------------
# RK4 stage times under a time-dependent velocity (Section 3.1): a uniform
# field a cos(pi t / T) with T comparable to a few steps, so that a stage
# evaluated at the wrong time changes the result at first order in dt.

@pytest.mark.parametrize("mk,p", [
    (lambda: S.quad_grid(5, jitter=0.1, seed=2, shuffle_seed=3, rotate_seed=4), 3),
    (lambda: S.tri_split(4, shuffle_seed=2), 2),
    (lambda: S.hex_grid(3, periodic=(True, True, True), jitter=0.1, seed=6), 2),
])
@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("mixed", 1e-5)])
def test_time_modulated_uniform_march_parity(G, mk, p, precision, tol):
    h = 0.25
    dim = mk().dim
    w = _workload(mk, p, S.Velocity("uniform", a=(1.0, 0.5, 0.25), T=0.05),
                  S.Circle((0.45, 0.55, 0.5)[:dim], 0.3, 3 * p / (4 * h)), h)
    w.dt = 0.01
    w.n_precond = 1000
    sol, F = _pair(G, w, precision=precision)
    for nsteps in (1, 5):
        F.step(nsteps)
        sol.step(nsteps)
        assert _rel(F.get(0), sol.phi.numpy()) < tol
        assert _rel(F.get(1), sol.psi.numpy()) < tol
    assert F.stats()["t"] == pytest.approx(sol.t, rel=1e-15)


# ---------------------------------------------------------------------------
# No-flux walls (an option beside the paper's copy ghost state)

@pytest.mark.parametrize("case", ["quad_walls_jitter_p4", "tri_delaunay_p3", "hex_walls_p3", "hex_rotated_walls_p3"])
@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("mixed", TOL32)])
def test_noflux_wall_rhs_parity(G, case, precision, tol):
    w = CASES[case]()
    w.wall = "noflux"
    sol, F = _pair(G, w, precision=precision)
    _perturb(sol, F)
    R = F.rhs(0.3).cpu().numpy()
    Ro = sol.rhs(sol.phi, sol.psi, 0.3)
    assert _rel(R[0], Ro[0].numpy()) < tol, case
    assert _rel(R[1], Ro[1].numpy()) < tol, case


@pytest.mark.parametrize("case", ["quad_walls_jitter_p4", "tri_delaunay_p3", "hex_walls_p3"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noflux_walls_conserve_mass(G, case, precision):
    w = CASES[case]()
    w.wall = "noflux"
    _, F = _pair(G, w, precision=precision)
    m0 = F.mass(0)
    F.step(60)
    assert F.sync() == 0
    assert abs(F.mass(0) - m0) < 1e-13 * abs(m0)
    _, F64 = _pair(G, w)
    with pytest.raises(G.FRError):
        F64.adjoint_record(4, 2)


# ---------------------------------------------------------------------------
# Kernel variants: triangle operator applies on tensor cores (float path)

@pytest.mark.parametrize("case", ["tri_delaunay_p3", "tri_delaunay_p5", "tri_split_periodic_p2"])
def test_triangle_tensor_core_variant_parity(G, case):
    w = CASES[case]()
    sol, F = _pair(G, w, precision="mixed", variant=1)
    assert F.params.variant == 1
    _perturb(sol, F)
    R = F.rhs(0.3).cpu().numpy()
    Ro = sol.rhs(sol.phi, sol.psi, 0.3)
    assert _rel(R[0], Ro[0].numpy()) < TOL32, case
    assert _rel(R[1], Ro[1].numpy()) < TOL32, case
    Rp = F.rhs_pseudo().cpu().numpy()
    assert _rel(Rp, sol.rhs_pseudo(sol.psi, sol.phi - 0.5).numpy()) < TOL32
    # both variants march with the oracle to float round-off
    _, F0 = _pair(G, w, precision="mixed", variant=0)
    F0.set(1, sol.psi.numpy())
    F.step(10)
    F0.step(10)
    sol.step(10)
    assert F.sync() == 0 and F0.sync() == 0
    assert _rel(F.get(0), sol.phi.numpy()) < 1e-5
    assert _rel(F0.get(0), sol.phi.numpy()) < 1e-5
    assert _rel(F.get(0), F0.get(0)) < 1e-5


def test_variant_counts_and_rejection(G):
    w = CASES["tri_delaunay_p3"]()
    M = G.Mesh.from_synthetic(w.mesh(), w.order)
    assert G.kernel_variants(M, "mixed") == 2 and G.kernel_variants(M, "fp64") == 1
    with pytest.raises(G.FRError):
        G.Field(M, G.make_params(w, "fp64", variant=1), ic=w.circle)
    wq = CASES["quad_periodic_jitter_p3"]()
    Mq = G.Mesh.from_synthetic(wq.mesh(), wq.order)
    assert G.kernel_variants(Mq, "mixed") == 4 and G.kernel_variants(Mq, "fp64") == 1


@pytest.mark.parametrize("case", ["quad_periodic_jitter_p3", "quad_walls_jitter_p4", "hex_periodic_jitter_p3",
                                  "hex_rotated_walls_p3"])
@pytest.mark.parametrize("variant", [1, 2, 3])
def test_tile_variants_march_with_the_oracle(G, case, variant):
    """The tile variants of the quad/hex physical-step kernels (half tiles
    for the residual and/or the update kernel) march with the oracle like the
    default tiles.  A variant is deterministic (two runs give the same bits);
    against the default tiles it agrees to float round-off only: a different
    tile is different compiled code, whose float operation order (for
    instance which products fuse into an FMA) need not be the same."""
    w = CASES[case]()
    sol, F = _pair(G, w, precision="mixed", variant=variant)
    _, F1 = _pair(G, w, precision="mixed", variant=variant)
    _, F0 = _pair(G, w, precision="mixed", variant=0)
    for f in (F, F1, F0):
        f.step(6)
    sol.step(6)
    assert F.sync() == 0
    assert _rel(F.get(0), sol.phi.numpy()) < 1e-5
    assert np.array_equal(F.get(0), F1.get(0)) and np.array_equal(F.get(1), F1.get(1))
    for fld in (0, 1):
        assert _rel(F.get(fld), F0.get(fld)) < 1e-6


def test_autotuner_measures_every_variant(G):
    from paper_2006_10967_gb300 import tune
    w = CASES["tri_delaunay_p3"]()
    table = tune.tune([w], "mixed", write=False, steps=20, warmup=5)
    ent = table[tune.key(1, w.order, "mixed")]
    assert set(ent["us_per_stage"]) == {"0", "1"}
    assert str(ent["variant"]) == min(ent["us_per_stage"], key=lambda k: ent["us_per_stage"][k])


# ---------------------------------------------------------------------------
# Full-size headline workload (64^3 hexes, p = 3, LeVeque field) in the
# benchmark's launch configuration, checked on sampled elements: the residual
# of an element depends on its neighbours and their neighbours, so the oracle
# evaluated on a 6^3 block cut from the same mesh (same nodes, same state)
# gives the exact residual of the block's central 2^3 elements.

def _hex_block(mesh, n, lo):
    """The 6^3 sub-block of an n^3 hex_grid mesh starting at element index lo
    (i, j, k), as a mesh of its own, and the global ids of its elements."""
    i, j, k = np.meshgrid(*[np.arange(l, l + 6) for l in lo], indexing="ij")
    ids = (i + n * (j + n * k)).ravel(order="F")
    conn = mesh.conn[ids]
    used, inv = np.unique(conn, return_inverse=True)
    sub = S.meshes.Mesh("hex", mesh.nodes[used], inv.reshape(conn.shape).astype(np.int64),
                        (False, False, False), (1.0, 1.0, 1.0), "block")
    ci, cj, ck = np.meshgrid(*[np.arange(l + 2, l + 4) for l in lo], indexing="ij")
    centre = (ci + n * (cj + n * ck)).ravel(order="F")
    local = np.array([int(np.nonzero(ids == g)[0][0]) for g in centre])
    return sub, centre, local


@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("mixed", TOL32)])
def test_full_size_c3_sampled_parity(G, precision, tol):
    w = S.workload("c3")
    n = 64
    mesh = w.mesh()
    M = G.Mesh.from_synthetic(mesh, w.order)
    F = G.Field(M, G.make_params(w, precision), ic=w.circle, precondition=False)
    t = 0.7
    R = F.rhs(t).cpu().numpy()
    scale = np.abs(R).max(axis=(1, 2))
    for lo in ((0, 0, 0), (20, 17, 18), (58, 29, 40), (23, 58, 0)):   # corners, edges and the interior
        sub, centre, local = _hex_block(mesh, n, lo)
        sol = Solver(sub, w.order, Params.from_workload(w), w.velocity)
        sol.initialize(w.circle, precondition=False)
        Ro = sol.rhs(sol.phi, sol.psi, t)
        for f in (0, 1):
            d = np.abs(R[f][centre] - Ro[f].numpy()[local]).max() / scale[f]
            assert d < tol, (lo, f, d)
    # mass conservation of the full field over a few steps with no-flux walls
    wn = w.with_(wall="noflux")
    Fn = G.Field(M, G.make_params(wn, precision), ic=wn.circle, precondition=True)
    m0 = Fn.mass(0)
    Fn.step(8)
    assert Fn.sync() == 0
    assert abs(Fn.mass(0) - m0) < 1e-12 * abs(m0)
