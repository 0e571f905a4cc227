"""Batched instances (fr_mesh_concat + fr_field_init_batch) against one
independent oracle run per instance: uneven sizes, per-instance time steps,
interface widths, viscosities, circles and random-phase velocities, with
preconditioning inside the window."""
import numpy as np
import pytest
import torch

import synthetic as S
from libutil import ensure_built
from oracle import Params, Solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    import paper_2006_10967_gb300 as G
    return G


def _instances(p, sizes, seed):
    rng = np.random.default_rng(seed)
    out = []
    for n in sizes:
        h = 1.0 / n
        vel = S.workloads.random_phase_stream(rng, n_modes=6, kmax=2.5, T=4.0)
        r = float(rng.uniform(0.2, 0.3))
        c = tuple(float(v) for v in rng.uniform(r, 1 - r, 2))
        w = S.Workload(f"i{n}", (lambda n=n: S.quad_grid(n, jitter=0.08, seed=n)), p, vel,
                       S.Circle(c, r, 3 * p / (4 * h)), t_end=4.0, h=h)
        w.eps = 0.06 * h / p
        w.nu_max = 0.15 * h / p
        w.pseudo_dtau = 0.1 * h / (p + 1)
        w.dt = 0.1 * h / (p + 1)
        w.n_precond = 3
        w.pseudo_kmax = 2
        out.append(w)
    return out


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 2e-5)])
def test_batch_matches_independent_oracle_runs(G, precision, tol):
    ws = _instances(2, [3, 5, 4], seed=11)
    (p, F, ranges), = G.batch_from_workloads(ws, precision=precision, pseudo_fixed=True)
    F.step(4)                    # preconditioning again before step 3
    assert F.sync() == 0
    phi = F.get(0)
    psi = F.get(1)
    for w, (b, e) in zip(ws, ranges):
        sol = Solver(w.mesh(), p, Params.from_workload(w, pseudo_fixed=True), w.velocity)
        sol.initialize(w.circle, precondition=True)
        sol.step(4)
        ref, refp = sol.phi.numpy(), sol.psi.numpy()
        assert np.abs(phi[b:e] - ref).max() / np.abs(ref).max() < tol
        assert np.abs(psi[b:e] - refp).max() / np.abs(refp).max() < tol


def test_batch_fields_have_no_adjoint(G):
    """The adjoint assumes one uniform time step: a batch field (per-instance
    steps) is rejected with FR_EUNSUPPORTED, before any work."""
    ws = _instances(2, [3, 4], seed=5)
    (p, F, ranges), = G.batch_from_workloads(ws, precision="fp64", pseudo_fixed=True)
    with pytest.raises(G.FRError) as e:
        F.adjoint_record(2, 1)
    assert e.value.code == -6
    F.step(1)
    assert F.sync() == 0


def test_ensemble_workload_builds_and_steps(G):
    """The 256-instance ensemble recipe, subsampled: one batch per order."""
    ws = S.ensemble_instances(16, seed=3)
    fields = G.batch_from_workloads(ws, precision="mixed")
    assert sorted(p for p, _, _ in fields) == sorted(set(w.order for w in ws))
    for p, F, ranges in fields:
        m0 = F.mass(0)
        F.step(5)
        assert F.sync() == 0
        assert abs(F.mass(0) - m0) < 1e-12 * abs(m0)   # periodic instances conserve mass


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 2e-5)])
def test_multi_order_ensemble_matches_independent_oracle_runs(G, precision, tol):
    """An ensemble with instances of orders 2, 3 and 4 (one batch field per
    order, as the 256-instance benchmark builds it) against one oracle run per
    instance, preconditioning inside the window."""
    ws = _instances(2, [3, 4], seed=5) + _instances(3, [3], seed=6) + _instances(4, [2, 3], seed=7)
    fields = G.batch_from_workloads(ws, precision=precision, pseudo_fixed=True)
    assert sorted(p for p, _, _ in fields) == [2, 3, 4]
    by_order = {}
    for w in ws:
        by_order.setdefault(w.order, []).append(w)
    for p, F, ranges in fields:
        F.step(4)
        assert F.sync() == 0
        phi = F.get(0)
        for w, (b, e) in zip(by_order[p], ranges):
            sol = Solver(w.mesh(), p, Params.from_workload(w, pseudo_fixed=True), w.velocity)
            sol.initialize(w.circle, precondition=True)
            sol.step(4)
            ref = sol.phi.numpy()
            assert np.abs(phi[b:e] - ref).max() / np.abs(ref).max() < tol, (p, b, e)


@pytest.mark.parametrize("precondition_every", [1000, 3])
def test_group_launch_matches_per_field_steps(G, precondition_every):
    """One launch per kernel per RK stage over the order groups of an
    ensemble (fr_group_step) gives the march of stepping each order's batch
    field on its own, with and without a preconditioning in the window: the
    same kernel bodies compiled into one kernel, equal to float round-off
    (launch bounds and register allocation differ, so not bit for bit)."""
    ws = _instances(2, [3, 4], seed=5) + _instances(3, [3], seed=6) + _instances(4, [2, 3], seed=7) + \
        _instances(5, [2], seed=8)
    for w in ws:
        w.n_precond = precondition_every
    fa = G.batch_from_workloads(ws, precision="mixed", pseudo_fixed=True)
    fb = G.batch_from_workloads(ws, precision="mixed", pseudo_fixed=True)
    grp = G.Group([F for _, F, _ in fa])
    for n in (5, 17):
        grp.step(n)
        for _, F, _ in fb:
            F.step(n)
    for (p, Fa, _), (_, Fb, _) in zip(fa, fb):
        assert Fa.sync() == 0 and Fb.sync() == 0
        for which in (0, 1):
            a, b = Fa.get(which), Fb.get(which)
            assert np.abs(a - b).max() <= 2e-6 * np.abs(b).max(), (p, which)
        assert Fa.stats()["t"] == Fb.stats()["t"]
        assert Fa.stats()["n_steps"] == Fb.stats()["n_steps"] == 22


def test_group_rejects_unsupported_fields(G):
    ws = _instances(2, [3], seed=5) + _instances(2, [4], seed=6)
    (p, F64, _), = G.batch_from_workloads(ws[:1], precision="fp64")
    with pytest.raises(G.FRError):
        G.Group([F64])
    a = G.batch_from_workloads(ws[:1], precision="mixed")[0][1]
    b = G.batch_from_workloads(ws[1:], precision="mixed")[0][1]
    with pytest.raises(G.FRError):
        G.Group([a, b])          # two fields of one order
