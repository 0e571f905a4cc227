"""Element-partitioned stepping on the device (paper_2006_10967_gb300.partition
with the library's fr_stage / fr_halo_pack / fr_halo_unpack / fr_traces).

Several ranks' local fields (owned elements plus two ghost layers, elements
in ascending global order) are held by one process on one GPU and stepped
stage by stage, each stage followed by the exchange of the ghosts' stage
values between the fields (device copies; the same pack/unpack calls a rank
makes around its NCCL send/receive).  The owned elements' state after
several RK4 steps equals the whole-mesh field's, bit for bit: every owned
element reads exactly the values it reads in the whole mesh, through the
same kernels.  The preconditioning, run one pseudo stage at a time with the
same exchange, does the same."""
import numpy as np
import pytest
import torch

import synthetic as S
from libutil import ensure_built
from test_gpu_parity import _workload

# meshes large enough that every rank's local mesh (owned elements and two
# ghost layers) is a proper part of the whole
CASES = {
    "quad_periodic_jitter_p3": lambda: _workload(
        lambda: S.quad_grid(12, jitter=0.12, seed=3, shuffle_seed=4, rotate_seed=5), 3,
        S.Velocity("rider_kothe", T=8.0), S.Circle((0.45, 0.55), 0.25, 3 * 3 / (4 / 12)), 1 / 12),
    "quad_walls_jitter_p4": lambda: _workload(
        lambda: S.quad_grid(11, 9, periodic=(False, False), jitter=0.1, seed=1, shuffle_seed=11, rotate_seed=12),
        4, S.Velocity("rider_kothe", T=8.0), S.Circle((0.5, 0.6), 0.25, 3 * 4 / (4 / 10)), 1 / 10),
    "tri_split_periodic_p2": lambda: _workload(
        lambda: S.tri_split(10, shuffle_seed=1), 2,
        S.Velocity("rotation", a=(0.5, 0.5)), S.Circle((0.5, 0.6), 0.25, 3 * 2 / (4 / 10)), 1 / 10),
    "tri_delaunay_p3": lambda: _workload(
        lambda: S.tri_delaunay(12, seed=2, shuffle_seed=13), 3,
        S.Velocity("rider_kothe", T=8.0), S.Circle((0.5, 0.6), 0.25, 3 * 3 / (4 / 11)), 1 / 11),
    "hex_rotated_walls_p3": lambda: _workload(
        lambda: S.hex_grid(7, shuffle_seed=2, rotate_seed=5), 3,
        S.Velocity("leveque", T=3.0), S.Circle((0.4, 0.45, 0.5), 0.3, 3 * 3 / (4 / 7)), 1 / 7),
    "hex_periodic_jitter_p2": lambda: _workload(
        lambda: S.hex_grid(8, periodic=(True, True, True), jitter=0.1, seed=4), 2,
        S.Velocity("leveque", T=3.0), S.Circle((0.4, 0.45, 0.5), 0.3, 3 * 2 / (4 / 8)), 1 / 8),
    "hex_axis_walls_p3": lambda: _workload(
        lambda: S.hex_grid(8, shuffle_seed=3), 3,
        S.Velocity("leveque", T=3.0), S.Circle((0.35, 0.35, 0.35), 0.15, 3 * 3 / (4 / 8)), 1 / 8),
}

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    import paper_2006_10967_gb300 as G
    return G


def _state(G, M, w, precision):
    """A whole-mesh field with a generic state (psi not aligned with phi);
    the arrays set into it are the ones the ranks receive."""
    P = G.make_params(w, precision, variant=0, n_precond=10**9)
    F = G.Field(M, P, ic=w.circle, precondition=False)
    x = M.solution_points()
    phi = F.get(0)
    psi = phi - 0.5 + 0.05 * np.sin(5.0 * x[..., 0] + 1.0) * np.cos(3.0 * x[..., 1])
    F.set(0, phi)
    F.set(1, psi)
    return F, phi, psi, P


@pytest.mark.parametrize("case,world", [
    ("quad_periodic_jitter_p3", 2),
    ("quad_walls_jitter_p4", 3),
    ("tri_split_periodic_p2", 2),
    ("tri_delaunay_p3", 3),
    ("hex_rotated_walls_p3", 3),
    ("hex_periodic_jitter_p2", 4),
    ("hex_axis_walls_p3", 4),
])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_partitioned_march_equals_whole_mesh(G, case, world, precision):
    from paper_2006_10967_gb300 import partition as PT
    w = CASES[case]()
    mesh = w.mesh()
    M = G.Mesh.from_synthetic(mesh, w.order)
    F, phi, psi, P = _state(G, M, w, precision)
    part = PT.partition(mesh, world)
    plans = PT.plans(mesh, part)
    fields = []
    for pl in plans:
        Ml = G.Mesh.from_synthetic(pl.mesh, w.order)
        Fl = G.Field(Ml, P, ic=w.circle, precondition=False)
        Fl.set(0, phi[pl.local])
        Fl.set(1, psi[pl.local])
        fields.append(Fl)
    n = 5
    F.step(n)
    PT.step_ranks(fields, plans, n)
    assert F.sync() == 0
    ref = [F.get(0), F.get(1)]
    covered = np.zeros(mesh.n_elems, dtype=bool)
    for pl, Fl in zip(plans, fields):
        assert Fl.sync() == 0
        assert Fl.stats()["n_steps"] == n
        for fld in (0, 1):
            got = Fl.get(fld)[pl.owned_local]
            assert np.array_equal(got, ref[fld][pl.owned]), (pl.rank, fld, np.abs(got - ref[fld][pl.owned]).max())
        covered[pl.owned] = True
    assert covered.all()
    # the ghosts really are refreshed: on a rank whose local mesh is a proper
    # part of the mesh, a march without the exchange differs
    assert all(len(pl.local) < mesh.n_elems for pl in plans)
    pl = plans[0]
    Fs = G.Field(G.Mesh.from_synthetic(pl.mesh, w.order), P, ic=w.circle, precondition=False)
    Fs.set(0, phi[pl.local])
    Fs.set(1, psi[pl.local])
    Fs.step(n)
    assert not np.array_equal(Fs.get(0)[pl.owned_local], ref[0][pl.owned])


@pytest.mark.parametrize("case,world", [
    ("quad_walls_jitter_p4", 3),
    ("tri_delaunay_p3", 2),
    ("hex_rotated_walls_p3", 3),
])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_partitioned_preconditioning_equals_whole_mesh(G, case, world, precision):
    """The preconditioning run one pseudo stage at a time with the ghost
    exchange after the reset and after every pseudo stage (fr_pseudo_begin,
    fr_pseudo_stage): at t = 0 and on fr_step's schedule (before steps 3 and
    6 of 7 here), the owned elements equal the whole-mesh field's, bit for
    bit; a rank preconditioned alone on its local mesh differs."""
    from paper_2006_10967_gb300 import partition as PT
    w = CASES[case]()
    mesh = w.mesh()
    M = G.Mesh.from_synthetic(mesh, w.order)
    P = G.make_params(w, precision, variant=0, n_precond=3, pseudo_kmax=4, pseudo_fixed=True)
    F = G.Field(M, P, ic=w.circle, precondition=False)
    phi = F.get(0)
    F.set(0, phi)                                    # the same set-up path as the ranks' fields
    F.precondition()
    psi_pre = F.get(1)
    part = PT.partition(mesh, world)
    plans = PT.plans(mesh, part)
    fields = []
    for pl in plans:
        Fl = G.Field(G.Mesh.from_synthetic(pl.mesh, w.order), P, ic=w.circle, precondition=False)
        Fl.set(0, phi[pl.local])
        fields.append(Fl)
    PT.precondition_ranks(fields, plans)
    for pl, Fl in zip(plans, fields):
        got = Fl.get(1)[pl.owned_local]
        assert np.array_equal(got, psi_pre[pl.owned]), (pl.rank, np.abs(got - psi_pre[pl.owned]).max())
    assert not np.array_equal(psi_pre, phi - 0.5)    # the iterations moved psi
    n = 7
    F.step(n)
    PT.step_ranks(fields, plans, n)
    assert F.sync() == 0
    ref = [F.get(0), F.get(1)]
    assert F.stats()["n_preconditions"] == 3
    for pl, Fl in zip(plans, fields):
        assert Fl.sync() == 0
        st = Fl.stats()
        assert st["n_steps"] == n and st["n_preconditions"] == 3
        for fld in (0, 1):
            got = Fl.get(fld)[pl.owned_local]
            assert np.array_equal(got, ref[fld][pl.owned]), (pl.rank, fld, np.abs(got - ref[fld][pl.owned]).max())
    pl = plans[0]
    Fs = G.Field(G.Mesh.from_synthetic(pl.mesh, w.order), P, ic=w.circle, precondition=False)
    Fs.set(0, phi[pl.local])
    Fs.precondition()
    assert not np.array_equal(Fs.get(1)[pl.owned_local], psi_pre[pl.owned])


def test_pseudo_stage_calls_need_the_fixed_iteration_count(G):
    """fr_pseudo_begin / fr_pseudo_stage refuse fields whose preconditioning
    stops on the RMS rule or that take the normal from phi
    (FR_EUNSUPPORTED), and stages outside 1..4 (FR_EINVAL)."""
    from paper_2006_10967_gb300 import _capi
    w = CASES["quad_periodic_jitter_p3"]()
    M = G.Mesh.from_synthetic(w.mesh(), w.order)
    for kw in ({}, {"pseudo_fixed": True, "normal": "phi"}):
        F = G.Field(M, G.make_params(w, "fp64", variant=0, **kw), ic=w.circle, precondition=False)
        with pytest.raises(_capi.FRError) as e:
            F.pseudo_begin()
        assert e.value.code == _capi.FR_EUNSUPPORTED
    F = G.Field(M, G.make_params(w, "fp64", variant=0, pseudo_fixed=True), ic=w.circle, precondition=False)
    with pytest.raises(_capi.FRError) as e:
        F.pseudo_stage(5)
    assert e.value.code == G.FR_EINVAL
    F.pseudo_begin()
    F.pseudo_stage(1)
    assert F.sync() == 0


def test_halo_rows_round_trip_and_index_check(G):
    """halo_pack gathers the listed elements' stage values in list order and
    halo_unpack scatters them back; an out-of-range element index is skipped
    on the device and reported as FR_EINVAL by the status word."""
    w = CASES["quad_periodic_jitter_p3"]()
    M = G.Mesh.from_synthetic(w.mesh(), w.order)
    F = G.Field(M, G.make_params(w, "fp64", variant=0), ic=w.circle, precondition=False)
    u = F.get(0)
    idx = torch.tensor([5, 0, 17, 5], dtype=torch.int64, device="cuda")
    rows = F.halo_pack(idx)
    assert rows.dtype == torch.float64 and rows.shape == (4, 2, M.info.nu)
    assert np.array_equal(rows[:, 0].cpu().numpy(), u[[5, 0, 17, 5]])
    F.halo_unpack(idx[1:3], torch.zeros_like(rows[1:3]))
    F.traces()
    got = F.halo_pack(idx[1:3])
    assert float(got.abs().max()) == 0.0
    assert F.sync() == 0
    bad = torch.tensor([M.info.n_elems], dtype=torch.int64, device="cuda")
    F.halo_pack(bad)
    assert F.sync() == G.FR_EINVAL
