"""Element partitioning with two-layer ghost halos (paper_2006_10967_gb300.partition)
on gloo ranks (CPU): each rank evaluates the FR residual on its local mesh
(owned elements and ghosts) with the ghosts' states received from their
owners, and marches RK4 with a ghost exchange before every stage; the owned
elements' residuals and states equal the single-domain ones.  The residual
here is the oracle's (CPU), which stands in for the per-rank kernels."""
import json
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(name):
    import synthetic as S
    if name == "quad":
        mesh = S.quad_grid(6, jitter=0.1, seed=3, shuffle_seed=4, rotate_seed=5)
        return mesh, 2, S.Velocity("rider_kothe", T=8.0), S.Circle((0.45, 0.55), 0.25, 6.0)
    if name == "hexp":
        mesh = S.hex_grid(5, periodic=(True, False, True), jitter=0.1, seed=8, rotate_seed=2, shuffle_seed=6)
    else:
        mesh = S.hex_grid(4, jitter=0.1, seed=2, rotate_seed=7)
    return mesh, 2, S.Velocity("leveque", T=3.0), S.Circle((0.45, 0.5, 0.4), 0.3, 6.0)


def _rank_main(rank, world, port, out_dir, name):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import Params, Solver
    from paper_2006_10967_gb300 import partition as PT
    mesh, p, vel, circ = _case(name)
    prm = Params(gamma=0.09, eps=0.01, tau=0.1, dt=2e-3)
    full = Solver(mesh, p, prm, vel)
    full.initialize(circ, precondition=False)
    full.psi = full.psi + 0.05 * torch.sin(5.0 * full.xu[..., 0])
    Rf = full.rhs(full.phi, full.psi, 0.3)
    part = PT.partition(mesh, world)
    plan = PT.plans(mesh, part)[rank]
    loc = Solver(plan.mesh, p, prm, vel)
    no = plan.n_owned
    ol = torch.as_tensor(plan.owned_local)
    gl = torch.as_tensor(np.searchsorted(plan.local, plan.ghosts))
    phi = torch.zeros_like(loc.xu[..., 0])
    psi = torch.zeros_like(phi)
    phi[ol] = full.phi[plan.owned]           # owners know their own elements only
    psi[ol] = full.psi[plan.owned]
    PT.exchange(phi, plan)
    PT.exchange(psi, plan)
    ghosts_ok = bool(torch.equal(phi[gl], full.phi[plan.ghosts]) and torch.equal(psi[gl], full.psi[plan.ghosts]))
    R = loc.rhs(phi, psi, 0.3)
    res_err = max(float((R[f][ol] - Rf[f][plan.owned]).abs().max() / Rf[f].abs().max()) for f in (0, 1))
    # RK4 with a ghost exchange before every stage, against the single domain
    dt = prm.dt
    u = torch.stack([phi, psi], 0)

    def rate(U, t):
        U = U.clone()
        PT.exchange(U[0], plan)
        PT.exchange(U[1], plan)
        a, b = loc.rhs(U[0], U[1], t)
        return torch.stack([a, b], 0)
    t = 0.0
    for _ in range(3):
        k1 = rate(u, t)
        k2 = rate(u + 0.5 * dt * k1, t + 0.5 * dt)
        k3 = rate(u + 0.5 * dt * k2, t + 0.5 * dt)
        k4 = rate(u + dt * k3, t + dt)
        u = u + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        t += dt
    full.prm.dt = dt
    for _ in range(3):
        full.rk4_step()
    step_err = max(float((u[f][ol] - s[plan.owned]).abs().max() / s.abs().max())
                   for f, s in ((0, full.phi), (1, full.psi)))
    with open(os.path.join(out_dir, f"{name}{rank}.json"), "w") as f:
        json.dump({"rank": rank, "owned": int(no), "ghosts": int(len(plan.ghosts)), "ghosts_ok": ghosts_ok,
                   "res_err": res_err, "step_err": step_err, "peers": sorted(plan.recv)}, f)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("name,world", [("quad", 2), ("quad", 3), ("hex", 2), ("hexp", 3)])
def test_partitioned_residual_and_march_equal_single_domain(tmp_path, name, world):
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path), name), nprocs=world,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"{name}{r}.json")) for r in range(world)]
    import synthetic  # noqa: F401
    sys.path.insert(0, ROOT)
    mesh = _case(name)[0]
    assert sum(r["owned"] for r in res) == mesh.n_elems
    for r in res:
        assert r["ghosts_ok"] and r["ghosts"] > 0 and r["peers"]
        assert r["res_err"] < 1e-13, r
        assert r["step_err"] < 1e-13, r


def _precond_rank_main(rank, world, port, out_dir, name):
    """The preconditioning (psi0 = phi - 1/2, RK4 in pseudo time) on a
    rank's local mesh with the stage values' ghosts exchanged before every
    pseudo residual, in the fixed-count form and with the stop rule's RMS
    over the owned points all-reduced across the ranks."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import Params, Solver
    from paper_2006_10967_gb300 import partition as PT
    mesh, p, vel, circ = _case(name)
    h = 1.0 / (6 if name == "quad" else 4)
    prm = Params(gamma=0.09, eps=0.01, tau=0.1, dt=2e-3, pseudo_kmax=6, pseudo_dtau=0.1 * h / (p + 1),
                 nu_max=0.02)
    full = Solver(mesh, p, prm, vel)
    full.initialize(circ, precondition=False)
    # the whole mesh's RMS after k iterations, k = 1..kmax; the adaptive
    # tolerance sits midway between iterations 2 and 3
    hist = []
    for k in range(1, prm.pseudo_kmax + 1):
        full.prm.pseudo_kmax = k
        hist.append(full.precondition(fixed=True)[1])
    full.prm.pseudo_kmax = 6
    tol = 0.5 * (hist[1] + hist[2])
    part = PT.partition(mesh, world)
    plan = PT.plans(mesh, part)[rank]
    loc = Solver(plan.mesh, p, prm, vel)
    ol = torch.as_tensor(plan.owned_local)
    phi = torch.zeros_like(loc.xu[..., 0])
    phi[ol] = full.phi[plan.owned]
    PT.exchange(phi, plan)
    psi0 = phi - 0.5
    dtau = prm.pseudo_dtau

    def rate(y):
        y = y.clone()
        PT.exchange(y, plan)
        return loc.rhs_pseudo(y, psi0)

    out = {"rank": rank, "hist": hist, "tol": tol}
    for fixed in (True, False):
        full.prm.pseudo_tol = tol
        it_f, rms_f = full.precondition(fixed=fixed)
        psi = psi0.clone()
        it, rms = 0, float("nan")
        for it in range(1, prm.pseudo_kmax + 1):
            k1 = rate(psi)
            k2 = rate(psi + 0.5 * dtau * k1)
            k3 = rate(psi + 0.5 * dtau * k2)
            k4 = rate(psi + dtau * k3)
            new = psi + dtau / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
            R = ((new - psi) / dtau)[ol]
            acc = torch.tensor([float((R * R).sum()), float(R.numel())], dtype=torch.float64)
            dist.all_reduce(acc)
            rms = float(torch.sqrt(acc[0] / acc[1]))
            psi = new
            if not fixed and rms <= tol:
                break
        key = "fixed" if fixed else "adaptive"
        out[key] = {"iters": it, "iters_full": it_f, "rms_rel": abs(rms - rms_f) / rms_f,
                    "err": float((psi[ol] - full.psi[plan.owned]).abs().max() / full.psi.abs().max())}
    with open(os.path.join(out_dir, f"pre{name}{rank}.json"), "w") as f:
        json.dump(out, f)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("name,world", [("quad", 3), ("hexp", 2)])
def test_partitioned_preconditioning_equals_single_domain(tmp_path, name, world):
    """The partitioned preconditioning (the pattern of partition.precondition:
    an exchange of the ghosts' stage values before every pseudo residual)
    gives the owned elements the single-domain psi, with the fixed count and
    with the stop rule, whose RMS over all points is an all-reduce of the
    ranks' sums over their owned points; the stop comes at the same
    iteration."""
    mp.start_processes(_precond_rank_main, args=(world, _free_port(), str(tmp_path), name), nprocs=world,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"pre{name}{r}.json")) for r in range(world)]
    h = res[0]["hist"]
    assert h[0] > res[0]["tol"] and h[1] > res[0]["tol"] > h[2]   # the rule stops after iteration 3
    for r in res:
        assert r["fixed"]["iters"] == r["fixed"]["iters_full"] == 6
        assert r["adaptive"]["iters"] == r["adaptive"]["iters_full"] == 3
        for key in ("fixed", "adaptive"):
            assert r[key]["err"] < 1e-13, r
            assert r[key]["rms_rel"] < 1e-12, r


def test_partition_is_balanced_and_plans_are_consistent():
    sys.path.insert(0, ROOT)
    import synthetic as S
    from paper_2006_10967_gb300 import partition as PT
    mesh = S.hex_grid(6, periodic=(True, False, True), rotate_seed=3, shuffle_seed=2)
    part = PT.partition(mesh, 4)
    counts = np.bincount(part, minlength=4)
    assert counts.min() >= mesh.n_elems // 4 - 1 and counts.max() <= mesh.n_elems // 4 + 1
    P = PT.plans(mesh, part)
    for p in P:
        for q, idx in p.send.items():
            # what p sends to q is, element for element, what q receives from p
            sent = p.local[idx]
            got = P[q].local[P[q].recv[p.rank]]
            assert np.array_equal(sent, got)
            assert np.all(part[sent] == p.rank)


@pytest.mark.parametrize("name,world", [("quad", 3), ("hex", 3), ("hexp", 4)])
def test_local_meshes_pair_faces_across_the_period(name, world):
    """A rank's local mesh covers part of a periodic domain, so its cell size
    no longer divides the period; faces that meet through the periodic
    boundary still pair (in the oracle's geometry and in the library's mesh
    builder), and the only boundary flux points are those whose neighbour in
    the whole mesh is not on the rank."""
    sys.path.insert(0, ROOT)
    from libutil import ensure_built
    from oracle.mesh import build_geometry
    from paper_2006_10967_gb300 import partition as PT
    ensure_built()
    import paper_2006_10967_gb300 as G
    mesh, p = _case(name)[:2]
    gfull = build_geometry(mesh, p)
    pe_full = gfull.pe
    partial = 0
    for plan in PT.plans(mesh, PT.partition(mesh, world)):
        here = np.zeros(mesh.n_elems, dtype=bool)
        here[plan.local] = True
        cut = ~here[pe_full[plan.local]]
        partial += int(cut.sum()) > 0
        expected = int((cut | gfull.boundary[plan.local]).sum())
        geo = build_geometry(plan.mesh, p)
        assert int(geo.boundary.sum()) == expected
        # partners map back to the whole mesh's partners
        inner = ~geo.boundary
        assert np.array_equal(plan.local[geo.pe][inner], pe_full[plan.local][inner])
        M = G.Mesh.from_synthetic(plan.mesh, p)
        assert M.info.n_boundary_fpts == expected
    assert partial > 0


def test_step_runs_the_preconditioning_on_fr_steps_schedule(monkeypatch):
    """partition.step on the host: before every step whose index is a
    positive multiple of n_precond, the preconditioning (the reset, then
    pseudo_kmax iterations of four pseudo stages), with a ghost exchange after
    the reset, after every pseudo stage and after every physical stage; none
    when the normal comes from phi."""
    from paper_2006_10967_gb300 import partition as PT
    calls = []

    class Params:
        normal, n_precond, pseudo_kmax = 0, 3, 2

    class FakeField:
        params = Params

        def stats(self):
            return {"n_steps": 0}

        def stage(self, s):
            calls.append(("stage", s))

        def pseudo_begin(self):
            calls.append(("begin",))

        def pseudo_stage(self, s):
            calls.append(("pseudo", s))

    monkeypatch.setattr(PT, "halo_exchange", lambda field, plan, dist=None: calls.append(("exchange",)))
    one_step = [c for s in (1, 2, 3, 4) for c in (("stage", s), ("exchange",))]
    pre = [("begin",), ("exchange",)] + [c for _ in range(2) for s in (1, 2, 3, 4)
                                         for c in (("pseudo", s), ("exchange",))]
    PT.step(FakeField(), None, 7)
    expect = []
    for i in range(7):
        expect += (pre if i in (3, 6) else []) + one_step
    assert calls == expect
    calls.clear()
    Params.normal = 1
    PT.step(FakeField(), None, 7)
    assert calls == one_step * 7


class _StencilField:
    """A stand-in for a rank's Field on the host: element rows of two
    fields, each stage (and pseudo stage) an explicit update that reads the
    face neighbours' rows, so a stale ghost changes the owned result.  It has
    the calls partition.step makes (stage, pseudo_begin, pseudo_stage,
    halo_pack, halo_unpack, traces, stats, params) with CPU tensors."""
    device = "cpu"

    class _Params:
        normal, n_precond, pseudo_kmax = 0, 2, 2

    params = _Params

    def __init__(self, rows, adj, glob):
        import types
        self.u = rows.clone()
        # neighbours in ascending global order, so that every rank sums them
        # in the same order as the whole mesh
        self.nbr = [sorted(a, key=lambda j: glob[j]) for a in adj]
        self.n = 0
        self.mesh = types.SimpleNamespace(info=types.SimpleNamespace(nu=rows.shape[2]))

    def _mix(self, fld, c):
        old = self.u[:, fld].clone()
        for e, nb in enumerate(self.nbr):
            if nb:
                m = sum(old[j] for j in nb) / len(nb)
                self.u[e, fld] = old[e] + c * (m - old[e])

    def stage(self, s):
        self._mix(0, 0.1 * s)
        self._mix(1, 0.05 * s)
        if s == 4:
            self.n += 1

    def pseudo_begin(self):
        self.u[:, 1] = self.u[:, 0] - 0.5

    def pseudo_stage(self, s):
        self._mix(1, 0.2)

    def stats(self):
        return {"n_steps": self.n}

    def halo_dtype(self):
        return self.u.dtype

    def halo_pack(self, ix):
        return self.u[ix].clone()

    def halo_unpack(self, ix, rows):
        self.u[ix] = rows

    def traces(self):
        pass


def _halo_rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2006_10967_gb300 import partition as PT
    mesh = _case("hexp")[0]
    g = torch.Generator().manual_seed(21)
    u0 = torch.rand(mesh.n_elems, 2, 5, generator=g, dtype=torch.float64)
    whole = _StencilField(u0, PT.face_adjacency(mesh), np.arange(mesh.n_elems))
    plan = PT.plans(mesh, PT.partition(mesh, world))[rank]
    mine = _StencilField(u0[torch.as_tensor(plan.local)], PT.face_adjacency(plan.mesh), plan.local)
    n = 5
    # the whole mesh on fr_step's schedule, no exchange
    for i in range(n):
        if i > 0 and i % whole.params.n_precond == 0:
            whole.pseudo_begin()
            for _ in range(whole.params.pseudo_kmax):
                for s in (1, 2, 3, 4):
                    whole.pseudo_stage(s)
        for s in (1, 2, 3, 4):
            whole.stage(s)
    PT.step(mine, plan, n, dist=dist)      # isend / irecv over gloo
    ol = torch.as_tensor(plan.owned_local)
    err = float((mine.u[ol] - whole.u[torch.as_tensor(plan.owned)]).abs().max())
    lone = _StencilField(u0[torch.as_tensor(plan.local)], PT.face_adjacency(plan.mesh), plan.local)
    for _ in range(n):
        for s in (1, 2, 3, 4):
            lone.stage(s)
    lone_err = float((lone.u[ol] - whole.u[torch.as_tensor(plan.owned)]).abs().max())
    with open(os.path.join(out_dir, f"halo{rank}.json"), "w") as f:
        json.dump({"err": err, "lone_err": lone_err, "steps": mine.n, "owned": int(plan.n_owned)}, f)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_step_and_halo_exchange_over_gloo(tmp_path, world):
    """partition.step and partition.halo_exchange, the calls a rank makes
    with one GPU per process, run with real point-to-point transport (gloo,
    one process per rank) on host stand-ins of the fields: after 5 steps
    with two scheduled preconditionings the owned rows equal the whole
    mesh's bit for bit, and a rank marched without the exchange differs."""
    mp.start_processes(_halo_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"halo{r}.json")) for r in range(world)]
    sys.path.insert(0, ROOT)
    assert sum(r["owned"] for r in res) == _case("hexp")[0].n_elems
    for r in res:
        assert r["steps"] == 5
        assert r["err"] == 0.0, r
        assert r["lone_err"] > 1e-6, r


def test_step_ranks_on_host_stand_ins():
    """partition.step_ranks (all ranks' fields in one process, the exchange
    a copy between them) on the host stand-ins: the owned rows after 5 steps
    with two scheduled preconditionings equal the whole mesh's bit for bit."""
    sys.path.insert(0, ROOT)
    from paper_2006_10967_gb300 import partition as PT
    mesh = _case("quad")[0]
    u0 = torch.rand(mesh.n_elems, 2, 4, generator=torch.Generator().manual_seed(5), dtype=torch.float64)
    whole = _StencilField(u0, PT.face_adjacency(mesh), np.arange(mesh.n_elems))
    for i in range(5):
        if i > 0 and i % 2 == 0:
            whole.pseudo_begin()
            for _ in range(2):
                for s in (1, 2, 3, 4):
                    whole.pseudo_stage(s)
        for s in (1, 2, 3, 4):
            whole.stage(s)
    plans = PT.plans(mesh, PT.partition(mesh, 3))
    fields = [_StencilField(u0[torch.as_tensor(p.local)], PT.face_adjacency(p.mesh), p.local) for p in plans]
    PT.step_ranks(fields, plans, 5)
    for p, f in zip(plans, fields):
        assert f.n == 5
        assert torch.equal(f.u[torch.as_tensor(p.owned_local)], whole.u[torch.as_tensor(p.owned)])


def test_partition_counts_edge_cases():
    """One part owns everything and has no ghosts or peers; as many parts as
    elements gives one element each; zero parts or more parts than elements
    are refused."""
    sys.path.insert(0, ROOT)
    import synthetic as S
    from paper_2006_10967_gb300 import partition as PT
    mesh = S.quad_grid(3, jitter=0.1, seed=1)
    one = PT.plans(mesh, PT.partition(mesh, 1))
    assert len(one) == 1 and len(one[0].ghosts) == 0 and not one[0].send and not one[0].recv
    assert np.array_equal(one[0].local, np.arange(mesh.n_elems))
    part = PT.partition(mesh, mesh.n_elems)
    assert np.array_equal(np.sort(part), np.arange(mesh.n_elems))
    for bad in (0, mesh.n_elems + 1):
        with pytest.raises(ValueError):
            PT.partition(mesh, bad)
