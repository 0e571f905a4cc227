"""Element partitioning and halo exchange plans for running one problem on
several GPUs, one rank per GPU.

The FR residual of an element needs its own state, its face neighbours'
traces (the common solution of Step 2) and, on faces where the neighbour is
the L side, the neighbour's corrected gradient at the face (the viscous
common flux of Step 5), which in turn needs the neighbour's neighbours.  A
rank therefore keeps, beside the elements it owns, the ghost elements within
two face-neighbour layers of them; with the ghosts' stage values received
from their owners before every RK stage, the residual of the owned elements
computed on the rank's local mesh equals the single-domain residual, and the
ghosts' own results are discarded (overwritten by the next exchange).

The local mesh keeps its elements in ascending global order: the L side of an
interior face (the side the LDG parameter beta = +1/2 refers to) is the one
with the lower element number, and a local numbering that preserves the
global order makes every rank pick the same L side as the single domain.

partition() splits the elements by recursive coordinate bisection of their
centroids (balanced counts, deterministic); plans() builds every rank's local
mesh and its send and receive lists; exchange() moves ghost values over
torch.distributed point-to-point calls (gloo on the host, NCCL on the device).

On the device a rank's field steps one RK stage at a time (Field.stage, the
library's fr_stage) and exchanges its ghosts' stage values between stages:
step() does that for one rank over torch.distributed, step_ranks() for
several ranks' fields held by one process on one device (the exchange is
then a device copy between the fields).  The preconditioning runs the same
way, one pseudo stage at a time (Field.pseudo_begin / pseudo_stage, the
library's fr_pseudo_begin / fr_pseudo_stage) with the ghost exchange after
the reset and after every pseudo stage: precondition() and
precondition_ranks(), called by step() and step_ranks() before every step
whose index is a positive multiple of params.n_precond, as fr_step does.
Only the fixed iteration count (params.pseudo_fixed): the stop rule's RMS is
taken over the whole mesh.
"""
from dataclasses import dataclass, field

import numpy as np

# face vertex lists per element type (local vertex numbers)
_FACES = {
    "quad": [(0, 1), (1, 2), (2, 3), (3, 0)],
    "tri": [(0, 1), (1, 2), (2, 0)],
    "hex": [(0, 1, 2, 3), (0, 1, 5, 4), (1, 2, 6, 5), (2, 3, 7, 6), (3, 0, 4, 7), (4, 5, 6, 7)],
}


def centroids(mesh):
    return mesh.nodes[mesh.conn].mean(axis=1)


def partition(mesh, nparts):
    """Part id per element: recursive bisection of the centroids along the
    axis of largest extent, with sizes proportional to the part counts.
    1 <= nparts <= the element count (no part is empty)."""
    nparts = int(nparts)
    if not 1 <= nparts <= mesh.n_elems:
        raise ValueError(f"nparts must lie in 1..{mesh.n_elems} (the element count), not {nparts}")
    cen = centroids(mesh)
    part = np.zeros(mesh.n_elems, dtype=np.int64)

    def split(ids, k, first):
        if k == 1 or len(ids) == 0:
            part[ids] = first
            return
        ext = cen[ids].max(0) - cen[ids].min(0)
        axis = int(np.argmax(ext))
        order = ids[np.argsort(cen[ids, axis], kind="stable")]
        k1 = k // 2
        n1 = int(round(len(ids) * k1 / k))
        split(order[:n1], k1, first)
        split(order[n1:], k - k1, first + k1)

    split(np.arange(mesh.n_elems), nparts, 0)
    return part


def face_adjacency(mesh, quantum=None):
    """Face neighbours of every element (faces matched by their vertex
    positions, modulo the period on periodic axes)."""
    nodes = np.asarray(mesh.nodes, dtype=np.float64)
    d = nodes.shape[1]
    span = nodes.max(0) - nodes.min(0)
    q0 = quantum if quantum is not None else 1e-9 * float(span.max())
    keyed = np.empty(nodes.shape, dtype=np.int64)
    for a in range(d):
        if mesh.periodic[a]:
            # a quantum that divides the period, so that a node and its
            # periodic image get the same key
            K = max(1, int(round(mesh.period[a] / q0)))
            keyed[:, a] = np.mod(np.round(nodes[:, a] * (K / mesh.period[a])).astype(np.int64), K)
        else:
            keyed[:, a] = np.round(nodes[:, a] / q0).astype(np.int64)
    table = {}
    for e in range(mesh.n_elems):
        for fv in _FACES[mesh.etype]:
            key = tuple(sorted(tuple(keyed[mesh.conn[e, v]]) for v in fv))
            table.setdefault(key, []).append(e)
    adj = [set() for _ in range(mesh.n_elems)]
    for lst in table.values():
        if len(lst) == 2 and lst[0] != lst[1]:
            adj[lst[0]].add(lst[1])
            adj[lst[1]].add(lst[0])
    return adj


@dataclass
class LocalMesh:
    """A rank's local mesh (the same fields as the meshes the binding and the
    tests take: element type, nodes, connectivity, periodicity)."""
    etype: str
    nodes: np.ndarray
    conn: np.ndarray
    periodic: tuple
    period: tuple
    name: str = ""

    @property
    def dim(self):
        return self.nodes.shape[1]

    @property
    def n_elems(self):
        return self.conn.shape[0]


@dataclass
class Plan:
    rank: int
    owned: np.ndarray                 # global ids, ascending
    ghosts: np.ndarray                # global ids, ascending
    local: np.ndarray                 # global id of every local element (owned and ghosts, ascending)
    mesh: object                      # the local mesh, elements in the order of local
    owned_local: np.ndarray = None    # local indices of the owned elements
    send: dict = field(default_factory=dict)   # peer -> local indices of owned elements the peer needs
    recv: dict = field(default_factory=dict)   # peer -> local indices of ghosts owned by the peer

    @property
    def n_owned(self):
        return len(self.owned)


def plans(mesh, part, depth=2):
    """Every rank's plan (each rank can build all of them from the global
    mesh and part ids; they are deterministic)."""
    adj = face_adjacency(mesh)
    nparts = int(part.max()) + 1
    out = []
    for r in range(nparts):
        owned = np.nonzero(part == r)[0]
        own = set(owned.tolist())
        ghosts, frontier = set(), set(owned.tolist())
        for _ in range(depth):
            nxt = set()
            for e in frontier:
                nxt |= adj[e]
            nxt -= own
            nxt -= ghosts
            ghosts |= nxt
            frontier = nxt
        gh = np.array(sorted(ghosts), dtype=np.int64)
        local = np.sort(np.concatenate([owned, gh]))
        conn = mesh.conn[local]
        used, inv = np.unique(conn, return_inverse=True)
        lm = LocalMesh(mesh.etype, mesh.nodes[used], inv.reshape(conn.shape).astype(np.int64),
                       tuple(mesh.periodic), tuple(mesh.period), f"{mesh.name}_part{r}")
        out.append(Plan(r, owned, gh, local, lm, np.searchsorted(local, owned)))
    pos = [{int(g): i for i, g in enumerate(p.local)} for p in out]
    for p in out:
        for q in range(nparts):
            if q == p.rank:
                continue
            need = [int(g) for g in out[q].ghosts if part[g] == p.rank]      # in q's ghost order
            if need:
                p.send[q] = np.array([pos[p.rank][g] for g in need], dtype=np.int64)
            have = [int(g) for g in p.ghosts if part[g] == q]
            if have:
                p.recv[q] = np.array([pos[p.rank][g] for g in have], dtype=np.int64)
    return out


def exchange(values, plan, dist=None):
    """Overwrite the ghost rows of values (local element-major tensor, first
    axis the local elements) with their owners' rows.  Point-to-point over
    torch.distributed (isend / irecv, all posted before waiting)."""
    import torch
    import torch.distributed as td
    d = dist or td
    reqs, bufs = [], {}
    for q, idx in sorted(plan.recv.items()):
        bufs[q] = torch.empty((len(idx),) + tuple(values.shape[1:]), dtype=values.dtype, device=values.device)
        reqs.append(d.irecv(bufs[q], src=q))
    for q, idx in sorted(plan.send.items()):
        reqs.append(d.isend(values[torch.as_tensor(idx)].contiguous(), dst=q))
    for r in reqs:
        r.wait()
    for q, idx in plan.recv.items():
        values[torch.as_tensor(idx)] = bufs[q]
    return values


def _device_lists(plan, device="cuda"):
    """The plan's send and receive lists as int64 tensors on `device`."""
    import torch
    cache = getattr(plan, "_dev", None)
    if cache is None:
        cache = plan._dev = {}
    if device not in cache:
        cache[device] = ({q: torch.as_tensor(ix, device=device) for q, ix in plan.send.items()},
                         {q: torch.as_tensor(ix, device=device) for q, ix in plan.recv.items()})
    return cache[device]


def halo_exchange(field, plan, dist=None):
    """Replace the ghost elements' stage values of a rank's field with their
    owners' (packed on the field's device, moved with isend/irecv,
    unpacked), then recompute the traces."""
    import torch
    import torch.distributed as td
    d = dist or td
    dev = field.device
    send, recv = _device_lists(plan, dev)
    packed = {q: field.halo_pack(ix) for q, ix in sorted(send.items())}
    bufs = {q: torch.empty((len(ix), 2, field.mesh.info.nu), dtype=field.halo_dtype(), device=dev)
            for q, ix in sorted(recv.items())}
    reqs = [d.irecv(bufs[q], src=q) for q in sorted(bufs)]
    reqs += [d.isend(packed[q], dst=q) for q in sorted(packed)]
    for r in reqs:
        r.wait()
    for q, ix in recv.items():
        field.halo_unpack(ix, bufs[q])
    field.traces()


def _precondition_due(field, n):
    """fr_step's schedule: a preconditioning before step n (the field's step
    count) when n is a positive multiple of params.n_precond and the normal
    comes from psi."""
    P = field.params
    return P.normal == 0 and n > 0 and n % P.n_precond == 0


def precondition(field, plan, dist=None):
    """The preconditioning of one rank's field: psi reset, then
    params.pseudo_kmax pseudo-time RK4 iterations, with a ghost exchange
    after the reset and after every pseudo stage."""
    field.pseudo_begin()
    halo_exchange(field, plan, dist)
    for _ in range(int(field.params.pseudo_kmax)):
        for s in (1, 2, 3, 4):
            field.pseudo_stage(s)
            halo_exchange(field, plan, dist)


def step(field, plan, n_steps=1, dist=None):
    """n physical RK4 steps of one rank's field with a ghost exchange after
    every stage, preconditioning on fr_step's schedule."""
    n0 = field.stats()["n_steps"]
    for i in range(int(n_steps)):
        if _precondition_due(field, n0 + i):
            precondition(field, plan, dist)
        for s in (1, 2, 3, 4):
            field.stage(s)
            halo_exchange(field, plan, dist)


def _exchange_ranks(fields, plans, lists):
    """Every rank's ghosts refreshed from their owners (device copies), then
    every rank's traces."""
    packed = {(p.rank, q): fields[p.rank].halo_pack(ix)
              for p, (send, _) in zip(plans, lists) for q, ix in sorted(send.items())}
    for p, (_, recv) in zip(plans, lists):
        for q, ix in sorted(recv.items()):
            fields[p.rank].halo_unpack(ix, packed[(q, p.rank)])
    for f in fields:
        f.traces()


def precondition_ranks(fields, plans):
    """precondition() for several ranks' fields held by this process on one
    device."""
    lists = [_device_lists(p, f.device) for p, f in zip(plans, fields)]
    for f in fields:
        f.pseudo_begin()
    _exchange_ranks(fields, plans, lists)
    for _ in range(int(fields[0].params.pseudo_kmax)):
        for s in (1, 2, 3, 4):
            for f in fields:
                f.pseudo_stage(s)
            _exchange_ranks(fields, plans, lists)


def step_ranks(fields, plans, n_steps=1):
    """n physical RK4 steps of several ranks' fields held by this process on
    one device: per stage every rank's stage, then every rank's ghosts
    refreshed from their owners by device copies, then the traces;
    preconditioning on fr_step's schedule."""
    lists = [_device_lists(p, f.device) for p, f in zip(plans, fields)]
    n0 = fields[0].stats()["n_steps"]
    for i in range(int(n_steps)):
        if _precondition_due(fields[0], n0 + i):
            precondition_ranks(fields, plans)
        for s in (1, 2, 3, 4):
            for f in fields:
                f.stage(s)
            _exchange_ranks(fields, plans, lists)
