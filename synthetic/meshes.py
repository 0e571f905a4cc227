"""Seeded mesh generators (node coordinates + connectivity only).

Vertex orders:
  quad: counter-clockwise, reference corners (-1,-1), (1,-1), (1,1), (-1,1)
  tri:  counter-clockwise, reference corners (-1,-1), (1,-1), (-1,1)
  hex:  bottom face counter-clockwise then top face, reference corners
        (+-1,+-1,+-1) with xi fastest, i.e. the quad order at zeta=-1 then +1.
Periodic axes keep duplicate image nodes on both ends; faces are matched
modulo the period by whoever consumes the mesh.
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class Mesh:
    etype: str                 # 'quad' | 'tri' | 'hex'
    nodes: np.ndarray          # (n_nodes, dim) float64
    conn: np.ndarray           # (n_elems, n_verts) int64
    periodic: tuple            # per-axis bool
    period: tuple              # per-axis period length (ignored if not periodic)
    name: str = ""

    @property
    def dim(self):
        return self.nodes.shape[1]

    @property
    def n_elems(self):
        return self.conn.shape[0]


def _grid_nodes(ns, lengths):
    axes = [np.linspace(0.0, L, n + 1) for n, L in zip(ns, lengths)]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([m.ravel(order="F") for m in mesh], axis=1)


def _jitter(nodes, ns, lengths, amount, rng, periodic):
    """Move nodes by U(-amount*h, amount*h) per coordinate.

    Nodes on a wall move only along that wall (corners stay put).  On a
    periodic axis a node and its periodic image receive the same displacement.
    """
    dim = len(ns)
    idx = np.stack(np.unravel_index(np.arange(nodes.shape[0]),
                                    [n + 1 for n in ns], order="F"), axis=1)
    # key each node by its index modulo the period on periodic axes
    key = idx.copy()
    for a in range(dim):
        if periodic[a]:
            key[:, a] = key[:, a] % ns[a]
    flat = np.ravel_multi_index(key.T, [n + 1 for n in ns], order="F")
    hs = np.array([L / n for n, L in zip(ns, lengths)])
    disp_all = rng.uniform(-amount, amount, size=(np.prod([n + 1 for n in ns]), dim)) * hs
    disp = disp_all[flat]
    for a in range(dim):
        if not periodic[a]:
            on_wall = (idx[:, a] == 0) | (idx[:, a] == ns[a])
            disp[on_wall, a] = 0.0
    return nodes + disp


def quad_grid(nx, ny=None, lengths=(1.0, 1.0), periodic=(True, True), jitter=0.0,
              seed=1, shuffle_seed=None, rotate_seed=None, name=""):
    """nx x ny quads on [0,Lx]x[0,Ly].

    jitter: interior node displacement as a fraction of h (uniform, seeded).
    shuffle_seed: permute element order (unstructured connectivity).
    rotate_seed: cyclically rotate each element's vertex list (CCW kept),
                 so that local face numbering differs between neighbours.
    """
    ny = nx if ny is None else ny
    ns = (nx, ny)
    nodes = _grid_nodes(ns, lengths)
    rng = np.random.default_rng(seed)
    if jitter > 0:
        nodes = _jitter(nodes, ns, lengths, jitter, rng, periodic)
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    i, j = i.ravel(order="F"), j.ravel(order="F")
    nid = lambda a, b: a + (nx + 1) * b
    conn = np.stack([nid(i, j), nid(i + 1, j), nid(i + 1, j + 1), nid(i, j + 1)], axis=1)
    conn = _reorder(conn, shuffle_seed, rotate_seed, 4)
    return Mesh("quad", nodes, conn.astype(np.int64), tuple(periodic), tuple(lengths), name)


def _hex_rotations():
    """The 24 proper rotations of the reference cube as permutations of the
    8 vertex slots: perm[k] is the old local vertex at R (ref corner k), so
    that the new map is x_old(R xi) and det J keeps its sign."""
    import itertools
    ref = [(-1, -1, -1), (1, -1, -1), (1, 1, -1), (-1, 1, -1),
           (-1, -1, 1), (1, -1, 1), (1, 1, 1), (-1, 1, 1)]
    index = {c: k for k, c in enumerate(ref)}
    out = []
    for axes in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            R = np.zeros((3, 3), dtype=int)
            for a in range(3):
                R[a, axes[a]] = signs[a]
            if round(np.linalg.det(R)) != 1:
                continue
            out.append([index[tuple(int(v) for v in R @ np.array(c))] for c in ref])
    return np.array(out, dtype=np.int64)


def hex_grid(nx, ny=None, nz=None, lengths=(1.0, 1.0, 1.0), periodic=(False, False, False),
             jitter=0.0, seed=1, shuffle_seed=None, rotate_seed=None, name=""):
    """nx x ny x nz hexahedra on [0,Lx]x[0,Ly]x[0,Lz].

    rotate_seed: give each element's vertex list one of the 24 proper
                 rotations of the reference cube (seeded), so that
                 neighbouring elements see a shared face in different
                 orientations (all 8 point orderings of a face occur).
    """
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    ns = (nx, ny, nz)
    nodes = _grid_nodes(ns, lengths)
    rng = np.random.default_rng(seed)
    if jitter > 0:
        nodes = _jitter(nodes, ns, lengths, jitter, rng, periodic)
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    i, j, k = i.ravel(order="F"), j.ravel(order="F"), k.ravel(order="F")
    nid = lambda a, b, c: a + (nx + 1) * (b + (ny + 1) * c)
    conn = np.stack([nid(i, j, k), nid(i + 1, j, k), nid(i + 1, j + 1, k), nid(i, j + 1, k),
                     nid(i, j, k + 1), nid(i + 1, j, k + 1), nid(i + 1, j + 1, k + 1),
                     nid(i, j + 1, k + 1)], axis=1)
    conn = _reorder(conn, shuffle_seed, None, 8)
    if rotate_seed is not None:
        rots = _hex_rotations()
        r = np.random.default_rng(rotate_seed).integers(0, len(rots), size=conn.shape[0])
        conn = np.take_along_axis(conn, rots[r], axis=1)
    return Mesh("hex", nodes, conn.astype(np.int64), tuple(periodic), tuple(lengths), name)


def tri_split(nx, ny=None, lengths=(1.0, 1.0), periodic=(True, True), shuffle_seed=None, name=""):
    """Each quad of an nx x ny grid split along its (0,0)-(1,1) diagonal."""
    q = quad_grid(nx, ny, lengths, periodic)
    a, b, c, d = q.conn.T
    conn = np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, d], 1)], 0)
    conn = _reorder(conn, shuffle_seed, None, 3)
    return Mesh("tri", q.nodes, conn.astype(np.int64), tuple(periodic), tuple(lengths), name)


def tri_delaunay(m, jitter=0.1, seed=2, shuffle_seed=None, name=""):
    """Delaunay triangulation of an m x m point lattice on [0,1]^2.

    Interior points move by U(-jitter*h, jitter*h); boundary points slide along
    their edge; corners stay.  Walls on all sides (not periodic).
    """
    from scipy.spatial import Delaunay
    ns = (m - 1, m - 1)
    nodes = _grid_nodes(ns, (1.0, 1.0))
    rng = np.random.default_rng(seed)
    nodes = _jitter(nodes, ns, (1.0, 1.0), jitter, rng, (False, False))
    tri = Delaunay(nodes).simplices.astype(np.int64)
    p = nodes[tri]
    area2 = ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1])
             - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1]))
    tri[area2 < 0] = tri[area2 < 0][:, [0, 2, 1]]
    # drop slivers of (near) zero area that a lattice can produce on the hull
    p = nodes[tri]
    area2 = ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1])
             - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1]))
    tri = tri[area2 > 1e-12]
    tri = _reorder(tri, shuffle_seed, None, 3)
    return Mesh("tri", nodes, tri, (False, False), (1.0, 1.0), name)


def _reorder(conn, shuffle_seed, rotate_seed, nv):
    if shuffle_seed is not None:
        perm = np.random.default_rng(shuffle_seed).permutation(conn.shape[0])
        conn = conn[perm]
    if rotate_seed is not None and nv == 4:
        r = np.random.default_rng(rotate_seed).integers(0, 4, size=conn.shape[0])
        cols = (np.arange(4)[None, :] + r[:, None]) % 4
        conn = np.take_along_axis(conn, cols, axis=1)
    return conn
