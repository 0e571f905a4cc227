"""Workload descriptions and seeded random draws.

Every workload is a plain record of numbers: a mesh, an order, a velocity
field, an initial circle/sphere and the run parameters.  The run parameters
follow the paper's settings (Section 2: gamma = 0.09, eps = 0.06 h/p;
Section 3.2: s0 = -5, nu_max = 0.15 h/p, precondition every 1000 steps, stop
norm 1/2; Section 4: beta = 3p/(4h)) with the readings stated beside them.
"""
from dataclasses import dataclass, field, replace
import math

import numpy as np

from . import meshes


@dataclass
class Velocity:
    """Analytic velocity field.

    kind: 'uniform'     u = a g(t)
          'rider_kothe' u = -sin^2(pi x) sin(2 pi y) g(t), v = sin(2 pi x) sin^2(pi y) g(t)
          'leveque'     3D deformation field of Section 4.3 times g(t)
          'stream'      u = dPsi/dy, v = -dPsi/dx with
                        Psi = g(t) sum_m A_m sin(2 pi k_m.x) + B_m cos(2 pi k_m.x)
          'rotation'    solid-body rotation about (a[0], a[1]): (a[1] - y, x - a[0])
                        (Section 4.1: Zalesak about (0.5, 0.5), Rudman about (2, 2))
    g(t) = cos(pi t / T) when T > 0, else 1.
    """
    kind: str
    a: tuple = (0.0, 0.0, 0.0)
    T: float = 0.0
    kx: np.ndarray = None
    ky: np.ndarray = None
    A: np.ndarray = None
    B: np.ndarray = None


@dataclass
class Circle:
    """Initial interface: phi = (1 + tanh(beta * (r - |x - c|))) / 2 (Section 4, discEq)."""
    centre: tuple
    radius: float
    beta: float


@dataclass
class SlottedDisk:
    """Initial interface of the solid-body rotation tests (Section 4.1): the disk
    |x - c| <= r with the slot |x - c_x| <= half_width, y <= top removed.

    The initial field is phi = (1 + tanh(beta d)) / 2 (Eq. initialCond) with d
    the signed distance of the slotted disk, positive inside, taken as the set
    difference min(r - |x - c|, -d_slot) where d_slot is the signed distance
    of the slot strip (positive inside it); this is exact at the interface and
    inside the shape, and saturates the tanh elsewhere."""
    centre: tuple
    radius: float
    half_width: float
    top: float
    beta: float

    def signed_distance(self, x):
        x = np.asarray(x, dtype=np.float64)
        dx = x[..., 0] - self.centre[0]
        dy = x[..., 1] - self.centre[1]
        d_disk = self.radius - np.sqrt(dx * dx + dy * dy)
        ax = np.abs(dx) - self.half_width            # > 0: beside the strip
        ay = x[..., 1] - self.top                    # > 0: above the strip
        inside = (ax <= 0) & (ay <= 0)
        d_slot = np.where(inside, np.minimum(-ax, -ay),
                          -np.sqrt(np.maximum(ax, 0.0) ** 2 + np.maximum(ay, 0.0) ** 2))
        return np.minimum(d_disk, -d_slot)

    def phi(self, x):
        """Initial phase field at the points x (..., 2)."""
        return 0.5 * (1.0 + np.tanh(self.beta * self.signed_distance(x)))


@dataclass
class Workload:
    name: str
    mesh_fn: object            # callable -> meshes.Mesh
    order: int
    velocity: Velocity
    circle: Circle
    t_end: float
    h: float
    gamma: float = 0.09
    eps: float = 0.0
    tau: float = 0.1           # LDG penalty on phi (not given in the paper)
    tau_psi: float = 0.1       # penalty on psi's jumps (the LDG penalty applies to u = [phi, psi])
    tau_pseudo: float = 0.1    # LDG penalty in the preconditioning equation
    dt: float = 0.0
    n_steps: int = 0
    n_precond: int = 1000
    pseudo_kmax: int = 20
    pseudo_dtau: float = 0.0
    pseudo_tol: float = 0.5
    s0: float = -5.0
    kappa: float = 5.0         # printed as 5e3; read as 5 (see the design notes)
    nu_max: float = 0.0
    delta: float = 1e-12
    precision: str = "fp64"
    wall: str = "copy"         # Section 3.3 copy ghost; "noflux": zero wall flux (an option)
    extra: dict = field(default_factory=dict)

    def mesh(self):
        return self.mesh_fn()

    def with_(self, **kw):
        return replace(self, **kw)


def _umax(vel, dim, n=257, length=1.0):
    """Max |u| at t = 0 on a fine lattice of [0, length]^dim (used only to size
    the time step)."""
    g = np.linspace(0.0, length, n)
    if dim == 2:
        x, y = np.meshgrid(g, g, indexing="ij")
        if vel.kind == "uniform":
            return float(np.hypot(vel.a[0], vel.a[1]))
        if vel.kind == "rider_kothe":
            u = -np.sin(np.pi * x) ** 2 * np.sin(2 * np.pi * y)
            v = np.sin(2 * np.pi * x) * np.sin(np.pi * y) ** 2
        elif vel.kind == "rotation":
            u, v = vel.a[1] - y, x - vel.a[0]
        elif vel.kind == "stream":
            u = np.zeros_like(x)
            v = np.zeros_like(x)
            for kx, ky, A, B in zip(vel.kx, vel.ky, vel.A, vel.B):
                arg = 2 * np.pi * (kx * x + ky * y)
                d = 2 * np.pi * (A * np.cos(arg) - B * np.sin(arg))
                u += ky * d
                v -= kx * d
        return float(np.sqrt(u * u + v * v).max())
    g = np.linspace(0.0, 1.0, 65)
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    if vel.kind == "uniform":
        return float(np.linalg.norm(vel.a))
    s = np.sin
    pi = np.pi
    u = 2 * s(pi * x) ** 2 * s(2 * pi * y) * s(2 * pi * z)
    v = -s(2 * pi * x) * s(pi * y) ** 2 * s(2 * pi * z)
    w = -s(2 * pi * x) * s(2 * pi * y) * s(pi * z) ** 2
    return float(np.sqrt(u * u + v * v + w * w).max())


def time_step(t_end, h, p, umax, cfl=0.1):
    """dt = CFL h / ((p+1) U_max), shortened so that an integer number of steps hits t_end."""
    dt = cfl * h / ((p + 1) * umax)
    n = int(math.ceil(t_end / dt - 1e-9))
    return t_end / n, n


def _finish(w, dim, cfl=0.1):
    p, h = w.order, w.h
    if w.eps == 0.0:
        w.eps = 0.06 * h / p
    w.nu_max = 0.15 * h / p
    w.pseudo_dtau = 0.1 * h / (p + 1)
    umax = _umax(w.velocity, dim, length=w.extra.get("length", 1.0))
    w.dt, w.n_steps = time_step(w.t_end, h, p, umax, cfl)
    w.extra.setdefault("umax", umax)
    return w


def _half_plane_vectors(kmax_norm):
    out = []
    r = int(math.floor(kmax_norm))
    for kx in range(0, r + 1):
        for ky in range(-r, r + 1):
            if kx == 0 and ky <= 0:
                continue
            if kx * kx + ky * ky <= kmax_norm * kmax_norm:
                out.append((kx, ky))
    out.sort(key=lambda k: (k[0] ** 2 + k[1] ** 2, k[0], k[1]))
    return out


def stream_coefficients(n_vectors=16, seed=4, sigma=0.1):
    """Stream function with n_vectors smallest half-plane integer wave vectors,
    sin and cos coefficients drawn from N(0, sigma^2)."""
    ks = _half_plane_vectors(4.0)[:n_vectors]
    rng = np.random.default_rng(seed)
    A = rng.normal(0.0, sigma, n_vectors)
    B = rng.normal(0.0, sigma, n_vectors)
    kx = np.array([k[0] for k in ks], dtype=np.float64)
    ky = np.array([k[1] for k in ks], dtype=np.float64)
    return kx, ky, A, B


def random_phase_stream(rng, n_modes=16, kmax=4.0, T=4.0):
    """Psi = sum a_k sin(2 pi k.x + theta_k), |k| <= kmax, a_k ~ 1/|k|^2,
    scaled so that max |u| = 1 at t = 0, times cos(pi t / T)."""
    pool = _half_plane_vectors(kmax)
    sel = rng.choice(len(pool), size=n_modes, replace=False)
    ks = np.array([pool[i] for i in sel], dtype=np.float64)
    kn2 = (ks ** 2).sum(1)
    a = 1.0 / kn2
    theta = rng.uniform(0.0, 2 * np.pi, n_modes)
    A = a * np.cos(theta)
    B = a * np.sin(theta)
    vel = Velocity("stream", T=T, kx=ks[:, 0].copy(), ky=ks[:, 1].copy(), A=A, B=B)
    s = 1.0 / _umax(vel, 2)
    vel.A = A * s
    vel.B = B * s
    return vel


def ensemble_instances(n_instances=256, seed=3):
    """Uneven-size periodic quad instances: n ~ U{16..96}, p ~ U{2,3,4,5},
    circles r ~ U[0.1, 0.2] at least r from the edges, random-phase velocity."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_instances):
        n = int(rng.integers(16, 97))
        p = int(rng.integers(2, 6))
        r = float(rng.uniform(0.1, 0.2))
        c = tuple(float(v) for v in rng.uniform(r, 1.0 - r, 2))
        vel = random_phase_stream(rng)
        h = 1.0 / n
        w = Workload(f"ens{i}", (lambda n=n: meshes.quad_grid(n)), p, vel,
                     Circle(c, r, 3 * p / (4 * h)), t_end=4.0, h=h, precision="mixed")
        out.append(_finish(w, 2))
    return out


def _c1():
    n, p = 16, 3
    h = 1.0 / n
    eps_b = 0.5 * h / (p + 1)
    w = Workload("c1_quad16_p3_translate", lambda: meshes.quad_grid(16, name="quad16"), p,
                 Velocity("uniform", a=(1.0, 0.5, 0.0)),
                 Circle((0.5, 0.5), 0.25, 1.0 / (2 * eps_b)), t_end=2.0, h=h)
    # The initial profile width eps_b is the equilibrium width eps/gamma.
    w.eps = w.gamma * eps_b
    return _finish(w, 2)


def _c2q(n=128):
    p = 4
    h = 1.0 / n
    w = Workload(f"c2q_quad{n}_jitter_p4_rider_kothe",
                 lambda: meshes.quad_grid(n, periodic=(False, False), jitter=0.1, seed=1,
                                          shuffle_seed=11, rotate_seed=12, name=f"quadjit{n}"),
                 p, Velocity("rider_kothe", T=8.0), Circle((0.5, 0.75), 0.15, 3 * p / (4 * h)),
                 t_end=8.0, h=h)
    return _finish(w, 2)


def _c2t(m=123):
    p = 3
    n_tri = 2 * (m - 1) ** 2
    h = math.sqrt(2.0 / n_tri)
    w = Workload(f"c2t_tri{n_tri}_p3_rider_kothe",
                 lambda: meshes.tri_delaunay(m, jitter=0.1, seed=2, shuffle_seed=13,
                                             name=f"tridel{m}"),
                 p, Velocity("rider_kothe", T=8.0), Circle((0.5, 0.75), 0.15, 3 * p / (4 * h)),
                 t_end=8.0, h=h)
    return _finish(w, 2)


def _c2s(n=128, p=3):
    """Rider-Kothe vortex on the paper's split-triangle family ("c" meshes of
    Section 4.2): an n x n grid with every square split along a diagonal,
    walls, element order shuffled (seed 14); h = sqrt(2 |Omega| / E) = 1/n."""
    h = 1.0 / n
    w = Workload(f"c2s_trisplit{n}_p{p}_rider_kothe",
                 lambda: meshes.tri_split(n, periodic=(False, False), shuffle_seed=14, name=f"trisplit{n}"),
                 p, Velocity("rider_kothe", T=8.0), Circle((0.5, 0.75), 0.15, 3 * p / (4 * h)),
                 t_end=8.0, h=h)
    return _finish(w, 2)


def _c3(n=64, p=3):
    h = 1.0 / n
    w = Workload(f"c3_hex{n}_p{p}_leveque",
                 lambda: meshes.hex_grid(n, name=f"hex{n}"), p, Velocity("leveque", T=3.0),
                 Circle((0.35, 0.35, 0.35), 0.15, 3 * p / (4 * h)), t_end=3.0, h=h,
                 precision="mixed")
    return _finish(w, 3)


def _c5():
    n, p = 64, 4
    h = 1.0 / n
    kx, ky, A, B = stream_coefficients(16, seed=4, sigma=0.1)
    vel = Velocity("stream", T=0.0, kx=kx, ky=ky, A=A, B=B)
    w = Workload("c5_quad64_p4_adjoint", lambda: meshes.quad_grid(n, name="quad64"), p, vel,
                 Circle((0.5, 0.5), 0.15, 3 * p / (4 * h)), t_end=0.0, h=h)
    w = _finish(w.with_(t_end=1.0), 2)
    w.n_steps = 400
    w.t_end = w.dt * 400
    rng = np.random.default_rng(5)
    off = rng.uniform(-0.1, 0.1, 2)
    w.extra["target"] = Circle((0.5 + float(off[0]), 0.5 + float(off[1])), 0.15, 3 * p / (4 * h))
    w.extra["ckpt_every"] = 20
    return w


def _zalesak(n=100, p=4):
    """Zalesak's slotted disk (Section 4.1): r = 0.15 at (0.5, 0.75), slot
    |x - 0.5| <= 0.025, y <= 0.85, solid-body rotation about (0.5, 0.5) for one
    revolution (t = 2 pi) on n x n uniform quads.

    The domain is periodic: the rotation crosses the unit square's edges, and
    with copy ghost states and the central inviscid flux an inflow edge
    amplifies round-off until the march fails; across opposite edges the
    rotation's normal component is the same, and the disk stays far from them."""
    h = 1.0 / n
    w = Workload(f"zalesak_quad{n}_p{p}",
                 lambda: meshes.quad_grid(n, periodic=(True, True), name=f"quadper{n}"), p,
                 Velocity("rotation", a=(0.5, 0.5, 0.0)),
                 SlottedDisk((0.5, 0.75), 0.15, 0.025, 0.85, 3 * p / (4 * h)), t_end=2 * math.pi, h=h)
    return _finish(w, 2)


def _rudman(n=200, p=4):
    """Rudman's slotted disk (Section 4.1): r = 0.5 at (2, 2.75) in [0, 4]^2,
    slot |x - 2| <= 0.06, y <= 2.65, rotation about (2, 2) for one revolution
    on n x n uniform quads (periodic, as for Zalesak's disk)."""
    h = 4.0 / n
    w = Workload(f"rudman_quad{n}_p{p}",
                 lambda: meshes.quad_grid(n, lengths=(4.0, 4.0), periodic=(True, True), name=f"quadper{n}L4"), p,
                 Velocity("rotation", a=(2.0, 2.0, 0.0)),
                 SlottedDisk((2.0, 2.75), 0.5, 0.06, 2.65, 3 * p / (4 * h)), t_end=2 * math.pi, h=h)
    w.extra["length"] = 4.0
    return _finish(w, 2)


def initial_phi(w, x):
    """The workload's initial phase field at the points x: the disk of Eq.
    discEq for a Circle, the slotted disk for a SlottedDisk."""
    c = w.circle
    if isinstance(c, SlottedDisk):
        return c.phi(x)
    x = np.asarray(x, dtype=np.float64)
    r = np.sqrt(((x - np.asarray(c.centre)[: x.shape[-1]]) ** 2).sum(-1))
    return 0.5 * (1.0 + np.tanh(c.beta * (c.radius - r)))


WORKLOADS = {
    "zalesak": _zalesak,
    "rudman": _rudman,
    "c1": _c1,
    "c2q": _c2q,
    "c2t": _c2t,
    "c2s": _c2s,
    "c3": _c3,
    "c5": _c5,
}


def workload(name, **kw):
    """Build a workload by short name ('c1', 'c2q', 'c2t', 'c3', 'c5');
    keyword arguments override size parameters (n=..., m=...)."""
    return WORKLOADS[name](**kw)
