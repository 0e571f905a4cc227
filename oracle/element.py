"""Reference elements and FR operators (oracle, test infrastructure only).

Section 3.1: solution points (Gauss-Legendre tensor points on quadrilaterals
and hexahedra; on triangles a symmetric interior point set, see below), the
nodal basis l_i = V^{-1} Psi (Vandermonde of an orthonormal basis Psi), flux
points on the element boundary, and the correction functions g_j with
n_i . g_j(x_i) = delta_ij.

Every operator is built densely, from the same generic recipe for all three
element types, so that it can be checked by eye:
  Lmat[k, i]   = l_i(x^f_k)                         (Step 1, Eq. extrapolateSoln)
  Dmat[a][j,i] = d l_i / d xi_a (x^u_j)              (Steps 3 and 6)
  LIFT[i, k]   = (div g_k)(x^u_i)                    (Steps 3 and 6)
The correction divergences are those of the DG-recovering choice (Huynh's
left/right Radau functions on tensor elements; the DG lift on triangles):
div g_k is the polynomial of degree <= p with
  int_elem (div g_k) v = int_face(k) lambda_k v  ds   for all v in P_p,
i.e. LIFT = M^{-1} E with M the nodal mass matrix (= (V V^T)^{-1} for an
orthonormal Psi) and E[i,k] = int l_i lambda_k ds, evaluated exactly by the
face Gauss-Legendre rule at the flux points.  The tests check that on tensor
elements this equals the Radau closed form g_L'(xi) along each line.

Triangle solution points: the Williams-Shunn tables are not available.  The
triangle uses the Blyth-Pozrikidis map of the 1D Gauss-Legendre nodes
v_0 < ... < v_p on [0, 1]: lattice index (i, j, k), i + j + k = p, goes to the
barycentric point l_a = (1 + 2 v_a - v_b - v_c)/3.  The set is symmetric,
interior and unisolvent, its interpolatory weights int l_i are positive for
p <= 5, and the advection operator on it (with the penalty tau = 0.1) is close
to energy neutral (the tests bound the largest real part of its spectrum); the same
map of equispaced nodes (the principal lattice) gives negative weights and
advection modes that grow by e^29 over one Rider-Kothe period at p = 3.  At
p = 5 the Gauss-Legendre set leaves a mode growing at Re lambda = 0.05 (the
Rider-Kothe march fails), so p = 5 maps the Chebyshev nodes of the second
kind instead, x_k = cos(k pi / (p + 2)), k = 1..p+1 (the Gauss-Jacobi(1/2, 1/2)
roots), whose advection spectrum keeps Re lambda below 0.01.
"""
import math
from dataclasses import dataclass

import numpy as np

from .polys import gauss_legendre, jacobi, jacobi_deriv, jacobi_norm


@dataclass
class RefElement:
    etype: str
    p: int
    dim: int
    verts: np.ndarray        # (nv, dim) reference vertex coordinates
    faces: list              # per face: dict(verts, normal, scale, npts)
    xu: np.ndarray           # (Nu, dim) solution points
    xf: np.ndarray           # (Nf, dim) flux points
    face_of: np.ndarray      # (Nf,) face id of each flux point
    nref: np.ndarray         # (Nf, dim) unit outward reference normals
    wf: np.ndarray           # (Nf,) face quadrature weights (reference measure)
    V: np.ndarray            # (Nu, Nu) V[j, m] = Psi_m(x^u_j)
    Vinv: np.ndarray
    L: np.ndarray            # (Nf, Nu)
    D: np.ndarray            # (dim, Nu, Nu)
    LIFT: np.ndarray         # (Nu, Nf)
    wq: np.ndarray           # (Nu,) int l_i over the reference element
    high: np.ndarray         # (Nu,) bool: modes removed by the truncation u_hat
    degrees: list            # per mode: multi-index

    @property
    def nu(self):
        return self.xu.shape[0]

    @property
    def nf(self):
        return self.xf.shape[0]

    def shape(self, x):
        """Geometric shape functions N_a(x) (n, nv) and gradients (n, nv, dim)."""
        x = np.atleast_2d(x)
        if self.etype == "tri":
            r, s = x[:, 0], x[:, 1]
            N = np.stack([-(r + s) / 2, (1 + r) / 2, (1 + s) / 2], 1)
            G = np.zeros((x.shape[0], 3, 2))
            G[:, 0] = [-0.5, -0.5]
            G[:, 1] = [0.5, 0.0]
            G[:, 2] = [0.0, 0.5]
            return N, G
        nv = self.verts.shape[0]
        N = np.ones((x.shape[0], nv))
        G = np.ones((x.shape[0], nv, self.dim))
        for a in range(nv):
            fac = [(1.0 + x[:, c] * self.verts[a, c]) / 2.0 for c in range(self.dim)]
            for c in range(self.dim):
                N[:, a] *= fac[c]
                for c2 in range(self.dim):
                    G[:, a, c2] *= (self.verts[a, c] / 2.0) if c == c2 else fac[c]
        return N, G


def _ortho_legendre(k, x):
    return jacobi(k, 0.0, 0.0, x) / math.sqrt(jacobi_norm(k, 0.0, 0.0))


def _ortho_legendre_d(k, x):
    return jacobi_deriv(k, 0.0, 0.0, x) / math.sqrt(jacobi_norm(k, 0.0, 0.0))


def _modal_tensor(p, dim, x):
    """Orthonormal tensor Legendre basis on [-1,1]^dim: values (n, Nm), grads (n, Nm, dim)."""
    n1 = p + 1
    idx = list(np.ndindex(*([n1] * dim)))
    idx = [tuple(reversed(t)) for t in idx]       # first index fastest
    P = np.zeros((x.shape[0], len(idx)))
    G = np.zeros((x.shape[0], len(idx), dim))
    for m, mi in enumerate(idx):
        vals = [_ortho_legendre(mi[c], x[:, c]) for c in range(dim)]
        ders = [_ortho_legendre_d(mi[c], x[:, c]) for c in range(dim)]
        P[:, m] = np.prod(vals, axis=0)
        for c in range(dim):
            g = ders[c].copy()
            for c2 in range(dim):
                if c2 != c:
                    g = g * vals[c2]
            G[:, m, c] = g
    return P, G, idx


def _modal_tri(p, x):
    """Orthonormal Dubiner basis on the triangle (-1,-1),(1,-1),(-1,1).

    psi_ij = sqrt(2) Phat_i(a) Phat_j^{(2i+1,0)}(b) (1-b)^i with collapsed
    coordinates a = 2(1+r)/(1-s) - 1, b = s; gradients by the chain rule.
    """
    r, s = x[:, 0], x[:, 1]
    a = 2.0 * (1.0 + r) / (1.0 - s) - 1.0
    b = s
    idx = [(i, j) for i in range(p + 1) for j in range(p + 1 - i)]
    P = np.zeros((x.shape[0], len(idx)))
    G = np.zeros((x.shape[0], len(idx), 2))
    for m, (i, j) in enumerate(idx):
        ni = math.sqrt(jacobi_norm(i, 0.0, 0.0))
        nj = math.sqrt(jacobi_norm(j, 2.0 * i + 1.0, 0.0))
        A = jacobi(i, 0.0, 0.0, a) / ni
        dA = jacobi_deriv(i, 0.0, 0.0, a) / ni
        B = jacobi(j, 2.0 * i + 1.0, 0.0, b) / nj
        dB = jacobi_deriv(j, 2.0 * i + 1.0, 0.0, b) / nj
        om = 1.0 - b
        P[:, m] = math.sqrt(2.0) * A * B * om ** i
        # d/dr: da/dr = 2/(1-b)
        G[:, m, 0] = math.sqrt(2.0) * dA * B * 2.0 * om ** (i - 1) if i > 0 else 0.0
        # d/ds: da/ds = (1+a)/(1-b), db/ds = 1
        t1 = dA * (1.0 + a) * B * om ** (i - 1) if i > 0 else 0.0 * a
        t2 = A * dB * om ** i
        t3 = -i * A * B * om ** (i - 1) if i > 0 else 0.0 * a
        G[:, m, 1] = math.sqrt(2.0) * (t1 + t2 + t3)
    return P, G, idx


def _faces(etype):
    s2 = math.sqrt(2.0)
    if etype == "quad":
        return [
            dict(map=lambda s: np.stack([s[:, 0], -np.ones(len(s))], 1), normal=(0.0, -1.0), verts=(0, 1), scale=1.0),
            dict(map=lambda s: np.stack([np.ones(len(s)), s[:, 0]], 1), normal=(1.0, 0.0), verts=(1, 2), scale=1.0),
            dict(map=lambda s: np.stack([-s[:, 0], np.ones(len(s))], 1), normal=(0.0, 1.0), verts=(2, 3), scale=1.0),
            dict(map=lambda s: np.stack([-np.ones(len(s)), -s[:, 0]], 1), normal=(-1.0, 0.0), verts=(3, 0), scale=1.0),
        ]
    if etype == "tri":
        return [
            dict(map=lambda s: np.stack([s[:, 0], -np.ones(len(s))], 1), normal=(0.0, -1.0), verts=(0, 1), scale=1.0),
            dict(map=lambda s: np.stack([-s[:, 0], s[:, 0]], 1), normal=(1 / s2, 1 / s2), verts=(1, 2), scale=s2),
            dict(map=lambda s: np.stack([-np.ones(len(s)), -s[:, 0]], 1), normal=(-1.0, 0.0), verts=(2, 0), scale=1.0),
        ]
    one = lambda s: np.ones(len(s))
    return [
        dict(map=lambda s: np.stack([s[:, 0], s[:, 1], -one(s)], 1), normal=(0.0, 0.0, -1.0), verts=(0, 1, 2, 3), scale=1.0),
        dict(map=lambda s: np.stack([s[:, 0], -one(s), s[:, 1]], 1), normal=(0.0, -1.0, 0.0), verts=(0, 1, 5, 4), scale=1.0),
        dict(map=lambda s: np.stack([one(s), s[:, 0], s[:, 1]], 1), normal=(1.0, 0.0, 0.0), verts=(1, 2, 6, 5), scale=1.0),
        dict(map=lambda s: np.stack([s[:, 0], one(s), s[:, 1]], 1), normal=(0.0, 1.0, 0.0), verts=(2, 3, 7, 6), scale=1.0),
        dict(map=lambda s: np.stack([-one(s), s[:, 0], s[:, 1]], 1), normal=(-1.0, 0.0, 0.0), verts=(3, 0, 4, 7), scale=1.0),
        dict(map=lambda s: np.stack([s[:, 0], s[:, 1], one(s)], 1), normal=(0.0, 0.0, 1.0), verts=(4, 5, 6, 7), scale=1.0),
    ]


_CACHE = {}


def ref_element(etype, p):
    key = (etype, p)
    if key in _CACHE:
        return _CACHE[key]
    n = p + 1
    g, w = gauss_legendre(n)
    if etype == "quad":
        dim = 2
        verts = np.array([[-1, -1], [1, -1], [1, 1], [-1, 1]], dtype=np.float64)
    elif etype == "hex":
        dim = 3
        q = [[-1, -1], [1, -1], [1, 1], [-1, 1]]
        verts = np.array([[a, b, -1] for a, b in q] + [[a, b, 1] for a, b in q], dtype=np.float64)
    elif etype == "tri":
        dim = 2
        verts = np.array([[-1, -1], [1, -1], [-1, 1]], dtype=np.float64)
    else:
        raise ValueError(etype)

    # solution points
    if etype in ("quad", "hex"):
        grids = np.meshgrid(*([g] * dim), indexing="ij")
        xu = np.stack([m.ravel(order="F") for m in grids], 1)
        P, Gm, degrees = _modal_tensor(p, dim, xu)
        high = np.array([max(d) == p for d in degrees])
        modal = lambda x: _modal_tensor(p, dim, x)[:2]
    else:
        # Blyth-Pozrikidis map of the 1D nodes v on [0, 1] (Gauss-Legendre;
        # Chebyshev of the second kind at p = 5):
        # lattice index (i, j, k), i + j + k = p, goes to the barycentric point
        # l_a = (1 + 2 v_a - v_b - v_c) / 3 (equispaced v would give the lattice)
        if p == 5:   # Chebyshev nodes of the second kind, ascending
            v = (np.cos(np.arange(n, 0, -1) * math.pi / (n + 1)) + 1.0) / 2.0
        else:
            v = (g + 1.0) / 2.0
        pts = []
        for j in range(p + 1):
            for i in range(p + 1 - j):
                k = p - i - j
                l1 = (1.0 + 2.0 * v[i] - v[j] - v[k]) / 3.0
                l2 = (1.0 + 2.0 * v[j] - v[i] - v[k]) / 3.0
                l0 = 1.0 - l1 - l2
                pts.append([l1 - l0 - l2, l2 - l0 - l1])   # vertices (-1,-1), (1,-1), (-1,1)
        xu = np.array(pts)
        P, Gm, degrees = _modal_tri(p, xu)
        high = np.array([i + j == p for (i, j) in degrees])
        modal = lambda x: _modal_tri(p, x)[:2]

    V = P
    Vinv = np.linalg.inv(V)

    # flux points: n^(dim-1) Gauss-Legendre points per face
    faces = _faces(etype)
    xf, face_of, nref, wf = [], [], [], []
    if dim == 2:
        s = g[:, None]
        ws = w
    else:
        sa, sb = np.meshgrid(g, g, indexing="ij")
        s = np.stack([sa.ravel(order="F"), sb.ravel(order="F")], 1)
        wa, wb = np.meshgrid(w, w, indexing="ij")
        ws = (wa * wb).ravel(order="F")
    for fi, f in enumerate(faces):
        xf.append(f["map"](s))
        face_of += [fi] * s.shape[0]
        nref.append(np.tile(np.array(f["normal"]), (s.shape[0], 1)))
        wf.append(ws * f["scale"])
        f["npts"] = s.shape[0]
    xf = np.concatenate(xf, 0)
    face_of = np.array(face_of)
    nref = np.concatenate(nref, 0)
    wf = np.concatenate(wf, 0)

    Pf, _ = modal(xf)
    L = Pf @ Vinv                                  # l_i(x^f_k)
    D = np.stack([Gm[:, :, a] @ Vinv for a in range(dim)], 0)
    Minv = V @ V.T
    E = L.T * wf[None, :]                          # int l_i lambda_k ds
    LIFT = Minv @ E
    # int psi_0 = psi_0 * |ref| with psi_0 constant = 1/sqrt(|ref|)
    ref_meas = 2.0 ** dim if etype != "tri" else 2.0
    wq = Vinv[0, :] * math.sqrt(ref_meas)
    el = RefElement(etype, p, dim, verts, faces, xu, xf, face_of, nref, wf, V, Vinv,
                    L, D, LIFT, wq, high, degrees)
    _CACHE[key] = el
    return el
