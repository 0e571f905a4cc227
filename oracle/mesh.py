"""Mesh geometry and face pairing (oracle, test infrastructure only).

Section 3.1: the mapping x = M(x~) from the standard element, its Jacobian
J = dM_i/dx~_j and det J (Eqs. maintranseq, maintranseq2), flux points that
"share the same physical coordinates with the corresponding points of
neighbouring elements", and Section 3.3's boundary faces (copy ghost states).

Pairing is geometric: faces are matched by their centroid (modulo the period
on periodic axes) and flux points by nearest physical position.  For every
interior face the side with the lower element number is the "L" side that
the LDG parameter beta = +1/2 refers to; a face of an element that meets
itself through a periodic boundary is ordered by the larger centroid
coordinate sum.  Boundary flux points are their own partners and count as
"L" (the ghost state equals the interior state).
"""
from dataclasses import dataclass

import numpy as np

from .element import ref_element


@dataclass
class Geometry:
    el: object
    xu: np.ndarray        # (E, Nu, d) physical solution points
    xf: np.ndarray        # (E, Nf, d) physical flux points
    Ju: np.ndarray        # (E, Nu, d, d) J[..., i, a] = dx_i / dxi_a
    detJu: np.ndarray     # (E, Nu)
    Jinvu: np.ndarray     # (E, Nu, d, d) Jinv[..., a, i] = dxi_a / dx_i
    pn: np.ndarray        # (E, Nf, d) det J J^{-T} n~ at flux points
    pn_mag: np.ndarray    # (E, Nf)
    nhat: np.ndarray      # (E, Nf, d) physical unit outward normal
    pe: np.ndarray        # (E, Nf) partner element
    pk: np.ndarray        # (E, Nf) partner flux point
    isL: np.ndarray       # (E, Nf) bool
    boundary: np.ndarray  # (E, Nf) bool
    h: float
    volume: float


def _map(el, verts_phys, x):
    """x(xi) and J(xi) for every element at reference points x (n, d)."""
    N, G = el.shape(x)
    X = np.einsum("na,ead->end", N, verts_phys)
    J = np.einsum("nac,ead->endc", G, verts_phys)
    return X, J


def build_geometry(mesh, p):
    el = ref_element(mesh.etype, p)
    d = el.dim
    verts = mesh.nodes[mesh.conn]                      # (E, nv, d)
    E = verts.shape[0]
    xu, Ju = _map(el, verts, el.xu)
    xf, Jf = _map(el, verts, el.xf)
    detJu = np.linalg.det(Ju)
    if np.any(detJu <= 0):
        raise ValueError("element with non-positive det J")
    Jinvu = np.linalg.inv(Ju)
    detJf = np.linalg.det(Jf)
    Jinvf = np.linalg.inv(Jf)
    # Nanson: n ds = det J J^{-T} n~ ds~
    pn = detJf[..., None] * np.einsum("ekai,ka->eki", Jinvf, el.nref)
    pn_mag = np.linalg.norm(pn, axis=-1)
    nhat = pn / pn_mag[..., None]

    volume = float(np.einsum("i,ei->", el.wq, detJu))
    if mesh.etype == "tri":
        h = float(np.sqrt(2.0 * volume / E))
    else:
        h = float((volume / E) ** (1.0 / d))

    # ---- face matching by centroid --------------------------------------
    per = np.array([mesh.period[a] if mesh.periodic[a] else 0.0 for a in range(d)])
    quantum = 1e-7 * h
    table = {}
    nfaces = len(el.faces)
    for f in range(nfaces):
        fv = list(el.faces[f]["verts"])
        cen = verts[:, fv, :].mean(axis=1)          # (E, d)
        keys = np.round(cen / quantum).astype(np.int64)
        for a in range(d):
            if per[a] > 0:
                # on a periodic axis the quantum is rounded to divide the
                # period, so a centroid and its periodic image share a key
                K = int(round(per[a] / quantum))
                keys[:, a] = np.mod(np.round(cen[:, a] * (K / per[a])).astype(np.int64), K)
        for e in range(E):
            table.setdefault(tuple(keys[e]), []).append((e, f))
    pe = np.tile(np.arange(E)[:, None], (1, el.nf))
    pk = np.tile(np.arange(el.nf)[None, :], (E, 1))
    isL = np.ones((E, el.nf), dtype=bool)
    boundary = np.ones((E, el.nf), dtype=bool)
    fpts_of_face = [np.nonzero(el.face_of == f)[0] for f in range(nfaces)]
    for key, lst in table.items():
        if len(lst) == 1:
            continue
        if len(lst) != 2:
            raise ValueError("face shared by more than two elements")
        (e1, f1), (e2, f2) = lst
        k1, k2 = fpts_of_face[f1], fpts_of_face[f2]
        dx = xf[e1, k1][:, None, :] - xf[e2, k2][None, :, :]
        for a in range(d):
            if per[a] > 0:
                dx[..., a] -= per[a] * np.round(dx[..., a] / per[a])
        dist = np.linalg.norm(dx, axis=-1)
        match = dist.argmin(axis=1)
        if dist[np.arange(len(k1)), match].max() > 1e-8 * h or len(set(match)) != len(k1):
            raise ValueError("flux points of a shared face do not coincide")
        if e1 != e2:
            first_is_L = e1 < e2
        else:
            c1 = verts[e1, list(el.faces[f1]["verts"])].mean(0).sum()
            c2 = verts[e2, list(el.faces[f2]["verts"])].mean(0).sum()
            first_is_L = c1 > c2
        pe[e1, k1] = e2
        pk[e1, k1] = k2[match]
        pe[e2, k2[match]] = e1
        pk[e2, k2[match]] = k1
        isL[e1, k1] = first_is_L
        isL[e2, k2[match]] = not first_is_L
        boundary[e1, k1] = False
        boundary[e2, k2] = False
    return Geometry(el, xu, xf, Ju, detJu, Jinvu, pn, pn_mag, nhat, pe, pk, isL, boundary,
                    h, volume)
