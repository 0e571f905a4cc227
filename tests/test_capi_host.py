"""Host-side checks of the C-ABI library: it builds, loads, exports every
declared entry point, and its mesh builder (points, quadrature, face pairing)
agrees with the oracle's independent construction.  No GPU needed."""
import ctypes as C

import numpy as np
import pytest

import synthetic as S
from libutil import ensure_built, header_functions


@pytest.fixture(scope="module")
def G():
    ensure_built()
    import paper_2006_10967_gb300 as G
    return G


def test_exports_every_declared_symbol(G):
    L = G.lib()
    names = header_functions()
    assert "fr_step" in names and "fr_mesh_create" in names and "fr_mass_integral" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


MESHES = [
    ("quad", lambda: S.quad_grid(5, jitter=0.12, seed=2, shuffle_seed=3, rotate_seed=4), 3),
    ("quad", lambda: S.quad_grid(6, periodic=(False, False), jitter=0.1, seed=1, shuffle_seed=11, rotate_seed=12), 4),
    ("tri", lambda: S.tri_delaunay(7, seed=2, shuffle_seed=13), 3),
    ("tri", lambda: S.tri_split(4, shuffle_seed=1), 2),
    ("hex", lambda: S.hex_grid(3, periodic=(True, False, True), jitter=0.1, seed=4, shuffle_seed=5), 2),
    ("quad", lambda: S.quad_grid(1), 2),
    # the highest order of each element type
    ("tri", lambda: S.tri_delaunay(5, seed=3, shuffle_seed=2), 5),
    ("quad", lambda: S.quad_grid(3, jitter=0.1, seed=6), 6),
    ("hex", lambda: S.hex_grid(2, jitter=0.1, seed=7), 5),
    # every hex carries one of the 24 rotations of its vertex list
    ("hex", lambda: S.hex_grid(3, periodic=(True, True, False), jitter=0.1, seed=4, rotate_seed=9), 3),
]


@pytest.mark.parametrize("et,mk,p", MESHES)
def test_mesh_geometry_matches_oracle(G, et, mk, p):
    from oracle.mesh import build_geometry
    m = mk()
    M = G.Mesh.from_synthetic(m, p)
    geo = build_geometry(m, p)
    assert M.info.n_elems == m.n_elems
    assert M.info.nu == geo.el.nu and M.info.nf == geo.el.nf
    assert np.allclose(M.solution_points(), geo.xu, atol=1e-13)
    assert np.allclose(M.quadrature(), geo.el.wq[None, :] * geo.detJu, atol=1e-14)
    assert M.info.h == pytest.approx(geo.h, rel=1e-12)
    assert M.info.n_boundary_fpts == int(geo.boundary.sum())


def test_invalid_meshes_are_rejected(G):
    m = S.quad_grid(3)
    with pytest.raises(G.FRError) as e:
        G.Mesh(m.nodes, np.where(m.conn == 5, 999, m.conn), "quad", 2)
    assert e.value.code == -1
    flipped = m.conn[:, ::-1].copy()            # clockwise elements: det J < 0
    with pytest.raises(G.FRError):
        G.Mesh(m.nodes, flipped, "quad", 2)
    with pytest.raises(G.FRError) as e:
        G.Mesh(m.nodes, m.conn, "quad", 9)      # order not built
    assert e.value.code == -6
    t = S.tri_split(2)
    with pytest.raises(G.FRError) as e:
        G.Mesh(t.nodes, t.conn, "tri", 6)
    assert e.value.code == -6
    h = S.hex_grid(2)
    with pytest.raises(G.FRError) as e:
        G.Mesh(h.nodes, h.conn, "hex", 6)
    assert e.value.code == -6
    bad = m.nodes.copy()
    bad[3, 0] = np.nan
    with pytest.raises(G.FRError):
        G.Mesh(bad, m.conn, "quad", 2)
    # three elements on one face
    conn = np.concatenate([m.conn, m.conn[:1]], 0)
    with pytest.raises(G.FRError):
        G.Mesh(m.nodes, conn, "quad", 2)


def test_workspace_size_and_param_validation(G):
    w = S.workload("c1")
    M = G.Mesh.from_synthetic(w.mesh(), w.order)
    p = G.make_params(w)
    n = C.c_size_t()
    assert G.lib().fr_field_workspace_bytes(M.handle, C.byref(p), C.byref(n)) == 0
    assert n.value > 16 * 16 * 16 * 2 * 8 * 4
    pm = G.make_params(w, precision="mixed")
    n2 = C.c_size_t()
    assert G.lib().fr_field_workspace_bytes(M.handle, C.byref(pm), C.byref(n2)) == 0
    assert n2.value < n.value
    p.dt = -1.0
    assert G.lib().fr_field_workspace_bytes(M.handle, C.byref(p), C.byref(n)) == -1
    assert G.lib().fr_strerror(-4) == b"non-finite value in the state"


def test_partner_index_width_is_guarded(G):
    """The packed partner index of a flux point (2 (e Nf + k) + L bit) is an
    int32: a mesh with E Nf >= 2^30 is refused before its arrays are read."""
    from paper_2006_10967_gb300 import _capi as capi
    d = capi.fr_mesh_desc()
    d.dim, d.etype, d.order = 3, 2, 5            # hex, p = 5: Nf = 216
    nodes = np.zeros(24)
    conn = np.zeros(8, dtype=np.int64)
    d.n_nodes = 8
    d.nodes = nodes.ctypes.data_as(C.POINTER(C.c_double))
    d.n_elems = (1 << 30) // 216 + 1               # the arrays are far shorter than this
    d.conn = conn.ctypes.data_as(C.POINTER(C.c_int64))
    h = C.c_void_p()
    assert G.lib().fr_mesh_create(C.byref(d), C.byref(h)) == -6
    assert not h.value
    d.n_elems = 1                                   # a one-element mesh with the same descriptor builds
    nodes[:] = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
                         [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]], dtype=float).ravel()
    conn[:] = np.arange(8)
    assert G.lib().fr_mesh_create(C.byref(d), C.byref(h)) == 0
    G.lib().fr_mesh_destroy(h)


def test_probe_rejects_bad_arguments_before_any_launch(G):
    """fr_probe_hex_apply validates its arguments on the host: unsupported
    order, unknown form, negative count, null or misaligned input, short
    output (none of these reaches the device)."""
    f = G.lib().fr_probe_hex_apply
    ok = C.c_void_p(256)                             # aligned, never dereferenced: every call below fails first
    assert f(2, 0, 0, ok, 1, ok, 576, None) == -6    # order 2: FR_EUNSUPPORTED
    assert f(3, 2, 0, ok, 1, ok, 576, None) == -1    # form 2
    assert f(3, 0, 0, ok, -1, ok, 576, None) == -1   # negative count
    assert f(3, 0, 0, None, 1, ok, 576, None) == -1  # null input
    assert f(3, 1, 0, C.c_void_p(260), 1, ok, 576, None) == -1  # input not on a 16-byte boundary
    assert f(3, 0, 0, ok, 1, ok, 575, None) == -1    # 1 x 2 x 288 values needed
    assert f(3, 1, 1, ok, 2, ok, 3, None) == -1      # reduce: 2 x 2 values needed
    assert f(3, 0, 0, None, 0, None, 0, None) == 0   # nothing to do


def test_partitioned_run_calls_reject_a_null_field(G):
    """The element-partitioned calls (fr_stage, fr_halo_*, fr_traces,
    fr_pseudo_begin, fr_pseudo_stage) return FR_EINVAL for a null field
    before touching the device."""
    L = G.lib()
    nb = C.c_size_t()
    assert L.fr_stage(None, 1, None) == -1
    assert L.fr_halo_row_bytes(None, C.byref(nb)) == -1
    assert L.fr_halo_pack(None, None, 0, None, None) == -1
    assert L.fr_halo_unpack(None, None, 0, None, None) == -1
    assert L.fr_traces(None, None) == -1
    assert L.fr_pseudo_begin(None, None) == -1
    assert L.fr_pseudo_stage(None, 1, None) == -1


def test_bounds_checked_build_exports_every_declared_symbol():
    """The bounds-checked build (FR_BOUNDS_CHECK) of the same sources links
    and exports the same entry points; its error code has a message."""
    from paper_2006_10967_gb300 import build
    path = build.build(checked=True)
    L = C.CDLL(path)
    missing = [n for n in header_functions() if not hasattr(L, n)]
    assert not missing, missing
    L.fr_strerror.restype = C.c_char_p
    assert b"bounds" in L.fr_strerror(-7)
