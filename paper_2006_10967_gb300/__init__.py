"""GB300-native FR-PCPF: the flux-reconstruction update of the preconditioned,
localised conservative phase field (arXiv 2006.10967) as hand-written sm_103a
CUDA kernels behind a C ABI (include/fr_pcpf.h, libfrpcpf.so).

This module is the thin Python binding: it marshals arguments, lets PyTorch
provide device memory (one workspace per field) and streams, and calls the
library.  Every step of the update runs in the library's kernels; if the
library is missing, importing Field/Mesh raises instead of falling back.
"""
import ctypes as C

import numpy as np

from . import _capi as capi
from ._capi import (FR_FP64, FR_MIXED, FR_QUAD, FR_TRI, FR_HEX, FR_IC_ARRAY, FR_IC_CIRCLE, FR_EINVAL,
                    FR_EBOUNDS, FRError, check, lib)

__all__ = ["Mesh", "Field", "make_params", "FRError", "FR_FP64", "FR_MIXED", "lib",
           "fr_mesh_create", "fr_field_init", "fr_step", "fr_adjoint_step", "fr_mass_integral"]

ETYPES = {"quad": FR_QUAD, "tri": FR_TRI, "hex": FR_HEX}
VELS = {"uniform": 0, "rider_kothe": 1, "leveque": 2, "stream": 3, "rotation": 4}
_dp = C.POINTER(C.c_double)


def _ptr(a):
    return a.ctypes.data_as(_dp)


class Mesh:
    """Host mesh (fr_mesh_create): operators, geometry, face pairing."""

    def __init__(self, nodes, conn, etype, order, periodic=(False, False, False), period=(1.0, 1.0, 1.0)):
        self._nodes = np.ascontiguousarray(nodes, dtype=np.float64)
        self._conn = np.ascontiguousarray(conn, dtype=np.int64)
        dim = self._nodes.shape[1]
        d = capi.fr_mesh_desc()
        d.dim = dim
        d.etype = ETYPES[etype] if isinstance(etype, str) else int(etype)
        d.order = int(order)
        d.n_nodes = self._nodes.shape[0]
        d.nodes = _ptr(self._nodes)
        d.n_elems = self._conn.shape[0]
        d.conn = self._conn.ctypes.data_as(C.POINTER(C.c_int64))
        for a in range(3):
            d.periodic[a] = int(bool(periodic[a])) if a < len(periodic) else 0
            d.period[a] = float(period[a]) if a < len(period) else 1.0
        h = C.c_void_p()
        check(lib().fr_mesh_create(C.byref(d), C.byref(h)), "fr_mesh_create")
        self.handle = h
        self.info = capi.fr_mesh_info()
        check(lib().fr_mesh_info_get(h, C.byref(self.info)), "fr_mesh_info_get")

    @classmethod
    def concat(cls, meshes):
        """Union mesh of a batch of instances (fr_mesh_concat)."""
        arr = (C.c_void_p * len(meshes))(*[m.handle for m in meshes])
        h = C.c_void_p()
        check(lib().fr_mesh_concat(arr, len(meshes), C.byref(h)), "fr_mesh_concat")
        obj = cls.__new__(cls)
        obj.handle = h
        obj.info = capi.fr_mesh_info()
        check(lib().fr_mesh_info_get(h, C.byref(obj.info)), "fr_mesh_info_get")
        obj.parts = [m.info.n_elems for m in meshes]
        return obj

    @classmethod
    def from_synthetic(cls, m, order):
        return cls(m.nodes, m.conn, m.etype, order, tuple(m.periodic) + (False,) * (3 - len(m.periodic)),
                   tuple(m.period) + (1.0,) * (3 - len(m.period)))

    @property
    def shape(self):
        return (self.info.n_elems, self.info.nu)

    def solution_points(self):
        out = np.empty((self.info.n_elems, self.info.nu, self.info.dim))
        check(lib().fr_mesh_solution_points(self.handle, _ptr(out)), "fr_mesh_solution_points")
        return out

    def quadrature(self):
        out = np.empty((self.info.n_elems, self.info.nu))
        check(lib().fr_mesh_quadrature(self.handle, _ptr(out)), "fr_mesh_quadrature")
        return out

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            lib().fr_mesh_destroy(h)
            self.handle = None


def make_params(w, precision="fp64", **kw):
    """fr_params from a workload-like object (attributes of synthetic.Workload)."""
    p = capi.fr_params()
    g = lambda k: kw.get(k, getattr(w, k))
    p.gamma = g("gamma")
    p.eps = g("eps")
    p.tau = g("tau")
    p.tau_psi = g("tau_psi")
    p.tau_pseudo = g("tau_pseudo")
    p.dt = g("dt")
    p.n_precond = int(g("n_precond"))
    p.pseudo_kmax = int(g("pseudo_kmax"))
    p.pseudo_dtau = g("pseudo_dtau")
    p.pseudo_tol = g("pseudo_tol")
    p.pseudo_fixed = int(bool(kw.get("pseudo_fixed", False)))
    p.precision = FR_MIXED if precision in ("mixed", FR_MIXED) else FR_FP64
    p.s0 = g("s0")
    p.kappa = g("kappa")
    p.nu_max = g("nu_max")
    p.delta = g("delta")
    p.vel_cache = int(bool(kw.get("vel_cache", True)))
    # interface normal: "psi" (preconditioned method) or "phi" (unpreconditioned CPF)
    normal = kw.get("normal", getattr(w, "normal", "psi"))
    if normal not in ("psi", "phi"):
        raise ValueError(f"normal must be 'psi' or 'phi', not {normal!r}")
    p.normal = 1 if normal == "phi" else 0
    # wall faces: "copy" (Section 3.3 copy ghost) or "noflux" (zero common normal flux)
    wall = kw.get("wall", getattr(w, "wall", "copy"))
    if wall not in ("copy", "noflux"):
        raise ValueError(f"wall must be 'copy' or 'noflux', not {wall!r}")
    p.wall = 1 if wall == "noflux" else 0
    # kernel variant: an explicit index, or "auto": the autotuner's table entry
    # for the field's mesh (resolved by Field), else 0
    variant = kw.get("variant", "auto")
    p._variant = variant
    p.variant = 0 if variant == "auto" else int(variant)
    vel = kw.get("velocity", w.velocity)
    p.vel.kind = VELS[vel.kind]
    p.vel.T = float(vel.T)
    for a in range(3):
        p.vel.a[a] = float(vel.a[a]) if a < len(vel.a) else 0.0
    keep = []
    if vel.kind == "stream":
        arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (vel.kx, vel.ky, vel.A, vel.B)]
        keep = arrs
        p.vel.n_modes = len(arrs[0])
        p.vel.kx, p.vel.ky, p.vel.A, p.vel.B = [_ptr(x) for x in arrs]
    p._keep = keep
    return p


def kernel_variants(mesh, precision):
    """Number of kernel variants built for the mesh's element type and order."""
    n = C.c_int32()
    check(lib().fr_kernel_variants(mesh.handle, FR_MIXED if precision in ("mixed", FR_MIXED) else FR_FP64,
                                   C.byref(n)), "fr_kernel_variants")
    return n.value


def _resolve_variant(mesh, params):
    if getattr(params, "_variant", None) == "auto":
        from . import tune
        params.variant = tune.lookup(mesh.info.etype, mesh.info.order, params.precision)


class Field:
    """Device state of one FR-PCPF problem (fr_field_init); PyTorch owns the workspace."""

    def __init__(self, mesh, params, ic=None, phi0=None, precondition=True, stream=None):
        import torch
        self.mesh = mesh
        self.params = params
        _resolve_variant(mesh, params)
        self.torch = torch
        nbytes = C.c_size_t()
        check(lib().fr_field_workspace_bytes(mesh.handle, C.byref(params), C.byref(nbytes)),
              "fr_field_workspace_bytes")
        self.workspace_bytes = nbytes.value
        self._ws = torch.empty(nbytes.value + 256, dtype=torch.uint8, device="cuda")
        base = self._ws.data_ptr()
        self._base = (base + 255) // 256 * 256
        icd = capi.fr_ic()
        icd.precondition = int(bool(precondition))
        self._phi0 = None
        if phi0 is not None:
            self._phi0 = np.ascontiguousarray(phi0, dtype=np.float64).reshape(-1)
            icd.kind = FR_IC_ARRAY
            icd.phi0 = _ptr(self._phi0)
        else:
            icd.kind = FR_IC_CIRCLE
            for a in range(3):
                icd.centre[a] = float(ic.centre[a]) if a < len(ic.centre) else 0.0
            icd.radius = float(ic.radius)
            icd.beta = float(ic.beta)
        h = C.c_void_p()
        check(lib().fr_field_init(mesh.handle, C.byref(params), C.byref(icd), C.c_void_p(self._base),
                                  nbytes.value, self._stream(stream), C.byref(h)), "fr_field_init")
        self.handle = h

    @classmethod
    def batch(cls, mesh, params, instances, precondition=True, stream=None):
        """A field over a batch of instances on a union mesh (fr_field_init_batch).

        instances: list of dicts with elem_begin, elem_end, dt, eps, nu_max,
        pseudo_dtau, velocity (synthetic.Velocity-like) and circle."""
        import torch
        obj = cls.__new__(cls)
        obj.mesh = mesh
        obj.params = params
        _resolve_variant(mesh, params)
        obj.torch = torch
        nbytes = C.c_size_t()
        check(lib().fr_field_workspace_bytes(mesh.handle, C.byref(params), C.byref(nbytes)),
              "fr_field_workspace_bytes")
        obj.workspace_bytes = nbytes.value
        obj._ws = torch.empty(nbytes.value + 256, dtype=torch.uint8, device="cuda")
        obj._base = (obj._ws.data_ptr() + 255) // 256 * 256
        arr = (capi.fr_instance * len(instances))()
        obj._keep = []
        for k, d in enumerate(instances):
            I = arr[k]
            I.elem_begin, I.elem_end = int(d["elem_begin"]), int(d["elem_end"])
            I.dt, I.eps, I.nu_max, I.pseudo_dtau = d["dt"], d["eps"], d["nu_max"], d["pseudo_dtau"]
            v = d["velocity"]
            I.vel.kind = VELS[v.kind]
            I.vel.T = float(v.T)
            for a in range(3):
                I.vel.a[a] = float(v.a[a]) if a < len(v.a) else 0.0
            if v.kind == "stream":
                arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (v.kx, v.ky, v.A, v.B)]
                obj._keep += arrs
                I.vel.n_modes = len(arrs[0])
                I.vel.kx, I.vel.ky, I.vel.A, I.vel.B = [_ptr(x) for x in arrs]
            c = d["circle"]
            I.ic.kind = FR_IC_CIRCLE
            for a in range(3):
                I.ic.centre[a] = float(c.centre[a]) if a < len(c.centre) else 0.0
            I.ic.radius, I.ic.beta = float(c.radius), float(c.beta)
        h = C.c_void_p()
        check(lib().fr_field_init_batch(mesh.handle, C.byref(params), len(instances), arr, int(bool(precondition)),
                                        C.c_void_p(obj._base), nbytes.value, obj._stream(stream), C.byref(h)),
              "fr_field_init_batch")
        obj.handle = h
        return obj

    def _stream(self, stream=None):
        s = stream if stream is not None else self.torch.cuda.current_stream()
        return C.c_void_p(s.cuda_stream)

    def step(self, n=1, stream=None):
        check(lib().fr_step(self.handle, int(n), self._stream(stream)), "fr_step")

    def precondition(self, stream=None):
        check(lib().fr_precondition(self.handle, self._stream(stream)), "fr_precondition")

    def sync(self, stream=None):
        return lib().fr_sync(self.handle, self._stream(stream))

    def stats(self, stream=None):
        s = capi.fr_stats()
        check(lib().fr_stats_get(self.handle, self._stream(stream), C.byref(s)), "fr_stats_get")
        return dict(n_steps=s.n_steps, t=s.t, last_pseudo_iters=s.last_pseudo_iters, status=s.status,
                    last_pseudo_rms=s.last_pseudo_rms, n_preconditions=s.n_preconditions)

    def mass(self, which=0, stream=None):
        out = C.c_double()
        check(lib().fr_mass_integral(self.handle, int(which), C.byref(out), self._stream(stream)),
              "fr_mass_integral")
        return out.value

    def get(self, which=0, stream=None):
        out = np.empty(self.mesh.shape)
        check(lib().fr_field_get(self.handle, int(which), _ptr(out), self._stream(stream)), "fr_field_get")
        return out

    def set(self, which, values, stream=None):
        arr = np.ascontiguousarray(values, dtype=np.float64).reshape(self.mesh.shape)
        check(lib().fr_field_set(self.handle, int(which), _ptr(arr), self._stream(stream)), "fr_field_set")

    def get_device(self, which, out, stream=None):
        check(lib().fr_field_get_device(self.handle, int(which), C.c_void_p(out.data_ptr()),
                                        self._stream(stream)), "fr_field_get_device")
        return out

    def set_device(self, which, values, stream=None):
        check(lib().fr_field_set_device(self.handle, int(which), C.c_void_p(values.data_ptr()),
                                        self._stream(stream)), "fr_field_set_device")

    def rhs(self, t, stream=None):
        out = self.torch.empty((2,) + self.mesh.shape, dtype=self.torch.float64, device="cuda")
        check(lib().fr_rhs(self.handle, float(t), C.c_void_p(out.data_ptr()), self._stream(stream)), "fr_rhs")
        return out

    def rhs_pseudo(self, stream=None):
        out = self.torch.empty(self.mesh.shape, dtype=self.torch.float64, device="cuda")
        check(lib().fr_rhs_pseudo(self.handle, C.c_void_p(out.data_ptr()), self._stream(stream)),
              "fr_rhs_pseudo")
        return out

    # ---- element-partitioned stepping (fr_stage, fr_halo_*, fr_traces) -----
    device = "cuda"  # where halo rows live (partition.halo_exchange allocates its buffers there)

    def stage(self, s, stream=None):
        """Stage s (1..4) of the physical RK4 step."""
        check(lib().fr_stage(self.handle, int(s), self._stream(stream)), "fr_stage")

    def halo_dtype(self):
        nb = C.c_size_t()
        check(lib().fr_halo_row_bytes(self.handle, C.byref(nb)), "fr_halo_row_bytes")
        return self.torch.float64 if nb.value == 2 * self.mesh.info.nu * 8 else self.torch.float32

    def halo_pack(self, elems, stream=None):
        """Stage values of the listed local elements (int64 device tensor) as
        an (n, 2, nu) device tensor of the bulk precision."""
        out = self.torch.empty((len(elems), 2, self.mesh.info.nu), dtype=self.halo_dtype(), device="cuda")
        check(lib().fr_halo_pack(self.handle, C.c_void_p(elems.data_ptr()), len(elems), C.c_void_p(out.data_ptr()),
                                 self._stream(stream)), "fr_halo_pack")
        return out

    def halo_unpack(self, elems, rows, stream=None):
        """Write rows (n, 2, nu; from halo_pack of the owners) into the listed
        local elements' stage values."""
        rows = rows.contiguous()
        assert rows.dtype == self.halo_dtype() and rows.shape == (len(elems), 2, self.mesh.info.nu)
        check(lib().fr_halo_unpack(self.handle, C.c_void_p(elems.data_ptr()), len(elems),
                                   C.c_void_p(rows.data_ptr()), self._stream(stream)), "fr_halo_unpack")

    def traces(self, stream=None):
        check(lib().fr_traces(self.handle, self._stream(stream)), "fr_traces")

    def pseudo_begin(self, stream=None):
        """psi_0 = psi = phi - 1/2 and psi's traces: the start of a
        preconditioning run one pseudo stage at a time (fr_pseudo_begin)."""
        check(lib().fr_pseudo_begin(self.handle, self._stream(stream)), "fr_pseudo_begin")

    def pseudo_stage(self, s, stream=None):
        """Stage s (1..4) of one pseudo-time RK4 iteration (fr_pseudo_stage)."""
        check(lib().fr_pseudo_stage(self.handle, int(s), self._stream(stream)), "fr_pseudo_stage")

    # ---- discrete adjoint -------------------------------------------------
    def adjoint_record(self, n_steps, ckpt_every, precondition=False, stream=None):
        """Advance n_steps keeping checkpoints for adjoint_step (fr_adjoint_record);
        with precondition, the window starts with the preconditioning of the
        current phi (psi is reset to phi - 1/2 first; FR_ADJ_PRECONDITION)."""
        flags = capi.FR_ADJ_PRECONDITION if precondition else 0
        nbytes = C.c_size_t()
        check(lib().fr_adjoint_workspace_bytes(self.handle, int(n_steps), int(ckpt_every), flags,
                                               C.byref(nbytes)), "fr_adjoint_workspace_bytes")
        self._adj_ws = self.torch.empty(nbytes.value + 256, dtype=self.torch.uint8, device="cuda")
        base = (self._adj_ws.data_ptr() + 255) // 256 * 256
        check(lib().fr_adjoint_record(self.handle, int(n_steps), int(ckpt_every), flags, C.c_void_p(base),
                                      nbytes.value, self._stream(stream)), "fr_adjoint_record")

    def adjoint_step(self, dJ_dphiT, dJ_dpsiT=None, n_coef=0, stream=None):
        """(dJ/du0 as a (2, E, Nu) tensor, dJ/dcoef (2M,) or None) via fr_adjoint_step."""
        t = self.torch
        gphi = dJ_dphiT.to(device="cuda", dtype=t.float64).contiguous()
        gpsi = None if dJ_dpsiT is None else dJ_dpsiT.to(device="cuda", dtype=t.float64).contiguous()
        out = t.empty((2,) + self.mesh.shape, dtype=t.float64, device="cuda")
        coef = t.zeros(n_coef, dtype=t.float64, device="cuda") if n_coef else None
        check(lib().fr_adjoint_step(self.handle, C.c_void_p(gphi.data_ptr()),
                                    C.c_void_p(gpsi.data_ptr()) if gpsi is not None else None,
                                    C.c_void_p(out.data_ptr()),
                                    C.c_void_p(coef.data_ptr()) if coef is not None else None,
                                    self._stream(stream)), "fr_adjoint_step")
        return out, coef

    def profile(self, enable=True):
        check(lib().fr_profile(self.handle, int(bool(enable))), "fr_profile")

    def profile_read(self, stream=None):
        ms = (C.c_double * 4)()
        n = (C.c_int64 * 4)()
        check(lib().fr_profile_read(self.handle, self._stream(stream), ms, n), "fr_profile_read")
        names = ("kb_phys", "ka_phys", "kb_pseudo", "ka_pseudo")
        return {k: (ms[i], n[i]) for i, k in enumerate(names)}

    def profile_kernel(self, kernel=0, n=400, stream=None):
        """Mean milliseconds per launch of kernel class `kernel` (0: physical
        residual + common flux), n launches replayed as one CUDA graph."""
        ms = C.c_double()
        check(lib().fr_profile_kernel(self.handle, int(kernel), int(n), self._stream(stream), C.byref(ms)),
              "fr_profile_kernel")
        return ms.value

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            if capi.CHECKED and lib().fr_sync(h, None) == capi.FR_EBOUNDS:
                capi.BOUNDS_FIRED.append(h.value)   # a fired index check is never lost
            lib().fr_field_destroy(h)
            self.handle = None


# C-ABI names of the hot path, for callers who want the raw entry points
def fr_mesh_create(*a):
    return lib().fr_mesh_create(*a)


def fr_field_init(*a):
    return lib().fr_field_init(*a)


def fr_step(*a):
    return lib().fr_step(*a)


def fr_mass_integral(*a):
    return lib().fr_mass_integral(*a)


def fr_adjoint_step(*a):
    return lib().fr_adjoint_step(*a)


class _PlaceholderIC:
    """Circle initial condition used only to set up a field whose state is
    then overwritten from device memory."""
    centre = (0.0, 0.0, 0.0)
    radius = 0.0
    beta = 1.0


_PLACEHOLDER_IC = _PlaceholderIC()


def flow_function(mesh, params_fn, n_steps, ckpt_every, precondition=False):
    """A torch.autograd.Function for phi_T = Flow(phi0, coef): the FR march of
    n_steps from phi0 (psi0 = phi0 - 1/2; with precondition, psi is then the
    fixed-count preconditioning of phi0 - 1/2 and the gradient follows it too)
    with a stream velocity whose coefficients are coef = (A_1..A_M, B_1..B_M).
    params_fn(coef) -> fr_params.  Backward is the hand-written adjoint
    (fr_adjoint_record / fr_adjoint_step).  phi0 (a CUDA float64 tensor of
    the mesh's shape) and phi_T stay on the device: the field is set up with a
    placeholder state and then loaded from phi0 by device copies."""
    import torch

    class _Flow(torch.autograd.Function):
        @staticmethod
        def forward(ctx, phi0, coef):
            P = params_fn(coef.detach().cpu().numpy())
            u0 = phi0.detach().to(device="cuda", dtype=torch.float64).reshape(mesh.shape).contiguous()
            F = Field(mesh, P, ic=_PLACEHOLDER_IC, precondition=False)
            F.set_device(0, u0)
            F.set_device(1, u0 - 0.5)
            F.set_device(2, u0 - 0.5)
            F.adjoint_record(n_steps, ckpt_every, precondition=precondition)
            ctx.field = F
            ctx.n_coef = coef.numel()
            out = torch.empty_like(u0)
            F.get_device(0, out)
            return out.to(phi0.device)

        @staticmethod
        def backward(ctx, g):
            du0, dc = ctx.field.adjoint_step(g, None, ctx.n_coef)
            gphi = (du0[0] + du0[1]).to(g.device)      # psi0 = phi0 - 1/2
            return gphi, dc.to(g.device)

    return _Flow.apply


class Group:
    """Fields stepped together, one launch per kernel per RK stage
    (fr_group_create / fr_group_step): the quad mixed-precision batch fields
    of distinct orders 2..5 of an ensemble."""

    def __init__(self, fields):
        import torch
        self.torch = torch
        self.fields = list(fields)
        arr = (C.c_void_p * len(self.fields))(*[f.handle for f in self.fields])
        h = C.c_void_p()
        check(lib().fr_group_create(arr, len(self.fields), C.byref(h)), "fr_group_create")
        self.handle = h

    def step(self, n=1, stream=None):
        s = stream if stream is not None else self.torch.cuda.current_stream()
        check(lib().fr_group_step(self.handle, int(n), C.c_void_p(s.cuda_stream)), "fr_group_step")

    def __del__(self):
        if getattr(self, "handle", None) is not None:
            try:
                lib().fr_group_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


def batch_from_workloads(workloads, precision="mixed", precondition=True, **kw):
    """Group workload records (synthetic.Workload, all quad or hex) by order and
    build one batch field per order.  Returns [(order, Field, [element ranges])]."""
    groups = {}
    for w in workloads:
        groups.setdefault(w.order, []).append(w)
    out = []
    for p in sorted(groups):
        ws = groups[p]
        meshes = [Mesh.from_synthetic(w.mesh(), p) for w in ws]
        U = Mesh.concat(meshes)
        inst, e = [], 0
        for w, m in zip(ws, meshes):
            n = m.info.n_elems
            inst.append(dict(elem_begin=e, elem_end=e + n, dt=w.dt, eps=w.eps, nu_max=w.nu_max,
                             pseudo_dtau=w.pseudo_dtau, velocity=w.velocity, circle=w.circle))
            e += n
        P = make_params(ws[0], precision, **kw)
        out.append((p, Field.batch(U, P, inst, precondition=precondition), [(d["elem_begin"], d["elem_end"]) for d in inst]))
    return out
