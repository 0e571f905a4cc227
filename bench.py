#!/usr/bin/env python
"""Benchmark of the FR-PCPF hot path: FR DOF-stage updates per second.

Default workload: the 3D deformation test of Section 4.3 on the unit cube,
64^3 hexahedra, p = 3 (16.8 M solution points), LeVeque field with T = 3,
sphere r = 0.15 at (0.35, 0.35, 0.35), the paper's parameters (gamma = 0.09,
eps = 0.06 h/p, precondition every 1000 steps with up to 20 pseudo
iterations, s0 = -5), mixed precision (FP32 bulk, float-float solution,
FP64 flux balance and mass integral).

One benchmark step = one pass of the whole hot path: the psi reset and
pseudo-time preconditioning, 1000 RK4 physical steps (4 FR residual + update
stages each) and the compensated mass integral.  value = (solution points x
4 stages x 1000 steps x K steps x ranks) / (max over ranks of the summed
device time of the K steps).  The L2 cache is flushed (a 512 MiB write)
before every timed step; the 64^3 working set (~1.8 GB) is larger than L2.

The roofline is the HBM bound with the algorithmic bytes per DOF-stage of
the two-array-pass model (RK4 registers plus the trace exchange): 82 B
mixed / 124 B FP64 for hex p = 3.  Secondary lines: the plain FP64 path on
the same workload, and the 128^2 jittered quad p = 4 Rider-Kothe workload.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (single RK4 steps on a 32^3 sub-grid of the
same problem), on the same metric.
"""
import argparse
import ctypes as C
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FR DOF-stage updates/s"
UNIT = "DOF-stage/s"
STEPS_PER_BENCH_STEP = 1000


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=100,
                    help="RK4 steps timed for the FP64 comparison on the same workload (0: skip)")
    ap.add_argument("--cpu-steps", type=int, default=3, help="oracle RK4 steps for cpu_baseline (0: skip)")
    ap.add_argument("--cpu-mesh-n", type=int, default=None,
                    help="elements per side of the oracle's sample (c3: 32, a sub-grid of the same problem)")
    ap.add_argument("--mesh-n", type=int, default=None,
                    help="elements per side (c3: 64, the benchmark workload; c2q: 128)")
    ap.add_argument("--no-secondary", action="store_true", help="skip the 128^2 quad p = 4 secondary line")
    ap.add_argument("--accuracy", action="store_true", help="also run both precisions to t = T and report E_L1")
    ap.add_argument("--accuracy-precision", default="both", choices=["both", "mixed", "fp64"],
                    help="precisions of the --accuracy runs")
    ap.add_argument("--no-vel-cache", action="store_true", help="evaluate the velocity in the kernels")
    ap.add_argument("--normal", default="psi", choices=["psi", "phi"],
                    help="interface normal: psi (preconditioned method) or phi (unpreconditioned CPF)")
    ap.add_argument("--wall", default=None, choices=["copy", "noflux"],
                    help="wall faces: the workload's own (copy ghost, Section 3.3) or zero normal flux")
    ap.add_argument("--order", type=int, default=None,
                    help="zalesak/rudman: polynomial order (default 4); c2s: (default 3)")
    ap.add_argument("--workload", default="c3", choices=["c2q", "c2t", "c2s", "c3", "c4", "zalesak", "rudman"],
                    help="c3: 64^3 hexes p=3 (LeVeque; the benchmark); c2q: 128^2 jittered quads p=4; "
                         "c2t: ~30k Delaunay triangles p=3; c4: 256-instance quad ensemble (200 steps per step); "
                         "zalesak / rudman: slotted disks in solid-body rotation (100^2 / 200^2 quads); "
                         "c2s: Rider-Kothe on split-triangle meshes (--mesh-n, --order <= 4)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint/forward timing")
    ap.add_argument("--ensemble-launch", default="streams", choices=["group", "streams"],
                    help="c4: one field per order on its own stream (faster, measured), or one launch per RK "
                         "stage over all orders (fr_group_step)")
    ap.add_argument("--probe", default=None, choices=["dense-hex"],
                    help="time the two forms of the hex p = 3 operator applies (fr_probe_hex_apply) and exit")
    ap.add_argument("--rk-steps", type=int, default=STEPS_PER_BENCH_STEP,
                    help="RK4 steps per benchmark step (profiling captures use fewer launches)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
def dist_init():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """Sample SM clocks and throttle reasons with nvidia-smi during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
KB_GRAPH_LAUNCHES = 400


def alg_bytes_per_dof(etype, p, precision):
    """Algorithmic HBM bytes per solution point per RK stage (a lower bound:
    every array touched once, geometry and velocity recomputed).

    RK4 registers of both fields over the 4 stages: 16 array passes per step
    (stage 1 reads u^n and writes acc and U_2; stages 2-3 read U_s, u^n, acc
    and write acc, U_s+1; stage 4 reads U_4, acc and writes u^n+1), 2 fields,
    / 4 stages: 8 P per DOF-stage in FP64 (64 B), 52 B in the mixed path
    (FP32 stage values, FP64 u^n and accumulator).  Trace exchange per element
    flux point: both fields' traces written and read by the neighbour (4 P_b)
    plus the one-sided viscous normal flux (P_b): 5 P_b Nf / Nu."""
    n = p + 1
    nu = {"quad": n * n, "hex": n ** 3, "tri": n * (n + 1) // 2}[etype]
    nf = {"quad": 4 * n, "hex": 6 * n * n, "tri": 3 * n}[etype]
    rk, pb = (52.0, 4) if precision == "mixed" else (64.0, 8)
    return rk + 5 * pb * nf / nu


def source_sha():
    h = hashlib.sha256()
    # the tensor kernels, their launch table and the field set-up that lays
    # out the arrays they read
    for fn in ("ktensor.cuh", "kcommon.cuh", "geom.cuh", "k_tensor_inst.cuh", "api.cu"):
        h.update(open(os.path.join(ROOT, "paper_2006_10967_gb300", "csrc", fn), "rb").read())
    return h.hexdigest()[:16]


def load_traffic(key):
    """Cold-cache DRAM bytes per solution point of one RK stage (kb + ka of
    the physical step) from the committed ncu summary, if its kernel source
    hash matches the current source (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    ent = d.get(key)
    if not ent or ent.get("source_sha") != source_sha():
        return None
    return ent.get("dram_bytes_per_dof")


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    d = json.load(open(path)) if os.path.exists(path) else {}
    return d


def make_field(G, S, M, P, w, precondition=True):
    """The workload's field: the disk through the library's circle initial
    condition, a slotted disk through its phi0 array at the solution points."""
    if isinstance(w.circle, S.SlottedDisk):
        return G.Field(M, P, phi0=S.initial_phi(w, M.solution_points()), precondition=precondition)
    return G.Field(M, P, ic=w.circle, precondition=precondition)


def oracle_init(sol, S, w):
    """The oracle's initial state for the workload (no preconditioning)."""
    import torch
    if isinstance(w.circle, S.SlottedDisk):
        sol.initialize(phi=torch.from_numpy(S.initial_phi(w, sol.xu.numpy())), precondition=False)
    else:
        sol.initialize(w.circle, precondition=False)


# ---------------------------------------------------------------------------
def run_path(G, S, w, mesh, precision, K, W, world, rank, flush, want_kernel=False, e2e=False, vel_cache=True,
             rk_steps=STEPS_PER_BENCH_STEP):
    """K timed steps of rk_steps RK4 steps (plus the preconditioning due among
    them and the mass integral), after W untimed ones."""
    import torch
    M = G.Mesh.from_synthetic(mesh, w.order)
    P = G.make_params(w, precision, vel_cache=vel_cache)
    F = make_field(G, S, M, P, w, precondition=True)
    ndof = M.info.n_dof
    stream = torch.cuda.current_stream()
    for _ in range(W):
        F.step(rk_steps)
        F.mass(0)
    torch.cuda.synchronize()
    out = {"ndof": ndof, "rk_steps": rk_steps}
    clocks = Clocks(torch.cuda.current_device())
    times = []
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    for _ in range(K):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        F.step(rk_steps)
        F.mass(0)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    barrier(world)
    out["clocks"] = clocks.stop()
    total_ms = max_over_ranks(sum(times), world)
    out["ms_per_step"] = total_ms / K
    out["value"] = world * K * rk_steps * 4 * ndof / (total_ms * 1e-3)
    out["status"] = F.sync()
    if want_kernel:
        flush.zero_()
        F.profile(True)
        F.step(rk_steps)
        prof = F.profile_read()
        F.profile(False)
        out["kernels"] = prof
        # steady-state duration of the residual kernel: a graph of back-to-back launches
        flush.zero_()
        out["kb_graph_ms"] = F.profile_kernel(0, KB_GRAPH_LAUNCHES)
    if e2e:
        # through the C ABI with host buffers: upload phi, psi (pinned), run, read phi back
        L = G.lib()
        phi = torch.from_numpy(F.get(0)).pin_memory()
        psi = torch.from_numpy(F.get(1)).pin_memory()
        res = torch.empty_like(phi).pin_memory()
        sp = C.c_void_p(stream.cuda_stream)
        dp = C.POINTER(C.c_double)
        ptr = lambda t: C.cast(C.c_void_p(t.data_ptr()), dp)
        m = C.c_double()
        times = []
        Ke = min(K, 3)   # end-to-end steps (each moves the state through host memory)
        for _ in range(Ke):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            G.check(L.fr_field_set(F.handle, 0, ptr(phi), sp), "fr_field_set")
            G.check(L.fr_field_set(F.handle, 1, ptr(psi), sp), "fr_field_set")
            G.check(L.fr_step(F.handle, rk_steps, sp), "fr_step")
            G.check(L.fr_mass_integral(F.handle, 0, C.byref(m), sp), "fr_mass_integral")
            G.check(L.fr_field_get(F.handle, 0, ptr(res), sp), "fr_field_get")
            times.append(time.perf_counter() - t0)
        tot = max_over_ranks(sum(times), world)
        out["e2e"] = {"value": world * Ke * rk_steps * 4 * ndof / tot, "unit": UNIT, "steps": Ke,
                      "h2d_bytes_per_step": 2 * ndof * 8, "d2h_bytes_per_step": ndof * 8 + 8}
    return out, F


def adjoint_ratio(G, S):
    """Wall time of the hand-written adjoint (checkpointed recompute + reverse
    sweep) over the forward march on the adjoint workload: 64^2 periodic quads,
    p = 4, 400 RK4 steps, 32 stream-function coefficients, checkpoints every 20."""
    import numpy as np
    import torch
    w = S.workload("c5")
    mesh = w.mesh()
    M = G.Mesh.from_synthetic(mesh, w.order)
    xu = M.solution_points()
    circ = lambda c: 0.5 * (1 + np.tanh(c.beta * (c.radius - np.sqrt(((xu - np.array(c.centre)) ** 2).sum(-1)))))
    phi0 = circ(w.circle)
    phis = torch.from_numpy(circ(w.extra["target"])).cuda()
    wq = torch.from_numpy(M.quadrature()).cuda()
    n, ck = w.n_steps, w.extra["ckpt_every"]
    res = {}
    F = G.Field(M, G.make_params(w), phi0=phi0, precondition=False)
    F.step(n)                      # warm-up (kernel attributes, caches)
    torch.cuda.synchronize()
    for rep in range(2):
        F = G.Field(M, G.make_params(w), phi0=phi0, precondition=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        F.step(n)
        F.sync()
        tf = time.perf_counter() - t0
        F = G.Field(M, G.make_params(w), phi0=phi0, precondition=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        F.adjoint_record(n, ck)
        phiT = torch.empty_like(wq)
        F.get_device(0, phiT)
        F.adjoint_step(wq * (phiT - phis), None, 32)
        ta = time.perf_counter() - t0
        res = {"forward_s": tf, "forward_plus_adjoint_s": ta, "adjoint_over_forward": (ta - tf) / tf,
               "workload": "stream-function quad64 p4 fp64, 400 RK4 steps, checkpoints every 20",
               "note": "adjoint = checkpointed forward recompute + reverse sweep; ratio excludes the recorded forward"}
    return res


def run_ensemble(G, S, K, W, world, flush, precision="mixed", n_inst=256, rk_steps=200, launch="group"):
    """The batched ensemble: 256 periodic quad instances (n ~ U{16..96},
    p ~ U{2..5}, random circles, random-phase stream-function velocities), one
    batch field per order, each on its own CUDA stream; one benchmark step =
    rk_steps RK4 steps of every instance.  Timed with CUDA events on the
    current stream, which the order streams join at the start and the end."""
    import torch
    ws = S.ensemble_instances(n_inst, seed=3)
    fields = G.batch_from_workloads(ws, precision=precision)
    streams = [torch.cuda.Stream() for _ in fields]
    ndof = sum(F.mesh.info.n_dof for _, F, _ in fields)
    cur = torch.cuda.current_stream()

    group = G.Group([F for _, F, _ in fields]) if launch == "group" else None

    def one():
        if group is not None:          # one launch per kernel per RK stage over all orders
            group.step(rk_steps, stream=cur)
            return
        start = torch.cuda.Event()
        start.record(cur)
        for (p, F, _), st in zip(fields, streams):
            st.wait_event(start)
            F.step(rk_steps, stream=st)
        for st in streams:
            done = torch.cuda.Event()
            done.record(st)
            cur.wait_event(done)
    for _ in range(W):
        one()
    torch.cuda.synchronize()
    times = []
    barrier(world)
    for _ in range(K):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(cur)
        one()
        e1.record(cur)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) * 1e-3)
    tot = max_over_ranks(sum(times), world)
    value = world * K * rk_steps * 4 * ndof / tot
    per_order = {str(p): {"instances": len(r), "dof": F.mesh.info.n_dof} for p, F, r in fields}
    status = max((F.sync() for _, F, _ in fields), key=abs)
    # HBM roofline: algorithmic bytes of every order group per stage
    b_stage = sum(alg_bytes_per_dof("quad", p, precision) * F.mesh.info.n_dof for p, F, _ in fields)
    stage_s = tot / (K * rk_steps * 4)
    pk = peaks()
    peak = pk.get("hbm_gbs") or 6800.0
    roof = {"bound": "hbm", "kernel": ("RK stage of all orders: kb_group + ka_group (one launch each)"
                                       if group is not None else
                                       "RK stage of every order group (kb_tensor + ka_tensor per order, 4 streams)"),
            "achieved": b_stage / stage_s / 1e9, "peak": peak, "unit": "GB/s",
            "frac": b_stage / stage_s / 1e9 / peak, "traffic": None,
            "alg_bytes_per_stage": b_stage, "stage_us": stage_s * 1e6,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs" if pk.get("hbm_gbs") else "fallback 6.8 TB/s",
            "timing": "CUDA events on the current stream around the joined order streams"}
    # end to end through the C ABI with host buffers (phi and psi up, phi down, every field)
    L = G.lib()
    dp = C.POINTER(C.c_double)
    ptr = lambda t: C.cast(C.c_void_p(t.data_ptr()), dp)
    host = [(torch.from_numpy(F.get(0)).pin_memory(), torch.from_numpy(F.get(1)).pin_memory(),
             torch.empty(F.mesh.shape, dtype=torch.float64).pin_memory()) for _, F, _ in fields]
    te = []
    Ke = min(K, 3)
    for _ in range(Ke):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if group is not None:
            sp = C.c_void_p(cur.cuda_stream)
            for ((p, F, _), (hphi, hpsi, hres)) in zip(fields, host):
                G.check(L.fr_field_set(F.handle, 0, ptr(hphi), sp), "fr_field_set")
                G.check(L.fr_field_set(F.handle, 1, ptr(hpsi), sp), "fr_field_set")
            G.check(L.fr_group_step(group.handle, rk_steps, sp), "fr_group_step")
            for ((p, F, _), (hphi, hpsi, hres)) in zip(fields, host):
                G.check(L.fr_field_get(F.handle, 0, ptr(hres), sp), "fr_field_get")
        else:
            for ((p, F, _), st, (hphi, hpsi, hres)) in zip(fields, streams, host):
                sp = C.c_void_p(st.cuda_stream)
                G.check(L.fr_field_set(F.handle, 0, ptr(hphi), sp), "fr_field_set")
                G.check(L.fr_field_set(F.handle, 1, ptr(hpsi), sp), "fr_field_set")
                G.check(L.fr_step(F.handle, rk_steps, sp), "fr_step")
            for ((p, F, _), st, (hphi, hpsi, hres)) in zip(fields, streams, host):
                G.check(L.fr_field_get(F.handle, 0, ptr(hres), C.c_void_p(st.cuda_stream)), "fr_field_get")
        te.append(time.perf_counter() - t0)
    e2e = {"value": world * Ke * rk_steps * 4 * ndof / max_over_ranks(sum(te), world), "unit": UNIT,
           "steps": Ke, "h2d_bytes_per_step": 2 * ndof * 8, "d2h_bytes_per_step": ndof * 8}
    return {"value": value, "ms_per_step": tot / K * 1e3, "ndof": ndof, "roofline": roof, "e2e": e2e, "launch": launch,
            "per_order": per_order, "status": status, "rk_steps": rk_steps, "instances": n_inst,
            "workloads": ws}


def ensemble_cpu_baseline(S, ws, n_sample=16, nsteps=1):
    """The FP64 oracle on the first n_sample instances of the ensemble, nsteps
    RK4 steps each, all host threads; DOF-stage/s over the sample."""
    import torch
    from oracle import Params, Solver
    tot_dof, tot_t = 0, 0.0
    for w in ws[:n_sample]:
        sol = Solver(w.mesh(), w.order, Params.from_workload(w), w.velocity)
        sol.initialize(w.circle, precondition=False)
        t0 = time.perf_counter()
        for _ in range(nsteps):
            sol.rk4_step()
        tot_t += time.perf_counter() - t0
        tot_dof += sol.E * sol.Nu
    return {"value": tot_dof * 4 * nsteps / tot_t, "unit": UNIT, "cores": torch.get_num_threads(),
            "os_cpu_count": os.cpu_count(), "kind": "oracle",
            "sample": f"{nsteps} RK4 step(s) of each of the first {n_sample} ensemble instances "
                      f"({tot_dof} solution points), FP64 torch-CPU oracle, {tot_t:.1f} s"}


def cpu_baseline(S, w, mesh, nsteps, sample_note):
    """The FP64 torch-CPU oracle on the host cores: nsteps RK4 steps with all
    threads, then one step on one thread, on `mesh` (the workload or a
    sub-grid of the same problem, described by sample_note)."""
    import torch
    from oracle import Params, Solver
    sol = Solver(mesh, w.order, Params.from_workload(w), w.velocity)
    oracle_init(sol, S, w)
    t0 = time.perf_counter()
    for _ in range(nsteps):
        sol.rk4_step()
    dt = time.perf_counter() - t0
    ndof = sol.E * sol.Nu
    nthr = torch.get_num_threads()
    torch.set_num_threads(1)
    try:
        t1 = time.perf_counter()
        sol.rk4_step()
        dt1 = time.perf_counter() - t1
    finally:
        torch.set_num_threads(nthr)
    return {"value": ndof * 4 * nsteps / dt, "unit": UNIT, "cores": nthr,
            "os_cpu_count": os.cpu_count(),
            "single_thread": {"value": ndof * 4 / dt1, "unit": UNIT, "steps": 1},
            "kind": "oracle",
            "sample": f"{nsteps} RK4 step(s) (4 residual stages) of {sample_note}, "
                      f"FP64 torch-CPU oracle, {dt:.1f} s; then 1 step on one thread, {dt1:.1f} s"}


def element_normals(M, order, psi):
    """Unit normal grad psi / |grad psi| at the solution points of tensor
    elements (quads, hexes) from the element-local gradient: the 1D
    Lagrange derivative at the Gauss-Legendre points along each reference
    axis (axis 0 fastest in the point index), mapped by J^{-T} with J the
    derivative of the points' coordinates (exact for multilinear maps).  A
    diagnostic of the state, computed on the host; None for triangles."""
    import numpy as np
    info = M.info
    if info.etype == 1:
        return None
    n, d = order + 1, info.dim
    x, _ = np.polynomial.legendre.leggauss(n)
    wb = np.array([1.0 / np.prod([x[j] - x[m] for m in range(n) if m != j]) for j in range(n)])
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = wb[j] / wb[i] / (x[i] - x[j])
        D[i, i] = -D[i].sum()
    E = info.n_elems
    shp = (E,) + (n,) * d                 # C order: [e][i_{d-1}]...[i_0]
    xu = M.solution_points().reshape((E, n ** d, d))
    u = np.asarray(psi).reshape(shp)

    def deriv(f, a):                      # along reference axis a (array axis d - a)
        return np.moveaxis(np.tensordot(D, f, axes=([1], [d - a])), 0, d - a)
    qt = np.stack([deriv(u, a).reshape(E, -1) for a in range(d)], -1)            # (E, NU, d)
    J = np.stack([np.stack([deriv(xu[..., c].reshape(shp), a).reshape(E, -1) for a in range(d)], -1)
                  for c in range(d)], -2)                                       # J[..., c, a]
    q = np.linalg.solve(np.swapaxes(J, -1, -2), qt[..., None])[..., 0]
    return q / np.maximum(np.linalg.norm(q, axis=-1, keepdims=True), 1e-12)


def accuracy(G, S, w, mesh, precisions=("fp64", "mixed")):
    """Run both precisions to t = T and report E_L1, E_r and E_m (Section 4)
    against the initial shape, which the flows return at t = T (Rider-Kothe
    reversal, one solid-body revolution)."""
    import numpy as np
    res = {}
    M = G.Mesh.from_synthetic(mesh, w.order)
    xu = M.solution_points()
    phi_e = S.initial_phi(w, xu)
    wq = M.quadrature()
    for prec in precisions:
        F = make_field(G, S, M, G.make_params(w, prec), w, precondition=True)
        m0 = F.mass(0)
        t0 = time.perf_counter()
        F.step(w.n_steps)
        F.sync()
        el = time.perf_counter() - t0
        phi = F.get(0)
        res.setdefault("_state", {})[prec] = (phi, F.get(1))
        res[prec] = {"E_L1": float((wq * np.abs(phi - phi_e)).sum()),
                     "E_r": float((wq * np.abs(phi - phi_e)).sum() / (wq * phi_e).sum()),
                     "E_m": float((F.mass(0) - m0) / (wq * phi_e).sum()),
                     "steps": w.n_steps, "wall_s": el}
    st = res.pop("_state")
    if "mixed" in res and "fp64" in res:
        res["ratio_L1_mixed_over_fp64"] = res["mixed"]["E_L1"] / res["fp64"]["E_L1"]
        n64 = element_normals(M, w.order, st["fp64"][1])
        n32 = element_normals(M, w.order, st["mixed"][1])
        if n64 is not None:
            band = (st["fp64"][0] > 0.05) & (st["fp64"][0] < 0.95)
            res["normal_error"] = {
                "mean_abs_diff": float(np.linalg.norm(n32 - n64, axis=-1)[band].mean()),
                "points": int(band.sum()),
                "definition": "mean |n_mixed - n_fp64| over solution points with 0.05 < phi_fp64 < 0.95, "
                              "n = grad psi / |grad psi| from the element-local gradient"}
    return res


def probe_dense_hex(args):
    """Steps 1 and 3's operator applies on 64^3 hexahedra of order 3 (traces
    and reference derivatives of both fields, no corrections), sum-factorised
    (form 0) against the dense 288 x 64 operator on the tensor cores (form 1),
    through fr_probe_hex_apply in its reducing mode (one sum per element and
    field written, so the output traffic is negligible).  Each launch is
    timed alone with CUDA events after an L2 flush; the median is reported."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2006_10967_gb300 as G
    from paper_2006_10967_gb300 import _capi
    L = G.lib()
    n = args.mesh_n or 64
    E = n ** 3
    u = torch.randn(E, 2, 64, device="cuda", generator=torch.Generator(device="cuda").manual_seed(7))
    out = {f: torch.empty(E * 2, device="cuda") for f in (0, 1)}
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    sp = C.c_void_p(stream.cuda_stream)

    def call(form):
        _capi.check(L.fr_probe_hex_apply(3, form, 1, C.c_void_p(u.data_ptr()), E, C.c_void_p(out[form].data_ptr()),
                                         E * 2, sp), "fr_probe_hex_apply")

    res = {}
    for form in (0, 1):
        for _ in range(max(args.warmup, 3)):
            call(form)
        ts = []
        for _ in range(max(args.steps, 5)):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            call(form)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b) * 1e3)
        res[form] = statistics.median(ts)
    agree = float((out[0] - out[1]).abs().max() / out[0].abs().max())
    cols = 2 * E
    useful = 2 * (96 * 4 + 192 * 4)          # FMAs x 2 per column, both forms' useful work
    dense_tc = 3 * 2 * 288 * 64              # three TF32 products of the dense operator per column
    pk = peaks()
    tf32_peak = pk.get("bf16_tflops", 1900.0) * (1.1 / 2.25)
    line = {"probe": "hex p=3 operator applies: flux-point traces and reference derivatives of both fields "
                     "(Steps 1 and 3 without corrections), reducing mode",
            "elements": E, "columns": cols, "input_bytes": u.numel() * 4,
            "sum_factorised_us": res[0], "dense_tensor_core_us": res[1], "dense_over_sf": res[1] / res[0],
            "sum_factorised": {"useful_tflops": useful * cols / (res[0] * 1e-6) / 1e12,
                               "input_gbs": u.numel() * 4 / (res[0] * 1e-6) / 1e9},
            "dense_tensor_core": {"tensor_tflops": dense_tc * cols / (res[1] * 1e-6) / 1e12,
                                  "tf32_peak_tflops": tf32_peak,
                                  "tf32_peak_source": "MEASURED_PEAKS bf16 burst x nominal TF32/BF16 ratio 1.1/2.25",
                                  "useful_tflops": useful * cols / (res[1] * 1e-6) / 1e12},
            "forms_agree_rel": agree,
            "timing": "median of per-launch CUDA events, L2 flushed (512 MiB write) before each launch"}
    line["dense_tensor_core"]["frac_of_tf32_peak"] = line["dense_tensor_core"]["tensor_tflops"] / tf32_peak
    print(json.dumps(line))


def main():
    args = parse()
    if args.probe == "dense-hex":
        probe_dense_hex(args)
        return
    rank, world = dist_init()
    import synthetic as S
    if args.workload == "c4" and args.impl == "ours":
        import torch
        import __graft_entry__
        __graft_entry__.build()
        import paper_2006_10967_gb300 as G
        flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
        out = run_ensemble(G, S, args.steps, max(args.warmup, 3), world, flush, args.precision,
                           launch=args.ensemble_launch)
        cpu = ensemble_cpu_baseline(S, out["workloads"]) if rank == 0 and world == 1 and args.cpu_steps > 0 else None
        line = {"metric": METRIC, "value": out["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(args.warmup, 3), "ms_per_step": out["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "mixed" else "f64",
                "data": "synthetic",
                "config": {"workload": "ensemble256_quad_p2to5_stream", "instances": out["instances"],
                           "solution_points": out["ndof"], "rk_steps_per_step": out["rk_steps"],
                           "per_order": out["per_order"], "precision": args.precision,
                           "launch": ("one launch per kernel per RK stage over the order groups (fr_group_step)"
                                      if out["launch"] == "group" else
                                      "one batch field per order, each on its own CUDA stream"),
                           "l2": "flushed before each timed step; working set larger than L2"},
                "roofline": out["roofline"], "e2e": out["e2e"], "cpu_baseline": cpu,
                "gpu_launches": 2 * 4 * out["rk_steps"] * len(out["per_order"]) * args.steps,
                "status": out["status"]}
        if rank == 0:
            print(json.dumps(line))
        return
    w, wname = select_workload(S, args.workload, args.mesh_n, args.order)
    w.normal = args.normal
    if args.normal == "phi":
        wname += "_unpreconditioned"
    if args.wall:
        w.wall = args.wall
        if args.wall == "noflux":
            wname += "_noflux_walls"
    mesh = w.mesh()
    workload_cfg = workload_config(w, wname, mesh, args.normal, world)
    workload_cfg["rk_steps_per_step"] = args.rk_steps
    # the oracle's bounded sample: the workload itself, or for the 64^3 hex
    # workload a 32^3 sub-grid of the same problem (same order, field and
    # parameters; the rate is per DOF-stage)
    cpu_n = args.cpu_mesh_n or (32 if args.workload == "c3" and (args.mesh_n or 64) > 32 else None)
    if cpu_n is not None:
        w_cpu, cpu_name = select_workload(S, args.workload, cpu_n, args.order)
        w_cpu.normal = args.normal
        if args.wall:
            w_cpu.wall = args.wall
        cpu_note = f"the same problem on a {cpu_n}^3 sub-grid ({cpu_name}, {cpu_n ** 3} elements)"
    else:
        w_cpu, cpu_note = w, f"the full workload ({wname})"

    if args.impl == "reference":
        if rank != 0:
            return
        import torch
        from oracle import Params, Solver
        mesh_cpu = w_cpu.mesh() if w_cpu is not w else mesh
        sol = Solver(mesh_cpu, w_cpu.order, Params.from_workload(w_cpu), w_cpu.velocity)
        oracle_init(sol, S, w_cpu)
        for _ in range(args.warmup):
            sol.rk4_step()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sol.rk4_step()
        dt = time.perf_counter() - t0
        ndof = sol.E * sol.Nu
        val = ndof * 4 * args.steps / dt
        line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 0,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": dict(workload_cfg, reference_step="one RK4 step of the oracle"),
                "cpu_baseline": {"value": val, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
                                 "sample": f"{args.steps} RK4 steps of {cpu_note} after {args.warmup} warm-up"},
                "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2006_10967_gb300 as G

    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    vc = not args.no_vel_cache
    main_out, F = run_path(G, S, w, mesh, args.precision, args.steps, max(args.warmup, 3), world, rank, flush,
                           want_kernel=True, e2e=True, vel_cache=vc, rk_steps=args.rk_steps)
    del F
    fp64_out = None
    if args.precision == "mixed" and args.fp64_steps > 0:
        fp64_out, F64 = run_path(G, S, w, mesh, "fp64", 1, 1, world, rank, flush, want_kernel=True,
                                 vel_cache=vc, rk_steps=args.fp64_steps)
        del F64
    torch.cuda.empty_cache()

    roof = roofline(main_out, mesh.etype, w.order, args.precision, args.workload)
    cpu = None
    if rank == 0 and world == 1 and args.cpu_steps > 0:
        cpu = cpu_baseline(S, w_cpu, w_cpu.mesh() if w_cpu is not w else mesh, args.cpu_steps, cpu_note)

    kern = main_out["kernels"]
    line = {"metric": METRIC, "value": main_out["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": main_out["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "mixed" else "f64",
            "data": "synthetic", "config": dict(workload_cfg, precision=args.precision, velocity_cache=vc),
            "clocks": main_out["clocks"], "e2e": main_out["e2e"],
            "gpu_launches": int(sum(v[1] for v in kern.values())) * args.steps + 3 * args.steps,
            "roofline": roof, "cpu_baseline": cpu, "status": main_out["status"]}
    if fp64_out is not None:
        line["fp64"] = {"value": fp64_out["value"], "rk_steps_timed": fp64_out["rk_steps"],
                        "roofline": roofline(fp64_out, mesh.etype, w.order, "fp64", args.workload),
                        "note": "the plain FP64 path on the same workload, one timed window of RK4 steps"}
        line["speedup_mixed_over_fp64"] = main_out["value"] / fp64_out["value"]
    if args.accuracy:
        line["accuracy"] = accuracy(G, S, w, mesh, {"both": ("fp64", "mixed"), "mixed": ("mixed",),
                                                    "fp64": ("fp64",)}[args.accuracy_precision])
    if not args.no_secondary and args.workload == "c3" and args.mesh_n in (None, 64) and args.order in (None, 3):
        w2, n2 = select_workload(S, "c2q", 128, None)
        sec, F2 = run_path(G, S, w2, w2.mesh(), args.precision, args.steps, max(args.warmup, 3), world, rank,
                           flush, want_kernel=True, vel_cache=vc)
        del F2
        line["secondary"] = {"workload": n2, "value": sec["value"], "unit": UNIT, "ms_per_step": sec["ms_per_step"],
                             "solution_points": sec["ndof"], "precision": args.precision,
                             "roofline": roofline(sec, "quad", 4, args.precision, "c2q"),
                             "note": "working set (~30 MB) L2-resident within a step; latency bound"}
    if not args.no_adjoint and world == 1:
        line["adjoint"] = adjoint_ratio(G, S)
    if rank == 0:
        print(json.dumps(line))


def select_workload(S, name, mesh_n, order):
    if name == "c2q":
        n = mesh_n or 128
        return S.workload("c2q", n=n), f"rider_kothe_quad{n}_jitter_p4"
    if name == "c2t":
        return S.workload("c2t"), "rider_kothe_tri_delaunay_p3"
    if name == "c2s":
        n = mesh_n or 128
        w = S.workload("c2s", n=n, p=order or 3)
        return w, f"rider_kothe_trisplit{n}_p{w.order}"
    if name in ("zalesak", "rudman"):
        n = mesh_n or (100 if name == "zalesak" else 200)
        w = S.workload(name, n=n, p=order or 4)
        return w, w.name
    n = mesh_n or 64
    w = S.workload("c3", n=n, p=order or 3)
    return w, f"leveque_hex{n}_p{w.order}"


def workload_config(w, wname, mesh, normal, world):
    nu_el = {"quad": (w.order + 1) ** 2, "tri": (w.order + 1) * (w.order + 2) // 2,
             "hex": (w.order + 1) ** 3}[mesh.etype]
    ndof = mesh.n_elems * nu_el
    big = ndof * 2 * 4 * 6 > 129e6
    return {"workload": wname, "normal": {"psi": "grad psi (preconditioned)",
                                          "phi": "grad phi (unpreconditioned CPF)"}[normal],
            "elements": mesh.n_elems, "order": w.order,
            "solution_points": ndof, "rk_steps_per_step": STEPS_PER_BENCH_STEP,
            "stages_per_rk_step": 4, "precondition_every": w.n_precond, "pseudo_kmax": w.pseudo_kmax,
            "l2": ("flushed before each timed step (512 MiB write); working set larger than L2" if big else
                   "flushed before each timed step (512 MiB write); working set L2-resident within a step"),
            "parallelism": f"replicas x{world}"}


def roofline(out, etype, p, precision, workload):
    """HBM roofline of one RK stage (the kb + ka launch pair of the physical
    step): algorithmic bytes per DOF-stage x solution points / stage time,
    with the stage time taken from the CUDA-event timed region (which also
    holds the preconditioning and the mass integral, so the figure is a lower
    bound), against the measured HBM copy bandwidth."""
    import torch
    ndof = out["ndof"]
    b_alg = alg_bytes_per_dof(etype, p, precision)
    stage_s = ndof / out["value"]                    # seconds per stage, all ranks' work per rank
    achieved = b_alg * ndof / stage_s / 1e9
    pk = peaks()
    peak = pk.get("hbm_gbs")
    src = "MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)"
    if not peak:
        peak, src = 6800.0, "fallback 6.8 TB/s"
    kern = out.get("kernels", {})
    stage_kern = {k: {"avg_us": v[0] / v[1] * 1e3, "launches": v[1]} for k, v in kern.items() if v[1]}
    tot = sum(v[0] for v in kern.values()) or 1.0
    for k, v in kern.items():
        if v[1]:
            stage_kern[k]["share_of_step"] = v[0] / tot
    traffic_dof = load_traffic(f"stage_{workload}_{etype}_p{p}_{precision}")
    return {"bound": "hbm", "kernel": "RK stage: kb_tensor + ka_tensor" if etype != "tri" else
            "RK stage: kb_tri + ka_tri",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic_dof * ndof if traffic_dof else None,
            "alg_bytes_per_dof_stage": b_alg, "stage_us": stage_s * 1e6,
            "peak_source": src, "sm_count": torch.cuda.get_device_properties(0).multi_processor_count,
            "timing": "stage time = timed region (CUDA events on the launching stream) / (RK steps x 4)",
            "kernels_profiled": stage_kern,
            "kb_graph_us": out["kb_graph_ms"] * 1e3 if out.get("kb_graph_ms") else None,
            "traffic_note": "cold-cache dram__bytes_read.sum + dram__bytes_write.sum of kb + ka per stage from "
                            "a small ncu capture, scaled by solution points (null: none at this source)"}


if __name__ == "__main__":
    main()
