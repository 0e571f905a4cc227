#!/usr/bin/env python
"""Benchmark of the FR-PCPF hot path: FR DOF-stage updates per second.

Workload: 128 x 128 jittered, shuffled quads on [0,1]^2, p = 4 (409,600
solution points), Rider-Kothe vortex with T = 8, disk r = 0.15 at (0.5, 0.75),
the paper's parameters (gamma = 0.09, eps = 0.06 h/p, precondition every
1000 steps with up to 20 pseudo iterations, s0 = -5).

One benchmark step = one pass of the whole hot path: the psi reset and
pseudo-time preconditioning, 1000 RK4 physical steps (4 FR residual + update
stages each) and the compensated mass integral.  value = (solution points x
4 stages x 1000 steps x K steps x ranks) / (max over ranks of the summed
device time of the K steps).  The L2 cache is flushed (a 512 MiB write)
before every timed step; within a step the working set (~30 MB) stays in L2.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (single RK4 steps), on the same metric.
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
    ap.add_argument("--fp64-steps", type=int, default=2, help="timed steps of the FP64 comparison (0: skip)")
    ap.add_argument("--cpu-steps", type=int, default=25, help="oracle RK4 steps for cpu_baseline (0: skip)")
    ap.add_argument("--mesh-n", type=int, default=None,
                    help="elements per side (c2q: 128, the benchmark workload; c3: 64)")
    ap.add_argument("--accuracy", action="store_true", help="also run both precisions to t = T and report E_L1")
    ap.add_argument("--accuracy-precision", default="both", choices=["both", "mixed", "fp64"],
                    help="precisions of the --accuracy runs")
    ap.add_argument("--no-vel-cache", action="store_true", help="evaluate the velocity in the kernels")
    ap.add_argument("--normal", default="psi", choices=["psi", "phi"],
                    help="interface normal: psi (preconditioned method) or phi (unpreconditioned CPF)")
    ap.add_argument("--order", type=int, default=None,
                    help="zalesak/rudman: polynomial order (default 4); c2s: (default 3)")
    ap.add_argument("--workload", default="c2q", choices=["c2q", "c2t", "c2s", "c3", "c4", "zalesak", "rudman"],
                    help="c2q: 128^2 jittered quads p=4 (the benchmark); c2t: ~30k Delaunay triangles p=3; "
                         "c3: 64^3 hexes p=3 (LeVeque); c4: 256-instance quad ensemble (200 steps per step); "
                         "zalesak / rudman: slotted disks in solid-body rotation (100^2 / 200^2 quads); "
                         "c2s: Rider-Kothe on split-triangle meshes (--mesh-n, --order <= 4)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint/forward timing")
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


def alg_flops_per_dof(dim, p):
    """Algorithmic flops per solution point per RK stage of the residual kernel
    (Steps 1-6, both fields, sum-factorised tensor operators; an FMA counts 2).
    Velocity evaluation and metric terms are excluded (they depend on whether
    they are stored or recomputed)."""
    n = p + 1
    nu = n ** dim
    nf = 2 * dim * n ** (dim - 1)
    r = nf / nu
    f = 0.0
    f += 2 * r * n * 2                       # Step 1 traces, 2 fields
    f += 2 * dim * (n * 2 + 2 * 2)           # Step 3 reference gradient + two line corrections
    f += 2 * dim * dim * 2                   # q = J^-T q~
    f += 0.5 * r * 2 * dim * n * 2           # q^f at L flux points
    f += 0.5 * r * (8 * dim + 14)            # Step 5 common flux (normal, speeds, fluxes, penalty)
    f += 6 * dim + 10                        # Step 4 pointwise fluxes (|v|, |q_psi|, sharpening)
    f += 2 * dim * dim * 2                   # f~ = det J J^-1 f
    f += 2 * r * n * 2 + 2 * r               # discontinuous normal flux and jump
    f += 2 * dim * (n * 2 + 2 * 2)           # Step 6 divergence + two line lifts
    return f


def source_sha():
    h = hashlib.sha256()
    for fn in ("ktensor.cuh", "kcommon.cuh", "geom.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2006_10967_gb300", "csrc", fn), "rb").read())
    return h.hexdigest()[:16]


def load_traffic(kernel_key):
    """DRAM bytes per launch from the committed ncu summary, if its kernel
    source hash matches the current source (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    ent = d.get(kernel_key)
    if not ent or ent.get("source_sha") != source_sha():
        return None
    return ent.get("dram_bytes_per_launch")


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
def run_path(G, S, w, mesh, precision, K, W, world, rank, flush, want_kernel=False, e2e=False, vel_cache=True):
    import torch
    M = G.Mesh.from_synthetic(mesh, w.order)
    P = G.make_params(w, precision, vel_cache=vel_cache)
    F = make_field(G, S, M, P, w, precondition=True)
    ndof = M.info.n_dof
    stream = torch.cuda.current_stream()
    for _ in range(W):
        F.step(STEPS_PER_BENCH_STEP)
        F.mass(0)
    torch.cuda.synchronize()
    out = {"ndof": ndof}
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
        F.step(STEPS_PER_BENCH_STEP)
        F.mass(0)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    barrier(world)
    out["clocks"] = clocks.stop()
    total_ms = max_over_ranks(sum(times), world)
    out["ms_per_step"] = total_ms / K
    out["value"] = world * K * STEPS_PER_BENCH_STEP * 4 * ndof / (total_ms * 1e-3)
    out["status"] = F.sync()
    if want_kernel:
        flush.zero_()
        F.profile(True)
        F.step(STEPS_PER_BENCH_STEP)
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
        for _ in range(K):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            G.check(L.fr_field_set(F.handle, 0, ptr(phi), sp), "fr_field_set")
            G.check(L.fr_field_set(F.handle, 1, ptr(psi), sp), "fr_field_set")
            G.check(L.fr_step(F.handle, STEPS_PER_BENCH_STEP, sp), "fr_step")
            G.check(L.fr_mass_integral(F.handle, 0, C.byref(m), sp), "fr_mass_integral")
            G.check(L.fr_field_get(F.handle, 0, ptr(res), sp), "fr_field_get")
            times.append(time.perf_counter() - t0)
        tot = max_over_ranks(sum(times), world)
        out["e2e"] = {"value": world * K * STEPS_PER_BENCH_STEP * 4 * ndof / tot, "unit": UNIT,
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


def run_ensemble(G, S, K, W, world, flush, precision="mixed", n_inst=256, rk_steps=200):
    """The batched ensemble: 256 periodic quad instances (n ~ U{16..96},
    p ~ U{2..5}, random circles, random-phase stream-function velocities), one
    batch field per order, each on its own CUDA stream; one benchmark step =
    rk_steps RK4 steps of every instance."""
    import torch
    ws = S.ensemble_instances(n_inst, seed=3)
    fields = G.batch_from_workloads(ws, precision=precision)
    streams = [torch.cuda.Stream() for _ in fields]
    ndof = sum(F.mesh.info.n_dof for _, F, _ in fields)
    def one():
        for (p, F, _), st in zip(fields, streams):
            F.step(rk_steps, stream=st)
        for st in streams:
            st.synchronize()
    for _ in range(W):
        one()
    torch.cuda.synchronize()
    times = []
    for _ in range(K):
        flush.zero_()
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        one()
        times.append(time.perf_counter() - t0)
    tot = max_over_ranks(sum(times), world)
    per_order = {str(p): {"instances": len(r), "dof": F.mesh.info.n_dof} for p, F, r in fields}
    status = max((F.sync() for _, F, _ in fields), key=abs)
    return {"value": world * K * rk_steps * 4 * ndof / tot, "ms_per_step": tot / K * 1e3, "ndof": ndof,
            "per_order": per_order, "status": status, "rk_steps": rk_steps, "instances": n_inst}


def cpu_baseline(S, w, mesh, nsteps):
    import torch
    from oracle import Params, Solver
    sol = Solver(mesh, w.order, Params.from_workload(w), w.velocity)
    oracle_init(sol, S, w)
    t0 = time.perf_counter()
    for _ in range(nsteps):
        sol.rk4_step()
    dt = time.perf_counter() - t0
    ndof = sol.E * sol.Nu
    # the same oracle on one thread, over a fifth of the sample
    nthr = torch.get_num_threads()
    n1 = max(1, nsteps // 5)
    torch.set_num_threads(1)
    try:
        t1 = time.perf_counter()
        for _ in range(n1):
            sol.rk4_step()
        dt1 = time.perf_counter() - t1
    finally:
        torch.set_num_threads(nthr)
    return {"value": ndof * 4 * nsteps / dt, "unit": UNIT, "cores": nthr,
            "os_cpu_count": os.cpu_count(),
            "single_thread": {"value": ndof * 4 * n1 / dt1, "unit": UNIT, "steps": n1},
            "kind": "oracle",
            "sample": f"{nsteps} RK4 step(s) (4 residual stages) of the full workload ({w.name}), "
                      f"FP64 torch-CPU oracle, {dt:.1f} s; then {n1} step(s) on one thread, {dt1:.1f} s"}


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
        res[prec] = {"E_L1": float((wq * np.abs(phi - phi_e)).sum()),
                     "E_r": float((wq * np.abs(phi - phi_e)).sum() / (wq * phi_e).sum()),
                     "E_m": float((F.mass(0) - m0) / (wq * phi_e).sum()),
                     "steps": w.n_steps, "wall_s": el}
    if "mixed" in res and "fp64" in res:
        res["ratio_L1_mixed_over_fp64"] = res["mixed"]["E_L1"] / res["fp64"]["E_L1"]
    return res


def main():
    args = parse()
    rank, world = dist_init()
    import synthetic as S
    if args.workload == "c4" and args.impl == "ours":
        import torch
        import __graft_entry__
        __graft_entry__.build()
        import paper_2006_10967_gb300 as G
        flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
        out = run_ensemble(G, S, args.steps, max(args.warmup, 3), world, flush, args.precision)
        line = {"metric": METRIC, "value": out["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(args.warmup, 3), "ms_per_step": out["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "mixed" else "f64",
                "data": "synthetic",
                "config": {"workload": "ensemble256_quad_p2to5_stream", "instances": out["instances"],
                           "solution_points": out["ndof"], "rk_steps_per_step": out["rk_steps"],
                           "per_order": out["per_order"], "precision": args.precision,
                           "launch": "one batch field per order, each on its own CUDA stream",
                           "l2": "flushed before each timed step; working set larger than L2"},
                "status": out["status"]}
        if rank == 0:
            print(json.dumps(line))
        return
    if args.workload == "c2q":
        n = args.mesh_n or 128
        w = S.workload("c2q", n=n)
        wname = f"rider_kothe_quad{n}_jitter_p4"
    elif args.workload == "c2t":
        w = S.workload("c2t")
        wname = "rider_kothe_tri_delaunay_p3"
    elif args.workload == "c2s":
        n = args.mesh_n or 128
        w = S.workload("c2s", n=n, p=args.order or 3)
        wname = f"rider_kothe_trisplit{n}_p{w.order}"
    elif args.workload in ("zalesak", "rudman"):
        n = args.mesh_n or (100 if args.workload == "zalesak" else 200)
        w = S.workload(args.workload, n=n, p=args.order or 4)
        wname = w.name
    else:
        n = args.mesh_n or 64
        w = S.workload("c3", n=n, p=args.order or 3)
        wname = f"leveque_hex{n}_p{w.order}"
    w.normal = args.normal
    if args.normal == "phi":
        wname += "_unpreconditioned"
    mesh = w.mesh()
    nu_el = {"quad": (w.order + 1) ** 2, "tri": (w.order + 1) * (w.order + 2) // 2, "hex": (w.order + 1) ** 3}[mesh.etype]
    workload_cfg = {"workload": wname, "normal": {"psi": "grad psi (preconditioned)",
                                                  "phi": "grad phi (unpreconditioned CPF)"}[args.normal],
                    "elements": mesh.n_elems, "order": w.order,
                    "solution_points": mesh.n_elems * nu_el, "rk_steps_per_step": STEPS_PER_BENCH_STEP,
                    "stages_per_rk_step": 4, "precondition_every": w.n_precond, "pseudo_kmax": w.pseudo_kmax,
                    "l2": "flushed before each timed step (512 MiB write); working set L2-resident within a step",
                    "parallelism": f"replicas x{world}"}

    if args.impl == "reference":
        if rank != 0:
            return
        import torch
        from oracle import Params, Solver
        sol = Solver(mesh, w.order, Params.from_workload(w), w.velocity)
        oracle_init(sol, S, w)
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
                                 "sample": f"{args.steps} RK4 steps of the full workload after {args.warmup} warm-up"},
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
                           want_kernel=True, e2e=True, vel_cache=vc)
    fp64_out = None
    if args.precision == "mixed" and args.fp64_steps > 0:
        fp64_out, _ = run_path(G, S, w, mesh, "fp64", args.fp64_steps, 1, world, rank, flush, want_kernel=True,
                               vel_cache=vc)

    # roofline of the dominant kernel (kb: the physical residual + common flux)
    kern = main_out["kernels"]
    dom = "kb_phys"
    ms_launch = main_out["kb_graph_ms"]
    pk = peaks()
    sm_max = pk.get("sm_max_mhz", 2070.0)
    if args.precision == "mixed":
        peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12   # FP32 lanes x FMA x clock
        peak_note = "FP32: 152 SM x 128 lanes x 2 flop x max SM clock"
    else:
        peak = 152 * 2 * 2 * sm_max * 1e6 / 1e12     # FP64: 2 DFMA/clk/SM
        peak_note = "FP64: 152 SM x 2 DFMA x 2 flop x max SM clock"
    ndof = main_out["ndof"]
    flops_launch = alg_flops_per_dof(mesh.dim, w.order) * ndof
    achieved = flops_launch / (ms_launch * 1e-3) / 1e12
    roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak,
            "traffic": load_traffic(f"kb_phys_{args.workload}_{args.precision}"),
            "peak_source": peak_note + " (derived, nominal units and clocks)",
            "avg_launch_us": ms_launch * 1e3,
            "timing": f"CUDA events around a CUDA graph of {KB_GRAPH_LAUNCHES} back-to-back launches on the "
                      "benchmark state, after the timed region",
            "event_pair_us": {k: v[0] / v[1] * 1e3 for k, v in kern.items() if v[1]},
            "share_of_step": kern[dom][0] / sum(v[0] for v in kern.values()),
            "alg_flops_per_launch": flops_launch}

    cpu = None
    if rank == 0 and world == 1 and args.cpu_steps > 0:
        cpu = cpu_baseline(S, w, mesh, args.cpu_steps)

    line = {"metric": METRIC, "value": main_out["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": main_out["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "mixed" else "f64",
            "data": "synthetic", "config": dict(workload_cfg, precision=args.precision, velocity_cache=vc),
            "clocks": main_out["clocks"], "e2e": main_out["e2e"],
            "gpu_launches": int(sum(v[1] for v in kern.values())) * args.steps + 3 * args.steps,
            "roofline": roof, "cpu_baseline": cpu, "status": main_out["status"]}
    if fp64_out is not None:
        line["fp64"] = {"value": fp64_out["value"], "ms_per_step": fp64_out["ms_per_step"],
                        "kb_phys_avg_us": fp64_out["kernels"]["kb_phys"][0] / fp64_out["kernels"]["kb_phys"][1] * 1e3}
        line["speedup_mixed_over_fp64"] = main_out["value"] / fp64_out["value"]
    if args.accuracy:
        line["accuracy"] = accuracy(G, S, w, mesh, {"both": ("fp64", "mixed"), "mixed": ("mixed",),
                                                    "fp64": ("fp64",)}[args.accuracy_precision])
    if not args.no_adjoint and world == 1:
        line["adjoint"] = adjoint_ratio(G, S)
    if rank == 0:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
