"""Kernel-variant autotuner.

Every element type, order and precision has one or more implementations of
the residual and update kernels (fr_params.variant; fr_kernel_variants gives
the count), all equal to round-off.  measure() times each variant on a field
of the caller's workload with CUDA events around a window of RK4 steps (after
warm-up steps), and tune() keeps the fastest per (element type, order,
precision) in tuning.json beside this file.  Fields built with
variant="auto" (the binding's default) take the table's entry, else 0.
"""
import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "tuning.json")
ETYPE_NAMES = {0: "quad", 1: "tri", 2: "hex"}


def key(etype, order, precision):
    et = ETYPE_NAMES.get(etype, etype)
    prec = "mixed" if precision in ("mixed", 1) else "fp64"
    return f"{et}_p{int(order)}_{prec}"


def load():
    if not os.path.exists(TABLE):
        return {}
    with open(TABLE) as f:
        return json.load(f)


def lookup(etype, order, precision):
    """The table's variant for the key, else 0."""
    ent = load().get(key(etype, order, precision))
    return int(ent["variant"]) if ent else 0


def measure(workload, precision="mixed", steps=400, warmup=100, mesh=None):
    """Microseconds per RK stage of every kernel variant on the workload's field."""
    import torch
    from . import Field, Mesh, kernel_variants, make_params
    m = mesh if mesh is not None else workload.mesh()
    M = Mesh.from_synthetic(m, workload.order)
    out = {}
    stream = torch.cuda.current_stream()
    for v in range(kernel_variants(M, precision)):
        F = Field(M, make_params(workload, precision, variant=v), ic=workload.circle, precondition=True)
        F.step(warmup)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        F.step(steps)
        e1.record(stream)
        e1.synchronize()
        if F.sync() != 0:
            raise RuntimeError(f"variant {v}: non-zero field status")
        out[v] = e0.elapsed_time(e1) * 1e3 / (4 * steps)
    return M.info, out


def tune(workloads, precision="mixed", write=True, **kw):
    """Measure every workload's variants and record the fastest; returns the table."""
    table = load()
    for w in workloads:
        info, us = measure(w, precision, **kw)
        best = min(us, key=us.get)
        table[key(info.etype, info.order, precision)] = {
            "variant": int(best), "us_per_stage": {str(v): t for v, t in us.items()},
            "elements": int(info.n_elems), "workload": getattr(w, "name", "")}
    if write:
        with open(TABLE, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
    return table


def _ensemble_probe(S, p, n=96, seed=3):
    """A periodic n^2 quad instance of order p with a random-phase stream
    velocity, the shape of the ensemble's instances."""
    import numpy as np
    rng = np.random.default_rng(seed)
    vel = S.workloads.random_phase_stream(rng)
    h = 1.0 / n
    w = S.Workload(f"ensemble_probe_quad{n}_p{p}", (lambda n=n: S.quad_grid(n)), p, vel,
                   S.Circle((0.5, 0.5), 0.15, 3 * p / (4 * h)), t_end=4.0, h=h, precision="mixed")
    return S.workloads._finish(w, 2)


if __name__ == "__main__":
    import sys
    sys.path.insert(0, os.path.dirname(HERE))
    import synthetic as S
    names = sys.argv[1:] or ["c3", "c2q", "c2t", "ens2", "ens3", "ens4", "ens5"]
    ws = []
    for n in names:
        ws.append(_ensemble_probe(S, int(n[3:])) if n.startswith("ens") else S.workload(n))
    print(json.dumps(tune(ws), indent=1))
