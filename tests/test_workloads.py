"""The synthetic workloads carry the paper's printed parameters (tests/golden/paper_parameters.json)."""
import json
import math
import os

import numpy as np
import pytest

import synthetic as S

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")))


@pytest.mark.parametrize("name", ["c2q", "c2t", "c3"])
def test_paper_parameters(name):
    w = S.workload(name)
    assert w.gamma == GOLD["gamma"]["value"]
    assert w.eps == pytest.approx(GOLD["eps_over_h_per_p"]["value"] * w.h / w.order)
    assert w.circle.beta == pytest.approx(GOLD["ic_beta_times_h_per_p"]["value"] * w.order / w.h)
    assert w.s0 == GOLD["s0"]["value"]
    assert w.nu_max == pytest.approx(GOLD["nu_max_over_h_per_p"]["value"] * w.h / w.order)
    assert w.n_precond == GOLD["precondition_every"]["value"]
    assert w.pseudo_tol == GOLD["pseudo_stop_rms"]["value"]
    lo, hi = GOLD["pseudo_iterations_typical"]["value"]
    assert w.pseudo_kmax == hi
    assert w.circle.radius == GOLD["disc_radius"]["value"]


def test_benchmark_geometry():
    w = S.workload("c2q")
    assert tuple(w.circle.centre) == tuple(GOLD["rider_kothe_centre"]["value"])
    assert w.velocity.T == GOLD["rider_kothe_period"]["value"]
    w3 = S.workload("c3")
    assert tuple(w3.circle.centre) == tuple(GOLD["leveque_centre"]["value"])
    assert w3.velocity.T == GOLD["leveque_period"]["value"]
    # the time step lands exactly on t_end
    assert w.dt * w.n_steps == pytest.approx(w.t_end, rel=1e-12)


def test_meshes_are_valid():
    m = S.workload("c2t").mesh()
    assert 29000 < m.n_elems < 30500
    p = m.nodes[m.conn]
    area2 = ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1])
             - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1]))
    assert (area2 > 0).all()
    q = S.quad_grid(8, jitter=0.1, seed=1, shuffle_seed=11, rotate_seed=12)
    assert q.n_elems == 64


@pytest.mark.parametrize("name,key", [("zalesak", "zalesak_disc"), ("rudman", "rudman_disc")])
def test_slotted_disk_workloads(name, key):
    """Section 4.1: slotted disks in solid-body rotation for one revolution."""
    g = GOLD[key]["value"]
    w = S.workload(name)
    c = w.circle
    assert isinstance(c, S.SlottedDisk)
    assert c.radius == g["radius"] and tuple(c.centre) == tuple(g["centre"])
    assert c.half_width == g["slot_half_width"] and c.top == g["slot_top"]
    assert tuple(w.velocity.a[:2]) == tuple(g["rotation_centre"])
    assert w.t_end == pytest.approx(2 * math.pi)
    assert w.h == pytest.approx(g["domain"] / 100 if name == "zalesak" else g["domain"] / 200)
    assert c.beta == pytest.approx(GOLD["ic_beta_times_h_per_p"]["value"] * w.order / w.h)
    assert w.eps == pytest.approx(GOLD["eps_over_h_per_p"]["value"] * w.h / w.order)
    m = w.mesh()
    assert np.allclose(m.nodes.max(0), g["domain"]) and np.allclose(m.nodes.min(0), 0.0)


def test_slotted_disk_signed_distance_closed_forms():
    c = S.SlottedDisk((0.5, 0.75), 0.15, 0.025, 0.85, 100.0)
    pts = np.array([[0.5, 0.75],      # in the slot: -distance to its nearer wall
                    [0.4, 0.75],      # beside the slot, inside the disk: distance to the circle
                    [0.5, 0.88],      # above the slot top: distance to the slot top
                    [0.51, 0.86],     # above the slot, near its top
                    [0.535, 0.85],    # beside the slot's top corner
                    [0.9, 0.1]])      # far outside
    d = c.signed_distance(pts)
    expect = [-0.025, 0.05, 0.02, 0.01, 0.01, 0.15 - math.hypot(0.4, 0.65)]
    assert np.allclose(d, expect, atol=1e-15)


def test_slotted_disk_area():
    """The region d > 0 has the slotted disk's area: pi r^2 minus the slot's part
    of the disk, int_{-w}^{w} (top - c_y + sqrt(r^2 - s^2)) ds."""
    from scipy.integrate import quad
    for cx, cy, r, w_, top, L in ((0.5, 0.75, 0.15, 0.025, 0.85, 1.0), (2.0, 2.75, 0.5, 0.06, 2.65, 4.0)):
        c = S.SlottedDisk((cx, cy), r, w_, top, 1.0)
        slot, _ = quad(lambda s: top - cy + math.sqrt(r * r - s * s), -w_, w_)
        area = math.pi * r * r - slot
        n = 4000
        g = (np.arange(n) + 0.5) * (L / n)
        X, Y = np.meshgrid(g, g, indexing="ij")
        inside = c.signed_distance(np.stack([X, Y], -1)) > 0
        assert inside.sum() * (L / n) ** 2 == pytest.approx(area, rel=2e-3)


def test_rotation_velocity_about_a_centre():
    """Solid-body rotation with unit angular velocity about (a0, a1) (Section 4.1)."""
    import torch
    from oracle.solver import velocity
    vel = S.Velocity("rotation", a=(2.0, 2.0, 0.0))
    x = torch.tensor([[2.0, 2.0], [3.0, 2.0], [2.0, 3.5], [0.5, 1.0]], dtype=torch.float64)
    v = velocity(vel, x, 0.7)
    expect = torch.tensor([[0.0, 0.0], [0.0, 1.0], [-1.5, 0.0], [1.0, -1.5]], dtype=torch.float64)
    assert torch.equal(v, expect)


def test_split_triangle_family():
    """Section 4.2's "c" meshes: n x n squares split along a diagonal, h = 1/n
    (sqrt(2 |Omega| / E))."""
    for n in (32, 64):
        w = S.workload("c2s", n=n, p=4)
        m = w.mesh()
        assert m.etype == "tri" and m.n_elems == 2 * n * n
        assert w.h == pytest.approx(math.sqrt(2.0 / m.n_elems))
        assert w.circle.beta == pytest.approx(GOLD["ic_beta_times_h_per_p"]["value"] * w.order / w.h)
        assert tuple(w.circle.centre) == tuple(GOLD["rider_kothe_centre"]["value"])
