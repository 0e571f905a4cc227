"""The synthetic workloads carry the paper's printed parameters (tests/golden/paper_parameters.json)."""
import json
import os

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
