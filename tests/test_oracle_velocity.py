"""Pins of the oracle's velocity fields (Sections 4.1-4.3) against their
defining properties, by central differences of independently written stream
functions: Rider-Kothe and the Fourier stream-function field are the rotated
gradients of their stream functions, every field is divergence free, and the
time factor cos(pi t / T) reverses the flow (u(T - t) = -u(t), u(T/2) = 0)."""
import math

import numpy as np
import pytest
import torch

import synthetic as S
from oracle.solver import velocity

H = 1e-5


def _pts(d, n=40, seed=0):
    return torch.as_tensor(np.random.default_rng(seed).random((n, d)), dtype=torch.float64)


def _fd_grad(f, x):
    g = []
    for a in range(x.shape[-1]):
        e = torch.zeros_like(x)
        e[..., a] = H
        g.append((f(x + e) - f(x - e)) / (2 * H))
    return torch.stack(g, -1)


def _divergence(vel, x, t):
    div = torch.zeros(x.shape[:-1], dtype=torch.float64)
    for a in range(x.shape[-1]):
        e = torch.zeros_like(x)
        e[..., a] = H
        div += (velocity(vel, x + e, t)[..., a] - velocity(vel, x - e, t)[..., a]) / (2 * H)
    return div


def test_rider_kothe_is_the_rotated_gradient_of_its_stream_function():
    vel = S.Velocity("rider_kothe", T=8.0)
    psi = lambda x: torch.sin(math.pi * x[..., 0]) ** 2 * torch.sin(math.pi * x[..., 1]) ** 2 / math.pi
    x = _pts(2)
    g = _fd_grad(psi, x)
    u = velocity(vel, x, 0.0)
    assert torch.allclose(u[..., 0], -g[..., 1], atol=1e-8)
    assert torch.allclose(u[..., 1], g[..., 0], atol=1e-8)


def test_stream_field_is_the_rotated_gradient_of_its_fourier_series():
    kx, ky, A, B = S.stream_coefficients(8, seed=4)
    vel = S.Velocity("stream", T=0.0, kx=kx, ky=ky, A=A, B=B)

    def Psi(x):
        out = torch.zeros(x.shape[:-1], dtype=torch.float64)
        for m in range(len(kx)):
            arg = 2 * math.pi * (kx[m] * x[..., 0] + ky[m] * x[..., 1])
            out += A[m] * torch.sin(arg) + B[m] * torch.cos(arg)
        return out
    x = _pts(2, seed=1)
    g = _fd_grad(Psi, x)
    u = velocity(vel, x, 0.0)
    scale = float(g.abs().max())
    assert torch.allclose(u[..., 0], g[..., 1], atol=1e-7 * scale)
    assert torch.allclose(u[..., 1], -g[..., 0], atol=1e-7 * scale)


@pytest.mark.parametrize("kind,d", [("rider_kothe", 2), ("leveque", 3), ("rotation", 2), ("stream", 2)])
def test_fields_are_divergence_free(kind, d):
    if kind == "stream":
        kx, ky, A, B = S.stream_coefficients(8, seed=4)
        vel = S.Velocity("stream", T=4.0, kx=kx, ky=ky, A=A, B=B)
    elif kind == "rotation":
        vel = S.Velocity("rotation", a=(0.5, 0.5))
    else:
        vel = S.Velocity(kind, T=3.0)
    x = _pts(d, seed=2)
    for t in (0.0, 0.37):
        u = velocity(vel, x, t)
        assert float(_divergence(vel, x, t).abs().max()) < 1e-7 * max(1.0, float(u.abs().max()))


@pytest.mark.parametrize("kind,d", [("rider_kothe", 2), ("leveque", 3)])
def test_time_factor_reverses_the_flow(kind, d):
    T = 3.0
    vel = S.Velocity(kind, T=T)
    x = _pts(d, seed=3)
    for t in (0.1, 0.9, 1.3):
        assert torch.allclose(velocity(vel, x, T - t), -velocity(vel, x, t), atol=1e-14)
    assert float(velocity(vel, x, T / 2).abs().max()) < 1e-15


def test_rotation_is_a_solid_body_rotation():
    c = (0.3, 0.6)
    vel = S.Velocity("rotation", a=c)
    x = _pts(2, seed=4)
    r = x - torch.tensor(c, dtype=torch.float64)
    u = velocity(vel, x, 0.0)
    # u = omega x r with unit angular velocity: perpendicular to r, |u| = |r|
    assert torch.allclose((u * r).sum(-1), torch.zeros(len(x), dtype=torch.float64), atol=1e-15)
    assert torch.allclose(u.norm(dim=-1), r.norm(dim=-1), atol=1e-15)
    assert torch.allclose(u[..., 1] * r[..., 0] - u[..., 0] * r[..., 1], r.norm(dim=-1) ** 2, atol=1e-15)
