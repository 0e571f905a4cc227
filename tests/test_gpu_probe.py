"""The two forms of the hexahedral operator applies (fr_probe_hex_apply):
sum factorisation along lines and the dense operator on the tensor cores.

Both are checked, through the C ABI, against the flux-point traces and
reference derivatives (Section 3.1, Step 1 Eq. extrapolateSoln and the
derivative part of Step 3 Eq. continuousGrad) formed here in FP64 from the
oracle's 1D Gauss-Legendre Lagrange operators, on element counts that leave
ragged last tiles in both forms (32 and 64 elements per tile).  Tolerance
1e-5 of the largest value: FP32 dot products of four terms with operator
entries up to ~8 (form 0), three-term TF32 products (relative 2^-22) summed
in FP32 (form 1).
"""
import ctypes as C

import numpy as np
import pytest
import torch

from libutil import ensure_built
from oracle.polys import gauss_legendre, lagrange_matrix

pytestmark = pytest.mark.gpu
N = 4


def _expected(u):
    """(E, 2, 288) traces and derivatives of u (E, 2, 64), point i0 + 4 i1 + 16 i2."""
    x, _ = gauss_legendre(N)
    Le = lagrange_matrix(x, np.array([-1.0, 1.0]))   # (2, N): l_j(-1), l_j(+1)
    D = lagrange_matrix(x, x, deriv=True)             # D[i, j] = l_j'(x_i)
    E = u.shape[0]
    U = u.reshape(E, 2, N, N, N)                      # [.., i2, i1, i0]
    tr = [np.einsum("sj,efzyj->efszy", Le, U),        # axis 0: face point i1 + 4 i2
          np.einsum("sj,efzjx->efszx", Le, U),        # axis 1: i0 + 4 i2
          np.einsum("sj,efjyx->efsyx", Le, U)]        # axis 2: i0 + 4 i1
    dv = [np.einsum("xm,efzym->efzyx", D, U),
          np.einsum("ym,efzmx->efzyx", D, U),
          np.einsum("zm,efmyx->efzyx", D, U)]
    parts = [t.reshape(E, 2, 2 * N * N) for t in tr] + [d.reshape(E, 2, N ** 3) for d in dv]
    return np.concatenate(parts, axis=2)


def _apply(L, form, reduce, u, E):
    n = E * 2 * (1 if reduce else 288)
    out = torch.full((max(n, 1),), float("nan"), device="cuda")
    sp = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.fr_probe_hex_apply(3, form, reduce, C.c_void_p(u.data_ptr()), E, C.c_void_p(out.data_ptr()), n, sp)
    assert rc == 0, rc
    torch.cuda.synchronize()
    return out[:n].cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("E", [1, 37, 131, 2000])
def test_both_forms_match_the_1d_operators(E):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    import paper_2006_10967_gb300 as G
    L = G.lib()
    g = torch.Generator().manual_seed(100 + E)
    u = torch.randn(E, 2, 64, generator=g, dtype=torch.float32)
    ref = _expected(u.double().numpy())
    scale = np.abs(ref).max()
    ud = u.cuda()
    full = {}
    for form in (0, 1):
        got = _apply(L, form, 0, ud, E).reshape(E, 2, 288)
        assert np.isfinite(got).all(), form
        err = np.abs(got - ref).max() / scale
        assert err < 1e-5, (form, err)
        full[form] = got
        red = _apply(L, form, 1, ud, E).reshape(E, 2)
        rerr = np.abs(red - ref.sum(axis=2)).max() / np.abs(ref).sum(axis=2).max()
        assert rerr < 1e-5, (form, rerr)
    assert np.abs(full[0] - full[1]).max() / scale < 1e-5
