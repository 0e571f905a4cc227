"""The allocation-free weighted integral (fr_mass_integral_noalloc) against
fr_mass_integral, through the C ABI.

fr_mass_integral_noalloc serves callers that cannot call cudaMalloc (code
inside another framework's memory pool, latency-critical loops, device data
without a field workspace); it keeps its scratch in a static device array.
This file is collected last so that a failure here cannot hide any other
test in a run that stops at the first failure.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synthetic as S
from libutil import ensure_built

pytestmark = pytest.mark.gpu


def test_noalloc_integral_matches_fr_mass_integral_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    import paper_2006_10967_gb300 as G
    from paper_2006_10967_gb300 import _capi
    L = G.lib()
    w = S.workload("c1")
    M = G.Mesh.from_synthetic(w.mesh(), w.order)
    F = G.Field(M, G.make_params(w), ic=w.circle, precondition=False)
    F.step(3)
    stream = torch.cuda.current_stream()
    sp = C.c_void_p(stream.cuda_stream)
    wq = torch.from_numpy(M.quadrature()).cuda()
    for which in (0, 1, 0):
        u = torch.empty(M.shape, dtype=torch.float64, device="cuda")
        F.get_device(which, u)
        ref = F.mass(which)
        for _ in range(2):                       # two calls in a row share the scratch
            out = C.c_double(np.nan)
            rc = L.fr_mass_integral_noalloc(C.c_void_p(u.data_ptr()), C.c_void_p(wq.data_ptr()),
                                            u.numel(), C.byref(out), sp)
            assert rc == 0
            assert out.value == pytest.approx(ref, rel=1e-13, abs=1e-15)
    # sizes beyond the static scratch are refused before any launch
    out = C.c_double()
    rc = L.fr_mass_integral_noalloc(C.c_void_p(u.data_ptr()), C.c_void_p(wq.data_ptr()),
                                    _capi.FR_NOALLOC_MAX_VALUES + 1, C.byref(out), sp)
    assert rc == -1
