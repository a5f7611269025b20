"""qa_density_static: the density without any device allocation.

Callers that cannot call cudaMalloc (host callbacks, error handlers,
plug-ins inside a framework that owns every device allocation, real-time
loops) use this entry point; its scratch is a static __device__ array.  The
test calls it through the C ABI on two different G's in a row and checks it
against qa_density (which uses the context's workspace).  The file name makes
pytest collect it last.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


def _static_density(L, ctx, G, stream):
    n = np.zeros(2 * ctx.norb * ctx.norb)
    N = C.c_double()
    status = L.qa_density_static(ctx.ctx, G.data_ptr(), n.ctypes.data, C.byref(N), stream)
    return status, n.view(np.complex128).reshape(ctx.norb, ctx.norb), N.value


def test_density_static_matches_workspace_path():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_22223_gb300 import build, qa
    build()
    L = qa.load()
    m = wl.config("five-orbital-6x5x1")
    ctx = qa.Context(m, "fp64")
    G0 = ctx.get(qa.QA_G0)
    G1, _, _, _ = ctx.step()
    stream = ctx._stream()
    for G in (G0, G1):                       # two calls in a row on different inputs
        status, n_static, N_static = _static_density(L, ctx, G, stream)
        assert status == 0, qa.strerror(status)
        n_ref, N_ref = ctx.density(G)
        assert np.abs(n_static - n_ref).max() <= 1e-12 * max(1.0, np.abs(n_ref).max())
        assert abs(N_static - N_ref) <= 1e-12 * max(1.0, abs(N_ref))
    # a context from qa_create alone (no workspace) works too
    prob = qa.Problem(m, "fp64")
    status, n_p, N_p = _static_density(L, prob, G1, stream)
    assert status == 0 and abs(N_p - N_ref) <= 1e-12 * max(1.0, abs(N_ref))
    # the 32x32x8 benchmark grid fits the 4 MiB static scratch (25 * 8192 * 16 B) ...
    big = qa.Problem(wl.five_orbital(n=(32, 32, 8), Lambda=100.0), "fp64")
    Gbig = torch.zeros((big.r, 5, 5, big.nk), dtype=torch.complex128, device="cuda")
    status, _, N_big = _static_density(L, big, Gbig, stream)
    assert status == 0 and N_big == 0.0
    # ... and a 32x32x12 grid (4.9 MB of n(k)) is rejected with QA_ENOMEM
    huge = qa.Problem(wl.five_orbital(n=(32, 32, 12), Lambda=100.0), "fp64")
    Ghuge = torch.zeros((huge.r, 5, 5, huge.nk), dtype=torch.complex128, device="cuda")
    status, _, _ = _static_density(L, huge, Ghuge, stream)
    assert status == 2
