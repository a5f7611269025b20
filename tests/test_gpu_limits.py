"""GPU runs at the limits the ABI accepts (include/qa.h): the largest k-grid
(N_k = 12288, mixed-radix FFT axes) and a DLR rank near the maximum of 128
(r = 98, where the mixed path leaves the tensor-core DLR kernel, 2r > 186, for the
SIMT one).

* Largest grid: the oracle is too slow there, so the two precisions are checked
  against each other (the FP64 path meets the oracle to 1e-10 elsewhere): mu,
  the local density and G of one iteration from G0, at the mixed path's bounds.
* Largest rank: one iteration of the two-orbital Peierls model (complex hoppings)
  against the oracle, element by element on the imaginary-time nodes (G(k, tau),
  Sigma^C(k, tau)) and mu.  At this Lambda the last Matsubara nodes the two sides
  pick can differ by one frequency where the pivoting meets near-ties (the library
  on an Arm host versus numpy), so Matsubara-node arrays are not compared; any
  such node set is a valid DLR basis and the tau-node results agree.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import gw

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_22223_gb300 import build
    build()


def rel(a, b):
    return float(np.abs(np.asarray(a) - b).max() / max(np.abs(b).max(), 1e-300))


def test_largest_grid_fp64_vs_fp32():
    from paper_2604_22223_gb300 import qa
    m = wl.config("peierls-3x3")
    m.n = (16, 32, 24)                        # N_k = 12288, the largest accepted grid
    out = {}
    for prec in ("fp64", "fp32"):
        ctx = qa.Context(m, prec)
        assert ctx.nk == 12288
        G, mu, n_loc, st = ctx.step()
        assert st["status"] == 0
        out[prec] = (G.cpu().numpy(), mu, n_loc, st["N"])
        del ctx
    G64, mu64, n64, N64 = out["fp64"]
    G32, mu32, n32, N32 = out["fp32"]
    assert abs(N64 - m.filling) <= 1e-10
    assert np.all(np.isfinite(G64)) and np.all(np.isfinite(G32))
    assert abs(mu32 - mu64) <= 2e-5 * max(1.0, abs(mu64))
    assert rel(G32, G64) <= 1e-4
    assert np.abs(n32 - n64).max() <= 2e-5


@pytest.fixture(scope="module")
def high_rank():
    m = wl.config("peierls-3x3")
    # Lambda 3e4 at the bench's eps 1e-12 (r = 98).  Tighter eps makes the DLR node
    # matrices too ill-conditioned for an FP64 reference (cond(K_tau) ~ 1e15 at 1e-14),
    # and the node selection's host cost grows with Lambda squared.
    m.Lambda, m.eps_dlr = 3.0e4, 1e-12
    d = gw.make_dlr(m)
    G0, mu0 = gw.g0(m, d)
    return m, d, gw.gw_step(m, d, G0)


@pytest.mark.parametrize("prec,bound", [("fp64", 1e-9), ("fp32", 1e-3)])
def test_largest_rank_against_oracle(high_rank, prec, bound):
    from paper_2604_22223_gb300 import qa
    m, d, o = high_rank
    ctx = qa.Context(m, prec)
    assert ctx.r == d.r and d.r > 93                  # beyond the tensor-core kernel's limit
    G, mu, n_loc, st = ctx.step()
    k_last = lambda x: np.moveaxis(x, 0, -1)
    grid = ctx.grid()
    assert np.array_equal(grid["t"], d.t) and np.array_equal(grid["x"], d.x)
    errs = {"G": rel(G.cpu().numpy(), k_last(o["G_ktau"])),
            "sigc_ktau": rel(ctx.get(qa.QA_SIGC_KTAU).cpu().numpy(), k_last(o["sigc_ktau"])),
            "mu": abs(mu - o["mu"]) / max(1.0, abs(o["mu"]))}
    print(prec, d.r, errs)
    assert max(errs.values()) <= bound, errs
