"""Failure paths of qa_gw_step, made to happen without any GPU fault.

* QA_ESINGULAR: a local interaction tuned on the host so that the screened-
  interaction system 1 - U P(q*, nu = 0) has an exactly cancelling pivot at the
  q* where the static bubble is largest (attractive U = 1 / P(q*, 0), the RPA
  instability of the single-band square lattice); the step reports the status
  and the failing system index nu * N_k + q*.
* QA_ETIMEOUT: qa_set_wait_limit(0) makes every pipeline wait of the tensor-core
  DLR kernels give up at once; the step reports the time-out, the kernels
  release their tensor memory and return, and the next step with the default
  limit reproduces a clean step.
* A non-finite input G: the step fails with a status (the NaN reaches the Dyson
  pivots), and the context stays usable.
"""
import copy

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

QA_ESINGULAR, QA_ERANGE, QA_ETIMEOUT = 3, 5, 6


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_22223_gb300 import build
    build()


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
def test_singular_screened_interaction_reported(prec):
    from paper_2604_22223_gb300 import qa
    m = wl.config("square-8x8")
    ctx = qa.Context(m, prec)
    _, _, _, st = ctx.step()
    assert st["status"] == 0
    mb = ctx.grid()["mb"]
    assert 0 in list(mb), "the bosonic DLR nodes include nu = 0"
    nu0 = list(mb).index(0)
    P = ctx.get(qa.QA_P_QNU).cpu().numpy()[nu0, 0, 0]          # P(q, nu = 0), [N_k]
    qs = int(np.argmax(np.abs(P)))
    assert abs(P[qs].imag) <= 1e-9 * abs(P[qs].real)
    Uc = 1.0 / P[qs].real                                        # 1 - Uc P(q*, 0) = 0
    m2 = copy.copy(m)
    m2.V = np.asarray(m.V) * (Uc / m.V[0][0, 0].real)
    ctx.set_params(m2)
    _, _, _, st = ctx.step(check=False)
    assert st["call_status"] == QA_ESINGULAR, st
    assert st["first_bad"] == nu0 * m.nk + qs, (st["first_bad"], nu0, qs)
    # back to the original interaction: the context is usable
    ctx.set_params(m)
    _, _, _, st = ctx.step()
    assert st["status"] == 0


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
def test_timeout_path_releases_and_recovers(prec):
    from paper_2604_22223_gb300 import qa
    m = wl.config("peierls-3x3")
    ref = qa.Context(m, prec)
    G_ref, mu_ref, _, _ = ref.step()
    ctx = qa.Context(m, prec)
    ctx.set_wait_limit(0)
    _, _, _, st = ctx.step(check=False)
    assert st["call_status"] == QA_ETIMEOUT, st
    ctx.set_wait_limit(None)
    G, mu, _, st = ctx.step()
    assert st["status"] == 0
    g, gr = G.cpu().numpy(), G_ref.cpu().numpy()
    assert np.abs(g - gr).max() <= 1e-9 * np.abs(gr).max()
    assert abs(mu - mu_ref) <= 1e-9 * max(1.0, abs(mu_ref))


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
def test_non_finite_input_fails_cleanly(prec):
    import torch
    from paper_2604_22223_gb300 import qa
    m = wl.config("peierls-3x3")
    ctx = qa.Context(m, prec)
    G_ref, _, _, _ = ctx.step()
    G = ctx.get(qa.QA_G0).clone()
    G[0, 0, 0, 0] = complex(float("nan"), 0.0)
    _, _, _, st = ctx.step(G, check=False)
    assert st["call_status"] in (QA_ESINGULAR, QA_ERANGE), st
    G1, _, _, st = ctx.step()
    assert st["status"] == 0
    assert torch.isfinite(torch.view_as_real(G1)).all()
    # the recovered step starts its mu search elsewhere: equal within the search's
    # tolerance (FP32 densities carry ~1e-6 noise on the FP32 path)
    tol = 1e-5 if prec == "fp32" else 1e-9
    assert np.abs(G1.cpu().numpy() - G_ref.cpu().numpy()).max() <= tol * np.abs(G_ref.cpu().numpy()).max()
