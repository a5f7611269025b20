"""GPU parity of the Hartree-Fock loop (qa_hf_solve) and the quasiparticle
quantities (qa_qp) against the oracle (oracle/qp.py).

Hartree-Fock: both sides iterate the same map from the Fermi-Dirac density of
H0 and stop at max |Sigma^HF_new - Sigma^HF_old| <= 1e-10, so their results
lie within ~1e-10 (times the contraction factor) of the same fixed point; the
iteration counts may differ by one where the last change sits next to tol.
All workloads below are metallic at their temperature (dN/dmu >= 0.24), so mu
is fixed to ~1e-11 by the filling and the HF Green's functions are comparable.

Quasiparticles: after one GW step from G0 on both sides (their Sigma's agree
to 1e-10, tests/test_gpu_parity.py), Z, Sigma(0), H_QP and the QP energies are
compared element by element.  Bounds: FP64 1e-8 relative (the Matsubara
difference quotient divides by 2 w0 = 2 pi / beta); mixed 1e-4 (Sigma^C(k, i w)
in complex64 carries 1e-5 relative error, test_gpu_parity.FP32_BOUND).
"""
import functools

import numpy as np
import pytest

import workloads as wl
from oracle import gw, lattice, qp

pytestmark = pytest.mark.gpu

HF_CASES = [("square-8x8", 1.0), ("peierls-3x3", 1.0), ("peierls-5x3x2", 1.0),
            ("graphene-6x6", 1.0), ("five-orbital-4x3x2", 0.5), ("five-orbital-6x5x1", 0.5),
            ("square-1x1", 1.0)]
QP_CASES = ["square-8x8", "peierls-3x3", "peierls-5x3x2", "graphene-6x6", "five-orbital-4x3x2",
            "five-orbital-6x5x1", "square-1x1"]
HF_TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_22223_gb300 import build
    build()


def rel(gpu, ref):
    return float(np.abs(np.asarray(gpu) - ref).max() / max(np.abs(ref).max(), 1e-300))


@functools.lru_cache(maxsize=None)
def oracle_hf(name, mix):
    m = wl.config(name)
    d = gw.make_dlr(m)
    res = qp.hf_loop(m, tol=HF_TOL, max_iter=500, mix=mix)
    G = qp.hf_green(m, d, res["mu"], res["sig_hf_k"])
    return m, d, res, G


@functools.lru_cache(maxsize=None)
def oracle_qp(name):
    m = wl.config(name)
    d = gw.make_dlr(m)
    G0, _ = gw.g0(m, d)
    o = gw.gw_step(m, d, G0)
    return m, d, o, qp.quasiparticle(m, d, o["sig_hf_k"], o["sigc_kiw"])


@pytest.mark.parametrize("name,mix", HF_CASES)
def test_hf_solve(name, mix):
    from paper_2604_22223_gb300 import qa
    m, d, res, G_ref = oracle_hf(name, mix)
    ctx = qa.Context(m, "fp64")
    G, mu, n_loc, iters, resid, status = ctx.hf_solve(500, HF_TOL, mix)
    assert status == 0 and resid <= HF_TOL
    assert abs(iters - res["iters"]) <= 1, (iters, res["iters"])
    sig = ctx.get(qa.QA_SIGHF_K).cpu().numpy()
    assert rel(sig, res["sig_hf_k"]) <= 1e-8
    assert abs(mu - res["mu"]) <= 1e-8 * max(1.0, abs(res["mu"]))
    n_ref = res["n_k"].mean(axis=0)
    assert np.abs(n_loc - n_ref).max() <= 1e-8
    assert rel(G.cpu().numpy(), np.moveaxis(G_ref, 0, -1)) <= 1e-8
    # filling of the HF solution
    assert abs(m.s_spin * np.trace(n_loc).real - m.filling) <= 1e-8


def test_hf_then_gw_step_and_qp():
    """The HF G starts a GW step; qa_qp after qa_hf_solve uses Sigma^HF alone (Z = 1)."""
    from paper_2604_22223_gb300 import qa
    m, d, res, G_ref = oracle_hf("peierls-3x3", 1.0)
    ctx = qa.Context(m, "fp64")
    G, mu, n_loc, iters, resid, status = ctx.hf_solve(500, HF_TOL, 1.0)
    q = ctx.qp()
    no = m.norb
    Z = q["Z"].cpu().numpy()
    assert np.abs(Z - np.eye(no)[None]).max() == 0.0
    ref = qp.quasiparticle(m, d, res["sig_hf_k"], np.zeros((m.nk, d.r, no, no), complex))
    assert rel(q["Hqp"].cpu().numpy(), ref["Hqp"]) <= 1e-8
    assert rel(q["eps"].cpu().numpy(), ref["eps"]) <= 1e-8
    # a GW step from the HF G against the oracle's step from its own HF G
    o = gw.gw_step(m, d, G_ref)
    G1, mu1, n1, st = ctx.step(G)
    assert rel(G1.cpu().numpy(), np.moveaxis(o["G_ktau"], 0, -1)) <= 1e-8
    assert abs(mu1 - o["mu"]) <= 1e-8 * max(1.0, abs(o["mu"]))


def test_hf_not_converged_reports_enoconv():
    from paper_2604_22223_gb300 import qa
    m, d, res, _ = oracle_hf("five-orbital-4x3x2", 0.5)
    assert res["iters"] > 3
    ctx = qa.Context(m, "fp64")
    _, _, _, iters, resid, status = ctx.hf_solve(3, HF_TOL, 0.5, check=False)
    assert status == 4 and iters == 3 and resid > HF_TOL
    with pytest.raises(qa.QAError):
        ctx.hf_solve(3, HF_TOL, 0.5)
    with pytest.raises(qa.QAError):
        ctx.hf_solve(10, HF_TOL, 0.0)       # mix outside (0, 1]


def _compare_qp(q, ref, bound):
    errs = {"Z": rel(q["Z"].cpu().numpy(), ref["Z"]),
            "sig0": rel(q["sig0"].cpu().numpy(), ref["sig0"]),
            "Hqp": rel(q["Hqp"].cpu().numpy(), ref["Hqp"]),
            "eps": rel(q["eps"].cpu().numpy(), ref["eps"])}
    assert max(errs.values()) <= bound, errs
    return errs


@pytest.mark.parametrize("name", QP_CASES)
def test_qp_fp64(name):
    from paper_2604_22223_gb300 import qa
    m, d, o, ref = oracle_qp(name)
    ctx = qa.Context(m, "fp64")
    with pytest.raises(qa.QAError):
        ctx.qp()                            # no self-energy yet
    ctx.step()
    q = ctx.qp()
    _compare_qp(q, ref, 1e-8)
    # Z is Hermitian positive definite with eigenvalues in (0, 1] for a causal Sigma
    Z = q["Z"].cpu().numpy()
    lam = np.linalg.eigvalsh(0.5 * (Z + np.conj(np.swapaxes(Z, 1, 2))))
    assert lam.min() > 0 and lam.max() <= 1 + 1e-12


@pytest.mark.parametrize("name", ["peierls-5x3x2", "five-orbital-4x3x2", "graphene-6x6"])
def test_qp_fp32(name):
    from paper_2604_22223_gb300 import qa
    m, d, o, ref = oracle_qp(name)
    ctx = qa.Context(m, "fp32")
    ctx.step()
    _compare_qp(ctx.qp(), ref, 1e-4)


def test_paper_graphene_workflow():
    """The paper's graphene validation model (t = 1, U = 2, V = 0.2 eV, 2000 K,
    25x25x1): HF -> GW step from the HF G -> quasiparticles, each against the
    oracle, with the particle-hole value mu = U/2 + 3V (tests/test_golden_paper.py)."""
    from paper_2604_22223_gb300 import qa
    m, d, res, G_ref = oracle_hf("graphene-paper-25x25", 1.0)
    mu_ph = 2.0 / 2 + 3 * 0.2
    ctx = qa.Context(m, "fp64")
    G, mu, n_loc, iters, resid, status = ctx.hf_solve(200, HF_TOL, 1.0)
    assert abs(mu - mu_ph) <= 1e-10
    assert rel(ctx.get(qa.QA_SIGHF_K).cpu().numpy(), res["sig_hf_k"]) <= 1e-9
    assert rel(G.cpu().numpy(), np.moveaxis(G_ref, 0, -1)) <= 1e-9
    o = gw.gw_step(m, d, G_ref)
    G1, mu1, n1, st = ctx.step(G)
    assert abs(mu1 - mu_ph) <= 1e-8
    assert rel(G1.cpu().numpy(), np.moveaxis(o["G_ktau"], 0, -1)) <= 1e-9
    ref = qp.quasiparticle(m, d, o["sig_hf_k"], o["sigc_kiw"])
    _compare_qp(ctx.qp(), ref, 1e-8)


@pytest.mark.parametrize("precision,bound", [("fp64", 1e-8), ("fp32", 1e-4)])
def test_paper_five_orbital_step_and_qp(precision, bound):
    """The paper's degenerate five-orbital benchmark model on a 3x3x2 grid."""
    from paper_2604_22223_gb300 import qa
    m, d, o, ref = oracle_qp("five-orbital-paper-3x3x2")
    ctx = qa.Context(m, precision)
    G1, mu1, n1, st = ctx.step()
    assert abs(mu1 - o["mu"]) <= (1e-10 if precision == "fp64" else 2e-5) * max(1.0, abs(o["mu"]))
    _compare_qp(ctx.qp(), ref, bound)


def test_paper_five_orbital_hf_half_filling():
    """qa_hf_solve on the paper's five-orbital model (8x8x8) reaches the
    particle-hole value mu = 9.5 (tests/test_golden_paper.py)."""
    from paper_2604_22223_gb300 import qa
    m = wl.config("five-orbital-paper-8x8x8")
    ctx = qa.Context(m, "fp32")
    G, mu, n_loc, iters, resid, status = ctx.hf_solve(200, 1e-12, 1.0)
    assert abs(mu - 9.5) <= 1e-10
    # n_loc is the DLR density -G(beta^-) of the HF G (eps = 1e-10 grid at beta Lambda = 2500)
    assert np.abs(np.diag(n_loc) - 0.5).max() <= 1e-8


def test_bench_size_hf_and_qp_properties():
    """The benchmark configuration (five-orbital 32x32x8, mixed context as bench.py runs
    it): qa_hf_solve against the oracle's loop element by element, and after one GW
    step the quasiparticle quantities satisfy what holds at any size: Z Hermitian with
    eigenvalues in (0, 1], H_QP Hermitian, eps ascending and equal to its eigenvalues."""
    from paper_2604_22223_gb300 import qa
    m = wl.config("five-orbital-32x32x8")
    res = qp.hf_loop(m, tol=HF_TOL, max_iter=200, mix=1.0)
    ctx = qa.Context(m, "fp32")
    G, mu, n_loc, iters, resid, status = ctx.hf_solve(200, HF_TOL, 1.0)
    assert status == 0 and abs(iters - res["iters"]) <= 1
    assert rel(ctx.get(qa.QA_SIGHF_K).cpu().numpy(), res["sig_hf_k"]) <= 1e-8
    assert abs(mu - res["mu"]) <= 1e-8 * max(1.0, abs(res["mu"]))
    ctx.step(G)
    q = {k: v.cpu().numpy() for k, v in ctx.qp().items()}
    herm = lambda X: np.abs(X - np.conj(np.swapaxes(X, 1, 2))).max() / np.abs(X).max()
    assert herm(q["Z"]) <= 1e-12 and herm(q["Hqp"]) <= 1e-12
    lam = np.linalg.eigvalsh(q["Z"])
    assert lam.min() > 0 and lam.max() <= 1 + 1e-6     # complex64 Sigma^C: ~1e-7 noise
    assert np.all(np.diff(q["eps"], axis=1) >= 0)
    assert np.abs(np.linalg.eigvalsh(q["Hqp"]) - q["eps"]).max() <= 1e-9 * np.abs(q["eps"]).max()
