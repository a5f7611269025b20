"""GPU parity on the full-size workloads.

* graphene-36x36 and five-orbital-16x16: one iteration from G0, every element of
  P(q, i nu), W^C(R, tau), Sigma^C, Sigma^HF, G and mu against the oracle.
* The mixed path runs on the reduced pair basis (its default): P is compared
  as B^H P B and W^C expanded as B Wt^C B^H.
* peierls-32x32x8 (the benchmark's 32x32x8 grid with the two-orbital Peierls
  model, which the oracle finishes in about a minute): every element of P(q, i nu),
  W^C(R, tau), Sigma^C(k, tau), Sigma^C(k, i w), G and mu in all three precisions,
  so the FFT kernels specialised to the 32x32x8 grid (q -> R, Sigma -> k and the
  fused bubble) are compared with the oracle element by element.
* five-orbital-32x32x8 (the benchmark workload, the launch configuration bench.py
  times): G0, mu0 and Sigma^HF in full; P(q, i nu) at sampled q from the
  oracle's explicit k-sum; and properties that hold at any size: the sum rule
  G(0+) + G(beta-) = -1 of the new G, the filling, and Sigma^C(-k, tau) =
  Sigma^C(k, tau)^T (the model's hoppings are real, t(-R) = t(R)^T).
"""
import numpy as np
import pytest

import workloads as wl
from oracle import gw, lattice

pytestmark = pytest.mark.gpu

FP64 = 1e-10
# The new G and mu depend on the chemical-potential root, which both sides find to
# |N - N_target| <= 1e-12; in the graphene semimetal dN/dmu is small at the Dirac
# points, so mu (and G) carry ~1e-10 of that root tolerance.
FP64_G = 1e-9
# Mixed path (double-float): the stated 1e-7 on Sigma, and on every other output.
MIXED = 1e-7
# FP32 path (the fast mode): FP32 rounding is amplified by the DLR Matsubara -> tau
# maps (W^C, G); G also inherits the mu root found on FP32 densities and refined by
# one FP64 step.
FP32 = {"P_qnu": 2e-6, "WC_Rtau": 2e-4, "sigc_ktau": 2e-4, "sigc_kiw": 2e-5, "sighf": 1e-9,
         "G": 1e-4, "mu": 5e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_22223_gb300 import build
    build()


def kl(x):
    return np.moveaxis(x, 0, -1)


def project_P(ctx, P):
    """B^H P B on the reduced pair basis (the tensor the GPU holds), else P."""
    if not ctx.reduced:
        return P
    return np.einsum("ai,...abk,bj->...ijk", ctx.basis.conj(), P, ctx.basis)


def expand_W(ctx, W):
    """B Wt B^H on the reduced pair basis, else W."""
    if not ctx.reduced:
        return W
    return np.einsum("ai,...ijk,bj->...abk", ctx.basis, W, ctx.basis.conj())


def rel(a, b):
    return float(np.abs(np.asarray(a) - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("name", ["graphene-36x36", "five-orbital-16x16"])
@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
def test_full_step(name, prec):
    from paper_2604_22223_gb300 import qa
    m = wl.config(name)
    d = gw.make_dlr(m)
    G0, mu0 = gw.g0(m, d)
    o = gw.gw_step(m, d, G0)
    ctx = qa.Context(m, prec)
    G, mu, n, st = ctx.step()
    errs = {
        "P_qnu": rel(ctx.get(qa.QA_P_QNU).cpu().numpy(), project_P(ctx, kl(o["P_qnu"]))),
        "WC_Rtau": rel(expand_W(ctx, ctx.get(qa.QA_WC_RTAU).cpu().numpy()), kl(o["WC_Rtau"])),
        "sigc_ktau": rel(ctx.get(qa.QA_SIGC_KTAU).cpu().numpy(), kl(o["sigc_ktau"])),
        "sigc_kiw": rel(ctx.get(qa.QA_SIGC_KIW).cpu().numpy(), kl(o["sigc_kiw"])),
        "sighf": rel(ctx.get(qa.QA_SIGHF_K).cpu().numpy(), o["sig_hf_k"]),
        "G": rel(G.cpu().numpy(), kl(o["G_ktau"])),
        "mu": abs(mu - o["mu"]) / max(1.0, abs(o["mu"])),
    }
    for k, e in errs.items():
        bound = {"fp64": FP64_G if k in ("G", "mu") else FP64, "mixed": MIXED, "fp32": FP32[k]}[prec]
        assert e <= bound, (k, e, bound, errs)


@pytest.fixture(scope="module")
def grid_oracle():
    m = wl.config("peierls-32x32x8")
    d = gw.make_dlr(m)
    G0, mu0 = gw.g0(m, d)
    return m, d, G0, gw.gw_step(m, d, G0)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
def test_benchmark_grid_elementwise(grid_oracle, prec):
    from paper_2604_22223_gb300 import qa
    m, d, G0, o = grid_oracle
    ctx = qa.Context(m, prec)
    G, mu, n, st = ctx.step()
    errs = {
        "P_qnu": rel(ctx.get(qa.QA_P_QNU).cpu().numpy(), project_P(ctx, kl(o["P_qnu"]))),
        "WC_Rtau": rel(expand_W(ctx, ctx.get(qa.QA_WC_RTAU).cpu().numpy()), kl(o["WC_Rtau"])),
        "sigc_ktau": rel(ctx.get(qa.QA_SIGC_KTAU).cpu().numpy(), kl(o["sigc_ktau"])),
        "sigc_kiw": rel(ctx.get(qa.QA_SIGC_KIW).cpu().numpy(), kl(o["sigc_kiw"])),
        "G": rel(G.cpu().numpy(), kl(o["G_ktau"])),
        "mu": abs(mu - o["mu"]) / max(1.0, abs(o["mu"])),
    }
    for k, e in errs.items():
        bound = {"fp64": FP64_G if k in ("G", "mu") else FP64, "mixed": MIXED, "fp32": FP32[k]}[prec]
        assert e <= bound, (k, e, bound, errs)


@pytest.fixture(scope="module")
def bench_oracle():
    m = wl.config("five-orbital-32x32x8")
    d = gw.make_dlr(m)
    G0, mu0 = gw.g0(m, d)
    return m, d, G0, mu0


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
def test_benchmark_grid_sampled(bench_oracle, prec):
    import torch
    from paper_2604_22223_gb300 import qa
    m, d, G0, mu0 = bench_oracle
    ctx = qa.Context(m, prec)
    g0 = ctx.get(qa.QA_G0).cpu().numpy()
    assert rel(g0, kl(G0)) <= FP64                        # G0 is built in FP64 in both modes
    assert abs(ctx.get(qa.QA_MU0) - mu0) <= 1e-10 * max(1.0, abs(mu0))
    G, mu, n, st = ctx.step()
    # Hartree + Fock from the input density, all k
    nk_in = gw.density_from_tau(d, G0)
    sig_h, sig_f = gw.hartree_fock(m, nk_in)
    assert rel(ctx.get(qa.QA_SIGHF_K).cpu().numpy(), sig_h[None] + sig_f) <= 1e-9
    # P(q, i nu) at sampled q by the oracle's explicit k-sum
    P = ctx.get(qa.QA_P_QNU)
    Grefl = gw.reflected(m, d, G0)
    rng = np.random.default_rng(3)
    for iq in [0, 1, int(rng.integers(2, m.nk))]:
        ref = gw.polarization_at_q(m, d, G0, iq, Grefl)
        if ctx.reduced:
            ref = np.einsum("ai,tab,bj->tij", ctx.basis.conj(), ref, ctx.basis)
        got = P[..., iq].cpu().numpy()
        assert rel(got, ref) <= {"fp64": FP64, "mixed": MIXED, "fp32": FP32["P_qnu"]}[prec], iq
    # sum rule and filling of the new G
    Gc = G.cpu().numpy()                                  # [r][a][b][k]
    c = np.linalg.solve(d.K_tau(), Gc.reshape(d.r, -1))
    g0p = (d.K_tau(np.array([0.0]))[0] @ c).reshape(m.norb, m.norb, m.nk)
    gbm = (d.K_beta() @ c).reshape(m.norb, m.norb, m.nk)
    tol = {"fp64": 1e-7, "mixed": 1e-6, "fp32": 1e-3}[prec]
    assert np.abs(g0p + gbm + np.eye(m.norb)[:, :, None]).max() <= tol
    assert abs(st["N"] - m.filling) <= (1e-5 if prec == "fp32" else 1e-11)
    # time reversal of a real-hopping model: Sigma^C(-k, tau) = Sigma^C(k, tau)^T
    S = ctx.get(qa.QA_SIGC_KTAU).cpu().numpy()
    mk = lattice.minus_R_index(m.n)
    Sm = S[..., mk]
    sym = np.abs(Sm - np.swapaxes(S, 1, 2)).max() / np.abs(S).max()
    assert sym <= (1e-12 if prec == "fp64" else 1e-5)
