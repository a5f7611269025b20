"""The GW grand potential (qa_free_energy) and its adjoint (qa_free_energy_backward).

* Parity: Omega and its four terms against the CPU oracle (oracle/free_energy.py)
  on the input G of the first and the second iteration, full and reduced pair
  basis, to 1e-10 relative.
* Gradient: qa_free_energy_backward against central differences (h = 1e-5) of
  qa_free_energy along seeded directions in t(R), U, J and G_in, within 1e-6
  relative; the t and U derivatives also against the oracle's differences.
* The five-orbital 16x16 workload: the gradient of Omega[G_10] + Re<c_n, n> after
  10 checkpointed self-consistent iterations (FreeEnergy and GWStep through
  torch.autograd) against central differences of the same loop.
"""
import copy

import numpy as np
import pytest

import workloads as wl
from oracle import free_energy as fe
from oracle import gw

pytestmark = pytest.mark.gpu
H = 1e-5
TOL = 1e-6
PARTS = ("omega_hf", "omega_dc", "omega_g", "omega_w")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_22223_gb300 import build
    build()


def _hop_direction(model, rng):
    idx = {tuple(R): i for i, R in enumerate(model.hop_R)}
    D = np.zeros_like(model.hop_t)
    done = set()
    for i, R in enumerate(model.hop_R):
        if i in done:
            continue
        j = idx[tuple(-R)]
        X = rng.normal(size=D.shape[1:]) + 1j * rng.normal(size=D.shape[1:])
        if i == j:
            X = 0.5 * (X + X.conj().T)
            np.fill_diagonal(X, 0)
        D[i] = X
        D[j] = X.conj().T if i != j else X
        done |= {i, j}
    return D


def _kanamori_dV(model, which):
    no = model.norb
    eU = wl.kanamori_local(no, 1.0, 0.0, 0.0)
    eUp = wl.kanamori_local(no, 0.0, 0.0, 1.0)
    eJ = wl.kanamori_local(no, 0.0, 1.0, 0.0)
    d = eU + eUp if which == "U" else eJ - 2.0 * eUp
    dV = np.zeros_like(model.V)
    i0 = [i for i, R in enumerate(model.V_R) if not np.any(R)][0]
    dV[i0] = d
    return dV


def _perturbed(model, dt=None, dV=None, h=0.0):
    m = copy.deepcopy(model)
    if dt is not None:
        m.hop_t = model.hop_t + h * dt
    if dV is not None:
        m.V = model.V + h * dV
    return m


@pytest.mark.parametrize("name,M", [("square-8x8", 48), ("peierls-3x3", 40), ("five-orbital-4x3x2", 24)])
@pytest.mark.parametrize("pairs", ["full", "reduced"])
def test_free_energy_matches_oracle(name, M, pairs):
    from paper_2604_22223_gb300 import qa
    model = wl.config(name)
    d = gw.make_dlr(model)
    G0o, mu0 = gw.g0(model, d)
    G1o = gw.gw_step(model, d, G0o)["G_ktau"]
    ctx = qa.Context(model, "fp64", pairs=pairs)
    G0 = ctx.get(qa.QA_G0)
    G1, _, _, _ = ctx.step(G0)
    for Gg, Go in ((G0, G0o), (G1, G1o)):
        om, parts = ctx.free_energy(Gg, mu0, M)
        ref = fe.grand_potential(model, d, Go, mu0, M)
        scale = max(abs(ref[k]) for k in PARTS)
        for k in PARTS:
            assert abs(parts[k] - ref[k]) <= 1e-10 * scale, (k, parts[k], ref[k])
        assert abs(om - ref["omega"]) <= 1e-10 * scale, (om, ref["omega"])


@pytest.mark.parametrize("name,M", [("peierls-3x3", 40), ("five-orbital-4x3x2", 24)])
def test_free_energy_gradient_matches_finite_differences(name, M):
    import torch
    from paper_2604_22223_gb300 import qa
    model = wl.config(name)
    rng = np.random.default_rng(17)
    d = gw.make_dlr(model)
    G0o, _ = gw.g0(model, d)
    o1 = gw.gw_step(model, d, G0o)
    G1o, mu = o1["G_ktau"], o1["mu"]          # the oracle's second-iteration G and mu
    ctx = qa.Context(model, "fp64", pairs="full")
    G0 = ctx.get(qa.QA_G0)
    G1, _, _, _ = ctx.step(G0)
    shape = tuple(G1.shape)
    Gb, gt, gV = ctx.free_energy_backward(G1, mu, M)

    def omega(m, G):
        ctx.set_params(m)
        return ctx.free_energy(G, mu, M)[0]

    dt = _hop_direction(model, rng)
    dU, dJ = _kanamori_dV(model, "U"), _kanamori_dV(model, "J")
    dG = torch.from_numpy(rng.normal(size=shape) + 1j * rng.normal(size=shape)).cuda() * 1e-2
    adj = {
        "t": float(np.sum(np.conj(gt) * dt).real),
        "U": float(np.sum(np.conj(gV) * dU).real),
        "J": float(np.sum(np.conj(gV) * dJ).real),
        "G": float(torch.sum(Gb.conj() * dG).real),
    }
    fd = {
        "t": (omega(_perturbed(model, dt=dt, h=H), G1) - omega(_perturbed(model, dt=dt, h=-H), G1)) / (2 * H),
        "U": (omega(_perturbed(model, dV=dU, h=H), G1) - omega(_perturbed(model, dV=dU, h=-H), G1)) / (2 * H),
        "J": (omega(_perturbed(model, dV=dJ, h=H), G1) - omega(_perturbed(model, dV=dJ, h=-H), G1)) / (2 * H),
        "G": (omega(model, G1 + H * dG) - omega(model, G1 - H * dG)) / (2 * H),
    }
    ctx.set_params(model)
    for k in adj:
        assert abs(adj[k] - fd[k]) <= TOL * max(1.0, abs(fd[k])), (k, adj[k], fd[k])

    # the oracle's derivative by its own differences, on its own second-iteration G
    def omega_or(m):
        return fe.grand_potential(m, d, G1o, mu, M)["omega"]

    fd_or_t = (omega_or(_perturbed(model, dt=dt, h=H)) - omega_or(_perturbed(model, dt=dt, h=-H))) / (2 * H)
    fd_or_U = (omega_or(_perturbed(model, dV=dU, h=H)) - omega_or(_perturbed(model, dV=dU, h=-H))) / (2 * H)
    assert abs(adj["t"] - fd_or_t) <= TOL * max(1.0, abs(fd_or_t)), (adj["t"], fd_or_t)
    assert abs(adj["U"] - fd_or_U) <= TOL * max(1.0, abs(fd_or_U)), (adj["U"], fd_or_U)


def test_five_orbital_16x16_free_energy_ten_checkpointed_iterations():
    """Gradient of L = Omega[G_10] + Re<c_n, n_local> (mu frozen at the forward
    values, Omega at the last iteration's mu, cutoff M = 64) with respect to
    every hopping matrix, U and J through 10 damped self-consistent iterations
    G <- G + alpha (F(G) - G), each checkpointed by torch.autograd, against
    central differences (h = 1e-5) of the same loop."""
    import torch
    from paper_2604_22223_gb300 import qa
    from paper_2604_22223_gb300.autograd import FreeEnergy, GWStep
    model = wl.config("five-orbital-16x16")
    n_iter, alpha, M = 10, 0.3, 64
    ctx = qa.Context(model, "fp64", pairs="full")
    rng = np.random.default_rng(23)
    mus = []
    G = ctx.get(qa.QA_G0)
    for _ in range(n_iter):
        F, mu, _, _ = ctx.step(G)
        G = G + alpha * (F - G)
        mus.append(mu)
    cn = rng.normal(size=(model.norb, model.norb)) + 1j * rng.normal(size=(model.norb, model.norb))

    def loop(m, grad=False):
        ctx.set_params(m)
        t = torch.tensor(m.hop_t, requires_grad=grad)
        V = torch.tensor(m.V, requires_grad=grad)
        G = ctx.get(qa.QA_G0)
        n = None
        for i in range(n_iter):
            ctx.set_mu(mus[i])
            F, _, n = GWStep.apply(G, t, V, ctx)
            G = G + alpha * (F - G)
        L = FreeEnergy.apply(G, t, V, ctx, mus[-1], M) + torch.sum(torch.from_numpy(cn).conj() * n).real
        return L, t, V

    L, t, V = loop(model, grad=True)
    L.backward()
    gt, gV = t.grad.numpy(), V.grad.numpy()
    dt = _hop_direction(model, rng).real.astype(model.hop_t.dtype)
    dU, dJ = _kanamori_dV(model, "U"), _kanamori_dV(model, "J")
    for k, (ddt, ddV) in {"t": (dt, None), "U": (None, dU), "J": (None, dJ)}.items():
        adj = 0.0
        if ddt is not None:
            adj += float(np.sum(np.conj(gt) * ddt).real)
        if ddV is not None:
            adj += float(np.sum(np.conj(gV) * ddV).real)
        Lp, _, _ = loop(_perturbed(model, dt=ddt, dV=ddV, h=H))
        Lm, _, _ = loop(_perturbed(model, dt=ddt, dV=ddV, h=-H))
        fd = (float(Lp.detach()) - float(Lm.detach())) / (2 * H)
        assert abs(adj - fd) <= TOL * max(1.0, abs(fd)), (k, adj, fd)
    ctx.set_params(model)
    ctx.set_mu(None)
