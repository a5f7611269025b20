"""The hand-written adjoint (qa_gw_backward) against central finite differences.

Loss: L = Re<C_G, G_out> + Re<C_S, Sigma^C(k, tau)> + Re<c_n, n_local> with seeded
random cotangents (<a, b> = sum conj(a) b), mu held at the forward value.
Directional derivatives along seeded random directions in the hopping
amplitudes t(R) (Hermitian pairs t(R), t(-R) moved together), in U and J of
the Kanamori interaction, and in G_in are compared with central differences
(h = 1e-5) of (a) the GPU FP64 forward and (b) the CPU oracle, within 1e-6
relative, on the full and on the reduced pair basis; the reduced basis'
gradients also match the full basis' ones element by element.
"""
import copy

import numpy as np
import pytest

import workloads as wl
from oracle import gw

pytestmark = pytest.mark.gpu
H = 1e-5
TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_22223_gb300 import build
    build()


def hop_direction(model, rng):
    """Random Hermitian-consistent perturbation of the listed t(R)."""
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


def kanamori_dV(model, which):
    """dV/dU or dV/dJ of the on-site Kanamori block (U' = U - 2J)."""
    no = model.norb
    eU = wl.kanamori_local(no, 1.0, 0.0, 0.0)          # V_(aa),(aa)
    eUp = wl.kanamori_local(no, 0.0, 0.0, 1.0)         # V_(aa),(cc), a != c
    eJ = wl.kanamori_local(no, 0.0, 1.0, 0.0)          # exchange + pair hopping
    d = eU + eUp if which == "U" else eJ - 2.0 * eUp
    dV = np.zeros_like(model.V)
    i0 = [i for i, R in enumerate(model.V_R) if not np.any(R)][0]
    dV[i0] = d
    return dV


def perturbed(model, dt=None, dV=None, h=0.0):
    m = copy.deepcopy(model)
    if dt is not None:
        m.hop_t = model.hop_t + h * dt
    if dV is not None:
        m.V = model.V + h * dV
    return m


@pytest.mark.parametrize("name,pairs", [("peierls-3x3", "full"), ("five-orbital-4x3x2", "full"),
                                        ("five-orbital-4x3x2", "reduced")])
def test_adjoint_matches_finite_differences(name, pairs):
    import torch
    from paper_2604_22223_gb300 import qa
    model = wl.config(name)
    rng = np.random.default_rng(11)
    d = gw.make_dlr(model)
    G0_or, _ = gw.g0(model, d)
    mu = gw.gw_step(model, d, G0_or)["mu"]   # the oracle's mu, frozen for both sides
    ctx = qa.Context(model, "fp64", pairs=pairs)
    assert ctx.reduced == (pairs == "reduced")
    G0 = ctx.get(qa.QA_G0)
    ctx.set_mu(mu)                      # frozen mu for the forward evaluations below
    shape = tuple(G0.shape)
    CG = torch.from_numpy(rng.normal(size=shape) + 1j * rng.normal(size=shape)).cuda()
    CS = torch.from_numpy(rng.normal(size=shape) + 1j * rng.normal(size=shape)).cuda()
    cn = rng.normal(size=(model.norb, model.norb)) + 1j * rng.normal(size=(model.norb, model.norb))

    def loss_gpu(m, G_in):
        ctx.set_params(m)
        G, _, n, _ = ctx.step(G_in)
        S = ctx.get(qa.QA_SIGC_KTAU)
        return float(torch.sum(CG.conj() * G).real + torch.sum(CS.conj() * S).real) + \
            float(np.sum(np.conj(cn) * n).real)

    Gb, gt, gV = ctx.backward(G0, mu, CG, CS, cn)
    # directions
    dt = hop_direction(model, rng)
    dG = torch.from_numpy(rng.normal(size=shape) + 1j * rng.normal(size=shape)).cuda() * 1e-2
    adj = {
        "t": float(np.sum(np.conj(gt) * dt).real),
        "U": float(np.sum(np.conj(gV) * kanamori_dV(model, "U")).real),
        "J": float(np.sum(np.conj(gV) * kanamori_dV(model, "J")).real),
        "G": float(torch.sum(Gb.conj() * dG).real),
    }
    fd = {
        "t": (loss_gpu(perturbed(model, dt=dt, h=H), G0) - loss_gpu(perturbed(model, dt=dt, h=-H), G0)) / (2 * H),
        "U": (loss_gpu(perturbed(model, dV=kanamori_dV(model, "U"), h=H), G0)
              - loss_gpu(perturbed(model, dV=kanamori_dV(model, "U"), h=-H), G0)) / (2 * H),
        "J": (loss_gpu(perturbed(model, dV=kanamori_dV(model, "J"), h=H), G0)
              - loss_gpu(perturbed(model, dV=kanamori_dV(model, "J"), h=-H), G0)) / (2 * H),
    }
    fd["G"] = (loss_gpu(model, G0 + H * dG) - loss_gpu(model, G0 - H * dG)) / (2 * H)
    for k in adj:
        assert abs(adj[k] - fd[k]) <= TOL * max(1.0, abs(fd[k])), (k, adj[k], fd[k])

    # the oracle's FP64 gradient by its own central differences (frozen mu)
    CGo = np.moveaxis(CG.cpu().numpy(), -1, 0)
    CSo = np.moveaxis(CS.cpu().numpy(), -1, 0)

    def loss_or(m):
        o = gw.gw_step(m, d, G0_or, mu_fixed=mu)
        return float(np.sum(np.conj(CGo) * o["G_ktau"]).real + np.sum(np.conj(CSo) * o["sigc_ktau"]).real
                     + np.sum(np.conj(cn) * o["n_local"]).real)

    fd_or_t = (loss_or(perturbed(model, dt=dt, h=H)) - loss_or(perturbed(model, dt=dt, h=-H))) / (2 * H)
    dU = kanamori_dV(model, "U")
    fd_or_U = (loss_or(perturbed(model, dV=dU, h=H)) - loss_or(perturbed(model, dV=dU, h=-H))) / (2 * H)
    assert abs(adj["t"] - fd_or_t) <= TOL * max(1.0, abs(fd_or_t)), (adj["t"], fd_or_t)
    assert abs(adj["U"] - fd_or_U) <= TOL * max(1.0, abs(fd_or_U)), (adj["U"], fd_or_U)


@pytest.mark.parametrize("name", ["five-orbital-4x3x2", "graphene-6x6", "four-orbital-3x2x2"])
def test_reduced_basis_adjoint_matches_full_basis(name):
    """The reduced pair basis is an exact rewriting of the iteration, so the
    adjoint on it (term-list bubble and self-energy adjoints, Dyson adjoint in
    the rho-dimensional subspace, Vbar = B Sbar B^H) must give the full basis'
    gradients up to rounding."""
    import torch
    from paper_2604_22223_gb300 import qa
    model = wl.config(name)
    rng = np.random.default_rng(5)
    full = qa.Context(model, "fp64", pairs="full")
    red = qa.Context(model, "fp64", pairs="reduced")
    assert red.reduced and red.rho < full.npair
    G0 = full.get(qa.QA_G0)
    _, mu, _, _ = full.step(G0, full.new_g())
    shape = tuple(G0.shape)
    CG = torch.from_numpy(rng.normal(size=shape) + 1j * rng.normal(size=shape)).cuda()
    CS = torch.from_numpy(rng.normal(size=shape) + 1j * rng.normal(size=shape)).cuda()
    cn = rng.normal(size=(model.norb, model.norb)) + 1j * rng.normal(size=(model.norb, model.norb))
    out_f = list(full.backward(G0, mu, CG, CS, cn))
    out_r = list(red.backward(G0, mu, CG, CS, cn))
    # the reduced iteration reads V through S = B^H V B (screening) and whole in
    # Sigma^H, Sigma^F: the two V cotangents agree on the subspace, Pi Vbar Pi
    # with Pi = B B^H (the directions a perturbation of the model can take
    # without changing the subspace; the finite-difference test covers U and J)
    Pi = red.basis @ red.basis.conj().T
    for o in (out_f, out_r):
        o[2] = np.einsum("ab,vbc,cd->vad", Pi, o[2], Pi)
    for what, a, b in zip(("G_in", "t", "V"), out_f, out_r):
        a = a.cpu().numpy() if hasattr(a, "cpu") else a
        b = b.cpu().numpy() if hasattr(b, "cpu") else b
        err = np.abs(a - b).max() / max(np.abs(a).max(), 1e-300)
        assert err <= 1e-9, (what, err)


def test_unrolled_autograd_density_gradient():
    """Gradient of the density after 3 checkpointed iterations w.r.t. the hoppings,
    through torch.autograd, against central differences of the same loop."""
    import torch
    from paper_2604_22223_gb300 import qa
    from paper_2604_22223_gb300.autograd import GWStep
    model = wl.config("peierls-3x3")
    ctx = qa.Context(model, "fp64")
    rng = np.random.default_rng(5)
    cn = rng.normal(size=(model.norb, model.norb))
    mus = []
    G = ctx.get(qa.QA_G0)
    for _ in range(3):                  # forward once to fix the mu of every iteration
        G, mu, _, _ = ctx.step(G)
        mus.append(mu)

    def loop(m, grad=False):
        ctx.set_params(m)
        t = torch.tensor(m.hop_t, requires_grad=grad)
        V = torch.tensor(m.V, requires_grad=grad)
        G = ctx.get(qa.QA_G0)
        n = None
        for i in range(3):
            ctx.set_mu(mus[i])
            G, S, n = GWStep.apply(G, t, V, ctx)
        L = torch.sum(torch.from_numpy(cn) * n.real)
        return L, t

    L, t = loop(model, grad=True)
    L.backward()
    dt = hop_direction(model, rng)
    adj = float(np.sum(np.conj(t.grad.numpy()) * dt).real)
    Lp, _ = loop(perturbed(model, dt=dt, h=H))
    Lm, _ = loop(perturbed(model, dt=dt, h=-H))
    fd = (float(Lp) - float(Lm)) / (2 * H)
    assert abs(adj - fd) <= TOL * max(1.0, abs(fd)), (adj, fd)


def test_five_orbital_16x16_ten_checkpointed_iterations():
    """The five-orbital 16x16 workload and its parameters (every listed hopping
    matrix t(R) of the eight in-plane neighbours, which holds the model's 75
    amplitudes, plus U and J of the Kanamori interaction): the gradient of
    L = Re<c_n, n_local> + Re<C_S, Sigma^C(k, tau)> after 10 self-consistent
    iterations G <- G + alpha (F(G) - G), each F = qa_gw_step checkpointed by
    torch.autograd (GWStep keeps only its input G and mu; the adjoint recomputes
    P and W), mu frozen at the forward values, against central differences
    (h = 1e-5) of the same loop along seeded directions: all hoppings at once, U,
    J, and a combination of all of them.  The linear mixing alpha = 0.3 keeps the
    frozen-mu iteration contracting: without it the perturbation grows about
    threefold per iteration on this workload (measured: d L / d t of 0.014, 0.20,
    -0.50, -9.9 after 1, 2, 3, 5 iterations, adjoint and differences agreeing to
    1e-7), so that after 10 iterations central differences no longer converge as
    h decreases."""
    import torch
    from paper_2604_22223_gb300 import qa
    from paper_2604_22223_gb300.autograd import GWStep
    model = wl.config("five-orbital-16x16")
    n_iter, alpha = 10, 0.3
    ctx = qa.Context(model, "fp64")
    rng = np.random.default_rng(21)
    mus = []
    G = ctx.get(qa.QA_G0)
    for _ in range(n_iter):             # forward once to fix the mu of every iteration
        F, mu, _, _ = ctx.step(G)
        G = G + alpha * (F - G)
        mus.append(mu)
    shape = tuple(G.shape)
    CS = torch.from_numpy(rng.normal(size=shape) + 1j * rng.normal(size=shape)).cuda() * 1e-2
    cn = rng.normal(size=(model.norb, model.norb)) + 1j * rng.normal(size=(model.norb, model.norb))

    def loop(m, grad=False):
        ctx.set_params(m)
        t = torch.tensor(m.hop_t, requires_grad=grad)
        V = torch.tensor(m.V, requires_grad=grad)
        G = ctx.get(qa.QA_G0)
        S = n = None
        for i in range(n_iter):
            ctx.set_mu(mus[i])
            F, S, n = GWStep.apply(G, t, V, ctx)
            G = G + alpha * (F - G)
        L = torch.sum(torch.from_numpy(cn).conj() * n).real + torch.sum(CS.conj() * S).real.cpu()
        return L, t, V

    L, t, V = loop(model, grad=True)
    L.backward()
    gt, gV = t.grad.numpy(), V.grad.numpy()
    dt = hop_direction(model, rng).real.astype(model.hop_t.dtype)   # the model's amplitudes are real
    dU, dJ = kanamori_dV(model, "U"), kanamori_dV(model, "J")
    cU, cJ = rng.normal(), rng.normal()
    dirs = {"t": (dt, None), "U": (None, dU), "J": (None, dJ), "all": (dt, cU * dU + cJ * dJ)}
    for k, (ddt, ddV) in dirs.items():
        adj = 0.0
        if ddt is not None:
            adj += float(np.sum(np.conj(gt) * ddt).real)
        if ddV is not None:
            adj += float(np.sum(np.conj(gV) * ddV).real)
        Lp, _, _ = loop(perturbed(model, dt=ddt, dV=ddV, h=H))
        Lm, _, _ = loop(perturbed(model, dt=ddt, dV=ddV, h=-H))
        fd = (float(Lp.detach()) - float(Lm.detach())) / (2 * H)
        assert abs(adj - fd) <= TOL * max(1.0, abs(fd)), (k, adj, fd)
    ctx.set_params(model)
    ctx.set_mu(None)
