"""Pins of the CPU oracle against results that the paper and the mathematics fix.

Each test compares the oracle with something computed a *different* way:
closed forms built from an eigendecomposition (G0, the Lindhard and
multi-band bubbles, W of a single band, the second-order self-energy), exact
pole sums (DLR), invariants (sum rules, filling), and a brute-force Fock-space
expectation value for the Hartree and Fock terms.  None of these re-uses the
oracle's own formula for the quantity under test.
"""
import itertools

import numpy as np
import pytest

import workloads as wl
from oracle import gw, lattice
from oracle.dlr import DLR, fermi, kfun


# ------------------------------------------------------------------ helpers

def _grid_index(n, pts):
    nn = np.asarray(n)
    p = np.asarray(pts) % nn
    return (p[..., 0] * nn[1] + p[..., 1]) * nn[2] + p[..., 2]


def _eig_model(model, mu):
    Hk = lattice.H_k(model)
    e, U = np.linalg.eigh(Hk)
    return e - mu, U


def _g0_closed_form_tau(model, dlr, mu, t_rel):
    """G0_ab(k, tau) = -sum_m U_am exp(-tau xi_m)/(1+exp(-beta xi_m)) U*_bm."""
    xi, U = _eig_model(model, mu)
    K = kfun(t_rel, (model.beta * xi).ravel()).reshape(len(t_rel), model.nk, model.norb)
    return -np.einsum("kam,tkm,kbm->ktab", U, K, U.conj())


def _pole_sum_bubble(model, dlr, mu, inu):
    """Bubble of G0 from its Lehmann form (s_spin/N) sum_k sum_mn ...

    P_{(ab),(cd)}(q, i nu) = (s/N) sum_k sum_{m,n} U_bm(k) U*_cm(k) U_dn(k') U*_an(k')
                             (f_n(k') - f_m(k)) / (i nu + xi_n(k') - xi_m(k)),  k' = k - q.
    Derived by inserting the eigen-decomposed G0 into the bubble and doing the tau
    integral analytically; the 0/0 limit is -beta f (1 - f).
    """
    xi, U = _eig_model(model, mu)
    f = fermi(model.beta * xi)
    pts = lattice.grid_points(model.n)
    no = model.norb
    out = np.zeros((model.nk, len(inu), no * no, no * no), dtype=np.complex128)
    for iq in range(model.nk):
        kp = _grid_index(model.n, pts - pts[iq])            # k - q for every k
        xm, xn = xi, xi[kp]                                  # [k, m], [k, n]
        fm, fn = f, f[kp]
        for j, nu in enumerate(inu):
            den = nu + xn[:, None, :] - xm[:, :, None]       # [k, m, n]
            num = fn[:, None, :] - fm[:, :, None]
            small = np.abs(den) < 1e-12
            lim = -model.beta * fm[:, :, None] * (1 - fm[:, :, None])
            frac = np.where(small, lim, num / np.where(small, 1.0, den))
            Ub, Ud = U, U[kp]
            T = np.einsum("kbm,kcm,kdn,kan,kmn->abcd", Ub, Ub.conj(), Ud, Ud.conj(), frac)
            out[iq, j] = model.s_spin * T.reshape(no * no, no * no) / model.nk
    return out


@pytest.fixture(scope="module")
def square():
    m = wl.config("square-8x8")
    d = gw.make_dlr(m)
    G0, mu0 = gw.g0(m, d)
    return m, d, G0, mu0, gw.gw_step(m, d, G0)


# ---------------------------------------------------------------- generator

def test_splitmix64_published_vectors():
    g = wl.SplitMix64(1234567)
    assert [g.next_u64() for _ in range(3)] == [6457827717110365317, 3203168211198807973,
                                                9817491932198370423]
    g = wl.SplitMix64(0)
    assert g.next_u64() == 0xE220A8397B1DCDAF


def test_models_hermitian():
    for name in ["square-8x8", "graphene-6x6", "five-orbital-4x3x2", "peierls-3x3"]:
        m = wl.config(name)
        Hk = lattice.H_k(m)
        assert np.abs(Hk - Hk.conj().transpose(0, 2, 1)).max() < 1e-14
        # V(-R) = V(R)^T (particle exchange) for every listed R
        idx = {tuple(R): i for i, R in enumerate(m.V_R)}
        for i, R in enumerate(m.V_R):
            j = idx[tuple(-R)]
            assert np.abs(m.V[j] - m.V[i].T).max() < 1e-15


# --------------------------------------------------------------------- DLR

@pytest.mark.parametrize("beta,Lam,eps", [(10.0, 100.0, 1e-10), (40.0, 1000.0, 1e-10),
                                          (8.0, 60.0, 1e-10), (10.0, 300.0, 1e-12)])
def test_dlr_reconstructs_pole_sums(beta, Lam, eps):
    """Random pole sums with poles in [-Lambda/beta, Lambda/beta]: tau and Matsubara
    values are exact closed forms; DLR interpolation must reproduce them to ~eps."""
    d = DLR(beta, Lam, eps)
    rng = np.random.default_rng(7)
    w = rng.uniform(-Lam / beta, Lam / beta, 30)
    c = rng.normal(size=30)

    def g_tau(t_rel):   # -sum_p c_p exp(-tau w_p)/(1+exp(-beta w_p)), closed form
        t = np.where(t_rel >= 0, t_rel, 1 + t_rel)
        val = np.zeros(len(t))
        for wp, cp in zip(w, c):
            if wp >= 0:
                val += -cp * np.exp(-t * beta * wp) / (1 + np.exp(-beta * wp))
            else:
                val += -cp * np.exp((1 - t) * beta * wp) / (1 + np.exp(beta * wp))
        return val

    tt = rng.uniform(-0.5, 0.5, 300)
    ref = g_tau(tt)
    scale = np.abs(ref).max()
    # tau -> tau
    coef = d.coef_from_tau(g_tau(d.t))
    assert np.abs(d.K_tau(tt) @ coef - ref).max() <= 50 * eps * scale
    # tau -> Matsubara (fermionic) at arbitrary n
    n = rng.integers(-5 * int(Lam), 5 * int(Lam), 200)
    iw = 1j * (2 * n + 1) * np.pi / beta
    ex = (1.0 / (iw[:, None] - w[None, :])) @ c
    assert np.abs(d.K_iw(n) @ coef - ex).max() <= 100 * eps * np.abs(ex).max()
    # Matsubara nodes -> tau
    giw = (1.0 / (d.iw()[:, None] - w[None, :])) @ c
    c2 = d.coef_from_iw(giw)
    # Matsubara-node interpolation has a larger Lebesgue constant than the tau one
    assert np.abs(d.K_tau(tt) @ c2 - ref).max() <= 1000 * eps * scale
    # bosonic nodes -> tau and tau -> bosonic (same real frequencies)
    m = rng.integers(-5 * int(Lam), 5 * int(Lam), 200)
    inu = 1j * 2 * m * np.pi / beta
    exb = (np.tanh(beta * w / 2) / (inu[:, None] - w[None, :])) @ c
    assert np.abs(d.K_inu(m) @ coef - exb).max() <= 100 * eps * np.abs(exb).max()
    gb = (np.tanh(beta * w / 2) / (d.inu()[:, None] - w[None, :])) @ c
    assert np.abs(d.K_tau(tt) @ d.coef_from_inu(gb) - ref).max() <= 1000 * eps * scale
    # reflection K(beta - tau, w) = K(tau, -w) and beta^- value = -f
    assert np.abs(d.K_tau_reflected() @ coef - g_tau(-d.t)).max() <= 50 * eps * scale


def test_dlr_rank_grows_with_lambda_and_precision():
    r1 = DLR(1.0, 100.0, 1e-10).r
    r2 = DLR(1.0, 1000.0, 1e-10).r
    r3 = DLR(1.0, 1000.0, 1e-12).r
    assert 20 <= r1 < r2 < r3 <= 80


# ---------------------------------------------------------------------- G0

@pytest.mark.parametrize("name", ["square-8x8", "peierls-3x3", "five-orbital-4x3x2"])
def test_g0_matches_closed_form(name):
    m = wl.config(name)
    d = gw.make_dlr(m)
    G0, mu0 = gw.g0(m, d)
    ref = _g0_closed_form_tau(m, d, mu0, d.t)
    assert np.abs(G0 - ref).max() <= 1e-7
    # G(0+) + G(beta-) = -1 and the density equals the Fermi function of H
    c = d.coef_from_tau(np.moveaxis(G0, 1, 0))
    g0p = np.einsum("l,lkab->kab", d.K_tau(np.array([0.0]))[0], c)
    gbm = np.einsum("l,lkab->kab", d.K_beta(), c)
    assert np.abs(g0p + gbm + np.eye(m.norb)[None]).max() <= 1e-7
    xi, U = _eig_model(m, mu0)
    n_exact = np.einsum("kam,km,kbm->kab", U, fermi(m.beta * xi), U.conj())
    assert np.abs(-gbm - n_exact).max() <= 1e-7
    N = m.s_spin * np.real(np.einsum("kaa->", n_exact)) / m.nk
    assert abs(N - m.filling) <= 1e-7


def test_half_filling_square_has_mu_zero(square):
    m, d, G0, mu0, out = square
    # particle-hole symmetry of the nearest-neighbour square lattice: mu0 = 0
    assert abs(mu0) < 1e-8
    # after one step at half filling the Hartree-Fock shift is U/2 (U n/2 * 2 - U n/2)
    assert abs(out["mu"] - 1.0) < 1e-6
    assert abs(out["N"] - 1.0) < 1e-11


# --------------------------------------------------------------- the bubble

def test_lindhard_single_band(square):
    """P(q, i nu) = (s/N) sum_k (f(k-q) - f(k)) / (i nu + xi(k-q) - xi(k))."""
    m, d, G0, mu0, out = square
    Hk = lattice.H_k(m)
    xi = np.real(Hk[:, 0, 0]) - mu0
    f = fermi(m.beta * xi)
    pts = lattice.grid_points(m.n)
    ref = np.zeros((m.nk, d.r), dtype=np.complex128)
    for iq in range(m.nk):
        kq = _grid_index(m.n, pts - pts[iq])
        for j, nu in enumerate(d.inu()):
            den = nu + xi[kq] - xi
            small = np.abs(den) < 1e-12
            val = np.where(small, -m.beta * f * (1 - f), (f[kq] - f) / np.where(small, 1, den))
            ref[iq, j] = m.s_spin * val.sum() / m.nk
    assert np.abs(out["P_qnu"][:, :, 0, 0] - ref).max() <= 1e-8 * np.abs(ref).max()
    # static charge response is negative, P(q, tau) = P(q, beta - tau) at half filling
    assert np.all(ref[:, np.argmin(np.abs(d.mb))].real < 0)
    Pq = out["P_qtau"][:, :, 0, 0]
    c = np.linalg.solve(d.K_tau(), Pq.T)
    assert np.abs(d.K_tau_reflected() @ c - Pq.T).max() <= 1e-8 * np.abs(Pq).max()


@pytest.mark.parametrize("name", ["peierls-3x3", "five-orbital-4x3x2"])
def test_multiband_bubble_lehmann(name):
    """Orbital orientation of P pinned by the Lehmann (eigenvector) form."""
    m = wl.config(name)
    d = gw.make_dlr(m)
    G0, mu0 = gw.g0(m, d)
    cG = gw._node_axis_solve(d.K_tau(), G0)
    GR = lattice.k_to_R(m.n, G0)
    GreflR = lattice.k_to_R(m.n, gw._node_axis_apply(d.K_tau_reflected(), cG))
    Pq = lattice.R_to_k(m.n, gw.polarization(m, d, GR, GreflR))
    Pqnu = gw._node_axis_apply(d.K_inu(), gw._node_axis_solve(d.K_tau(), Pq))
    ref = _pole_sum_bubble(m, d, mu0, d.inu())
    assert np.abs(Pqnu - ref).max() <= 1e-8 * np.abs(ref).max()


def test_charge_conservation_q0():
    """sum_{a,c} P_{(aa),(cc)}(q=0, i nu != 0) = 0 (total charge commutes with H0)."""
    m = wl.config("peierls-3x3")
    d = gw.make_dlr(m)
    G0, _ = gw.g0(m, d)
    out = gw.gw_step(m, d, G0)
    no = m.norb
    diag = [a * no + a for a in range(no)]
    s = out["P_qnu"][0][:, diag][:, :, diag].sum(axis=(1, 2))
    nz = d.mb != 0
    assert np.abs(s[nz]).max() <= 1e-8 * np.abs(out["P_qnu"]).max()


# -------------------------------------------------------------------------- W

def test_single_band_W(square):
    """Local U, single band: W(q, i nu) = U / (1 - U P(q, i nu)) with the Lindhard P."""
    m, d, G0, mu0, out = square
    U = 2.0
    P = out["P_qnu"][:, :, 0, 0]
    ref = U / (1 - U * P)
    assert np.abs(out["W_qnu"][:, :, 0, 0] - ref).max() <= 1e-13 * abs(U)
    # W^C vanishes at large |nu| (P ~ 1/nu^2)
    big = np.argmax(np.abs(d.mb))
    assert np.abs(out["WC_qnu"][:, big]).max() < 0.05 * np.abs(out["WC_qnu"]).max()


def test_W_dyson_residual():
    m = wl.config("five-orbital-4x3x2")
    d = gw.make_dlr(m)
    G0, _ = gw.g0(m, d)
    out = gw.gw_step(m, d, G0)
    Vq = lattice.V_q(m)
    W, P = out["W_qnu"], out["P_qnu"]
    res = W - Vq[:, None] - np.einsum("qAB,qnBC,qnCD->qnAD", Vq, P, W)
    assert np.abs(res).max() <= 1e-12 * np.abs(Vq).max()


# ------------------------------------------------------------ self-energy

def _second_order_sigma(model, dlr, mu):
    """Sigma^(2)_{ad}(k, tau) = -(1/N) sum_q sum_bc G0_bc(k-q, tau) [V P0 V]_(ab),(cd)(q, tau)

    with G0 and P0(q, tau) = -(s/N) sum_k' G0(k', tau) (x) G0(k'-q, beta - tau)
    from the exact exponentials of the eigendecomposition (no DLR)."""
    no = model.norb
    Gt = _g0_closed_form_tau(model, dlr, mu, dlr.t)            # [k, t, a, b]
    Gb = _g0_closed_form_tau(model, dlr, mu, -dlr.t)           # at beta - tau
    pts = lattice.grid_points(model.n)
    Vq = lattice.V_q(model).reshape(model.nk, no, no, no, no)
    P0 = np.zeros((model.nk, dlr.r, no, no, no, no), dtype=np.complex128)
    for iq in range(model.nk):
        kq = _grid_index(model.n, pts - pts[iq])
        P0[iq] = -model.s_spin * np.einsum("ktbc,ktda->tabcd", Gt, Gb[kq]) / model.nk
    VPV = np.einsum("qabef,qtefgh,qghcd->qtabcd", Vq, P0, Vq)
    S = np.zeros((model.nk, dlr.r, no, no), dtype=np.complex128)
    for ik in range(model.nk):
        kmq = _grid_index(model.n, pts[ik] - pts)               # k - q for every q
        S[ik] = -np.einsum("qtbc,qtabcd->tad", Gt[kmq], VPV) / model.nk
    return S


@pytest.mark.parametrize("name", ["square-1x1", "peierls-3x3"])
def test_second_order_self_energy(name):
    """Sigma^C(lam V) = lam^2 Sigma^(2) + O(lam^3); Richardson in lam removes lam^3."""
    base = wl.config(name)
    d = gw.make_dlr(base)
    G0, mu0 = gw.g0(base, d)

    def sig(lam):
        m = wl.config(name)
        m.V = base.V * lam
        return gw.gw_step(m, d, G0)["sigc_ktau"]

    lam = 1e-4      # the expansion parameter is lam * |V| * beta, not lam
    s1, s2 = sig(lam), sig(2 * lam)
    est = (8 * s1 - s2) / (4 * lam ** 2)
    ref = _second_order_sigma(base, d, mu0)
    assert np.abs(est - ref).max() <= 1e-5 * np.abs(ref).max()


def test_sum_rule_after_step(square):
    m, d, G0, mu0, out = square
    c = gw._node_axis_solve(d.K_tau(), out["G_ktau"])
    g0p = np.einsum("l,kl...->k...", d.K_tau(np.array([0.0]))[0], c)
    gbm = np.einsum("l,kl...->k...", d.K_beta(), c)
    assert np.abs(g0p + gbm + np.eye(m.norb)[None]).max() <= 1e-7


# ------------------------------------------------- Hartree-Fock, brute force

def _fock_space_energy(V, C, no):
    """<Phi| (1/2) sum V_{(il),(jk)} c+_is c+_js' c_ks' c_ls |Phi> by brute force.

    Spin orbitals (x, s) -> mode 2x + s; Jordan-Wigner matrices on 2^(2 no) states;
    |Phi> = prod_o (sum_x C_xo c+_x,up) prod_o (sum_x C_xo c+_x,dn) |0>.
    """
    nm = 2 * no
    dim = 1 << nm

    def ann(mode):
        A = np.zeros((dim, dim))
        for st in range(dim):
            if st >> mode & 1:
                sign = (-1) ** bin(st & ((1 << mode) - 1)).count("1")
                A[st ^ (1 << mode), st] = sign
        return A

    c = [ann(mm) for mm in range(nm)]
    cd = [a.T for a in c]
    vac = np.zeros(dim, dtype=np.complex128)
    vac[0] = 1
    phi = vac
    for s in (0, 1):
        for o in range(C.shape[1]):
            op = sum(C[x, o] * cd[2 * x + s] for x in range(no))
            phi = op @ phi
    E = 0.0
    for i, l, j, k in itertools.product(range(no), repeat=4):
        v = V[i * no + l, j * no + k]
        if v == 0:
            continue
        for s, sp in itertools.product((0, 1), repeat=2):
            op = cd[2 * i + s] @ cd[2 * j + sp] @ c[2 * k + sp] @ c[2 * l + s]
            E += 0.5 * v * np.vdot(phi, op @ phi)
    return E / np.vdot(phi, phi)


def test_hartree_fock_fock_space():
    """E_HF = (s/2) Tr[(Sigma^H + Sigma^F) n] equals the exact <Phi|H_int|Phi> for
    Slater determinants, with a random complex interaction of the right symmetry."""
    no = 3
    rng = np.random.default_rng(3)
    npair = no * no
    V = rng.normal(size=(npair, npair)) + 1j * rng.normal(size=(npair, npair))
    sw = V.T                                              # particle exchange
    V = 0.5 * (V + sw)
    herm = np.zeros_like(V)                               # V_(il),(jk)* = V_(li),(kj)
    for i, l, j, k in itertools.product(range(no), repeat=4):
        herm[i * no + l, j * no + k] = np.conj(V[l * no + i, k * no + j])
    V = 0.5 * (V + herm)
    m = wl.Model("cluster", (1, 1, 1), no, np.zeros((0, 3), np.int64),
                 np.zeros((0, no, no), complex), np.zeros(no), np.zeros((1, 3), np.int64),
                 V[None], 1.0, 10.0, 1e-10, 1.0)
    for nocc in (1, 2):
        for trial in range(2):
            Q, _ = np.linalg.qr(rng.normal(size=(no, no)) + 1j * rng.normal(size=(no, no)))
            C = Q[:, :nocc]
            n = C @ C.conj().T                      # n_xy = <c+_y c_x> per spin
            sig_h, sig_f = gw.hartree_fock(m, n[None])
            E_hf = 0.5 * m.s_spin * np.trace((sig_h + sig_f[0]) @ n)
            E_ex = _fock_space_energy(V, C, no)
            assert abs(E_hf - E_ex) <= 1e-12 * max(1.0, abs(E_ex))


# ------------------------------------------- explicit-sum forms and the G Dyson step

@pytest.mark.parametrize("name", ["peierls-3x3", "five-orbital-4x3x2"])
def test_polarization_at_q_matches_real_space_bubble(name):
    """The explicit k-sum bubble -(s/N) sum_k G_bc(k, tau) G_da(k - q, beta - tau)
    (Eq. for the polarizability written as a convolution) equals, at every q, the
    real-space product G(R) G(-R) followed by the FFT R -> q that gw_step uses.
    A wrong k - q index or pair orientation in either form breaks the agreement
    (peierls-3x3 has complex hoppings, so G(k) != G(-k))."""
    m = wl.config(name)
    d = gw.make_dlr(m)
    G0, _ = gw.g0(m, d)
    o = gw.gw_step(m, d, G0)
    Grefl = gw.reflected(m, d, G0)
    for iq in range(m.nk):
        got = gw.polarization_at_q(m, d, G0, iq, Grefl)
        ref = o["P_qnu"][iq]
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(o["P_qnu"]).max(), iq


@pytest.mark.parametrize("name", ["peierls-3x3", "five-orbital-4x3x2"])
def test_self_energy_at_k_matches_real_space_product(name):
    """The explicit q-sum -(1/N) sum_q G_bc(k - q, tau) W^C_(ab),(cd)(q, tau) (Eq. for
    the GW self-energy as a convolution) equals, at every k, the real-space
    product -G(R) W^C(R) followed by the FFT that gw_step uses."""
    m = wl.config(name)
    d = gw.make_dlr(m)
    G0, _ = gw.g0(m, d)
    o = gw.gw_step(m, d, G0)
    scale = np.abs(o["sigc_ktau"]).max()
    for ik in range(m.nk):
        got = gw.self_energy_at_k(m, G0, o["WC_qtau"], ik)
        assert np.abs(got - o["sigc_ktau"][ik]).max() <= 1e-12 * scale, ik


def test_dyson_g_with_pole_self_energy_closed_form():
    """G(k, i w) = (i w + mu - H(k) - Sigma(i w))^-1 (Eq. for the full Green's
    function) with a frequency-dependent Sigma(i w) = V V^H / (i w - w0) is the
    upper-left block of the resolvent of the Hermitian matrix
    M = [[H - mu, V], [V^H, w0]] (Schur complement), so G(k, tau) is the pole sum
    sum_m U_am U*_bm K(tau, lambda_m) over M's eigenpairs.  Complex, non-commuting
    H(k) and V make a sign error in Sigma or a transposed Sigma fail."""
    rng = np.random.default_rng(5)
    no, nk, beta, mu, w0 = 2, 3, 10.0, 0.3, -0.7
    d = DLR(beta, 200.0, 1e-12)
    A = rng.normal(size=(nk, no, no)) + 1j * rng.normal(size=(nk, no, no))
    Hk = 0.5 * (A + np.conj(np.swapaxes(A, 1, 2)))
    V = 0.6 * (rng.normal(size=(no, no)) + 1j * rng.normal(size=(no, no)))
    iw = d.iw()
    sig = (V @ V.conj().T)[None, None] / (iw[None, :, None, None] - w0)
    sig = np.broadcast_to(sig, (nk, d.r, no, no))
    Giw = gw.g_iw(d, Hk, mu, None, sig)
    Gtau = gw._node_axis_apply(d.K_tau(), gw._node_axis_solve(d.K_iw(), Giw))
    for k in range(nk):
        M = np.zeros((2 * no, 2 * no), dtype=np.complex128)
        M[:no, :no] = Hk[k] - mu * np.eye(no)
        M[:no, no:] = V
        M[no:, :no] = V.conj().T
        M[no:, no:] = w0 * np.eye(no)
        lam, U = np.linalg.eigh(M)
        Uo = U[:no]
        # Matsubara nodes: sum_m U_am U*_bm / (i w - lambda_m)
        ref_iw = np.einsum("am,nm,bm->nab", Uo, 1.0 / (iw[:, None] - lam[None, :]), Uo.conj())
        assert np.abs(Giw[k] - ref_iw).max() <= 1e-12 * np.abs(ref_iw).max()
        # tau nodes: sum_m U_am U*_bm K(tau, lambda_m), K = -k(t, beta lambda)
        K = -kfun(d.t, beta * lam)                             # [tau, m]
        ref_tau = np.einsum("am,tm,bm->tab", Uo, K, Uo.conj())
        assert np.abs(Gtau[k] - ref_tau).max() <= 1e-9 * np.abs(ref_tau).max()


@pytest.mark.parametrize("name", ["peierls-3x3", "five-orbital-4x3x2"])
def test_bubble_of_interacting_pole_sum(name):
    """P(q, i nu) of an interacting G against the bubble's exact Matsubara sum over
    its DLR pole form.  With G(k, i w) = sum_l c_l(k) / (i w - w_l) (an expansion on
    the DLR real frequencies), the fermionic sum in (Eqs. for the polarizability
    and the k <-> R transform)
      P_(ab),(cd)(q, i nu) = (s / (beta N)) sum_{k,n} G_bc(k, i w_n + i nu) G_da(k - q, i w_n)
    is done in closed form term by term:
      (1/beta) sum_n 1 / ((i w_n + i nu - w_l)(i w_n - w_m)) = (f(w_m) - f(w_l)) / (i nu + w_m - w_l),
    with the limit -beta f (1 - f) at nu = 0, w_l = w_m.  G is the oracle's G after
    one iteration with its DLR weight kept on the poles |w_l| <= Lambda / (2 beta):
    generic coefficient matrices c_l(k) (not the rank-one eigenprojectors of the G0
    test) whose bubble stays inside the cutoff, so the fit on the tau nodes is exact
    to the DLR tolerance.  This pins the bubble's pair orientation, the k - q index
    and the tau -> i nu fit for an interacting G."""
    m = wl.config(name)
    d = gw.make_dlr(m)
    G0, _ = gw.g0(m, d)
    G1 = gw.gw_step(m, d, G0)["G_ktau"]
    c = gw._node_axis_solve(d.K_tau(), G1)               # [k][l][a][b], G = sum_l c_l K(tau, w_l)
    c[:, np.abs(d.x) > 0.5 * m.Lambda] = 0.0
    assert np.abs(c).max() > 0.1 * np.abs(gw._node_axis_solve(d.K_tau(), G1)).max()
    Gh = gw._node_axis_apply(d.K_tau(), c)
    P = gw.gw_step(m, d, Gh)["P_qnu"]                   # [q][nu][(ab)][(cd)]
    w = d.omega
    f = fermi(m.beta * w)
    pts = lattice.grid_points(m.n)
    no = m.norb
    inu = d.inu()
    jsel = range(len(inu)) if m.nk * len(inu) <= 400 else np.linspace(0, len(inu) - 1, 6).astype(int)
    scale = np.abs(P).max()
    for iq in range(m.nk):
        kp = _grid_index(m.n, pts - pts[iq])
        for j in jsel:
            den = inu[j] + w[None, :] - w[:, None]             # [l, m]
            num = f[None, :] - f[:, None]
            small = np.abs(den) < 1e-12
            frac = np.where(small, -m.beta * f[:, None] * (1 - f[:, None]), num / np.where(small, 1.0, den))
            A = np.einsum("klbc,lm->kmbc", c, frac)
            T = np.einsum("kmbc,kmda->abcd", A, c[kp])
            ref = m.s_spin * T.reshape(no * no, no * no) / m.nk
            assert np.abs(P[iq, j] - ref).max() <= 1e-8 * scale, (iq, j)


def test_screened_interaction_tau_by_direct_matsubara_sum():
    """W^C(q, tau) of the oracle (the DLR fit of W^C(q, i nu) on the bosonic nodes,
    evaluated at the tau nodes; Eq. for the screened interaction with the static V
    removed before the i nu -> tau step) against the direct bosonic sum
      W^C(q, tau) = (1/beta) sum_m exp(-i nu_m tau) W^C(q, i nu_m),  |m| <= M,
    with W^C = (1 - V P)^-1 V P V at every nu_m and P(q, i nu_m) the exact Matsubara
    sum over G0's pole form (as in the bubble pins).  W^C decays like T1/(i nu) +
    T2/(i nu)^2 (T1 = V A1 V, T2 = -V A2 V + V A1 V A1 V from P = A1/(i nu) -
    A2/(i nu)^2 + ...); these tails are summed in closed form,
      (1/beta) sum_{m != 0} exp(-i nu_m tau) / (i nu_m)   = tau/beta - 1/2,
      (1/beta) sum_{m != 0} exp(-i nu_m tau) / (i nu_m)^2 = -(beta/2) B_2(tau/beta),
    B_2(x) = x^2 - x + 1/6, and the rest converges as 1/M^2.  Complex hoppings
    (peierls-3x3) keep every pair entry independent."""
    m = wl.config("peierls-3x3")
    d = gw.make_dlr(m)
    G0, _ = gw.g0(m, d)
    o = gw.gw_step(m, d, G0)
    c = gw._node_axis_solve(d.K_tau(), G0)
    Vq = lattice.V_q(m)
    beta, no = m.beta, m.norb
    npair = no * no
    w = d.omega
    f = fermi(beta * w)
    Dlm = w[None, :] - w[:, None]
    num = f[None, :] - f[:, None]
    M = 3000
    mm = np.arange(-M, M + 1)
    nu = 2j * np.pi * mm / beta
    nz = mm != 0
    taus = d.tau_abs()
    x = taus / beta
    S1 = x - 0.5
    S2 = -(beta / 2) * (x * x - x + 1.0 / 6.0)
    ph = np.exp(-np.outer(taus, nu))
    pts = lattice.grid_points(m.n)
    scale = np.abs(o["WC_qtau"]).max()
    for iq in range(m.nk):
        kp = _grid_index(m.n, pts - pts[iq])
        den = nu[:, None, None] + Dlm[None]
        small = np.abs(den) < 1e-12
        frac = np.where(small, (-beta * f[:, None] * (1 - f[:, None]))[None], num[None] / np.where(small, 1.0, den))
        P = m.s_spin * np.einsum("vkmbc,kmda->vabcd", np.einsum("klbc,vlm->vkmbc", c, frac),
                                 c[kp]).reshape(len(nu), npair, npair) / m.nk
        A1 = m.s_spin * np.einsum("klbc,lm,kmda->abcd", c, num, c[kp]).reshape(npair, npair) / m.nk
        A2 = m.s_spin * np.einsum("klbc,lm,kmda->abcd", c, num * Dlm, c[kp]).reshape(npair, npair) / m.nk
        V = Vq[iq]
        VP = np.einsum("ab,vbc->vac", V, P)
        W = np.linalg.solve(np.eye(npair)[None] - VP, np.einsum("vab,bc->vac", VP, V))
        T1 = V @ A1 @ V
        T2 = -V @ A2 @ V + V @ A1 @ V @ A1 @ V
        W[nz] -= T1[None] / nu[nz, None, None] + T2[None] / nu[nz, None, None] ** 2
        Wt = np.einsum("tv,vab->tab", ph, W) / beta + S1[:, None, None] * T1[None] + S2[:, None, None] * T2[None]
        assert np.abs(Wt - o["WC_qtau"][iq]).max() <= 1e-6 * scale, iq
