"""One GW iteration, written as the paper states it (test infrastructure only).

Array layout throughout: axis 0 = lattice point (k, q or R, linear index of
lattice.py), axis 1 = DLR node (tau_j, i w_n or i nu_m), then orbital indices.
Pair index A = (a, b) -> a*norb + b.

Readings of the paper used here (each also listed in the design notes):
  * Fourier conventions: X(k) = sum_R exp(-i k.R) X(R) (Eq. for the k<->R
    transform) and X(i w) = int_0^beta exp(+i w tau) X(tau) dtau, so that
    G0(k, i w_n) = (i w_n + mu - H(k))^-1 (Eqs. for the bare Green's function).
    The exponents printed in the equations for P and Sigma^GW carry the other
    signs; with one convention used everywhere this is a relabelling k -> -k,
    w -> -w.
  * Bubble (Eq. for the polarizability, pairs (i,l) x (j,k)): per spin
    P_{(ab),(cd)}(R, tau) = G_{bc}(R, tau) G_{da}(-R, -tau)
                          = -G_{bc}(R, tau) G_{da}(-R, beta - tau),
    using G(-tau) = -G(beta - tau).  The spin sum of W's Dyson equation (spin
    independent V, paramagnetic) multiplies it by s_spin = 2.
  * Screened interaction (Eq. for W): W = V + V P W as a matrix product in the
    pair basis, W = (1 - V P)^-1 V per (q, i nu); W^C = W - V.
  * Self-energy (Eq. for Sigma^GW, Wick contraction of the interaction term):
    Sigma^C_{ad}(R, tau) = - sum_{bc} G_{bc}(R, tau) W^C_{(ab),(cd)}(R, tau).
  * Hartree (Eq. for Sigma^H): Sigma^H_{ab} = s_spin sum_{cd} V_{(ab),(cd)}(q=0) n_{dc}(R=0).
    Fock (Eq. for Sigma^F): Sigma^F_{ad}(R) = - sum_{bc} V_{(ab),(cd)}(R) n_{bc}(R),
    Sigma^F(k) = sum_R exp(-i k.R) Sigma^F(R), with n = -G(beta^-).
  * Dyson for G (Eq. for the full Green's function):
    G(k, i w_n) = (i w_n + mu - H(k) - Sigma^HF(k) - Sigma^C(k, i w_n))^-1.
  * mu is found by bisection on N(mu) = (s_spin/N_k) sum_k Tr n(k) = filling.
"""
from __future__ import annotations

import numpy as np

from . import lattice
from .dlr import DLR

MU_TOL_N = 1e-12     # |N - N_target| <= MU_TOL_N * max(1, N_target)
MU_TOL_BRACKET = 2e-13


def _node_axis_apply(K: np.ndarray, X: np.ndarray) -> np.ndarray:
    """out[k, j, ...] = sum_l K[j, l] X[k, l, ...]."""
    return np.einsum("jl,kl...->kj...", K, X)


def _node_axis_solve(K: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Solve K c = X along the node axis (axis 1)."""
    Xt = np.moveaxis(X, 1, 0)
    sh = Xt.shape
    c = np.linalg.solve(K, Xt.reshape(sh[0], -1)).reshape(sh)
    return np.moveaxis(c, 0, 1)


def make_dlr(model) -> DLR:
    return DLR(model.beta, model.Lambda, model.eps_dlr)


# --------------------------------------------------------------- G and density

def g_iw(dlr: DLR, Hk: np.ndarray, mu: float, sig_hf_k=None, sig_iw=None) -> np.ndarray:
    """Dyson: G(k, i w_n) = (i w_n + mu - H(k) - Sigma^HF(k) - Sigma^C(k, i w_n))^-1."""
    nk, no = Hk.shape[0], Hk.shape[1]
    iw = dlr.iw()
    A = (iw[None, :, None, None] + mu) * np.eye(no)[None, None] - Hk[:, None]
    if sig_hf_k is not None:
        A = A - sig_hf_k[:, None]
    if sig_iw is not None:
        A = A - sig_iw
    return np.linalg.inv(A)


def density_from_iw(dlr: DLR, Giw: np.ndarray) -> np.ndarray:
    """n(k) = -G(k, beta^-) from Matsubara-node values (DLR fit, then evaluation)."""
    c = _node_axis_solve(dlr.K_iw(), Giw)
    return -np.einsum("l,kl...->k...", dlr.K_beta(), c)


def density_from_tau(dlr: DLR, Gtau: np.ndarray) -> np.ndarray:
    """n(k) = -G(k, beta^-) from tau-node values."""
    c = _node_axis_solve(dlr.K_tau(), Gtau)
    return -np.einsum("l,kl...->k...", dlr.K_beta(), c)


def total_density(model, nk: np.ndarray) -> float:
    """N = (s_spin / N_k) sum_k Tr n(k)  (electrons per cell)."""
    return float(model.s_spin * np.real(np.einsum("kaa->", nk)) / nk.shape[0])


def mu_bracket(Hk, sig_hf_k, sig_iw, beta):
    """A bracket for mu from Gershgorin discs of H + Sigma^HF, widened by
    max ||Sigma^C(i w)||_inf + 1 + 10/beta."""
    M = Hk if sig_hf_k is None else Hk + sig_hf_k
    d = np.real(np.einsum("kaa->ka", M))
    off = np.abs(M).sum(axis=2) - np.abs(np.einsum("kaa->ka", M))
    lo = float((d - off).min())
    hi = float((d + off).max())
    wid = 1.0 + 10.0 / beta
    if sig_iw is not None:
        wid += float(np.abs(sig_iw).sum(axis=3).max())
    return lo - wid, hi + wid


def solve_mu(model, dlr, Hk, sig_hf_k=None, sig_iw=None):
    """Bisection on mu until |N - filling| <= 1e-12 max(1, filling) or the
    bracket is narrower than 2e-13.  Returns (mu, N, iterations)."""
    lo, hi = mu_bracket(Hk, sig_hf_k, sig_iw, model.beta)
    target = model.filling
    mid, N = 0.5 * (lo + hi), None
    for it in range(400):
        mid = 0.5 * (lo + hi)
        N = total_density(model, density_from_iw(dlr, g_iw(dlr, Hk, mid, sig_hf_k, sig_iw)))
        if abs(N - target) <= MU_TOL_N * max(1.0, target):
            break
        if N < target:
            lo = mid
        else:
            hi = mid
        if hi - lo < MU_TOL_BRACKET:
            mid = 0.5 * (lo + hi)
            N = total_density(model, density_from_iw(dlr, g_iw(dlr, Hk, mid, sig_hf_k, sig_iw)))
            break
    return mid, N, it + 1


def g0(model, dlr: DLR):
    """Non-interacting G0(k, tau_j) at the mu0 that gives the target filling.

    G0(k, i w_n) = (i w_n + mu0 - H(k))^-1 at the DLR Matsubara nodes, then DLR
    fit and evaluation at the tau nodes.  Returns (G0_tau, mu0)."""
    Hk = lattice.H_k(model)
    mu0, _, _ = solve_mu(model, dlr, Hk)
    Giw = g_iw(dlr, Hk, mu0)
    c = _node_axis_solve(dlr.K_iw(), Giw)
    return _node_axis_apply(dlr.K_tau(), c), mu0


# ------------------------------------------------------------ Hartree & Fock

def hartree_fock(model, nk: np.ndarray):
    """Sigma^H (k independent) and Sigma^F(k) from n(k)."""
    no = model.norb
    s = model.s_spin
    pts = lattice.grid_points(model.n)
    # n(R) = (1/N_k) sum_k exp(+i k.R) n(k) at the interaction's R vectors
    E = lattice.phase(model.n, pts, model.V_R, +1)          # [k, nV]
    nR = np.einsum("kr,kab->rab", E, nk) / model.nk          # [nV, no, no]
    n0 = nk.sum(axis=0) / model.nk
    Vq0 = model.V.sum(axis=0).reshape(no, no, no, no)        # (a,b,c,d)
    sig_h = s * np.einsum("abcd,dc->ab", Vq0, n0)
    VR = model.V.reshape(-1, no, no, no, no)
    sig_f_R = -np.einsum("rabcd,rbc->rad", VR, nR)
    Em = lattice.phase(model.n, pts, model.V_R, -1)          # [k, nV]
    sig_f_k = np.einsum("kr,rad->kad", Em, sig_f_R)
    return sig_h, sig_f_k


# --------------------------------------------------------------------- GW step

def polarization(model, dlr, GR: np.ndarray, GreflR: np.ndarray) -> np.ndarray:
    """P_{(ab),(cd)}(R, tau) = -s_spin G_{bc}(R, tau) G_{da}(-R, beta - tau)."""
    no = model.norb
    mR = lattice.minus_R_index(model.n)
    P = -model.s_spin * np.einsum("Rtbc,Rtda->Rtabcd", GR, GreflR[mR])
    return P.reshape(model.nk, dlr.r, no * no, no * no)


def screened_interaction(Vq: np.ndarray, Pqnu: np.ndarray):
    """W = (1 - V P)^-1 V per (q, i nu); returns (W, W^C = W - V)."""
    npair = Vq.shape[1]
    A = np.eye(npair)[None, None] - np.einsum("qAC,qnCB->qnAB", Vq, Pqnu)
    W = np.linalg.solve(A, np.broadcast_to(Vq[:, None], A.shape))
    return W, W - Vq[:, None]


def self_energy_c(model, GR: np.ndarray, WCR: np.ndarray) -> np.ndarray:
    """Sigma^C_{ad}(R, tau) = - sum_{bc} G_{bc}(R, tau) W^C_{(ab),(cd)}(R, tau)."""
    no = model.norb
    W6 = WCR.reshape(WCR.shape[0], WCR.shape[1], no, no, no, no)
    return -np.einsum("Rtbc,Rtabcd->Rtad", GR, W6)


def gw_step(model, dlr: DLR, Gtau: np.ndarray, mu_fixed=None) -> dict:
    """One G -> P -> W -> Sigma -> G iteration (paper Fig. 3(b)) from G(k, tau_j).

    mu_fixed: use this chemical potential instead of the bisection (the frozen-mu
    reading used for gradients, where mu is held at its forward value)."""
    n = model.n
    out = {}
    # DLR coefficients of the input G; G at beta - tau_j; density n(k)
    cG = _node_axis_solve(dlr.K_tau(), Gtau)
    Grefl = _node_axis_apply(dlr.K_tau_reflected(), cG)
    nk_in = -np.einsum("l,kl...->k...", dlr.K_beta(), cG)
    out["n_k_in"] = nk_in
    # Hartree and Fock
    sig_h, sig_f_k = hartree_fock(model, nk_in)
    sig_hf_k = sig_h[None] + sig_f_k
    out["sig_h"], out["sig_f_k"], out["sig_hf_k"] = sig_h, sig_f_k, sig_hf_k
    # real space
    GR = lattice.k_to_R(n, Gtau)
    GreflR = lattice.k_to_R(n, Grefl)
    out["G_Rtau"], out["Grefl_Rtau"] = GR, GreflR
    # polarizability
    PR = polarization(model, dlr, GR, GreflR)
    Pq = lattice.R_to_k(n, PR)
    Pqnu = _node_axis_apply(dlr.K_inu(), _node_axis_solve(dlr.K_tau(), Pq))
    out["P_qtau"], out["P_qnu"] = Pq, Pqnu
    del PR
    # screened interaction
    Vq = lattice.V_q(model)
    W, WC = screened_interaction(Vq, Pqnu)
    out["W_qnu"], out["WC_qnu"] = W, WC
    WCq = _node_axis_apply(dlr.K_tau(), _node_axis_solve(dlr.K_inu(), WC))
    WCR = lattice.k_to_R(n, WCq)
    out["WC_qtau"], out["WC_Rtau"] = WCq, WCR
    # self-energy
    sigR = self_energy_c(model, GR, WCR)
    sigk = lattice.R_to_k(n, sigR)
    sigiw = _node_axis_apply(dlr.K_iw(), _node_axis_solve(dlr.K_tau(), sigk))
    out["sigc_Rtau"], out["sigc_ktau"], out["sigc_kiw"] = sigR, sigk, sigiw
    # Dyson for G and the chemical potential
    Hk = lattice.H_k(model)
    if mu_fixed is None:
        mu, N, nit = solve_mu(model, dlr, Hk, sig_hf_k, sigiw)
    else:
        mu, nit = float(mu_fixed), 0
        N = total_density(model, density_from_iw(dlr, g_iw(dlr, Hk, mu, sig_hf_k, sigiw)))
    Giw = g_iw(dlr, Hk, mu, sig_hf_k, sigiw)
    cnew = _node_axis_solve(dlr.K_iw(), Giw)
    Gnew = _node_axis_apply(dlr.K_tau(), cnew)
    nk_out = -np.einsum("l,kl...->k...", dlr.K_beta(), cnew)
    out.update(mu=mu, N=N, mu_iterations=nit, G_kiw=Giw, G_ktau=Gnew, n_k=nk_out,
               n_local=nk_out.sum(axis=0) / model.nk)
    return out


def reflected(model, dlr: DLR, Gtau: np.ndarray) -> np.ndarray:
    """G(k, beta - tau_j) from G(k, tau_j) through the DLR coefficients."""
    return _node_axis_apply(dlr.K_tau_reflected(), _node_axis_solve(dlr.K_tau(), Gtau))


def _k_minus(model, iq: int) -> np.ndarray:
    """Linear index of k - q for every k (q given by its index)."""
    pts = lattice.grid_points(model.n)
    nn = np.asarray(model.n)
    kq = (pts - pts[iq]) % nn
    return (kq[:, 0] * nn[1] + kq[:, 1]) * nn[2] + kq[:, 2]


def polarization_at_q(model, dlr: DLR, Gtau: np.ndarray, iq: int, Grefl=None) -> np.ndarray:
    """P(q, i nu_m) for one q by the explicit k-sum of the bubble.

    P_{(ab),(cd)}(q, tau) = sum_R exp(-i q.R) P(R, tau)
                          = -(s_spin/N_k) sum_k G_{bc}(k, tau) G_{da}(k - q, beta - tau),
    then the DLR tau -> i nu transform.  Used for sampled checks on grids
    where the full R-space evaluation is too large.  Returns [r, npair, npair].
    """
    no = model.norb
    if Grefl is None:
        Grefl = reflected(model, dlr, Gtau)
    P = -model.s_spin * np.einsum("ktbc,ktda->tabcd", Gtau, Grefl[_k_minus(model, iq)]) / model.nk
    P = P.reshape(dlr.r, no * no, no * no)
    c = np.linalg.solve(dlr.K_tau(), P.reshape(dlr.r, -1))
    return (dlr.K_inu() @ c).reshape(dlr.r, no * no, no * no)


def self_energy_at_k(model, Gtau: np.ndarray, WCq_tau: np.ndarray, ik: int) -> np.ndarray:
    """Sigma^C(k, tau_j) for one k by the explicit q-sum (convolution form).

    Sigma^C_{ad}(k, tau) = sum_R exp(-i k.R) Sigma^C_{ad}(R, tau)
                         = -(1/N_k) sum_q sum_bc G_{bc}(k - q, tau) W^C_{(ab),(cd)}(q, tau).
    WCq_tau: [N_k, r, npair, npair].  Returns [r, norb, norb].
    """
    no = model.norb
    pts = lattice.grid_points(model.n)
    nn = np.asarray(model.n)
    kq = (pts[ik] - pts) % nn
    kq = (kq[:, 0] * nn[1] + kq[:, 1]) * nn[2] + kq[:, 2]
    W6 = WCq_tau.reshape(WCq_tau.shape[0], WCq_tau.shape[1], no, no, no, no)
    return -np.einsum("qtbc,qtabcd->tad", Gtau[kq], W6) / model.nk
