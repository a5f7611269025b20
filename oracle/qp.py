"""Hartree-Fock self-consistency and quasiparticle quantities, as the paper
states them (test infrastructure only; nothing in the product imports this).

Hartree-Fock loop (Sec. "Hartree-Fock self-consistency", Fig. 3(a)):
  H(k) = H0(k) + Sigma^H + Sigma^F(k) (Eqs. for Sigma^H and Sigma^F from the
  density matrix n), mu set to the filling, n(k) = 1/(exp(beta (H(k) - mu)) + 1)
  (Fermi-Dirac of the matrix H(k) - mu), repeated until Sigma^H + Sigma^F stops
  changing.  Readings: the loop starts from the Fermi-Dirac density of H0 at
  its own mu; convergence is max |Sigma^HF_new - Sigma^HF_old| <= tol; the
  paper names no mixing, so the default is the plain iteration (mix = 1), and
  mix < 1 replaces Sigma^HF by Sigma^HF + mix (Sigma^HF_new - Sigma^HF).

Quasiparticle quantities (Secs. on the Z and SigStc classes and the
quasiparticle Hamiltonian of the graphene results):
  Z(k)^-1 = 1 - d Sigma(k, i w) / d(i w) at w = 0,
  H_QP(k) = sqrt(Z) (H0(k) + Sigma(k, w = 0)) sqrt(Z).
  Reading of "at w = 0" for a Matsubara function: the DLR pole form
  sum_l c_l / (z - w_l) reproduces Sigma at every Matsubara frequency but not
  at z = 0 (its smallest real poles lie next to the origin, so continuing the
  fit off the imaginary axis is ill-conditioned; the pins show an error of
  order 1e-1 at z = 0).  The limit is therefore taken on the Matsubara axis,
  from the DLR evaluation at the two lowest fermionic frequencies
  +-i w0 = +-i pi / beta:
    Sigma(0)        = (Sigma(i w0) + Sigma(-i w0)) / 2,
    dSigma/d(iw)|0  = (Sigma(i w0) - Sigma(-i w0)) / (2 i w0),
  which for one orbital is the usual Z^-1 = 1 - Im Sigma(i w0) / w0 and which
  tends to the derivative at the origin as the temperature goes to zero.
  Further readings: Sigma in H_QP is the whole static self-energy Sigma^H +
  Sigma^F + Sigma^C(k, 0) (H0 is the bare Hamiltonian); Z^-1 and
  H0 + Sigma(0) are Hermitian for an exact self-energy and their Hermitian
  parts are used; sqrt(Z) is the positive square root through the
  eigendecomposition of the Hermitian Z.
"""
from __future__ import annotations

import numpy as np

from . import lattice
from .dlr import DLR
from .gw import _node_axis_apply, _node_axis_solve, g_iw, hartree_fock

MU_TOL_N = 1e-12


def fermi(x: np.ndarray) -> np.ndarray:
    """1 / (exp(x) + 1) without overflow."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    pos = x > 0
    ex = np.exp(-x[pos])
    out[pos] = ex / (1.0 + ex)
    out[~pos] = 1.0 / (1.0 + np.exp(x[~pos]))
    return out


def fd_density(model, Hk_eff: np.ndarray, mu: float):
    """n(k) = U f(beta (E - mu)) U^H of each Hermitian H(k); returns (n_k, N)."""
    Hh = 0.5 * (Hk_eff + np.conj(np.swapaxes(Hk_eff, 1, 2)))
    E, U = np.linalg.eigh(Hh)
    f = fermi(model.beta * (E - mu))
    nk = np.einsum("kai,ki,kbi->kab", U, f, U.conj())
    N = model.s_spin * float(f.sum()) / model.nk
    return nk, N


def solve_mu_fd(model, Hk_eff: np.ndarray):
    """Bisection on N(mu) = (s/N_k) sum_{k,i} f(beta (E_ki - mu)) = filling."""
    Hh = 0.5 * (Hk_eff + np.conj(np.swapaxes(Hk_eff, 1, 2)))
    E = np.linalg.eigvalsh(Hh)
    lo = float(E.min()) - 1.0 - 40.0 / model.beta
    hi = float(E.max()) + 1.0 + 40.0 / model.beta
    target = model.filling
    for _ in range(300):
        mid = 0.5 * (lo + hi)
        N = model.s_spin * float(fermi(model.beta * (E - mid)).sum()) / model.nk
        if abs(N - target) <= MU_TOL_N * max(1.0, target) or hi - lo < 1e-14 * max(1.0, abs(mid)):
            break
        if N < target:
            lo = mid
        else:
            hi = mid
    return mid


def hf_loop(model, tol: float = 1e-10, max_iter: int = 500, mix: float = 1.0) -> dict:
    """Self-consistent Hartree-Fock solution; returns mu, Sigma^HF(k), n(k),
    the number of iterations and the last change of Sigma^HF."""
    Hk = lattice.H_k(model)
    mu = solve_mu_fd(model, Hk)
    nk, _ = fd_density(model, Hk, mu)
    sig = np.zeros_like(Hk)
    resid = np.inf
    it = 0
    for it in range(1, max_iter + 1):
        sh, sfk = hartree_fock(model, nk)
        new = sh[None] + sfk
        resid = float(np.abs(new - sig).max())
        sig = sig + mix * (new - sig)
        mu = solve_mu_fd(model, Hk + sig)
        nk, _ = fd_density(model, Hk + sig, mu)
        if resid <= tol:
            break
    return {"mu": mu, "sig_hf_k": sig, "n_k": nk, "iters": it, "resid": resid}


def hf_green(model, dlr: DLR, mu: float, sig_hf_k: np.ndarray) -> np.ndarray:
    """The Hartree-Fock Green's function on the tau nodes, [k, node, a, b]:
    Dyson with the static Sigma^HF at mu, DLR fit at the Matsubara nodes,
    evaluation at the tau nodes."""
    Giw = g_iw(dlr, lattice.H_k(model), mu, sig_hf_k)
    return _node_axis_apply(dlr.K_tau(), _node_axis_solve(dlr.K_iw(), Giw))


def sigma_static(dlr: DLR, sig_iw: np.ndarray):
    """Sigma(w = 0) and d Sigma / d(i w) at w = 0 (Matsubara-axis reading
    above) from values at the DLR Matsubara nodes (node axis 1 of
    sig_iw [k, node, ...])."""
    Xt = np.moveaxis(sig_iw, 1, 0)
    sh = Xt.shape
    c = np.linalg.solve(dlr.K_iw(), Xt.reshape(sh[0], -1)).reshape(sh)   # pole weights
    w0 = np.pi / dlr.beta
    sp = np.einsum("l,l...->...", 1.0 / (1j * w0 - dlr.omega), c)        # Sigma(+i w0)
    sm = np.einsum("l,l...->...", 1.0 / (-1j * w0 - dlr.omega), c)       # Sigma(-i w0)
    return 0.5 * (sp + sm), (sp - sm) / (2j * w0)


def _herm(A: np.ndarray) -> np.ndarray:
    return 0.5 * (A + np.conj(np.swapaxes(A, -1, -2)))


def quasiparticle(model, dlr: DLR, sig_hf_k: np.ndarray, sig_iw: np.ndarray) -> dict:
    """Z(k), Sigma(k, 0) (= Sigma^HF + Sigma^C(0)), H_QP(k) and its eigenvalues."""
    no = model.norb
    s0, s1 = sigma_static(dlr, sig_iw)
    Zi = _herm(np.eye(no)[None] - s1)
    Z = np.linalg.inv(Zi)
    lam, U = np.linalg.eigh(_herm(Z))
    if np.any(lam <= 0):
        raise ValueError("Z(k) is not positive definite")
    sqZ = np.einsum("kai,ki,kbi->kab", U, np.sqrt(lam), U.conj())
    sig0 = sig_hf_k + s0
    Hs = _herm(lattice.H_k(model) + sig0)
    Hqp = _herm(sqZ @ Hs @ sqZ)
    return {"Z": Z, "sig0": sig0, "Hqp": Hqp, "eps": np.linalg.eigvalsh(Hqp), "dsig": s1}
