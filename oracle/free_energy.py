"""GW grand potential in the Luttinger-Ward form (test infrastructure only).

The paper names the Luttinger-Ward functional in its introduction, as the
quantity whose gradients a differentiable GW code gives access to, but does
not write it down.  The reading used here (also listed in the design notes):
the Luttinger-Ward grand potential per unit cell of the GW approximation,

  Omega[G] = -Tr ln(-G_D^-1) - Tr[Sigma G] + Phi[G],
  Phi[G]   = Phi_HF[G] + (1/2) Tr_b [ln(1 - V P) + V P]     (the GW ring sum),

evaluated on the input G of one iteration (Sigma = Sigma^HF + Sigma^C and P
computed from G exactly as gw.gw_step does, mu held fixed).  It is split into
four terms, each finite on its own:

  Omega_HF = -(s/(beta N_k)) sum_k sum_i ln(1 + exp(-beta (e_i(k) - mu))),
             e_i(k) the eigenvalues of the Hermitian part of H(k) + Sigma^HF(k)
             (= -Tr ln(-G_HF^-1) for the static Hartree-Fock G_HF);
  Omega_dc = -(1/2) (s/N_k) sum_k Re tr[Sigma^HF(k) n(k)]
             (= Phi_HF - Tr[Sigma^HF G], Phi_HF = (1/2) Tr[Sigma^HF[n] n]);
  Omega_G  = -(s/(beta N_k)) sum_k sum_{n=-M}^{M-1}
             Re{ ln det[1 - G_HF Sigma^C] + tr[Sigma^C G] }(k, i w_n)
             (= -Tr ln(1 - G_HF Sigma^C) - Tr[Sigma^C G]);
  Omega_W  = (1/(2 beta N_k)) sum_q sum_{m=-M}^{M}
             Re{ ln det[1 - V(q) P(q, i nu_m)] + tr[V(q) P(q, i nu_m)] }.

The Matsubara traces run over the first 2M fermionic and 2M+1 bosonic
frequencies (w_n = (2n+1) pi/beta, nu_m = 2 m pi/beta); the terms kept in
them decay as 1/w^2, so no convergence factor is needed, and the cutoff M is
part of the definition.  Only Re ln det = ln|det| enters (no branch of the
logarithm is chosen).  Sigma^C(k, i w_n), G(k, i w_n) and P(q, i nu_m) at the
uniform frequencies come from their DLR expansions (the fermionic kernel at
i w_n, the bosonic form of the same kernel at i nu_m).
"""
from __future__ import annotations

import numpy as np

from . import gw, lattice
from .dlr import DLR


def uniform_fermi_map(dlr: DLR, M: int) -> np.ndarray:
    """E[n, j]: X(i w_n) = sum_j E[n, j] X(tau_j) for n = -M .. M-1."""
    n = np.arange(-M, M)
    return np.linalg.solve(dlr.K_tau().T, dlr.K_iw(n).T).T


def uniform_bose_map(dlr: DLR, M: int) -> np.ndarray:
    """E[m, j]: X(i nu_m) = sum_j E[m, j] X(i nu_j) (DLR bosonic nodes) for m = -M .. M."""
    m = np.arange(-M, M + 1)
    return np.linalg.solve(dlr.K_inu().T, dlr.K_inu(m).T).T


def _logabsdet(A: np.ndarray) -> np.ndarray:
    return np.linalg.slogdet(A)[1]


def grand_potential(model, dlr: DLR, Gtau: np.ndarray, mu: float, M: int, step=None) -> dict:
    """Omega[G] and its four terms for the input G(k, tau_j) at fixed mu.

    step: the output of gw.gw_step(model, dlr, Gtau, mu_fixed=mu) if already at hand."""
    o = step if step is not None else gw.gw_step(model, dlr, Gtau, mu_fixed=mu)
    s, nk, beta = model.s_spin, model.nk, model.beta
    no = model.norb
    eye = np.eye(no)
    Hk = lattice.H_k(model)
    A = Hk + o["sig_hf_k"]
    Ah = 0.5 * (A + np.conj(np.swapaxes(A, 1, 2)))
    e = np.linalg.eigvalsh(Ah)
    omega_hf = -(s / (beta * nk)) * float(np.sum(np.logaddexp(0.0, -beta * (e - mu))))
    omega_dc = -0.5 * (s / nk) * float(np.real(np.einsum("kab,kba->", o["sig_hf_k"], o["n_k_in"])))
    # fermionic trace
    EF = uniform_fermi_map(dlr, M)
    iw = 1j * (2 * np.arange(-M, M) + 1) * np.pi / beta
    Sn = gw._node_axis_apply(EF, o["sigc_ktau"])
    Gn = gw._node_axis_apply(EF, Gtau)
    Aw = (iw[None, :, None, None] + mu) * eye - A[:, None]
    tg = _logabsdet(Aw - Sn) - _logabsdet(Aw) + np.real(np.einsum("knab,knba->kn", Sn, Gn))
    omega_g = -(s / (beta * nk)) * float(np.sum(tg))
    # bosonic trace
    EB = uniform_bose_map(dlr, M)
    Pm = gw._node_axis_apply(EB, o["P_qnu"])
    Vq = lattice.V_q(model)
    npair = Vq.shape[-1]
    VP = np.einsum("qab,qmbc->qmac", Vq, Pm)
    tw = _logabsdet(np.eye(npair) - VP) + np.real(np.einsum("qmaa->qm", VP))
    omega_w = float(np.sum(tw)) / (2.0 * beta * nk)
    return dict(omega=omega_hf + omega_dc + omega_g + omega_w, omega_hf=omega_hf, omega_dc=omega_dc,
                omega_g=omega_g, omega_w=omega_w)
