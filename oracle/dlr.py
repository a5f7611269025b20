"""Discrete Lehmann representation (DLR), oracle version (test infrastructure).

Follows the construction of Kaye, Chen & Parcollet, "Discrete Lehmann
representation of imaginary time Green's functions", PRB 105, 235115 (2022),
which the paper cites for its imaginary-time/Matsubara sampling (Sec.
"Methods", DLR paragraph after the bare Green's function equations):

  1. Work with the dimensionless kernel k(t, x) = exp(-t x) / (1 + exp(-x)),
     t = tau/beta in [0, 1], x = beta*omega in [-Lambda, Lambda].
  2. Discretise x on composite Chebyshev panels refined dyadically toward
     x = 0, and t on panels refined dyadically toward t = 0 and t = 1.
  3. Select the DLR real frequencies x_l by pivoted Gram-Schmidt on the
     columns of the discretised kernel, stopping at relative tolerance eps.
  4. Select r imaginary-time nodes by pivoted Gram-Schmidt on the rows of
     k(t, x_l), and r fermionic / bosonic Matsubara nodes the same way on the
     rows of the Matsubara kernels.

Readings where the description leaves choices open (stated once here):
  * p = 24 first-kind Chebyshev points per panel; ceil(log2 Lambda) panels on
    [0, Lambda] and on [0, 1/2] (mirrored); Matsubara candidates |n| <= ceil(Lambda).
  * Column norms are plain (unweighted) 2-norms; the stopping rule is
    max residual norm <= eps * (largest initial column norm).
  * Ties in the pivot choice go to the lowest index among the columns whose
    residual norm is within a relative 1e-12 of the maximum.
  * Imaginary times are kept in *relative format*: a node t > 1/2 is stored as
    the negative number t - 1, so nodes close to beta keep full precision.
  * Bosonic quantities use the same real frequencies and tau nodes (the
    fermionic kernel in tau); their Matsubara kernel is
    tanh(x/2)/(i 2 pi m - x), which is the exact bosonic Fourier transform of
    the fermionic tau kernel.

Physical conventions (shared with gw.py):
  X(i w) = int_0^beta exp(+i w tau) X(tau) dtau,
  K(tau, omega)   = -k(tau/beta, beta*omega),
  K_F(i w_n, w)   = 1/(i w_n - w),                w_n = (2n+1) pi / beta,
  K_B(i nu_m, w)  = tanh(beta w / 2)/(i nu_m - w), nu_m = 2 m pi / beta.
"""
from __future__ import annotations

import math

import numpy as np

P_CHEB = 24
TIE_REL = 1e-12


# ---------------------------------------------------------------- fine grids

def _cheb_panel(a: float, b: float, p: int) -> np.ndarray:
    k = np.arange(p, dtype=np.float64)
    return 0.5 * (a + b) - 0.5 * (b - a) * np.cos(np.pi * (k + 0.5) / p)


def n_panels(Lambda: float) -> int:
    return max(1, int(math.ceil(math.log2(Lambda))))


def fine_x(Lambda: float, p: int = P_CHEB) -> np.ndarray:
    """Composite Chebyshev grid on [-Lambda, Lambda], dyadic toward 0."""
    npan = n_panels(Lambda)
    edges = [0.0] + [Lambda / 2.0 ** (npan - i) for i in range(1, npan + 1)]
    pos = np.concatenate([_cheb_panel(edges[i], edges[i + 1], p) for i in range(npan)])
    return np.concatenate([-pos[::-1], pos])


def fine_t(Lambda: float, p: int = P_CHEB) -> np.ndarray:
    """Composite Chebyshev grid on [0, 1] in relative format (t>1/2 stored as t-1)."""
    npan = n_panels(Lambda)
    edges = [0.0] + [2.0 ** (i - npan - 1) for i in range(1, npan + 1)]
    left = np.concatenate([_cheb_panel(edges[i], edges[i + 1], p) for i in range(npan)])
    return np.concatenate([left, -left[::-1]])


# ------------------------------------------------------------------- kernels

def kfun(t_rel: np.ndarray, x: np.ndarray) -> np.ndarray:
    """k(t, x) = exp(-t x)/(1+exp(-x)) for relative-format t, evaluated stably.

    Returns the outer array [len(t_rel), len(x)].
    """
    t_rel = np.asarray(t_rel, dtype=np.float64)[:, None]
    x = np.asarray(x, dtype=np.float64)[None, :]
    out = np.empty(np.broadcast(t_rel, x).shape)
    left = t_rel >= 0.0            # t = t_rel
    # t measured from 0 (t in [0, 1/2]): exponent -t x for x >= 0, (1-t) x for x < 0
    t = np.where(left, t_rel, 1.0 + t_rel)
    s = np.where(left, 1.0 - t_rel, -t_rel)   # 1 - t, exact for the right half
    xp = x >= 0.0
    with np.errstate(over="ignore", under="ignore", invalid="ignore"):
        out = np.where(xp, np.exp(-t * x) / (1.0 + np.exp(-x)),
                       np.exp(s * x) / (1.0 + np.exp(x)))
    return out


def fermi(x: np.ndarray) -> np.ndarray:
    """1/(exp(x)+1), the value k(t=1, x)."""
    x = np.asarray(x, dtype=np.float64)
    with np.errstate(over="ignore", under="ignore", invalid="ignore"):
        return np.where(x >= 0.0, np.exp(-x) / (1.0 + np.exp(-x)), 1.0 / (1.0 + np.exp(x)))


def kmats_fermi(n: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Dimensionless fermionic Matsubara kernel 1/(i(2n+1)pi - x), [len(n), len(x)]."""
    n = np.asarray(n, dtype=np.float64)[:, None]
    x = np.asarray(x, dtype=np.float64)[None, :]
    return 1.0 / (1j * (2.0 * n + 1.0) * np.pi - x)


def kmats_bose(m: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Dimensionless bosonic Matsubara kernel tanh(x/2)/(i 2 pi m - x), [len(m), len(x)].

    At m = 0 and x = 0 the limit is -1/2.
    """
    m = np.asarray(m, dtype=np.float64)[:, None]
    x = np.asarray(x, dtype=np.float64)[None, :]
    num = np.tanh(0.5 * x) + 0.0 * m
    den = 1j * 2.0 * np.pi * m - x
    with np.errstate(invalid="ignore", divide="ignore"):
        out = num / den
    out = np.where((m == 0) & (x == 0), -0.5 + 0j, out)
    return out


# ------------------------------------------------------- pivoted Gram-Schmidt

def pivoted_gram_schmidt(A: np.ndarray, eps: float | None = None, rank: int | None = None):
    """Column-pivoted Gram-Schmidt (with one re-orthogonalisation pass).

    At each step the remaining column of largest residual 2-norm is chosen
    (ties to the lowest index within TIE_REL), normalised, and projected out of
    every column.  Stops after `rank` columns, or when the largest residual
    norm falls to eps * (largest initial column norm).  Returns the selected
    column indices in selection order.
    """
    R = np.array(A, dtype=np.complex128 if np.iscomplexobj(A) else np.float64, copy=True)
    ncol = R.shape[1]
    ref = float(np.sqrt((np.abs(R) ** 2).sum(axis=0)).max())
    chosen = np.zeros(ncol, dtype=bool)
    sel = []
    limit = min(R.shape) if rank is None else rank
    while len(sel) < limit:
        nrm = np.sqrt((np.abs(R) ** 2).sum(axis=0))
        nrm[chosen] = -1.0
        m = float(nrm.max())
        if rank is None and m <= eps * ref:
            break
        j = int(np.flatnonzero(nrm >= m * (1.0 - TIE_REL))[0])
        q = R[:, j] / nrm[j]
        for _ in range(2):
            R -= np.outer(q, q.conj() @ R)
        chosen[j] = True
        sel.append(j)
    return sel


# ------------------------------------------------------------------ the grid

class DLR:
    """A DLR basis for given beta, Lambda (= beta*omega_max) and eps."""

    def __init__(self, beta: float, Lambda: float, eps: float):
        self.beta = float(beta)
        self.Lambda = float(Lambda)
        self.eps = float(eps)
        xf = fine_x(Lambda)
        tf = fine_t(Lambda)
        A = kfun(tf, xf)
        isel = pivoted_gram_schmidt(A, eps=eps)
        self.x = np.sort(xf[isel])                      # dimensionless real poles
        r = len(self.x)
        self.r = r
        B = kfun(tf, self.x)                             # [n_t, r]
        it = pivoted_gram_schmidt(B.T, rank=r)
        self.t = np.array(sorted(tf[it], key=lambda v: v if v >= 0 else 1.0 + v))
        nmax = int(math.ceil(Lambda))
        nf_cand = np.arange(-nmax, nmax, dtype=np.int64)
        jf = pivoted_gram_schmidt(kmats_fermi(nf_cand, self.x).T, rank=r)
        self.nf = np.sort(nf_cand[jf])
        mb_cand = np.arange(-nmax, nmax + 1, dtype=np.int64)
        jb = pivoted_gram_schmidt(kmats_bose(mb_cand, self.x).T, rank=r)
        self.mb = np.sort(mb_cand[jb])

    # physical node values --------------------------------------------------
    @property
    def omega(self) -> np.ndarray:
        return self.x / self.beta

    def tau_abs(self) -> np.ndarray:
        """Node times in [0, beta] (loses the relative-format precision)."""
        return self.beta * np.where(self.t >= 0, self.t, 1.0 + self.t)

    def iw(self) -> np.ndarray:
        return 1j * (2 * self.nf + 1) * np.pi / self.beta

    def inu(self) -> np.ndarray:
        return 1j * 2 * self.mb * np.pi / self.beta

    # kernel matrices (physical units) --------------------------------------
    def K_tau(self, t_rel=None) -> np.ndarray:
        """K(tau, omega_l) = -k(t, x_l) at relative-format times t (default: nodes)."""
        t = self.t if t_rel is None else np.asarray(t_rel, dtype=np.float64)
        return -kfun(t, self.x)

    def K_tau_reflected(self) -> np.ndarray:
        """K(beta - tau_j, omega_l) = K(tau_j, -omega_l)."""
        return -kfun(self.t, -self.x)

    def K_beta(self) -> np.ndarray:
        """K(beta^-, omega_l) = -f(beta omega_l)."""
        return -fermi(self.x)

    def K_iw(self, n=None) -> np.ndarray:
        n = self.nf if n is None else np.asarray(n)
        return self.beta * kmats_fermi(n, self.x)

    def K_inu(self, m=None) -> np.ndarray:
        m = self.mb if m is None else np.asarray(m)
        return self.beta * kmats_bose(m, self.x)

    # fits (the DLR coefficient solves) -------------------------------------
    def coef_from_tau(self, vals: np.ndarray) -> np.ndarray:
        """DLR coefficients from values at the tau nodes (axis 0 = node)."""
        sh = vals.shape
        c = np.linalg.solve(self.K_tau(), vals.reshape(self.r, -1))
        return c.reshape(sh)

    def coef_from_iw(self, vals: np.ndarray) -> np.ndarray:
        sh = vals.shape
        c = np.linalg.solve(self.K_iw(), vals.reshape(self.r, -1))
        return c.reshape(sh)

    def coef_from_inu(self, vals: np.ndarray) -> np.ndarray:
        sh = vals.shape
        c = np.linalg.solve(self.K_inu(), vals.reshape(self.r, -1))
        return c.reshape(sh)

    @staticmethod
    def apply(K: np.ndarray, coef: np.ndarray) -> np.ndarray:
        """Evaluate sum_l K[:, l] coef[l, ...]."""
        sh = coef.shape
        out = K @ coef.reshape(sh[0], -1)
        return out.reshape((K.shape[0],) + sh[1:])
