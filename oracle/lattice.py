"""Lattice grids and explicit Fourier sums, oracle version (test infrastructure).

Paper, Methods, Eq. for the k <-> R transform: X(k) = sum_R X(R) exp(-i k.(R + tau_p - tau_q)),
X(R) = (1/N_k) sum_k X(k) exp(+i k.(R + tau_p - tau_q)).

Readings:
  * Gamma-centred grid: k = sum_d (i_d / N_d) b_d, i_d in [0, N_d); q = 0 is on
    the grid (the Hartree term needs V(q=0)).
  * Cell gauge: the basis-position phase exp(-i k.(tau_p - tau_q)) is dropped.
    It is a k-dependent diagonal unitary; R-space quantities, eigenvalues, the
    density and mu do not depend on it.
  * Linear index of a grid point (i1, i2, i3): (i1*N2 + i2)*N3 + i3; the same
    order is used for k, q and for the R cells j_d in [0, N_d).
All sums here are explicit O(N_k^2) sums over a phase matrix.
"""
from __future__ import annotations

import numpy as np


def grid_points(n) -> np.ndarray:
    """Integer grid points [N_k, 3] in linear-index order."""
    n1, n2, n3 = n
    i1, i2, i3 = np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij")
    return np.stack([i1.ravel(), i2.ravel(), i3.ravel()], axis=1).astype(np.int64)


def kR_fraction(n, kpts: np.ndarray, R: np.ndarray) -> np.ndarray:
    """k.R / (2 pi) as the fraction sum_d i_d R_d / N_d, for all pairs [len(k), len(R)]."""
    nn = np.asarray(n, dtype=np.float64)
    return (kpts[:, None, :] * R[None, :, :] / nn[None, None, :]).sum(axis=2)


def phase(n, kpts: np.ndarray, R: np.ndarray, sign: int) -> np.ndarray:
    """exp(sign * i k.R) for all (k, R)."""
    return np.exp(sign * 2j * np.pi * kR_fraction(n, kpts, R))


def minus_R_index(n) -> np.ndarray:
    """Linear index of the cell -R (mod N) for every cell R."""
    pts = grid_points(n)
    nn = np.asarray(n)
    neg = (-pts) % nn
    return (neg[:, 0] * nn[1] + neg[:, 1]) * nn[2] + neg[:, 2]


def k_to_R(n, Xk: np.ndarray) -> np.ndarray:
    """X(R) = (1/N_k) sum_k exp(+i k.R) X(k), axis 0 = grid point."""
    pts = grid_points(n)
    E = phase(n, pts, pts, +1).T            # [R, k]
    sh = Xk.shape
    return (E @ Xk.reshape(sh[0], -1) / sh[0]).reshape(sh)


def R_to_k(n, XR: np.ndarray) -> np.ndarray:
    """X(k) = sum_R exp(-i k.R) X(R), axis 0 = grid point."""
    pts = grid_points(n)
    E = phase(n, pts, pts, -1)              # [k, R]
    sh = XR.shape
    return (E @ XR.reshape(sh[0], -1)).reshape(sh)


def H_k(model) -> np.ndarray:
    """H(k) = sum_R H(R) exp(-i k.R), H(R) = -t(R) + delta_{R0} diag(eps)  [N_k, norb, norb]."""
    pts = grid_points(model.n)
    E = phase(model.n, pts, model.hop_R, -1)            # [k, nH]
    Hk = -np.einsum("kr,rab->kab", E, model.hop_t)
    Hk = Hk + np.diag(model.eps.astype(np.complex128))[None]
    return Hk


def V_q(model) -> np.ndarray:
    """V(q) = sum_R V(R) exp(-i q.R) in the pair basis  [N_k, npair, npair]."""
    pts = grid_points(model.n)
    E = phase(model.n, pts, model.V_R, -1)
    return np.einsum("kr,rAB->kAB", E, model.V)
