"""Pins of the Hartree-Fock loop and the quasiparticle quantities of the
oracle (oracle/qp.py) against closed forms, invariants and an independent
second route (no GPU)."""
import numpy as np
import pytest

import workloads as wl
from oracle import gw, lattice, qp


def test_hf_half_filled_square_closed_form():
    """Single band, local U, half filling: Sigma^H = s U n = U, Sigma^F = -U n
    = -U/2, so Sigma^HF = U/2 at every k and particle-hole symmetry puts
    mu at U/2 with n = 1/2 per spin."""
    m = wl.config("square-8x8")
    U = float(np.real(m.V[0, 0, 0]))
    out = qp.hf_loop(m, tol=1e-13)
    assert out["resid"] <= 1e-13
    assert np.abs(out["sig_hf_k"] - U / 2).max() <= 1e-12
    assert abs(out["mu"] - U / 2) <= 1e-10
    n_loc = out["n_k"].mean(axis=0)
    assert abs(n_loc[0, 0].real - 0.5) <= 1e-12


@pytest.mark.parametrize("name,mix", [("five-orbital-4x3x2", 0.5), ("graphene-6x6", 1.0),
                                      ("peierls-3x3", 1.0)])
def test_hf_fixed_point_and_second_route(name, mix):
    """At convergence n(k) = f(H0 + Sigma^HF[n] - mu) holds, N equals the
    filling, Sigma^HF(k) is Hermitian, and the DLR route to the density
    (-G(beta^-) of (i w + mu - H - Sigma^HF)^-1 at the Matsubara nodes)
    gives the same n(k)."""
    m = wl.config(name)
    out = qp.hf_loop(m, tol=1e-12, max_iter=2000, mix=mix)
    assert out["resid"] <= 1e-12, out["iters"]
    Hk = lattice.H_k(m)
    sh, sf = gw.hartree_fock(m, out["n_k"])
    # the fixed-point residual is the last change times the map's gain (<= 100)
    assert np.abs(sh[None] + sf - out["sig_hf_k"]).max() <= 1e-10
    n2, N = qp.fd_density(m, Hk + out["sig_hf_k"], out["mu"])
    assert abs(N - m.filling) <= 1e-11 * max(1, m.filling)
    assert np.abs(n2 - out["n_k"]).max() <= 1e-12
    S = out["sig_hf_k"]
    assert np.abs(S - np.conj(np.swapaxes(S, 1, 2))).max() <= 1e-12
    d = gw.make_dlr(m)
    n_dlr = gw.density_from_iw(d, gw.g_iw(d, Hk, out["mu"], out["sig_hf_k"]))
    assert np.abs(n_dlr - out["n_k"]).max() <= 1e-8


@pytest.mark.parametrize("w0,s", [(0.7, 0.3), (-1.3, 0.05), (0.15, 1.2)])
def test_sigma_static_single_pole(w0, s):
    """Sigma(i w) = s/(i w - w0) with the lowest Matsubara frequency wm = pi/beta:
    (Sigma(i wm) + Sigma(-i wm))/2 = -s w0/(w0^2 + wm^2) and
    (Sigma(i wm) - Sigma(-i wm))/(2 i wm) = -s/(w0^2 + wm^2), from DLR values at
    the nodes only."""
    m = wl.config("square-8x8")
    d = gw.make_dlr(m)
    wm = np.pi / m.beta
    sig = (s / (d.iw() - w0))[None, :, None, None]         # [k=1, node, 1, 1]
    s0, s1 = qp.sigma_static(d, sig)
    assert abs(s0[0, 0, 0] - (-s * w0 / (w0 ** 2 + wm ** 2))) <= 1e-10
    assert abs(s1[0, 0, 0] - (-s / (w0 ** 2 + wm ** 2))) <= 1e-10


def test_sigma_static_pole_form_fails_at_origin():
    """Why the limit is taken on the Matsubara axis: the DLR pole form, exact at
    the Matsubara frequencies, is far off at z = 0 for a pole not on the DLR grid."""
    m = wl.config("square-8x8")
    d = gw.make_dlr(m)
    w0, s = 0.7, 0.3
    c = np.linalg.solve(d.K_iw(), s / (d.iw() - w0))
    zn = 1j * 7 * np.pi / m.beta                            # a Matsubara frequency off the nodes
    assert abs(np.sum(c / (zn - d.omega)) - s / (zn - w0)) <= 1e-10
    assert abs(np.sum(c / (0.0 - d.omega)) - s / (0.0 - w0)) > 1e-3


def test_quasiparticle_limits():
    """Without self-energy Z = 1 and H_QP = H0 (eigenvalues = the bands); with a
    k-independent single-pole Sigma^C the scalar Z of the closed form, and H_QP
    = Z (H0 + Sigma(0)) for one orbital."""
    m = wl.config("square-8x8")
    d = gw.make_dlr(m)
    Hk = lattice.H_k(m)
    zero_iw = np.zeros((m.nk, d.r, 1, 1), dtype=complex)
    out = qp.quasiparticle(m, d, np.zeros_like(Hk), zero_iw)
    assert np.abs(out["Z"] - 1).max() <= 1e-14
    assert np.abs(out["eps"] - np.linalg.eigvalsh(Hk)).max() <= 1e-13
    w0, s = 0.9, 0.4
    wm = np.pi / m.beta
    sig = np.broadcast_to((s / (d.iw() - w0))[None, :, None, None], (m.nk, d.r, 1, 1)).copy()
    out = qp.quasiparticle(m, d, np.zeros_like(Hk), sig)
    Z = 1.0 / (1.0 + s / (w0 ** 2 + wm ** 2))
    sig0 = -s * w0 / (w0 ** 2 + wm ** 2)
    assert np.abs(out["Z"] - Z).max() <= 1e-10
    assert np.abs(out["eps"][:, 0] - Z * (Hk[:, 0, 0].real + sig0)).max() <= 1e-10
