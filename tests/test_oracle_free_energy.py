"""Pins of the oracle's GW grand potential (oracle/free_energy.py).

Each check compares the functional with something fixed independently:
  * the uniform-frequency DLR maps against the closed-form G0(k, i w_n) and the
    Lindhard bubble at i nu_m (frequency convention, normalisation);
  * the noninteracting limit, the free-fermion grand potential computed from
    the square-lattice dispersion;
  * d Omega / d mu = -N of the Dyson G (the thermodynamic identity of a grand
    potential), to the truncation of the Matsubara traces;
  * the second-order coefficient of the ring term against the Lindhard sum;
  * stationarity, the defining property of a Luttinger-Ward functional: at a
    self-consistent G (fixed mu) the derivative of Omega along a physical
    direction vanishes as the cutoff M grows, while it is of order one away
    from self-consistency.  This fixes the normalisation and sign of every term
    against the self-energy the iteration computes.
"""
import copy

import numpy as np
import pytest

import workloads as wl
from oracle import free_energy as fe
from oracle import gw, lattice
from oracle.dlr import fermi


def _square_dispersion(model):
    pts = lattice.grid_points(model.n)
    k = 2.0 * np.pi * pts[:, :2] / np.asarray(model.n[:2], dtype=np.float64)
    return -2.0 * (np.cos(k[:, 0]) + np.cos(k[:, 1]))


@pytest.fixture(scope="module")
def square():
    m = wl.config("square-8x8")
    d = gw.make_dlr(m)
    G0, mu0 = gw.g0(m, d)
    return m, d, G0, mu0


def test_uniform_fermi_map_gives_closed_form_g0(square):
    m, d, G0, mu0 = square
    M = 64
    Gn = gw._node_axis_apply(fe.uniform_fermi_map(d, M), G0)
    iw = 1j * (2 * np.arange(-M, M) + 1) * np.pi / m.beta
    eps = _square_dispersion(m)
    Gc = 1.0 / (iw[None, :] + mu0 - eps[:, None])
    assert np.abs(Gn[:, :, 0, 0] - Gc).max() <= 1e-9 * np.abs(Gc).max()


def _lindhard(model, mu, inu):
    """(s/N) sum_k (f(xi_{k-q}) - f(xi_k)) / (i nu + xi_{k-q} - xi_k), 0/0 -> -beta f (1 - f)."""
    pts = lattice.grid_points(model.n)
    nn = np.asarray(model.n)
    xi = _square_dispersion(model) - mu
    f = fermi(model.beta * xi)
    out = np.zeros((model.nk, len(inu)), dtype=np.complex128)
    for iq in range(model.nk):
        p = (pts - pts[iq]) % nn
        kp = (p[:, 0] * nn[1] + p[:, 1]) * nn[2] + p[:, 2]
        den = inu[None, :] + xi[kp][:, None] - xi[:, None]
        num = (f[kp] - f)[:, None] + 0.0 * den
        small = np.abs(den) < 1e-12
        lim = (-model.beta * f * (1.0 - f))[:, None] + 0.0 * den
        out[iq] = model.s_spin * np.where(small, lim, num / np.where(small, 1.0, den)).sum(axis=0) / model.nk
    return out


def test_uniform_bose_map_gives_lindhard(square):
    m, d, G0, mu0 = square
    M = 16
    inu = 1j * 2.0 * np.pi * np.arange(-M, M + 1) / m.beta
    Pm = gw._node_axis_apply(fe.uniform_bose_map(d, M), gw.gw_step(m, d, G0, mu_fixed=mu0)["P_qnu"])
    P = _lindhard(m, mu0, inu)
    assert np.abs(Pm[:, :, 0, 0] - P).max() <= 1e-9 * np.abs(P).max()


def test_noninteracting_limit_is_free_fermion_grand_potential(square):
    m, d, G0, mu0 = square
    m0 = copy.deepcopy(m)
    m0.V = 0.0 * m.V
    o = fe.grand_potential(m0, d, G0, mu0, 32)
    xi = _square_dispersion(m) - mu0
    ref = -m.s_spin / (m.beta * m.nk) * np.sum(np.logaddexp(0.0, -m.beta * xi))
    assert abs(o["omega"] - ref) <= 1e-13 * abs(ref)
    for k in ("omega_dc", "omega_g", "omega_w"):
        assert abs(o[k]) <= 1e-14, (k, o[k])


@pytest.mark.parametrize("name,tol", [("square-8x8", 1e-7), ("peierls-3x3", 1e-5)])
def test_mu_derivative_is_minus_density(name, tol):
    """d Omega / d mu at fixed G equals -N of the Dyson G at that mu, up to the
    truncation of the fermionic trace, which falls as the cutoff M grows."""
    m = wl.config(name)
    d = gw.make_dlr(m)
    G0, mu0 = gw.g0(m, d)
    N = gw.gw_step(m, d, G0, mu_fixed=mu0)["N"]
    h = 1e-5
    err = []
    for M in (64, 512):
        op = fe.grand_potential(m, d, G0, mu0 + h, M)
        om = fe.grand_potential(m, d, G0, mu0 - h, M)
        err.append(abs((op["omega"] - om["omega"]) / (2 * h) + N))
    assert err[1] <= tol * max(1.0, N), err
    assert err[1] < err[0] / 8, err


def test_ring_term_second_order(square):
    """Omega_W(lambda V) = -(lambda^2 / (4 beta N)) sum_{q,m} (U P_m(q))^2 + O(lambda^3)
    for the single band with local U, P the Lindhard bubble of G0."""
    m, d, G0, mu0 = square
    M = 16
    inu = 1j * 2.0 * np.pi * np.arange(-M, M + 1) / m.beta
    U = float(m.V[0][0, 0].real)
    a_ref = -float(np.sum((U * _lindhard(m, mu0, inu)) ** 2).real) / (4.0 * m.beta * m.nk)

    def a(lam):
        ml = copy.deepcopy(m)
        ml.V = lam * m.V
        return fe.grand_potential(ml, d, G0, mu0, M)["omega_w"] / lam ** 2

    a_rich = 2.0 * a(5e-3) - a(1e-2)       # removes the O(lambda) term
    assert abs(a_rich - a_ref) <= 2e-4 * abs(a_ref), (a_rich, a_ref)


def _self_consistent(model, dlr, mu, alpha=0.3, tol=1e-12, max_iter=400):
    G, _ = gw.g0(model, dlr)
    for _ in range(max_iter):
        Gn = gw.gw_step(model, dlr, G, mu_fixed=mu)["G_ktau"]
        dG = np.abs(Gn - G).max()
        G = G + alpha * (Gn - G)
        if dG < tol:
            return G
    raise AssertionError(f"no self-consistency: |dG| = {dG}")


@pytest.mark.parametrize("name,M,rel", [("square-1x1", 256, 1e-6), ("peierls-3x3", 1024, 1e-2)])
def test_stationary_at_self_consistency(name, M, rel):
    """Along the physical direction D = G0 - G* (products of such functions stay
    in the DLR space; a random perturbation of the node values does not, and
    the iteration's node-wise products then differ from the continuum ones),
    d Omega / d G at the self-consistent G* is small against its value at G0 and
    falls as the Matsubara cutoff M grows."""
    m = wl.config(name)
    d = gw.make_dlr(m)
    G0, mu0 = gw.g0(m, d)
    mu = gw.gw_step(m, d, G0)["mu"]
    Gs = _self_consistent(m, d, mu)
    D = G0 - Gs
    h = 1e-5

    def deriv(G, MM):
        return (fe.grand_potential(m, d, G + h * D, mu, MM)["omega"]
                - fe.grand_potential(m, d, G - h * D, mu, MM)["omega"]) / (2 * h)

    ref = abs(deriv(G0, M))
    lo, hi = abs(deriv(Gs, M // 4)), abs(deriv(Gs, M))
    assert hi <= rel * ref, (hi, ref)
    assert hi < lo / 2, (lo, hi)
