"""Pins from the values the paper prints for its two worked models
(tests/golden/paper_models.json: the graphene validation model of Sec.
"Validation: Electronic structure of graphene" and the degenerate five-orbital
benchmark model of Table 1).

The named workloads graphene-paper-* and five-orbital-paper-* must carry the
printed parameters, and on the graphene model the oracle must reproduce what
particle-hole symmetry fixes at half filling: with nearest-neighbour hopping
and interactions on the bipartite honeycomb lattice, every site holds half an
electron per spin and the chemical potential equals the static local shift,
  mu = Sigma^HF_aa(R = 0) = s (U + 3 V) / 2 - U / 2 = U/2 + 3V
(Hartree from the on-site U and the three nearest neighbours, minus the
on-site Fock term), for Hartree-Fock and, since the GW self-energy keeps the
symmetry, for a GW step as well.
"""
import json
import os

import numpy as np
import pytest

import workloads as wl
from oracle import gw, lattice, qp

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_models.json")))


def test_table1_row_sums_match_the_quoted_totals():
    tab = GOLD["table1_seconds_per_iteration"]
    for row in ("MF+Loop", "DLR+Vec"):
        r = tab[row]
        assert abs(r["G"] + r["P"] + r["W"] + r["Sigma"] - r["total"]) < 0.011


def _bond_values(model, R_list, a, b):
    return {tuple(R): model.V[i][a * model.norb + a, b * model.norb + b]
            for i, R in enumerate(model.V_R) if tuple(R) in R_list}


@pytest.mark.parametrize("name", ["graphene-paper-25x25", "graphene-paper-6x6"])
def test_graphene_model_carries_the_printed_parameters(name):
    g = GOLD["graphene"]
    m = wl.config(name)
    if name.endswith("25x25"):
        assert list(m.n) == g["k_grid"]
    assert abs(m.beta * wl.KB_EV_PER_K * g["temperature_K"] - 1.0) < 1e-12
    assert abs(m.Lambda / m.beta - g["Lambda_eV"]) < 1e-9
    assert m.norb == 2 and m.filling == 2.0                       # half filling of 2 sites x 2 spins
    # every hopping is the nearest-neighbour t, three bonds per site
    nz = np.abs(m.hop_t[np.abs(m.hop_t) > 0])
    assert np.all(np.abs(nz - g["t"]) < 1e-15) and len(nz) == 6
    # on-site U, nearest-neighbour V, nothing beyond
    i0 = [i for i, R in enumerate(m.V_R) if not np.any(R)][0]
    assert m.V[i0][0, 0] == g["U"] and m.V[i0][3, 3] == g["U"]
    vals = np.abs(m.V[np.abs(m.V) > 0])
    assert set(np.round(vals, 14)) == {g["U"], g["V_nearest_neighbour"]}


def test_five_orbital_model_carries_the_printed_parameters():
    g = GOLD["five_orbital_degenerate"]
    m = wl.config("five-orbital-paper-8x8x8")
    assert list(m.n) == g["k_grid"] and m.norb == g["norb"]
    assert m.beta == g["beta_per_eV"] and abs(m.Lambda / m.beta - g["Lambda_eV"]) < 1e-12
    for t in m.hop_t:                                             # degenerate orbitals
        assert np.array_equal(t, g["t"] * np.eye(5))
    i0 = [i for i, R in enumerate(m.V_R) if not np.any(R)][0]
    V0 = m.V[i0]
    U, J = g["U"], g["J"]
    assert V0[0, 0] == U and abs(V0[0, 6] - (U - 2 * J)) < 1e-15 and V0[1, 5] == J
    nn = _bond_values(m, {(1, 0, 0), (0, 0, -1)}, 0, 3)
    assert set(nn.values()) == {g["V_nearest_neighbour"]}


@pytest.mark.parametrize("name", ["graphene-paper-6x6", "graphene-paper-25x25"])
def test_graphene_hf_particle_hole_closed_form(name):
    g = GOLD["graphene"]
    m = wl.config(name)
    res = qp.hf_loop(m, tol=1e-12, max_iter=200)
    mu_ph = g["U"] / 2 + 3 * g["V_nearest_neighbour"]
    assert abs(res["mu"] - mu_ph) <= 1e-12
    nloc = res["n_k"].mean(axis=0)
    assert np.abs(np.diag(nloc).real - 0.5).max() <= 1e-12
    sig_loc = res["sig_hf_k"].mean(axis=0)
    assert np.abs(np.diag(sig_loc).real - mu_ph).max() <= 1e-12


def test_graphene_gw_step_particle_hole_and_z():
    g = GOLD["graphene"]
    m = wl.config("graphene-paper-6x6")
    d = gw.make_dlr(m)
    G0, mu0 = gw.g0(m, d)
    assert abs(mu0) <= 1e-8                                       # tight binding: mu0 = 0
    o = gw.gw_step(m, d, G0)
    assert abs(o["mu"] - (g["U"] / 2 + 3 * g["V_nearest_neighbour"])) <= 1e-8
    q = qp.quasiparticle(m, d, o["sig_hf_k"], o["sigc_kiw"])
    lam = np.linalg.eigvalsh(q["Z"])
    assert lam.min() > 0 and lam.max() < 1


def test_five_orbital_hf_half_filling_closed_form():
    """The paper's five-orbital model at half filling on the even 8x8x8 grid
    (particle-hole symmetric: orbital-diagonal nearest-neighbour hopping on a
    bipartite lattice): every spin-orbital holds 1/2 and mu equals the local
    HF shift  s/2 (U + (N-1) U' + 6 N V) - (U + (N-1) J)/2  with U' = U - 2J
    (Hartree over all orbitals of the site and its six neighbours, minus the
    on-site Fock terms U and the exchange J)."""
    g = GOLD["five_orbital_degenerate"]
    m = wl.config("five-orbital-paper-8x8x8")
    U, J, V, N = g["U"], g["J"], g["V_nearest_neighbour"], g["norb"]
    res = qp.hf_loop(m, tol=1e-12, max_iter=200)
    mu_ph = m.s_spin / 2 * (U + (N - 1) * (U - 2 * J) + 6 * N * V) - (U + (N - 1) * J) / 2
    assert abs(mu_ph - 9.5) < 1e-12
    assert abs(res["mu"] - mu_ph) <= 1e-10
    assert np.abs(np.diag(res["n_k"].mean(axis=0)).real - 0.5).max() <= 1e-12
