"""Host-side checks of the C ABI (no GPU): the library loads, exports every
symbol of include/qa.h, validates its inputs, and its host planner produces
the same DLR grid as the oracle and bit-identical integer plan tables."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as wl
from oracle import lattice
from oracle.dlr import DLR
from paper_2604_22223_gb300.builder import build as build_lib
from paper_2604_22223_gb300 import qa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def lib():
    build_lib()
    return qa.load()


def test_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "qa.h")).read()
    declared = set(re.findall(r"^\s*(?:int|void|const char\*)\s+(qa_[a-z_]+)\s*\(", hdr, re.M))
    declared -= {"qa_ctx", "qa_step_stats", "qa_lattice", "qa_hoppings", "qa_interaction"}
    L = ctypes.CDLL(qa.LIB_PATH)
    for name in sorted(declared):
        assert hasattr(L, name), name
    assert declared >= set(qa.EXPORTED)


@pytest.mark.parametrize("name", ["square-8x8", "graphene-36x36", "five-orbital-16x16",
                                  "five-orbital-6x5x1", "peierls-3x3"])
def test_dlr_grid_matches_oracle(name):
    m = wl.config(name)
    p = qa.Problem(m)
    g = p.grid()
    d = DLR(m.beta, m.Lambda, m.eps_dlr)
    assert g["r"] == d.r
    assert np.abs(g["x"] - d.x).max() <= 1e-12 * m.Lambda
    assert np.array_equal(g["t"], d.t) or np.abs(g["t"] - d.t).max() <= 1e-16
    assert np.array_equal(g["nf"], d.nf)
    assert np.array_equal(g["mb"], d.mb)


@pytest.mark.slow
def test_dlr_grid_matches_oracle_large():
    m = wl.config("five-orbital-32x32x8")
    g = qa.Problem(m).grid()
    d = DLR(m.beta, m.Lambda, m.eps_dlr)
    assert g["r"] == d.r == 86
    assert np.array_equal(g["nf"], d.nf) and np.array_equal(g["mb"], d.mb)
    assert np.abs(g["x"] - d.x).max() <= 1e-12 * m.Lambda


@pytest.mark.parametrize("n", [(8, 8, 1), (5, 3, 2), (36, 36, 1), (32, 32, 8), (1, 1, 1), (6, 7, 9)])
def test_plan_tables_bit_identical(n):
    m = wl.square_single_band(n=n)
    p = qa.Problem(m)
    pl = p.plan()
    # -R map by brute force
    assert np.array_equal(pl["minus_R"], lattice.minus_R_index(n).astype(np.int32))
    # mixed-radix digit reversal: applying the stages to a basis vector in
    # exact arithmetic must put frequency f at position pos[f]
    off = 0
    for d, L in enumerate(n):
        fac = [int(v) for v in pl["fac"][d][:pl["nfac"][d]]]
        assert int(np.prod(fac)) == L
        pos = pl["pos"][off:off + L]
        off += L
        assert sorted(pos) == list(range(L))
        for f in range(L):
            x = np.exp(-2j * np.pi * f * np.arange(L) / L)     # spectrum: delta at f
            y = x.copy()
            Ls = L
            for rad in fac:
                Lp = Ls // rad
                z = y.copy()
                for blk in range(L // Ls):
                    for jp in range(Lp):
                        xs = [y[blk * Ls + j1 * Lp + jp] for j1 in range(rad)]
                        for k1 in range(rad):
                            acc = sum(xs[j1] * np.exp(-2j * np.pi * j1 * k1 / rad) for j1 in range(rad))
                            z[blk * Ls + k1 * Lp + jp] = acc * np.exp(-2j * np.pi * jp * k1 / Ls)
                y = z
                Ls = Lp
            # the conjugate-free DFT of exp(-2 pi i f j / L) is L at frequency (-f) mod L
            target = (-f) % L
            assert abs(y[pos[target]] - L) < 1e-9 * L


def test_invalid_inputs_rejected():
    m = wl.config("peierls-3x3")
    bad = wl.config("peierls-3x3")
    bad.hop_t = bad.hop_t.copy()
    bad.hop_t[0, 0, 1] += 0.5          # breaks t(-R) = t(R)^dagger
    with pytest.raises(qa.QAError) as e:
        qa.Problem(bad)
    assert e.value.status == 1
    for field, val in [("norb", 6), ("beta", -1.0), ("Lambda", 0.5), ("eps_dlr", 2.0),
                       ("filling", 0.0), ("n", (17, 1, 1)), ("n", (128, 128, 1))]:
        mm = wl.config("peierls-3x3")
        setattr(mm, field, val)
        if field == "norb":
            continue   # array shapes would not match; covered by the size check below
        with pytest.raises(qa.QAError):
            qa.Problem(mm)
    p = qa.Problem(m)
    assert p.workspace_size() > 0


def subspace_projector(Vs, tol=1e-12):
    """Projector on the span of the columns of every V(R) and V(R)^H, from an
    SVD of the stacked matrix (independent of the library's construction)."""
    X = np.concatenate([np.concatenate([V, V.conj().T], axis=1) for V in Vs], axis=1)
    U, s, _ = np.linalg.svd(X)
    k = int(np.sum(s > tol * s[0])) if s.size and s[0] > 0 else 0
    return U[:, :k] @ U[:, :k].conj().T, k


@pytest.mark.parametrize("name,rho", [("five-orbital-6x5x1", 15), ("five-orbital-32x32x8", 15),
                                      ("graphene-36x36", 2), ("peierls-3x3", 3),
                                      ("three-orbital-4x3x2", 6), ("four-orbital-3x2x2", 10),
                                      ("square-8x8", 1)])
def test_pair_basis(name, rho):
    """The reduced pair basis: its rank, orthonormality, the subspace it spans
    (against an SVD), V(R) = Pi V(R) Pi, and the rank of the Kanamori plus
    density-density interaction, norb + norb(norb - 1)/2 (one density per orbital
    and one symmetric exchange/pair-hopping combination per orbital pair)."""
    m = wl.config(name)
    p = qa.Problem(m, "fp32")
    assert p.rho == rho
    B = p.basis
    assert B.shape == (m.norb ** 2, rho)
    assert np.abs(B.conj().T @ B - np.eye(rho)).max() <= 1e-14
    Pi_svd, k = subspace_projector(list(m.V))
    assert k == rho
    Pi = B @ B.conj().T
    assert np.abs(Pi - Pi_svd).max() <= 1e-12
    for V in m.V:
        assert np.abs(Pi @ V @ Pi - V).max() <= 1e-14 * max(1.0, np.abs(V).max())
    # default choice: reduced on the mixed path when it is smaller, full on FP64
    assert p.reduced == (rho < m.norb ** 2)
    assert not qa.Problem(m, "fp64").reduced
    assert qa.Problem(m, "fp64", pairs="reduced").reduced == (rho < m.norb ** 2)
    assert not qa.Problem(m, "fp32", pairs="full").reduced
    # the reduced workspace is smaller
    if rho < m.norb ** 2:
        assert qa.Problem(m, "fp32").workspace_size() < qa.Problem(m, "fp32", pairs="full").workspace_size()


def _canonical_pattern(norb):
    """Supports of the canonical reduced basis: the diagonal pairs as unit vectors,
    then {(a,b), (b,a)} for each a < b in lexicographic order."""
    supp = [[a * norb + a] for a in range(norb)]
    supp += [[a * norb + b, b * norb + a] for a in range(norb) for b in range(a + 1, norb)]
    return supp


@pytest.mark.parametrize("name,canonical", [("five-orbital-6x5x1", True), ("five-orbital-32x32x8", True),
                                            ("peierls-3x3", True), ("three-orbital-4x3x2", True),
                                            ("four-orbital-3x2x2", True), ("graphene-36x36", False)])
def test_pair_basis_canonical_shape(name, canonical):
    """Kanamori-type interactions give the canonical basis shape for which the
    mixed path's Sigma contraction runs with compile-time indices (norb 2 to 5);
    the GPU parity tests of these workloads therefore exercise that kernel, and
    graphene's density-density basis exercises the generic term-list kernel."""
    m = wl.config(name)
    B = qa.Problem(m, "fp32").basis
    supp = [sorted(np.flatnonzero(np.abs(B[:, j]) > 0).tolist()) for j in range(B.shape[1])]
    match = supp == _canonical_pattern(m.norb)
    assert match == canonical
    if match:
        for j, s in enumerate(supp):
            assert np.allclose(np.abs(B[s, j]), len(s) ** -0.5, rtol=0, atol=1e-15)


def test_pair_basis_rank_deficient_block():
    """A model whose only coupling is a rank-1 block on the pairs (01), (10)
    gets the single vector (e_01 + e_10)/sqrt 2 (up to sign), not the unit vectors."""
    m = wl.config("peierls-3x3")
    V = np.zeros_like(m.V)
    V[0][1, 1] = V[0][1, 2] = V[0][2, 1] = V[0][2, 2] = 0.7
    m.V = V
    p = qa.Problem(m, "fp32")
    assert p.rho == 1 and p.reduced
    b = p.basis[:, 0] * np.sign(p.basis[1, 0].real)
    assert np.allclose(b, [0, 2 ** -0.5, 2 ** -0.5, 0], atol=1e-15)
