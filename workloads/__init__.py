"""Seeded synthetic lattice models for the GW iteration (inputs only).

This module builds the *problem statement* of a GW run: the lattice (grid
sizes), the hopping amplitudes t(R), on-site energies, the two-body
interaction V(R) in the orbital-pair ("product") basis, beta, the DLR cutoff
Lambda, the DLR tolerance eps and the electron filling.  It holds no GW
arithmetic: no Green's functions, no Fourier transforms, no DLR.  Both the
CPU oracle and the CUDA library are fed from here, so both see identical
numbers.

Conventions (paper, Methods, Eq. for the many-body Hamiltonian):
  * H_ab(R) = <a,R|H|b,0> = -t_ab(R) + delta_{R,0} delta_ab eps_a  (the paper's
    hopping enters with a minus sign).  Every model lists both R and -R and
    satisfies t(-R) = t(R)^dagger.
  * V_{(ab),(cd)}(R) is the product-basis matrix of the interaction
    (1/2) sum V_ijkl c+_i c+_j c_k c_l with pair A=(i,l)=(a,b) living on the cell
    R and pair B=(j,k)=(c,d) on the cell 0; pair index A = a*norb + b.
  * Random numbers come from SplitMix64 (Steele, Lea & Flood 2014) with a
    Box-Muller transform, in double precision, so the stream is reproducible
    on any machine.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

DEFAULT_SEED = 2604222230
_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator (Steele, Lea & Flood, OOPSLA 2014)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def normal(self) -> float:
        """Standard normal by Box-Muller (one variate per two uniforms)."""
        u1 = 1.0 - self.uniform()  # (0, 1]
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)

    def normals(self, n: int, sigma: float) -> np.ndarray:
        return np.array([sigma * self.normal() for _ in range(n)], dtype=np.float64)


@dataclass
class Model:
    """One GW problem: lattice, one-body part, interaction and thermodynamics."""

    name: str
    n: tuple            # k-grid (N1, N2, N3), Gamma-centred
    norb: int
    hop_R: np.ndarray   # int64 [nH, 3]
    hop_t: np.ndarray   # complex128 [nH, norb, norb], H(R) = -t(R)
    eps: np.ndarray     # float64 [norb], on-site energies
    V_R: np.ndarray     # int64 [nV, 3]
    V: np.ndarray       # complex128 [nV, npair, npair]
    beta: float
    Lambda: float       # dimensionless DLR cutoff beta * omega_max
    eps_dlr: float
    filling: float      # electrons per cell, both spins
    s_spin: int = 2
    avec: np.ndarray = field(default_factory=lambda: np.eye(3))
    orb_pos: np.ndarray | None = None   # [norb, 3] cartesian

    @property
    def nk(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    @property
    def npair(self) -> int:
        return self.norb * self.norb


# --------------------------------------------------------------------------
# interaction builders (model definitions, product basis)
# --------------------------------------------------------------------------

def kanamori_local(norb: int, U: float, J: float, Up: float | None = None) -> np.ndarray:
    """Kanamori on-site interaction in the pair basis V_{(ab),(cd)}.

    U on V_{(aa),(aa)}, U' = U - 2J on V_{(aa),(cc)} (a != c), J on the exchange
    element V_{(ab),(ba)} and on the pair-hopping element V_{(ab),(ab)} (a != b).
    """
    if Up is None:
        Up = U - 2.0 * J
    npair = norb * norb
    V = np.zeros((npair, npair), dtype=np.complex128)
    for a in range(norb):
        for c in range(norb):
            V[a * norb + a, c * norb + c] = U if a == c else Up
    for a in range(norb):
        for b in range(norb):
            if a != b:
                V[a * norb + b, b * norb + a] = J
                V[a * norb + b, a * norb + b] = J
    return V


def density_density(norb: int, Vmat: np.ndarray) -> np.ndarray:
    """Density-density coupling V_{(aa),(cc)} = Vmat[a, c] in the pair basis."""
    npair = norb * norb
    V = np.zeros((npair, npair), dtype=np.complex128)
    for a in range(norb):
        for c in range(norb):
            V[a * norb + a, c * norb + c] = Vmat[a, c]
    return V


def _finish(hops: dict, Vs: dict, norb: int):
    hop_R = np.array(sorted(hops.keys()), dtype=np.int64).reshape(-1, 3)
    hop_t = np.array([hops[tuple(R)] for R in hop_R], dtype=np.complex128).reshape(-1, norb, norb)
    V_R = np.array(sorted(Vs.keys()), dtype=np.int64).reshape(-1, 3)
    V = np.array([Vs[tuple(R)] for R in V_R], dtype=np.complex128).reshape(-1, norb * norb, norb * norb)
    return hop_R, hop_t, V_R, V


# --------------------------------------------------------------------------
# models
# --------------------------------------------------------------------------

def square_single_band(n=(8, 8, 1), t=1.0, U=2.0, beta=10.0, Lambda=100.0, eps_dlr=1e-10,
                       filling=1.0, name="square-1band") -> Model:
    """Single-band square lattice, nearest-neighbour t, local U (half filling)."""
    hops = {}
    for R in [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0)]:
        hops[R] = np.array([[t]], dtype=np.complex128)
    Vs = {(0, 0, 0): np.array([[U]], dtype=np.complex128)}
    hop_R, hop_t, V_R, V = _finish(hops, Vs, 1)
    return Model(name, tuple(n), 1, hop_R, hop_t, np.zeros(1), V_R, V, beta, Lambda, eps_dlr,
                 filling, orb_pos=np.zeros((1, 3)))


def honeycomb(n=(36, 36, 1), t=2.7, U=9.3, V1=5.5, beta=40.0, Lambda=1000.0, eps_dlr=1e-10,
              filling=2.0, name="graphene", v_range=2.0) -> Model:
    """Graphene p_z model: two sublattices, nearest-neighbour hopping t.

    Interaction: on-site U and a 1/r density-density tail V(r) = V1 * d / r for
    r <= v_range (d = carbon-carbon distance = 1; 2.0 reaches the third
    neighbours, 1.0 keeps the nearest neighbours only).
    """
    s3 = math.sqrt(3.0)
    a1 = np.array([s3, 0.0, 0.0])
    a2 = np.array([s3 / 2.0, 1.5, 0.0])
    a3 = np.array([0.0, 0.0, 10.0])
    pos = np.array([[0.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    hops, Vs = {}, {}
    for R1 in range(-3, 4):
        for R2 in range(-3, 4):
            R = (R1, R2, 0)
            T = np.zeros((2, 2), dtype=np.complex128)
            Vd = np.zeros((2, 2))
            for a in range(2):
                for b in range(2):
                    d = np.linalg.norm(pos[a] + R1 * a1 + R2 * a2 - pos[b])
                    if abs(d - 1.0) < 1e-9:
                        T[a, b] = t
                    if d < 1e-9:
                        Vd[a, b] = U
                    elif d < v_range + 1e-9:
                        Vd[a, b] = V1 * 1.0 / d
            if np.any(T != 0):
                hops[R] = T
            if np.any(Vd != 0):
                Vs[R] = density_density(2, Vd)
    hop_R, hop_t, V_R, V = _finish(hops, Vs, 2)
    return Model(name, tuple(n), 2, hop_R, hop_t, np.zeros(2), V_R, V, beta, Lambda, eps_dlr,
                 filling, avec=np.stack([a1, a2, a3]), orb_pos=pos)


def five_orbital(n=(16, 16, 1), seed=DEFAULT_SEED, U=3.0, J=0.6, Vnn=0.5, beta=40.0,
                 Lambda=2000.0, eps_dlr=1e-10, filling=6.0, sig_nn=0.5, sig_nnn=0.15,
                 name="five-orbital") -> Model:
    """Five-orbital extended Hund-Hubbard model with seeded random real hoppings.

    Draw order (SplitMix64 + Box-Muller): t(x) 25 normals (sigma sig_nn),
    t(y) 25 (sig_nn), t(x+y) = t(x-y) 25 (sig_nnn), crystal field 5 uniforms in
    [-0.3, 0.3), then t(z) 25 (sig_nn) only when N3 > 1 (a simple-tetragonal
    stack).  t(-R) = t(R)^T.  Interaction: Kanamori (U, J, U' = U - 2J) on site,
    density-density Vnn between in-plane nearest-neighbour cells (+-x, +-y), as in
    the 2-D model; the stack adds interlayer hopping only.
    """
    norb = 5
    rng = SplitMix64(seed)
    tx = rng.normals(25, sig_nn).reshape(5, 5)
    ty = rng.normals(25, sig_nn).reshape(5, 5)
    tnn = rng.normals(25, sig_nnn).reshape(5, 5)
    cf = np.array([-0.3 + 0.6 * rng.uniform() for _ in range(5)])
    three_d = n[2] > 1
    tz = rng.normals(25, sig_nn).reshape(5, 5) if three_d else None
    hops = {
        (1, 0, 0): tx, (-1, 0, 0): tx.T,
        (0, 1, 0): ty, (0, -1, 0): ty.T,
        (1, 1, 0): tnn, (-1, -1, 0): tnn.T,
        (1, -1, 0): tnn, (-1, 1, 0): tnn.T,
    }
    if three_d:
        hops[(0, 0, 1)] = tz
        hops[(0, 0, -1)] = tz.T
    hops = {k: np.asarray(v, dtype=np.complex128) for k, v in hops.items()}
    Vs = {(0, 0, 0): kanamori_local(norb, U, J)}
    nn = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0)]
    for R in nn:
        Vs[R] = density_density(norb, np.full((norb, norb), Vnn))
    hop_R, hop_t, V_R, V = _finish(hops, Vs, norb)
    return Model(name, tuple(n), norb, hop_R, hop_t, cf, V_R, V, beta, Lambda, eps_dlr, filling,
                 orb_pos=np.zeros((norb, 3)))


def hund_hubbard(norb, n=(4, 3, 2), seed=DEFAULT_SEED + 11, U=3.0, J=0.6, Vnn=0.5, beta=10.0,
                 Lambda=200.0, eps_dlr=1e-10, filling=None, sig_nn=0.5, name=None) -> Model:
    """norb-orbital extended Hund-Hubbard model with seeded random real hoppings on a
    simple-tetragonal lattice (the five-orbital model's construction for any norb).

    Draw order (SplitMix64 + Box-Muller): t(x) norb^2 normals (sigma sig_nn), t(y)
    norb^2, t(z) norb^2, crystal field norb uniforms in [-0.3, 0.3).  t(-R) = t(R)^T.
    Kanamori (U, J, U' = U - 2J) on site, density-density Vnn between nearest-neighbour
    cells along x and y.  Default filling 1.2 electrons per orbital.
    """
    rng = SplitMix64(seed)
    tx = rng.normals(norb * norb, sig_nn).reshape(norb, norb)
    ty = rng.normals(norb * norb, sig_nn).reshape(norb, norb)
    tz = rng.normals(norb * norb, sig_nn).reshape(norb, norb)
    cf = np.array([-0.3 + 0.6 * rng.uniform() for _ in range(norb)])
    hops = {(1, 0, 0): tx, (-1, 0, 0): tx.T, (0, 1, 0): ty, (0, -1, 0): ty.T,
            (0, 0, 1): tz, (0, 0, -1): tz.T}
    hops = {k: np.asarray(v, dtype=np.complex128) for k, v in hops.items()}
    Vs = {(0, 0, 0): kanamori_local(norb, U, J)}
    for R in [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0)]:
        Vs[R] = density_density(norb, np.full((norb, norb), Vnn))
    hop_R, hop_t, V_R, V = _finish(hops, Vs, norb)
    return Model(name or "hund-hubbard-%d" % norb, tuple(n), norb, hop_R, hop_t, cf, V_R, V, beta,
                 Lambda, eps_dlr, 1.2 * norb if filling is None else filling,
                 orb_pos=np.zeros((norb, 3)))


def degenerate_cubic(n=(8, 8, 8), norb=5, t=1.0, U=1.0, J=0.1, Vnn=0.2, beta=100.0,
                     Lambda=2500.0, eps_dlr=1e-10, filling=5.0,
                     name="five-orbital-degenerate") -> Model:
    """Degenerate multi-orbital extended Hund-Hubbard model on a simple cubic
    lattice: orbital-diagonal nearest-neighbour hopping t (six neighbours),
    Kanamori (U, J, U' = U - 2J) on site, density-density Vnn between all
    orbitals of nearest-neighbour cells.  No random draws."""
    nn = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    hops = {R: t * np.eye(norb, dtype=np.complex128) for R in nn}
    Vs = {(0, 0, 0): kanamori_local(norb, U, J)}
    for R in nn:
        Vs[R] = density_density(norb, np.full((norb, norb), Vnn))
    hop_R, hop_t, V_R, V = _finish(hops, Vs, norb)
    return Model(name, tuple(n), norb, hop_R, hop_t, np.zeros(norb), V_R, V, beta, Lambda, eps_dlr,
                 filling, orb_pos=np.zeros((norb, 3)))


KB_EV_PER_K = 8.617333262e-5          # Boltzmann constant (CODATA 2018), eV/K


def peierls_two_orbital(n=(3, 3, 1), seed=DEFAULT_SEED + 7, U=2.0, J=0.4, Vnn=0.3, beta=8.0,
                        Lambda=60.0, eps_dlr=1e-10, filling=1.3, name="peierls-2orb") -> Model:
    """Two-orbital square-lattice model with complex (Peierls-phase) hoppings.

    Complex, non-symmetric hoppings make G(k, tau) complex and orbital-asymmetric,
    so any transposed pair index in P, W or Sigma changes the result.
    """
    norb = 2
    rng = SplitMix64(seed)

    def cmat(sig):
        re = rng.normals(4, sig).reshape(2, 2)
        im = rng.normals(4, sig).reshape(2, 2)
        return re + 1j * im

    tx = cmat(0.6)
    ty = cmat(0.6)
    t0 = np.zeros((2, 2), dtype=np.complex128)
    t0[0, 1] = complex(rng.normal() * 0.4, rng.normal() * 0.4)
    t0[1, 0] = np.conj(t0[0, 1])
    hops = {(1, 0, 0): tx, (-1, 0, 0): tx.conj().T, (0, 1, 0): ty, (0, -1, 0): ty.conj().T,
            (0, 0, 0): t0}
    Vs = {(0, 0, 0): kanamori_local(norb, U, J)}
    for R in [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0)]:
        Vs[R] = density_density(norb, np.full((norb, norb), Vnn))
    cf = np.array([0.25, -0.15])
    hop_R, hop_t, V_R, V = _finish(hops, Vs, norb)
    return Model(name, tuple(n), norb, hop_R, hop_t, cf, V_R, V, beta, Lambda, eps_dlr, filling,
                 orb_pos=np.zeros((norb, 3)))


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

def config(name: str) -> Model:
    """Named workloads.

    square-8x8            single band, 8x8x1, beta 10, Lambda 100, eps 1e-10, U 2
    graphene-36x36        two sublattices, 36x36x1, beta 40, Lambda 1000, eps 1e-10
    five-orbital-16x16    5 orbitals, 16x16x1, beta 40, Lambda 2000, eps 1e-10
    five-orbital-32x32x8  5 orbitals, 32x32x8, beta 100, Lambda 1e4, eps 1e-12
    plus small parity cases (ragged and 3-D grids).
    """
    if name == "square-8x8":
        return square_single_band()
    if name == "graphene-36x36":
        return honeycomb()
    if name == "five-orbital-16x16":
        return five_orbital()
    if name == "five-orbital-32x32x8":
        return five_orbital(n=(32, 32, 8), beta=100.0, Lambda=1.0e4, eps_dlr=1e-12,
                            name="five-orbital-32x32x8")
    if name == "five-orbital-16x16x8":      # same beta/Lambda/eps at 1/4 of the k-points
        return five_orbital(n=(16, 16, 8), beta=100.0, Lambda=1.0e4, eps_dlr=1e-12,
                            name="five-orbital-16x16x8")
    # the paper's own models (Sec. "Validation: Electronic structure of graphene"
    # and the five-orbital benchmark of Table 1); parameters in eV, beta = 1/(k_B T),
    # dimensionless Lambda = beta * (cutoff energy)
    if name == "graphene-paper-25x25":
        beta = 1.0 / (KB_EV_PER_K * 2000.0)
        return honeycomb(n=(25, 25, 1), t=1.0, U=2.0, V1=0.2, v_range=1.0, beta=beta,
                         Lambda=100.0 * beta, name="graphene-paper-25x25")
    if name == "five-orbital-paper-8x8x8":
        return degenerate_cubic(n=(8, 8, 8), t=1.0, U=1.0, J=0.1, Vnn=0.2, beta=100.0,
                                Lambda=25.0 * 100.0, name="five-orbital-paper-8x8x8")
    if name == "graphene-paper-6x6":          # the paper's graphene parameters on a small grid
        beta = 1.0 / (KB_EV_PER_K * 2000.0)
        return honeycomb(n=(6, 6, 1), t=1.0, U=2.0, V1=0.2, v_range=1.0, beta=beta,
                         Lambda=100.0 * beta, name="graphene-paper-6x6")
    if name == "five-orbital-paper-3x3x2":    # the paper's five-orbital parameters, small grid
        return degenerate_cubic(n=(3, 3, 2), t=1.0, U=1.0, J=0.1, Vnn=0.2, beta=100.0,
                                Lambda=25.0 * 100.0, name="five-orbital-paper-3x3x2")
    # small parity cases
    if name == "five-orbital-6x5x1":
        return five_orbital(n=(6, 5, 1), beta=10.0, Lambda=200.0, name="five-orbital-6x5x1")
    if name == "five-orbital-4x3x2":
        return five_orbital(n=(4, 3, 2), beta=10.0, Lambda=200.0, name="five-orbital-4x3x2")
    if name == "graphene-6x6":
        return honeycomb(n=(6, 6, 1), beta=10.0, Lambda=300.0, name="graphene-6x6")
    if name == "peierls-3x3":
        return peierls_two_orbital()
    if name == "peierls-5x3x2":
        return peierls_two_orbital(n=(5, 3, 2), name="peierls-5x3x2")
    if name == "peierls-4x4x2":               # power-of-two 3-D grids (register FFT passes)
        return peierls_two_orbital(n=(4, 4, 2), name="peierls-4x4x2")
    if name == "five-orbital-2x4x4":
        return five_orbital(n=(2, 4, 4), beta=10.0, Lambda=200.0, name="five-orbital-2x4x4")
    if name == "peierls-32x32x8":             # the bench grid shape (specialised FFT kernels)
        return peierls_two_orbital(n=(32, 32, 8), name="peierls-32x32x8")
    if name == "peierls-16x16x8":
        return peierls_two_orbital(n=(16, 16, 8), name="peierls-16x16x8")
    if name == "three-orbital-4x3x2":         # 3- and 4-orbital Kanamori (ragged 3-D grids)
        return hund_hubbard(3, n=(4, 3, 2), name="three-orbital-4x3x2")
    if name == "four-orbital-3x2x2":
        return hund_hubbard(4, n=(3, 2, 2), name="four-orbital-3x2x2")
    if name == "square-16x1x1":               # one non-trivial axis
        return square_single_band(n=(16, 1, 1), name="square-16x1x1")
    if name == "square-1x1":
        return square_single_band(n=(1, 1, 1), name="square-1x1")
    raise KeyError(name)


CONFIG_NAMES = ["square-8x8", "graphene-36x36", "five-orbital-16x16", "five-orbital-32x32x8"]
