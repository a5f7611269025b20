"""Plain, slow FP64 CPU oracle for the GW iteration (TEST INFRASTRUCTURE ONLY).

Only the test-suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA
library never calls it and shares no code, tables or constants with it.

Contents
  dlr.py      discrete Lehmann representation built from its published
              definition (Kaye, Chen & Parcollet, PRB 105, 235115 (2022)):
              composite-Chebyshev fine grids, pivoted Gram-Schmidt selection
              of real frequencies, imaginary-time and Matsubara nodes.
  lattice.py  k- and R-grids, explicit (O(N_k^2)) lattice Fourier sums,
              H(k) and V(q) (paper Eq. for the k<->R transform).
  gw.py       one GW iteration written as the paper states it: G0 (Eqs. for
              the bare Green's function), the bubble P (Eq. for the
              polarizability), W = V + VPW (Eq. for the screened Coulomb
              interaction), Sigma^C = -G W^C (Eq. for the GW self-energy),
              Hartree and Fock terms (Eqs. for Sigma^H, Sigma^F), the Dyson
              equation for G, the chemical-potential bisection and the density
              n = -G(beta^-) (Sec. "GW self-consistency").
  qp.py       Hartree-Fock loop and quasiparticle quantities.
  free_energy.py  the GW grand potential in the Luttinger-Ward form (named in
              the paper's introduction, defined here on truncated Matsubara
              traces) on the input G of one iteration.

Every floating-point quantity is complex128/float64.  Library primitives
(matrix products, linear solves, eigh) are used as single steps; nothing is
blocked, fused or reordered.
"""
