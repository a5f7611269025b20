/*
 * qa.h -- C ABI of the GB300 GW-iteration library (libqa.so).
 *
 * One call of qa_gw_step performs one self-consistent GW iteration on a
 * k-grid with a discrete-Lehmann-representation (DLR) imaginary-time grid,
 * as described in the QAssemble paper (arXiv 2604.22223), Sec. "GW
 * self-consistency" and Fig. 3(b):
 *
 *   G(k,tau) -> G(R,tau)                 lattice FFT, Eq. (k<->R transform)
 *   P(R,tau) = -s G(R,tau) G(-R,beta-tau) bubble, Eq. (polarizability)
 *   P(q,tau) -> P(q,i nu)                DLR transform (ref. Kaye et al. 2022)
 *   W = V + V P W,  W^C = W - V          Dyson, Eq. (screened Coulomb)
 *   W^C(q,i nu) -> W^C(R,tau)            DLR + FFT
 *   Sigma^C(R,tau) = -G(R,tau) W^C(R,tau) Eq. (GW self-energy)
 *   Sigma^H, Sigma^F from n = -G(beta^-) Eqs. (Hartree, Fock self-energy)
 *   G(k,i w) = [i w + mu - H - Sigma]^-1  Eq. (Dyson for G), mu bisection
 *
 * Conventions (all arrays complex = interleaved (re, im) doubles unless noted):
 *   * k-grid (N1,N2,N3), Gamma-centred; linear index (i1*N2 + i2)*N3 + i3.
 *     The same index labels real-space cells R (j_d in [0, N_d)).
 *   * Orbital index a in [0, norb); pair index A = (a,b) -> a*norb + b;
 *     npair = norb*norb.
 *   * H_ab(R) = <a,R|H|b,0> = -t_ab(R) + delta_{R0} delta_ab eps_a.
 *     X(k) = sum_R exp(-i k.R) X(R) (cell gauge), X(i w) = int_0^beta exp(+i w tau) X(tau).
 *   * V_{(ab),(cd)}(R): interaction in the pair basis, paper V_ijkl = V_{(il),(jk)},
 *     pair (ab) on cell R, pair (cd) on cell 0.
 *   * Green's function arrays ("G layout"): [r][norb][norb][N_k] complex128,
 *     k fastest, at the r DLR imaginary-time nodes tau_j (qa_get_grid).
 *
 * Memory and execution:
 *   * qa_create copies every input; it touches no GPU and allocates no device
 *     memory.  The caller then obtains qa_workspace_size bytes of device
 *     memory (e.g. from PyTorch's allocator) and hands it over with qa_bind,
 *     which uploads the tables and builds G0.  The context owns nothing on the
 *     device; the workspace must outlive the context's use.  qa_bind also
 *     allocates one small pinned host buffer (cudaHostAlloc, mapped, < 1 KB)
 *     through which the kernels hand over scalar results (reductions, the
 *     error word, the local density); qa_destroy frees it.
 *   * Device pointers passed to calls are borrowed for the duration of the call.
 *   * All GPU work is enqueued on the caller's stream (cudaStream_t passed as
 *     void*; NULL = legacy default stream).  Calls that return host scalars
 *     (mu, densities, status) synchronise that stream before returning.
 *   * Every call returns a status code; no call aborts or traps.  Device-side
 *     failures (a singular Dyson pivot, a non-finite value) are reported
 *     through a device error word read back at the end of the call.
 *
 * Limits: 1 <= norb <= 5 (npair <= 25 fits one warp per Dyson system);
 *         N_k * 16 bytes (FP64, mixed) or * 8 bytes (FP32) must fit the FFT's
 *         shared-memory tile (N_k <= 12288); 1 <= r <= 128.
 */
#ifndef QA_H
#define QA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
enum {
  QA_OK = 0,
  QA_EINVAL = 1,      /* bad argument, size or layout                       */
  QA_ENOMEM = 2,      /* workspace too small                                */
  QA_ESINGULAR = 3,   /* a Dyson pivot below threshold (first index in stats) */
  QA_ENOCONV = 4,     /* chemical-potential search did not converge          */
  QA_ERANGE = 5,      /* non-finite values or spectrum outside the DLR window */
  QA_ETIMEOUT = 6,    /* a bounded device wait ran out                       */
  QA_ECUDA = 7,       /* a CUDA runtime call failed                          */
  QA_ESTATE = 8,      /* call out of order (e.g. step before qa_bind)        */
  QA_EBOUNDS = 9      /* an index-map gather out of range (only in a library
                         built with QA_CHECK_BOUNDS; the access was skipped)  */
};

/* arithmetic of the GPU path */
enum {
  QA_FP64 = 0,        /* complex128 storage and FP64 arithmetic everywhere   */
  QA_MIXED = 1,       /* every tensor stored as double-float (a pair of FP32
                         values hi + lo per real number, 16 bytes per complex)
                         and computed from FP32 instructions: error-free FP32
                         transformations for the FFTs, products and small
                         solves, the Dyson solve for W in FP32 refined by one
                         residual step (its dense product on the tensor cores
                         from exact fixed-point bf16 slices, the rest in
                         double-float), and the DLR maps on the tensor cores
                         from fixed-point bf16 slices; FP64 for
                         the DLR matrices, the chemical potential and density
                         sums.  Agrees with QA_FP64 to ~1e-9 relative.       */
  QA_FP32 = 2         /* complex64 storage of P, W^C and the G/Sigma stages,
                         FP32 arithmetic, split-bf16 tensor-core DLR maps
                         (the fast mode: ~1e-6 - 1e-5 relative to QA_FP64)  */
};

/* pair basis of the big tensors P(q, i nu) and W^C (qa_set_pair_basis) */
enum {
  QA_PAIRS_AUTO = 0,     /* reduced on QA_MIXED / QA_FP32, full on QA_FP64    */
  QA_PAIRS_FULL = 1,     /* all npair^2 entries (the paper's product basis)    */
  QA_PAIRS_REDUCED = 2   /* the rho^2 entries of the interaction subspace      */
};

typedef struct qa_ctx qa_ctx;

/* Crystal: the k-grid and the orbital count (paper Sec. "Crystal"). */
typedef struct {
  int n[3];           /* N1, N2, N3 >= 1                                      */
  int norb;           /* orbitals per cell (basis sites x orbitals merged)    */
  int nspin;          /* spin degeneracy s (2 = paramagnetic spin-1/2)        */
} qa_lattice;

/* One-body part H0[t, eps] (paper Eq. for the many-body Hamiltonian, first term). */
typedef struct {
  int nR;             /* number of listed lattice vectors                     */
  const int* R;       /* [nR][3] integer lattice vectors; both R and -R listed */
  const double* t;    /* [nR][norb][norb] complex: t_ab(R), H(R) = -t(R)       */
  const double* eps;  /* [norb] real on-site energies                          */
} qa_hoppings;

/* Two-body part (paper Eq. for the many-body Hamiltonian, second term). */
typedef struct {
  int nR;             /* number of listed lattice vectors                     */
  const int* R;       /* [nR][3]                                              */
  const double* V;    /* [nR][npair][npair] complex V_{(ab),(cd)}(R)           */
} qa_interaction;

/* Per-step report. */
typedef struct {
  double mu;            /* chemical potential after the step                   */
  double N;             /* electrons per cell at mu (mixed path: the FP64
                           density, linearised over the final Newton step)     */
  int mu_evals;         /* density evaluations used by the mu search           */
  int status;           /* QA_OK or the first error code seen                  */
  long long first_bad;  /* first failing system index (nu*N_k + q) or -1       */
  int launches;         /* kernels this call launched                          */
  float stage_ms[16];   /* per-stage GPU times when timing is enabled          */
} qa_step_stats;

/* qa_create: validate and copy the problem (paper Sec. "Results": Crystal, DLR,
 * H0, V), build the DLR grid (Lambda = beta*omega_max dimensionless, eps = DLR
 * tolerance; Kaye, Chen & Parcollet 2022) and the FFT plans on the host.
 * filling = electrons per cell (both spins).  precision = QA_FP64, QA_MIXED or QA_FP32.
 * Returns QA_EINVAL for sizes outside the limits above or a non-Hermitian H.
 * *out receives a new context (free with qa_destroy). */
int qa_create(const qa_lattice* lat, const qa_hoppings* hop, const qa_interaction* inter,
              double beta, double Lambda, double eps, double filling, int precision,
              qa_ctx** out);

/* qa_set_pair_basis: choose the basis of the big tensors before qa_bind
 * (QA_ESTATE afterwards; the workspace size depends on it).
 * The interaction matrices V(R) all act inside one subspace of the pair space:
 * the span of the columns of every V(R) and V(R)^H, of dimension rho (15 of 25
 * pairs for Kanamori plus density-density interactions on five orbitals, 2 of
 * 4 for a two-site density-density model).  With B an orthonormal basis of it,
 * V(q) = B S(q) B^H, the Dyson equation W = V + V P W of the paper's screened
 * interaction closes on Pt = B^H P B and S, and W^C = B Wt^C B^H exactly
 * (up to rounding): the reduced basis carries rho^2 instead of npair^2 entries
 * per (q, nu) through the bubble, both FFTs, both DLR maps and the Dyson solve.
 * This is an exact instance of the rank reduction of the orbital-index
 * contraction that the paper proposes for the O(N_orb^4) polarizability (Sec.
 * "Results", five-orbital benchmark).  QA_PAIRS_REDUCED takes effect when
 * 0 < rho < npair and the contraction term lists have at most 4096 entries;
 * otherwise the full basis is used.  qa_free_energy_backward needs the full basis. */
int qa_set_pair_basis(qa_ctx* ctx, int mode);

/* The interaction subspace: *rho its dimension, *active 1 when the big tensors
 * use it, B (may be NULL) [npair][rho] complex (interleaved doubles), the
 * orthonormal basis (columns), real and sparse for real interactions: a
 * component of pairs whose V columns have full rank keeps its unit vectors.
 * Available right after qa_create (no GPU needed). */
int qa_get_pair_basis(const qa_ctx* ctx, int* rho, int* active, double* B);

/* Bytes of device workspace qa_bind needs (tables, intermediates, G0). */
int qa_workspace_size(const qa_ctx* ctx, size_t* bytes);

/* Attach a device workspace (>= qa_workspace_size bytes, 256-byte aligned),
 * upload tables, build H(k), V(q) and the noninteracting G0 at the mu0 that
 * gives the filling (paper Eqs. for G0; "G0 class").  Synchronises `stream`. */
int qa_bind(qa_ctx* ctx, void* workspace, size_t bytes, void* stream);

/* DLR grid: r nodes; x = beta*omega_l (dimensionless real poles) [r];
 * t_rel = tau_j/beta in relative format (t>1/2 stored as t-1) [r];
 * nf = fermionic Matsubara integers n (w_n=(2n+1)pi/beta) [r];
 * mb = bosonic Matsubara integers m (nu_m = 2 m pi/beta) [r].
 * Any output pointer may be NULL. */
int qa_get_grid(const qa_ctx* ctx, int* r, double* x, double* t_rel, int* nf, int* mb);

/* Host-side plan tables (no GPU needed): minus_R [N_k] = linear index of the
 * cell -R mod N for every cell R; fft_pos [N1+N2+N3] = per axis, the
 * in-place position of frequency f after the mixed-radix stages; fft_nfac [3]
 * radix counts; fft_fac [3][16] radices in stage order.  Any pointer may be NULL. */
int qa_get_plan(const qa_ctx* ctx, int* minus_R, int* fft_pos, int* fft_nfac, int* fft_fac);

/* Sizes: N_k, norb, r.  Any pointer may be NULL. */
int qa_get_sizes(const qa_ctx* ctx, int* nk, int* norb, int* r);

/* One GW iteration (paper Fig. 3(b)).
 *   G_in   device, G layout, complex128; NULL = the context's G0.
 *   G_out  device, G layout, complex128 (may equal G_in): the new G(k, tau_j).
 *   mu_out host, new chemical potential;  n_out host [norb][norb] complex,
 *          local density matrix n(R=0) = -G(R=0, beta^-) of the new G.
 * Intermediates (P, W^C, Sigma^C, Sigma^HF) stay in the workspace; read them
 * with qa_get.  Returns QA_ESINGULAR / QA_ENOCONV / QA_ERANGE on failure. */
int qa_gw_step(qa_ctx* ctx, const void* G_in, void* G_out, double* mu_out, double* n_out,
               qa_step_stats* stats, void* stream);

/* Hold the chemical potential fixed (fixed = 1: every qa_gw_step uses `mu`
 * instead of the search; fixed = 0: search again).  The frozen-mu reading is
 * the one the adjoint differentiates. */
int qa_set_mu(qa_ctx* ctx, int fixed, double mu);

/* Replace the hopping amplitudes, on-site energies and interaction values of a
 * bound context (same R lists, same order as at qa_create); rebuilds H(k) and
 * V(q) on the device.  Used for finite differences and for optimisation loops. */
int qa_set_params(qa_ctx* ctx, const qa_hoppings* hop, const qa_interaction* inter, void* stream);

/* qa_gw_backward: hand-written adjoint of one qa_gw_step at fixed chemical
 * potential `mu` (the value the forward step used), FP64 contexts only.
 * For a real loss L of the step's outputs the caller passes the cotangents
 * (Xbar = dL/dRe X + i dL/dIm X, each may be NULL = zero):
 *   Gbar_out  device, G layout complex128: cotangent of the new G(k, tau_j);
 *   Sigbar    device, [r][norb][norb][N_k] complex128: cotangent of Sigma^C(k, tau_j);
 *   nbar      host [norb][norb] complex: cotangent of the local density n(R=0).
 * Outputs (each may be NULL):
 *   Gbar_in   device, G layout complex128: cotangent of G_in (chains iterations);
 *   grad_t    host [nR_hop][norb][norb] complex: dL/dRe t(R) + i dL/dIm t(R) per
 *             listed hopping matrix (t(R) and t(-R) are separate entries);
 *   grad_V    host [nR_V][npair][npair] complex: the same for V(R).
 * The forward stages are recomputed from G_in (nothing is kept from an earlier
 * step), so an unrolled loop checkpoints only its G's and mu's.  Adjoints:
 * FFT -> inverse FFT, DLR map -> conjugate transpose, Dyson -> -G^H Gbar G^H,
 * W Dyson -> Pbar = W^H Wbar W^H, Vbar = (1-VP)^-H Wbar (1+PW)^H - Wbar, with the
 * LU factors of 1 - VP that the recomputed forward W Dyson solve keeps (one per
 * (q, i nu), in the workspace).  Either pair basis: on the reduced one the
 * bubble and self-energy adjoints walk the forward's term lists, the Dyson
 * adjoint runs in the rho-dimensional subspace (S = B^H V B) and grad_V is
 * B Sbar B^H plus the Hartree-Fock part; on the subspace (Pi grad_V Pi,
 * Pi = B B^H, the directions in which V can move without changing the
 * subspace) it equals the full basis' gradient.
 * Synchronises `stream`. */
int qa_gw_backward(qa_ctx* ctx, const void* G_in, double mu, const void* Gbar_out,
                   const void* Sigbar, const double* nbar, void* Gbar_in, double* grad_t,
                   double* grad_V, void* stream);

/* qa_free_energy: the GW grand potential per unit cell in the Luttinger-Ward
 * form, evaluated on the input G of one iteration at fixed chemical potential
 * `mu` (the paper's introduction names the Luttinger-Ward functional as the
 * target of a differentiable GW code without writing it down; this is the
 * reading used, with truncated Matsubara traces):
 *   Omega = Omega_HF + Omega_dc + Omega_G + Omega_W, parts[] in this order,
 *   Omega_HF = -(s/(beta N_k)) sum_{k,i} ln(1 + exp(-beta (e_i(k) - mu))), e_i the
 *              eigenvalues of the Hermitian part of H(k) + Sigma^HF(k);
 *   Omega_dc = -(1/2)(s/N_k) sum_k Re tr[Sigma^HF(k) n(k)];
 *   Omega_G  = -(s/(beta N_k)) sum_k sum_{n=-M}^{M-1}
 *              Re{ln det[1 - G_HF Sigma^C] + tr[Sigma^C G]}(k, i w_n),
 *              G_HF = (i w_n + mu - H - Sigma^HF)^-1;
 *   Omega_W  = (1/(2 beta N_k)) sum_q sum_{m=-M}^{M}
 *              Re{ln det[1 - V(q) P(q, i nu_m)] + tr[V(q) P(q, i nu_m)]},
 * with Sigma = Sigma^HF + Sigma^C and P computed from G_in as qa_gw_step does,
 * and Sigma^C, G, P at the uniform frequencies from their DLR expansions.
 *   G_in   device, G layout complex128, or NULL = G0;
 *   M      Matsubara cutoff (1 .. 2^20); part of the definition;
 *   omega  host scalar, parts host [4] (either may be NULL).
 * FP64 contexts only (QA_EINVAL otherwise); either pair basis.  The first call
 * for a cutoff allocates the uniform-frequency maps and a scratch (cudaMalloc,
 * kept until qa_destroy; QA_ENOMEM if it fails); a singular 1 - V P or
 * Dyson matrix gives QA_ESINGULAR.  Synchronises `stream`. */
int qa_free_energy(qa_ctx* ctx, const void* G_in, double mu, int M, double* omega, double* parts,
                   void* stream);

/* qa_free_energy_backward: gradient of omega_bar * Omega (qa_free_energy, same
 * G_in, mu, M) through the adjoint of the iteration's stages (qa_gw_backward's
 * chain, with Omega's explicit cotangents added where its terms read Sigma^HF,
 * n, H, Sigma^C, G, P and V).  Outputs as qa_gw_backward (Gbar_in device,
 * grad_t and grad_V host; each may be NULL).  FP64 contexts, full pair basis
 * (QA_ESTATE otherwise).  Synchronises `stream`. */
int qa_free_energy_backward(qa_ctx* ctx, const void* G_in, double mu, int M, double omega_bar,
                            void* Gbar_in, double* grad_t, double* grad_V, void* stream);

/* qa_hf_solve: self-consistent Hartree-Fock (paper Sec. "Hartree-Fock
 * self-consistency" and Fig. 3(a), the first stage of the QAssemble workflow).
 * Starting from the Fermi-Dirac density of H0 at its own chemical potential,
 * each iteration builds Sigma^HF(k) = Sigma^H + Sigma^F(k) from n(k) (the same
 * Hartree and Fock equations as qa_gw_step), mixes it,
 *   Sigma^HF <- Sigma^HF_old + mix (Sigma^HF_new - Sigma^HF_old),
 * diagonalises H(k) + Sigma^HF(k) per k (FP64 Jacobi rotations), sets mu to
 * the filling (s/N_k) sum_{k,i} f(beta (E_ki - mu)) = filling, and takes
 * n(k) = U f(beta (E - mu)) U^H.  It stops when max |Sigma^HF_new -
 * Sigma^HF_old| <= tol or after max_iter iterations.  Arguments: max_iter >= 1;
 * tol >= 0; 0 < mix <= 1 (1 = plain iteration).  Outputs (each may be NULL):
 *   G_out     device, G layout complex128: the HF Green's function
 *             G(k, i w) = (i w + mu - H - Sigma^HF)^-1 on the tau nodes, the
 *             usual starting point of qa_gw_step;
 *   mu_out, iters_out, resid_out: host scalars (last change of Sigma^HF);
 *   n_out     host [norb][norb] complex: local density matrix of the result.
 * Sigma^HF stays in the workspace (qa_get QA_SIGHF_K), mu becomes the warm
 * start of the next mu search, and qa_qp then uses Sigma^HF alone (Z = 1).
 * Returns QA_ENOCONV (outputs filled) when tol was not reached.  Needs the
 * workspace scratch of three N_k norb^2 complex arrays (r >= 3: QA_ENOMEM
 * otherwise).  Synchronises `stream`. */
int qa_hf_solve(qa_ctx* ctx, int max_iter, double tol, double mix, void* G_out, double* mu_out,
                int* iters_out, double* resid_out, double* n_out, void* stream);

/* qa_qp: quasiparticle quantities from the self-energy of the last qa_gw_step
 * (Sigma^HF and Sigma^C(k, i w) of that step; after qa_hf_solve, Sigma^HF
 * alone) and the current H(k) (paper Secs. on the renormalisation factor and
 * the static self-energy, and the quasiparticle Hamiltonian of the graphene
 * results):
 *   Sigma(+-i w0), w0 = pi/beta, from the DLR expansion of Sigma^C(k, i w_n);
 *   Sig0 = Sigma^HF + (Sigma(i w0) + Sigma(-i w0)) / 2          (Sigma at w = 0)
 *   Z    = [1 - (Sigma(i w0) - Sigma(-i w0)) / (2 i w0)]^-1      (Hermitian part inverted)
 *   Hqp  = sqrt(Z) (H0 + Sig0) sqrt(Z)  (Hermitian parts; sqrt(Z) the positive root)
 *   eps  = eigenvalues of Hqp, ascending.
 * The limit w -> 0 is taken on the Matsubara axis at the lowest fermionic
 * frequencies (continuing the DLR pole form to w = 0 is ill-conditioned).
 * Outputs: device, [N_k][norb][norb] complex128 (eps: [N_k][norb] double); each
 * may be NULL.  QA_ESTATE before any step or HF solve; QA_ERANGE when some
 * Z(k)^-1 is not positive definite.  Synchronises `stream`. */
int qa_qp(qa_ctx* ctx, void* Z, void* Sig0, void* Hqp, double* eps, void* stream);

/* Density of a G in G layout (device): n_out [norb][norb] complex local density
 * matrix -G(R=0, beta^-), *N_total = s * Tr n (electrons per cell). */
int qa_density(qa_ctx* ctx, const void* G, double* n_out, double* N_total, void* stream);

/* qa_density_static: the result of qa_density without any device allocation.
 * The paper has no counterpart; this entry point exists for callers that cannot
 * call cudaMalloc (host callbacks, error handlers, plug-ins inside a framework
 * that owns every device allocation, real-time loops where an allocation may
 * block).  It needs only a context from qa_create (no qa_bind, no workspace) and
 * the caller's device G (G layout, complex128).  Its scratch is a file-scope
 * static __device__ array of 4 MiB that every GPU loading the library holds
 * until process exit; problems with (r + norb^2 * (N_k + 1)) * 16 bytes (each
 * part rounded up to 256) above 4 MiB are rejected with QA_ENOMEM (five orbitals
 * fit up to N_k = 10,480).  All calls
 * on a device share that array and it keeps the last call's contents: calls
 * whose GPU work overlaps (other streams or threads) race and give wrong
 * results.  The first call on a device looks up the array's address.
 * Synchronises `stream`. */
int qa_density_static(const qa_ctx* ctx, const void* G, double* n_out, double* N_total,
                      void* stream);

/* qa_fma_probe: arithmetic-rate probe (a measurement utility; the paper has no
 * counterpart).  Enqueues on `stream` one kernel of 8 blocks per SM x 256
 * threads in which every thread runs eight independent chains of `iters` fused
 * multiply-adds in FP64 (precision = QA_FP64) or FP32 (QA_FP32), writing one
 * value per thread to `out` (device, *out_elems doubles or floats, caller
 * owned).  *flops receives the kernel's floating-point operations (2 per FMA);
 * the caller times the launch to obtain the GPU's FMA rate.  out = NULL only
 * reports *out_elems and *flops.  QA_EINVAL for iters < 1 or another precision. */
int qa_fma_probe(int precision, int iters, void* out, long long* out_elems, double* flops,
                 void* stream);

/* Intermediates of the last step / of qa_bind, copied to dst (host or device):
 * element type complex128 for QA_FP64, double-float complex for QA_MIXED (four
 * floats re.hi, re.lo, im.hi, im.lo; value = hi + lo) and complex64 for
 * QA_FP32, except where noted.  bytes must equal the array size.  With the reduced pair basis active
 * (qa_get_pair_basis) the two big tensors are held and returned as
 * B^H P B and B^H W^C B: [r][rho][rho][N_k]. */
enum {
  QA_P_QNU = 1,       /* P(q, i nu_m)        [r][npair][npair][N_k]           */
  QA_WC_RTAU = 2,     /* W^C(R, tau_j)       [r][npair][npair][N_k]           */
  QA_SIGC_KTAU = 3,   /* Sigma^C(k, tau_j)   [r][norb][norb][N_k]             */
  QA_SIGC_KIW = 4,    /* Sigma^C(k, i w_n)   [r][norb][norb][N_k]             */
  QA_SIGHF_K = 5,     /* Sigma^H + Sigma^F   [N_k][norb][norb], complex128    */
  QA_G0 = 6,          /* G0(k, tau_j)        G layout, complex128             */
  QA_HK = 7,          /* H(k)                [N_k][norb][norb], complex128    */
  QA_MU0 = 8          /* mu0 of G0, one double                                */
};
int qa_get(const qa_ctx* ctx, int which, void* dst, size_t bytes, void* stream);

/* qa_set_wait_limit: a diagnostics control of the tensor-core DLR kernels (the
 * paper has no counterpart).  Their producer/consumer pipeline waits on shared
 * memory barriers, each wait bounded by `polls` polls (default 2^24; polls < 0
 * restores it).  A wait that runs out takes the kernel's time-out path: the
 * error word becomes QA_ETIMEOUT (returned by the call), the kernel lets the
 * tensor-core operations it already issued finish (with the default bound),
 * releases its tensor memory and returns, so the context stays usable.
 * polls = 0 makes every pipeline wait give up at once: a way to exercise that
 * path without any fault.  Host only; takes effect from the next call. */
int qa_set_wait_limit(qa_ctx* ctx, long long polls);

/* Enable per-stage CUDA-event timing in qa_step_stats (0/1). */
int qa_set_timing(qa_ctx* ctx, int enable);

void qa_destroy(qa_ctx* ctx);
const char* qa_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* QA_H */
