// Internal declarations shared by the host planner (qa_api.cpp, qa_dlr.cpp)
// and the CUDA kernels (qa_*.cu).  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <complex>
#include <vector>

#include <cuda_runtime.h>

struct qa_ctx;

namespace qa {

struct dfl;   // double-float real (qa_df.cuh); complex arrays of it are dfc

// Device-side copy of the public status code for a singular pivot.
constexpr int QA_ESINGULAR_CODE = 3;
constexpr int QA_ETIMEOUT_CODE = 6;
constexpr int QA_EBOUNDS_CODE = 9;

// ------------------------------------------------------------------- DLR
// Discrete Lehmann representation (Kaye, Chen & Parcollet, PRB 105, 235115
// (2022)); dimensionless real poles x_l = beta*omega_l, imaginary-time nodes
// t_j = tau_j/beta in relative format (t > 1/2 stored as t - 1), fermionic
// and bosonic Matsubara integers.
struct DlrGrid {
  int r = 0;
  std::vector<double> x, t;
  std::vector<int> nf, mb;
};
int build_dlr(double Lambda, double eps, DlrGrid* out);

// Transform matrices composed in extended precision on the host, physical
// units, row-major [rows][r], complex interleaved as std::complex<double>.
struct DlrMatrices {
  std::vector<std::complex<double>> Trefl;  // G(k, beta - tau_j) from G(k, tau)
  std::vector<std::complex<double>> Ttn;    // tau -> i nu (bosonic)
  std::vector<std::complex<double>> Tnt;    // i nu -> tau
  std::vector<std::complex<double>> Ttw;    // tau -> i w (fermionic)
  std::vector<std::complex<double>> Twt;    // i w -> tau
  std::vector<std::complex<double>> dtau;   // n = sum_j dtau_j G(tau_j)
  std::vector<std::complex<double>> dw;     // n = sum_n dw_n G(i w_n)
  std::vector<std::complex<double>> wq_p;   // X(+i pi/beta) = sum_n wq_p[n] X(i w_n)
  std::vector<std::complex<double>> wq_m;   // X(-i pi/beta) = sum_n wq_m[n] X(i w_n)
  std::vector<double> iw;                   // w_n values (imaginary parts)
};
void build_dlr_matrices(const DlrGrid& g, double beta, DlrMatrices* m);
// Uniform-frequency evaluation of DLR expansions, physical units, row-major:
// EF [2M][r]: X(i w_n) = sum_j EF[n+M][j] X(tau_j), n = -M .. M-1;
// EB [2M+1][r]: X(i nu_m) = sum_j EB[m+M][j] X(i nu_j) (bosonic DLR nodes).
void build_uniform_maps(const DlrGrid& g, double beta, int M, std::vector<std::complex<double>>* EF,
                        std::vector<std::complex<double>>* EB);

// ------------------------------------------------------------ pair basis
// Orthonormal basis B (npair x rho, row-major [A][j]) of the subspace that the
// interaction matrices V(R) act in (qa_basis.cpp); returns rho (0: no V).
int reduced_pair_basis(const std::vector<std::complex<double>>& VR, int nV, int npair,
                       std::vector<std::complex<double>>* B);

// Term lists of the reduced bubble and self-energy contractions, one list per
// reduced output entry o = i*rho + j (terms off[o] .. off[o+1]-1).
//   bubble: Pt_ij += coef * G[idx & 255] * G^refl[idx >> 8]
//   sigma:  Sigma[idx >> 8] += coef * G[idx & 255] * Wt_ij
struct PairTerms {
  std::vector<int> off;
  std::vector<int> idx;
  std::vector<std::complex<double>> coef;
  bool distinct_targets = false;   // no output list holds two terms with the same idx >> 8
};
void pair_basis_terms(const std::vector<std::complex<double>>& B, int norb, int rho, double s,
                      PairTerms* bubble, PairTerms* sigma);

// ------------------------------------------------------------------- FFT
// Mixed-radix decimation-in-frequency plan for one axis of length L: the
// radices in stage order, and pos[f] = position of frequency f after the
// in-place stages (a mixed-radix digit reversal).
struct FftAxisPlan {
  int L = 1;
  int nfac = 0;
  int fac[16] = {0};
};
void plan_fft_axis(int L, FftAxisPlan* p, std::vector<int>* pos);

constexpr int kMaxFac = 16;

struct FftDev {            // passed by value to the FFT kernel
  int n[3];
  int nfac[3];
  int fac[3][kMaxFac];
  int tw_off[3];           // offset of each axis' twiddle table in tw[]
  int pos_off[3];          // offset of each axis' position table in pos[]
  const void* tw;          // complex (precision of the kernel) exp(-2 pi i m / L)
  const int* pos;
};

// ------------------------------------------------------------- kernels
// All launchers enqueue on `st` and return cudaGetLastError().
// Complex arrays are double2 (FP64), float2 (FP32) or dfc (double-float, qa_df.cuh);
// the template argument T is double, float or dfl.

// out[j][c] = sum_l T[j][l] in[l][c], j < rows_out, l < r, c < ncol.
// in and out may alias (each block stages its columns before writing).
// accumulate != 0: out[j][c] += ... (in and out must not alias then).
template <typename T>
cudaError_t launch_dlr_apply(const void* Tm, int rows_out, int r, const void* in, void* out,
                             long long ncol, cudaStream_t st, int accumulate = 0);

// Tensor-core (tcgen05) DLR transform of FP32 complex columns, in place allowed.
// Bsplit: the packed operand of pack_dlr_tc.  Supported when 2r <= 186.
bool dlr_tc_supported(int r, size_t* smem_bytes);
void pack_dlr_tc(const std::complex<double>* T, int r, std::vector<uint16_t>* dst);
// out_c128: store the result as complex128 (out must not alias in then).
// wait_limit: polls of each pipeline mbarrier wait (< 0: the default, 2^24).
cudaError_t launch_dlr_tc(const void* Bsplit, int r, const void* in, void* out, long long ncol,
                          int* err, cudaStream_t st, bool out_c128 = false, long long wait_limit = -1);

// Accurate DLR transform of double-float (dfc) columns on the tensor cores from
// fixed-point bf16 slices (qa_dlr_oz.cu); out must not alias in.  The packed
// operand (pack_dlr_oz) holds, per part of at most 96 output rows of the real
// embedding, five slices [Nw][Kp] in the canonical layout, then the row
// exponents.  Supported when 2r <= 192.
struct DlrOzLayout {
  int nparts = 0, Kp = 0;
  int n0[2] = {0, 0}, Nw[2] = {0, 0};
  long long off[2] = {0, 0};
  long long rexp_off = 0, bytes = 0;
  size_t smem = 0;
};
DlrOzLayout dlr_oz_layout(int r);
bool dlr_oz_supported(int r);
void pack_dlr_oz(const std::complex<double>* T, int r, std::vector<uint8_t>* dst);
// out_c128: store complex128 instead of double-float.  colscale: device scratch of
// ncol floats (the per-column slice grid, written by a streaming pass that this
// call launches first: two kernels per call).  code (optional, [r][ncol] bytes):
// the grid codes (oz_grid_code) that the kernel producing `in` stored beside it;
// the pass then reads them instead of the values.
cudaError_t launch_dlr_oz(const void* pack, int r, const void* in, void* out, long long ncol,
                          int* err, cudaStream_t st, bool out_c128, long long wait_limit, float* colscale,
                          const uint8_t* code = nullptr);

// Batched 3-D FFT of contiguous lines of N_k points (in place allowed).
// sign = -1: X(k) = sum_R e^{-ikR} X(R); sign = +1: (1/N_k) sum_k e^{+ikR} X(k).
// scale > 0 replaces the default factor (1 for sign -1, 1/N_k for sign +1).
template <typename T>
cudaError_t launch_fft3d(const FftDev& plan, int sign, const void* in, void* out, long long nlines,
                         cudaStream_t st, double scale = 0.0);

// Bubble and R -> q transform in one pass (power-of-two axes <= 32, see
// fft3d_bubble_supported): line (t, o) of out = FFT over R of
// sum_{terms of o} coef G[t][g1][R] Grefl[t][g2][mR[R]] (term lists as for
// launch_bubble_reduced, at most max_terms terms per output, <= 640).
// code (optional, double-float only): [r][nout N_k] bytes, the grid code of every
// stored value (oz_grid_code), written where fft3d_bubble_codes(plan) holds and
// left untouched otherwise.
bool fft3d_bubble_supported(const FftDev& plan);
bool fft3d_bubble_codes(const FftDev& plan);
template <typename T>
cudaError_t launch_fft3d_bubble(const FftDev& plan, const void* GR, const void* GreflR,
                                const int* mR, const int* terms, const void* coef, int max_terms,
                                int nout, int norb, void* out, int r, cudaStream_t st, int* err = nullptr,
                                bool real_coef = false, unsigned char* code = nullptr);

// P[t][(ab)][(cd)][R] = -s G[t][b][c][R] Grefl[t][d][a][mR[R]]
template <typename T>
cudaError_t launch_bubble(const void* GR, const void* GreflR, const int* mR, void* P, int r,
                          int norb, int nk, double s, cudaStream_t st);

// Diagonal blocks of V(q) (or S(q)): index i couples only to [lo[i], hi[i]);
// nblk = 0: no block structure known.
struct DysonBlocks {
  int nblk = 0;
  unsigned char lo[16] = {0}, hi[16] = {0};
};

// W^C(q, i nu) from P(q, i nu) and V(q): per (nu, q) system of size npair.  blk
// (optional, FP32 systems of size <= 16): V(q)'s block structure, used to skip
// its zero blocks in V P and V P V.  lu, piv (optional, FP64 only): keep the
// LU factors of 1 - V P (row-pivoted, unit L below the diagonal; layout of P)
// and the pivot row of each column ([r][npair][N_k] bytes) for the adjoint.
template <typename T>
cudaError_t launch_dyson_w(const void* P, const void* Vq, void* WC, int r, int npair, int nk,
                           int* err, long long* first_bad, cudaStream_t st,
                           const DysonBlocks* blk = nullptr, void* lu = nullptr,
                           unsigned char* piv = nullptr);

// Accurate mixed path (qa_dyson_df.cu): W^C from double-float P and S(q), an FP32
// Gauss-Jordan solve refined by one double-float residual step; n <= 16, out of
// place.
bool dyson_w_df_supported(int n);
// real_s: S(q) is real for every q (its imaginary parts are not read).  code
// (optional): [r][n^2 N_k] bytes, the grid code of every stored value (oz_grid_code).
cudaError_t launch_dyson_w_df(const void* P, const void* Vq, void* WC, int r, int n, int nk,
                              int* err, long long* first_bad, cudaStream_t st,
                              const DysonBlocks* blk = nullptr, bool real_s = false,
                              unsigned char* code = nullptr);

// Sigma^C[t][a][d][R] = -sum_bc G[t][b][c][R] W^C[t][(ab)][(cd)][R]
template <typename T>
cudaError_t launch_sigma(const void* GR, const void* WC, void* Sig, int r, int norb, int nk,
                         cudaStream_t st);

// Reduced-basis bubble and self-energy (qa_reduced.cu).  terms: int
// off[nout + 1] followed by int idx[nterm]; coef: cplx<T>[nterm].
//   Pt[t][o][R] = sum_terms coef * GR[t][g1][R] * GreflR[t][g2][mR[R]]
//   Sig[t][e][R] = sum_o sum_terms coef * GR[t][g][R] * Wt[t][o][R]
constexpr int kMaxPairTerms = 4096;
template <typename T>
cudaError_t launch_bubble_reduced(const void* GR, const void* GreflR, const int* mR,
                                  const int* terms, const void* coef, int nterm, void* Pt, int r,
                                  int norb, int rho, int nk, cudaStream_t st);
// distinct != 0 (PairTerms::distinct_targets): the terms of one output entry
// update distinct Sigma entries and run in parallel.
template <typename T>
cudaError_t launch_sigma_reduced(const void* GR, const void* Wt, const int* terms, const void* coef,
                                 int nterm, void* Sig, int r, int norb, int rho, int nk,
                                 cudaStream_t st, int distinct = 0);
// The Sigma term list of the canonical reduced basis (the norb diagonal pairs as
// unit vectors, then one vector on {(a,b), (b,a)} per a < b in lexicographic
// order; Kanamori-type interactions) has a fixed index pattern.  Returns norb
// when off/idx (PairTerms of pair_basis_terms) follow it and a compile-time
// kernel exists for norb (2 to 5), else 0.
int sigma_canonical_norb(const int* off, const int* idx, int nout, int nterm, int norb);
// FP32 Sigma on such a basis: same inputs, outputs and bits as
// launch_sigma_reduced<float>; coef: the list's norb^4 coefficients (host).
cudaError_t launch_sigma_canonical(const void* GR, const void* Wt, const std::complex<double>* coef,
                                   int norb, void* Sig, int r, int nk, cudaStream_t st);
// Sigma in double-float (dfc G, Wt and Sigma; accurate mixed path) from the sigma
// term lists regrouped by target entry: toff[norb^2 + 1], tidx[nterm] = (Wt entry,
// G entry) as int2, tcoef[nterm] dfc.  Any pair basis (nout = nb^2 entries of Wt).
cudaError_t launch_sigma_target_df(const void* GR, const void* Wt, const int* toff, const void* tidx,
                                   const void* tcoef, void* Sig, int r, int norb, int nout, int nk,
                                   cudaStream_t st, int* err = nullptr, bool real_coef = false);

// Dyson for G.  prep: Bm[n][a][b][k] = (mu_ref - H(k) - SigHF(k))_ab - SigIw[n][a][b][k]
// (SigHF FP64 [N_k][norb][norb] and SigIw may be null) and per-block bounds
// part[2 b] of the row-sum norm of H + Sigma - mu_ref over all (k, n).
template <typename T>
cudaError_t launch_dyson_g_prep(const double2* Hk, const double2* SigHF, const void* SigIw,
                                double mu_ref, int r, int norb, int nk, void* Bm, double* part,
                                int nblocks, cudaStream_t st);
// G = (i w_n + dmu + Bm)^-1 with dmu = mu - mu_ref (mus non-null: mus[0] -
// mus[1] read on the device).  mode 0: per-block partial sums of
// Re(dw_n Tr G) and Re(dw_n Tr G^2) into part[2*blocks]; mode 1: also store
// G(k, i w_n) in Giw [r][norb][norb][N_k].
template <typename T>
cudaError_t launch_dyson_g(const void* Bm, const void* dw, const double* iw, double dmu, int r,
                           int norb, int nk, void* Giw, double* part, int nblocks, int mode,
                           int* err, cudaStream_t st, const double* mus = nullptr);

// State of the device-side chemical-potential search (qa_mu.cu); mu and
// mu_ref come first (the density kernel reads them).
struct MuState {
  double mu, mu_ref;
  double target, tolN, wid, wlo, whi;
  double N, dN, f, d, mu0, f0, d0;
  double a, fa, b, fb, db, step, dir;
  double lo, hi, dx, dxold;
  int phase, count, status, it, m, fp64, nt;
};
// Start the search at mu_s (the density table Bm folded with mu_ref = mu_s);
// bound[0]: the bound of ||H + Sigma - mu_s|| that sets the window.
cudaError_t launch_mu_init(MuState* s, const double* bound, double mu_s, double target, double beta,
                           int fp64, cudaStream_t st);
// Reduce the density sums of the last evaluation, advance the search and set
// the while-node condition `cond` (non-zero while the search goes on).  Only
// inside a graph with that conditional node.
cudaError_t launch_mu_update(const double* part, int nblocks, MuState* s, double nspin, int nk,
                             cudaGraphConditionalHandle cond, cudaStream_t st);
int dyson_g_blocks(int r, int nk);
// FP64-accurate density sums (mode 0) at mu with Sigma^C(k, i w) stored as
// complex64, from FP32 arithmetic: FP32 inverse and one residual correction in
// double-float (two launches; hs = scratch of N_k * norb^2 * 16 bytes).
cudaError_t launch_dyson_g_refine(const double2* Hk, const double2* SigHF, const void* SigIw,
                                  const void* dw, const double* iw, double mu, int r, int norb,
                                  int nk, void* hs, double* part, int nblocks, int* err,
                                  cudaStream_t st);

// Deterministic final reduction of `n` partial pairs (sum or max).
cudaError_t launch_reduce_pairs(const double* part, int n, int op_max, double* out,
                                cudaStream_t st);

// H(k) and V(q) tables from their R lists (FP64).
cudaError_t launch_ft_table(const int* R, const double2* XR, int nR, int msize, const int* kpts,
                            int nk, int n1, int n2, int n3, double2* out, cudaStream_t st);

// ph[v][k] = e^{+i k.R_v} (FP64) for a list of R.
cudaError_t launch_phase_table(const int* R, int nR, int nk, int n1, int n2, int n3, double2* ph,
                               cudaStream_t st);

// n(R_v) = (1/N_k) sum_k e^{+i k.R_v} n(k) for the interaction's R list,
// n(k) given as [norb^2][N_k] FP64; phases from ph ([nRv][N_k]) when given.
cudaError_t launch_density_R(const double2* nk_, const int* R, int nRv, int norb2, const int* kpts,
                             int nk, int n1, int n2, int n3, double2* nR_out, cudaStream_t st,
                             const double2* ph = nullptr);

// Sigma^H and Sigma^F(R_v) (one block), then Sigma^HF(k) per k (phases from ph when given).
cudaError_t launch_hf(const double2* VR, const double2* nR_in, const int* R, int nRv, int norb,
                      double s, const int* kpts, int nk, int n1, int n2, int n3, double2* sigF_R,
                      double2* SigHF, cudaStream_t st, const double2* ph = nullptr);

// n(k) = sum_j dtau_j G(k, tau_j) (FP64, [ncol]) of a complex128 G [r][ncol], and
// its complex64 copy G32 when G32 != null (one pass; r <= 128).  real_w: every
// dtau_j is real (the DLR weights f K_tau^-1 are), so each term takes two FP64
// FMAs instead of four (same values).
cudaError_t launch_g_input(const double2* G, const double2* dtau, int r, long long ncol,
                           float2* G32, double2* nk_out, cudaStream_t st, bool real_w = false);

// The same with a double-float (dfc: re.hi, re.lo, im.hi, im.lo) copy of G.
cudaError_t launch_g_input_df(const double2* G, const double2* dtau, int r, long long ncol,
                              void* Gdf, double2* nk_out, cudaStream_t st, bool real_w = false);

// Local average over k: out[e] = (1/N_k) sum_k x[e][k], e < m (FP64 out).
template <typename T>
cudaError_t launch_k_average(const void* x, int m, int nk, double2* out, cudaStream_t st);

// ---- adjoint (FP64), qa_adjoint.cu
cudaError_t launch_dyson_g_bwd(const double2* Hk, const double2* SigHF, const double2* SigIw,
                               const double* iw, double mu, int r, int norb, int nk,
                               const double2* Gbar_iw, double2* SigCbar_iw, double2* Sbar,
                               cudaStream_t st);
cudaError_t launch_sigma_bwd(const double2* GR, const double2* SigbarR, double2* W, double2* GRbar,
                             int r, int norb, int nk, cudaStream_t st);
cudaError_t launch_bubble_bwd(const double2* GR, const double2* GL, const int* mR,
                              const double2* Pbar, double2* GRbar, double2* GLbar, int r, int norb,
                              int nk, double s, cudaStream_t st);
// Reduced pair basis: adjoints of the term-list bubble and self-energy
// (terms: off[nb2 + 1] then idx[]; coef complex128), one thread per (tau, R).
cudaError_t launch_sigma_bwd_terms(const double2* GR, const double2* SigbarR, double2* W, double2* GRbar,
                                   const int* terms, const double2* coef, int r, int nb2, int norb, int nk,
                                   cudaStream_t st);
cudaError_t launch_bubble_bwd_terms(const double2* GR, const double2* GL, const int* mR, const double2* Pbar,
                                    double2* GRbar, double2* GLbar, const int* terms, const double2* coef,
                                    int r, int nb2, int norb, int nk, cudaStream_t st);
// lu, piv (may be NULL): the factors kept by launch_dyson_w for the same P and
// V; without them the kernel factorises 1 - V P itself.
cudaError_t launch_dyson_w_bwd(const double2* P, const double2* Vq, double2* Wb, double* Vqbar,
                               int r, int npair, int nk, int* err, cudaStream_t st,
                               const double2* lu = nullptr, const unsigned char* piv = nullptr);
cudaError_t launch_hf_bwd(const double2* VR, const double2* nR, const double2* X, int nV, int norb,
                          double s, int nk, double2* VbarHF, double2* nbarR, cudaStream_t st);
cudaError_t launch_nbar_k(const double2* nbarR, const int* R, int nV1, int np, int nk, int n1,
                          int n2, int n3, double2* nbk, cudaStream_t st);
cudaError_t launch_add_dw_nbar(double2* Gbar_iw, const double2* dw, const double2* nbar, int r,
                               int np, int nk, cudaStream_t st);
cudaError_t launch_axpy(double2* y, const double2* x, double a, long long n, cudaStream_t st);
cudaError_t launch_scale(double2* y, double a, long long n, cudaStream_t st);

// ---- Hartree-Fock loop and quasiparticle quantities (FP64), qa_qp.cu
// E[k][i] (ascending) and U[k][a][i] of the Hermitian part of H(k) + SigHF(k)
// (SigHF may be null); both [N_k][norb][norb].
cudaError_t launch_hf_eig(const double2* Hk, const double2* SigHF, int norb, int nk, double* E,
                          double2* U, cudaStream_t st);
// part[2b] >= max E, part[2b+1] >= max(-E) (bounds for a bracket), n = N_k norb
cudaError_t launch_fd_range(const double* E, long long n, double* part, int nblocks,
                            cudaStream_t st);
// part[2b], part[2b+1]: block sums of f(beta (E - mu)) and beta f (1 - f)
cudaError_t launch_fd_sum(const double* E, long long n, double beta, double mu, double* part,
                          int nblocks, cudaStream_t st);
// n(k) = U f(beta (E - mu)) U^H into nk_out [norb^2][N_k]
cudaError_t launch_fd_density(const double* E, const double2* U, int norb, int nk, double beta,
                              double mu, double2* nk_out, cudaStream_t st);
// part[2b] = block max |cur - old|; then cur = old = old + mix (cur - old)
cudaError_t launch_mix(double2* cur, double2* old, double mix, long long n, double* part,
                       int nblocks, cudaStream_t st);
// Z, Sigma(0), H_QP ([N_k][norb][norb]) and eps ([N_k][norb]) per k from
// Sigma^C(k, i w) (storage TS, [r][norb][norb][N_k]; r = 0: none), SigHF and
// the weights wp, wm of Sigma(+-i w0); S = scratch of 2 N_k norb^2 complex128;
// any output may be null; err = 5 where Z^-1 is not positive definite.
template <typename TS>
cudaError_t launch_qp(const double2* Hk, const double2* SigHF, const void* SigIw,
                      const double2* wp, const double2* wm, int r, int norb, int nk, double w0,
                      double2* S, double2* Z, double2* S0, double2* Hqp, double* eps, int* err,
                      cudaStream_t st);

// ---- GW grand potential in the Luttinger-Ward form (FP64), qa_free_energy.cu
// Per k: part[k] = sum_i ln(1 + e^{-beta (E_ki - mu)}), part[nk + k] =
// Re tr[SigHF(k) n(k)] (n [norb^2][N_k]); nhf (may be null) = scale f(A - mu).
cudaError_t launch_omega_hf(const double* E, const double2* U, const double2* SigHF,
                            const double2* nk_in, int norb, int nk, double beta, double mu,
                            double* part, double2* nhf, double scale, cudaStream_t st);
// Fermionic-trace terms of rows j = 0..rows-1 (i w_{n0+j}) of S = Sigma^C and G
// ([rows][norb^2][N_k]): part[j][k]; with abar (may be null) the cotangents
// S <- cs (G - G_D)^H, G <- cs S^H (in place), abar = ca (G_D - G_HF)^H.
cudaError_t launch_omega_g(const double2* Hk, const double2* SigHF, double2* S, double2* G, int n0,
                           int rows, int norb, int nk, double beta, double mu, double* part,
                           double2* abar, double cs, double ca, int* err, cudaStream_t st);
// Bosonic-trace terms of rows of P ([rows][nb^2][N_k]) with V(q) ([N_k][nb^2]):
// part[j][q] = ln|det(1 - V P)| + Re tr[V P]; with vbar (may be null)
// P <- cw (W - V)^H in place and vbar = cw (P W P)^H, W = (1 - V P)^-1 V.
cudaError_t launch_omega_w(double2* P, const double2* Vq, int nb, int nk, int rows, double* part,
                           double2* vbar, double cw, int* err, cudaStream_t st);
// out[(a,b)][k] = coef conj(in_(b,a)(k)); in [N_k][norb^2] (kmajor) or [norb^2][N_k]
cudaError_t launch_herm_scale(const double2* in, int kmajor, int norb, int nk, double coef, double2* out,
                              cudaStream_t st);
// out[e] (+)= sum_j buf[j][e], j < rows, e < n
cudaError_t launch_sum_rows(const double2* buf, int rows, long long n, double2* out, int accumulate,
                            cudaStream_t st);
// acc[slot] += scale * sum part[0 .. n) (fixed order)
cudaError_t launch_sum_scalar(const double* part, long long n, double scale, double* acc, int slot,
                              cudaStream_t st);

// Host copies a density call needs (valid for the context's lifetime).
int density_tables(const ::qa_ctx* ctx, const std::complex<double>** dtau, int* r, int* norb,
                   int* nk, int* nspin);

// Precision conversions.
cudaError_t launch_c128_to_c64(const double2* in, float2* out, long long n, cudaStream_t st);
cudaError_t launch_c64_to_c128(const float2* in, double2* out, long long n, cudaStream_t st);
cudaError_t launch_c128_to_df(const double2* in, void* out, long long n, cudaStream_t st);
cudaError_t launch_df_to_c128(const void* in, double2* out, long long n, cudaStream_t st);

}  // namespace qa
