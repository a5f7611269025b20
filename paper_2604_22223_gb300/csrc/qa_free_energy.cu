// GW grand potential in the Luttinger-Ward form and the pieces of its adjoint
// (FP64).  The paper's introduction names the Luttinger-Ward functional as the
// object whose gradients a differentiable GW code provides; it is evaluated
// here on the input G of one iteration (Sigma and P from G as in qa_gw_step,
// mu fixed), with the Matsubara traces truncated at a cutoff M:
//   Omega = Omega_HF + Omega_dc + Omega_G + Omega_W,
//   Omega_HF = -(s/(beta N_k)) sum_{k,i} ln(1 + e^{-beta (e_i(k) - mu)}),
//              e_i the eigenvalues of the Hermitian part of H(k) + Sigma^HF(k);
//   Omega_dc = -(1/2)(s/N_k) sum_k Re tr[Sigma^HF(k) n(k)];
//   Omega_G  = -(s/(beta N_k)) sum_k sum_{n=-M}^{M-1}
//              Re{ln det[1 - G_HF Sigma^C] + tr[Sigma^C G]}(k, i w_n);
//   Omega_W  = (1/(2 beta N_k)) sum_q sum_{m=-M}^{M}
//              Re{ln det[1 - V P] + tr[V P]}(q, i nu_m).
// Only ln|det| enters.  The kernels below produce per-point terms (summed in a
// fixed order, so repeated evaluations give the same bits) and, for the
// adjoint, the cotangents of Sigma^C, G, H + Sigma^HF, P and V at the uniform
// frequencies; the caller maps those back to the DLR nodes.
//
// Layouts: node-major [rows][entries][N_k] for the frequency chunks (as the
// DLR maps produce them), [N_k][norb^2] for H(k) and Sigma^HF(k),
// [N_k][nb^2] for V(q).
#include "qa_common.cuh"

namespace qa {
namespace {

__device__ __forceinline__ double softplus(double x) {      // ln(1 + e^x)
  return x > 0.0 ? x + log1p(exp(-x)) : log1p(exp(x));
}

// Gauss-Jordan inverse of an NO x NO complex matrix in registers with partial
// pivoting (largest |a|, lowest row on ties); returns ln|det a| and sets
// *bad when a pivot is zero or not finite.
template <int NO>
__device__ __forceinline__ double inv_logdet(double2 (&a)[NO][NO], double2 (&x)[NO][NO], bool* bad) {
#pragma unroll
  for (int i = 0; i < NO; ++i)
#pragma unroll
    for (int j = 0; j < NO; ++j) x[i][j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  double ld = 0.0;
#pragma unroll
  for (int c = 0; c < NO; ++c) {
    int p = c;
    double best = cabs2(a[c][c]);
#pragma unroll
    for (int i = c + 1; i < NO; ++i) {
      const double v = cabs2(a[i][c]);
      if (v > best) { best = v; p = i; }
    }
    if (!(best > 0.0) || !isfinite(best)) *bad = true;
    // swap rows c and p (predicated: indices stay compile-time)
#pragma unroll
    for (int i = c + 1; i < NO; ++i) {
      const bool sw = (i == p);
#pragma unroll
      for (int j = 0; j < NO; ++j) {
        const double2 ac = a[c][j], ai = a[i][j], xc = x[c][j], xi = x[i][j];
        a[c][j] = sw ? ai : ac; a[i][j] = sw ? ac : ai;
        x[c][j] = sw ? xi : xc; x[i][j] = sw ? xc : xi;
      }
    }
    ld += 0.5 * log(best);
    const double2 inv = cinv(a[c][c]);
#pragma unroll
    for (int j = 0; j < NO; ++j) {
      a[c][j] = cmul(a[c][j], inv);
      x[c][j] = cmul(x[c][j], inv);
    }
#pragma unroll
    for (int i = 0; i < NO; ++i) {
      if (i == c) continue;
      const double2 f = a[i][c];
#pragma unroll
      for (int j = 0; j < NO; ++j) {
        a[i][j] = cfms(f, a[c][j], a[i][j]);
        x[i][j] = cfms(f, x[c][j], x[i][j]);
      }
    }
  }
  return ld;
}

// Per k: part[k] = sum_i ln(1 + e^{-beta (e_i - mu)}), part[nk + k] =
// Re tr[Sigma^HF(k) n(k)]; with nhf: the Hartree-Fock density matrix
// f(A - mu) = U f(E) U^H, scaled by `scale`, [norb^2][N_k].
template <int NO>
__global__ void omega_hf_kernel(const double* __restrict__ E, const double2* __restrict__ U,
                                const double2* __restrict__ SigHF, const double2* __restrict__ nk_in,
                                double beta, double mu, int nk, double* __restrict__ part,
                                double2* __restrict__ nhf, double scale) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nk) return;
  double f[NO], sp = 0.0;
#pragma unroll
  for (int i = 0; i < NO; ++i) {
    const double x = -beta * (E[static_cast<size_t>(k) * NO + i] - mu);
    sp += softplus(x);
    f[i] = 1.0 / (1.0 + exp(-x));
  }
  double tr = 0.0;
  const double2* s = SigHF + static_cast<size_t>(k) * NO * NO;
#pragma unroll
  for (int a = 0; a < NO; ++a)
#pragma unroll
    for (int b = 0; b < NO; ++b) {
      const double2 sab = s[a * NO + b], nba = nk_in[static_cast<size_t>(b * NO + a) * nk + k];
      tr += sab.x * nba.x - sab.y * nba.y;
    }
  part[k] = sp;
  part[nk + k] = tr;
  if (nhf) {
    const double2* u = U + static_cast<size_t>(k) * NO * NO;
#pragma unroll
    for (int a = 0; a < NO; ++a)
#pragma unroll
      for (int b = 0; b < NO; ++b) {
        double2 acc = make_double2(0.0, 0.0);
#pragma unroll
        for (int i = 0; i < NO; ++i) acc = cfma(cscale(u[a * NO + i], f[i]), cconj(u[b * NO + i]), acc);
        nhf[static_cast<size_t>(a * NO + b) * nk + k] = cscale(acc, scale);
      }
  }
}

// One thread per (k, row j of the chunk), i w = (2 (n0 + j) + 1) pi / beta:
//   A = i w + mu - H(k) - Sigma^HF(k), G_HF = A^-1, G_D = (A - S)^-1 with
//   S = Sigma^C(k, i w), G = G(k, i w);
//   part = ln|det(A - S)| - ln|det A| + Re tr[S G].
// With abar (adjoint, coefficients cs = -c Omegabar, ca = c Omegabar,
// c = s / (beta N_k)): S <- cs (G - G_D)^H and G <- cs S^H in place, and
// abar[j] = ca (G_D - G_HF)^H, the cotangent of H + Sigma^HF from this point.
template <int NO>
__global__ void omega_g_kernel(const double2* __restrict__ Hk, const double2* __restrict__ SigHF,
                               double2* __restrict__ S, double2* __restrict__ G, int n0, int rows,
                               double beta, double mu, int nk, double* __restrict__ part,
                               double2* __restrict__ abar, double cs, double ca, int* err) {
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<long long>(rows) * nk) return;
  const int j = static_cast<int>(idx / nk), k = static_cast<int>(idx - static_cast<long long>(j) * nk);
  const double w = (2.0 * (n0 + j) + 1.0) * 3.14159265358979323846 / beta;
  const size_t base = static_cast<size_t>(j) * NO * NO * nk + k;
  double2 A[NO][NO], Ms[NO][NO], s[NO][NO], g[NO][NO], ghf[NO][NO], gd[NO][NO];
#pragma unroll
  for (int a = 0; a < NO; ++a)
#pragma unroll
    for (int b = 0; b < NO; ++b) {
      const double2 h = Hk[static_cast<size_t>(k) * NO * NO + a * NO + b];
      const double2 sh = SigHF[static_cast<size_t>(k) * NO * NO + a * NO + b];
      double2 v = make_double2(-h.x - sh.x, -h.y - sh.y);
      if (a == b) { v.x += mu; v.y += w; }
      A[a][b] = v;
      s[a][b] = S[base + static_cast<size_t>(a * NO + b) * nk];
      g[a][b] = G[base + static_cast<size_t>(a * NO + b) * nk];
      Ms[a][b] = csub(v, s[a][b]);
    }
  bool bad = false;
  const double ldm = inv_logdet<NO>(Ms, gd, &bad);
  const double lda = inv_logdet<NO>(A, ghf, &bad);
  double tr = 0.0;
#pragma unroll
  for (int a = 0; a < NO; ++a)
#pragma unroll
    for (int b = 0; b < NO; ++b) tr += s[a][b].x * g[b][a].x - s[a][b].y * g[b][a].y;
  part[idx] = ldm - lda + tr;
  if (bad) atomicCAS(err, 0, QA_ESINGULAR_CODE);
  if (abar) {
#pragma unroll
    for (int a = 0; a < NO; ++a)
#pragma unroll
      for (int b = 0; b < NO; ++b) {
        const size_t o = base + static_cast<size_t>(a * NO + b) * nk;
        S[o] = cscale(cconj(csub(g[b][a], gd[b][a])), cs);
        G[o] = cscale(cconj(s[b][a]), cs);
        abar[o] = cscale(cconj(csub(gd[b][a], ghf[b][a])), ca);
      }
  }
}

// One warp per (q, row j of the chunk): A = 1 - V(q) P (nb x nb), Gauss-Jordan
// elimination of [A | V] with partial pivoting (pivot search across the lanes,
// lowest row on ties) gives ln|det A| and W = A^-1 V;
//   part = ln|det A| + Re tr[V P].
// With vbar (adjoint, coefficient cw = -(1/(2 beta N_k)) Omegabar):
// P <- cw (W - V)^H in place and vbar[j] = cw (P W P)^H.  Lane c owns columns
// c of A and of V (nb <= 32); the matrices sit in shared memory, padded rows.
constexpr int kOwWarps = 2;

__global__ void __launch_bounds__(kOwWarps * 32) omega_w_kernel(double2* __restrict__ P,
                                                                const double2* __restrict__ Vq, int nb,
                                                                int nk, int rows, double* __restrict__ part,
                                                                double2* __restrict__ vbar, double cw,
                                                                int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long sys = static_cast<long long>(blockIdx.x) * kOwWarps + wid;
  const int ld = nb + 1;                                   // padded row stride
  double2* Ps = reinterpret_cast<double2*>(smem_raw) + static_cast<size_t>(wid) * 4 * nb * ld;
  double2* Vs = Ps + nb * ld;
  double2* As = Vs + nb * ld;                              // A, then P W
  double2* Ws = As + nb * ld;                              // V, then W
  if (sys >= static_cast<long long>(rows) * nk) return;   // whole warps leave together
  const int j = static_cast<int>(sys / nk), q = static_cast<int>(sys - static_cast<long long>(j) * nk);
  const int nn = nb * nb;
  const size_t base = static_cast<size_t>(j) * nn * nk + q;
  for (int e = lane; e < nn; e += 32) {
    const int a = e / nb, b = e - a * nb;
    Ps[a * ld + b] = P[base + static_cast<size_t>(e) * nk];
    const double2 v = Vq[static_cast<size_t>(q) * nn + e];
    Vs[a * ld + b] = v;
    Ws[a * ld + b] = v;
  }
  __syncwarp();
  const bool own = lane < nb;
  const int c0 = own ? lane : 0;
  // column c0 of A = 1 - V P; lane i: row i of V times column i of P for tr[V P]
  double trv = 0.0;
  if (own) {
    for (int i = 0; i < nb; ++i) {
      double2 acc = make_double2(i == c0 ? 1.0 : 0.0, 0.0);
      for (int l = 0; l < nb; ++l) acc = cfms(Vs[i * ld + l], Ps[l * ld + c0], acc);
      As[i * ld + c0] = acc;
    }
    for (int l = 0; l < nb; ++l) {
      const double2 v = Vs[c0 * ld + l], p = Ps[l * ld + c0];
      trv += v.x * p.x - v.y * p.y;
    }
  }
  __syncwarp();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) trv += __shfl_xor_sync(0xffffffffu, trv, o);
  double lda = 0.0;
  bool bad = false;
  for (int c = 0; c < nb; ++c) {
    // pivot: the largest |A_ic| over rows i >= c (lane i), lowest row on ties
    double v = (own && lane >= c) ? cabs2(As[lane * ld + c]) : -1.0;
    int p = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double vo = __shfl_xor_sync(0xffffffffu, v, o);
      const int po = __shfl_xor_sync(0xffffffffu, p, o);
      if (vo > v || (vo == v && po < p)) { v = vo; p = po; }
    }
    if (!(v > 0.0) || !isfinite(v)) bad = true;
    lda += 0.5 * log(v);
    if (own && p != c) {
      double2 t = As[c * ld + c0]; As[c * ld + c0] = As[p * ld + c0]; As[p * ld + c0] = t;
      t = Ws[c * ld + c0]; Ws[c * ld + c0] = Ws[p * ld + c0]; Ws[p * ld + c0] = t;
    }
    __syncwarp();
    const double2 inv = cinv(As[c * ld + c]);
    __syncwarp();
    double2 ra = make_double2(0.0, 0.0), rw = make_double2(0.0, 0.0);
    if (own) {
      ra = cmul(As[c * ld + c0], inv);
      rw = cmul(Ws[c * ld + c0], inv);
    }
    __syncwarp();
    if (own) {
      for (int i = 0; i < nb; ++i) {
        if (i == c) continue;
        const double2 f = As[i * ld + c];                    // column c is rewritten after the sync
        if (c0 != c) As[i * ld + c0] = cfms(f, ra, As[i * ld + c0]);
        Ws[i * ld + c0] = cfms(f, rw, Ws[i * ld + c0]);
      }
    }
    __syncwarp();
    if (own) {
      As[c * ld + c0] = ra;
      Ws[c * ld + c0] = rw;
      if (c0 == c)
        for (int i = 0; i < nb; ++i) As[i * ld + c] = make_double2(i == c ? 1.0 : 0.0, 0.0);
    }
    __syncwarp();
  }
  if (lane == 0) {
    part[sys] = lda + trv;
    if (bad) atomicCAS(err, 0, QA_ESINGULAR_CODE);
  }
  if (!vbar) return;
  // P <- cw (W - V)^H
  for (int e = lane; e < nn; e += 32) {
    const int a = e / nb, b = e - a * nb;
    P[base + static_cast<size_t>(e) * nk] = cscale(cconj(csub(Ws[b * ld + a], Vs[b * ld + a])), cw);
  }
  // X = P W into As (column c0), then Y = X P (column c0 in registers) -> vbar = cw Y^H
  if (own)
    for (int i = 0; i < nb; ++i) {
      double2 acc = make_double2(0.0, 0.0);
      for (int l = 0; l < nb; ++l) acc = cfma(Ps[i * ld + l], Ws[l * ld + c0], acc);
      As[i * ld + c0] = acc;
    }
  __syncwarp();
  if (own)
    for (int i = 0; i < nb; ++i) {
      double2 acc = make_double2(0.0, 0.0);
      for (int l = 0; l < nb; ++l) acc = cfma(As[i * ld + l], Ps[l * ld + c0], acc);
      // Y_{i c0} -> vbar entry (c0, i)
      vbar[base + static_cast<size_t>(c0 * nb + i) * nk] = cscale(cconj(acc), cw);
    }
}

// out[e] (+)= sum_j buf[j][e] over the rows of a chunk, in row order
__global__ void sum_rows_kernel(const double2* __restrict__ buf, int rows, long long n,
                                double2* __restrict__ out, int accumulate) {
  const long long e = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= n) return;
  double2 s = accumulate ? out[e] : make_double2(0.0, 0.0);
  for (int j = 0; j < rows; ++j) s = cadd(s, buf[static_cast<size_t>(j) * n + e]);
  out[e] = s;
}

// acc[slot] += scale * sum of part[0 .. n): one block, a fixed summation order
constexpr int kSumThreads = 1024;
__global__ void __launch_bounds__(kSumThreads) sum_scalar_kernel(const double* __restrict__ part,
                                                                 long long n, double scale,
                                                                 double* acc, int slot) {
  __shared__ double sh[kSumThreads];
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += kSumThreads) s += part[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = kSumThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) acc[slot] += scale * sh[0];
}

// out[(a,b)][k] = coef conj(in_(b,a)(k)), in k-major ([N_k][norb^2]) or
// entry-major ([norb^2][N_k]); out entry-major
__global__ void herm_scale_kernel(const double2* __restrict__ in, int kmajor, int norb, int nk,
                                  double coef, double2* __restrict__ out) {
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int no2 = norb * norb;
  if (idx >= static_cast<long long>(no2) * nk) return;
  const int e = static_cast<int>(idx / nk), k = static_cast<int>(idx - static_cast<long long>(e) * nk);
  const int a = e / norb, b = e - a * norb, t = b * norb + a;
  const double2 v = kmajor ? in[static_cast<size_t>(k) * no2 + t] : in[static_cast<size_t>(t) * nk + k];
  out[idx] = cscale(cconj(v), coef);
}

}  // namespace

cudaError_t launch_omega_hf(const double* E, const double2* U, const double2* SigHF,
                            const double2* nk_in, int norb, int nk, double beta, double mu,
                            double* part, double2* nhf, double scale, cudaStream_t st) {
  const unsigned g = static_cast<unsigned>((nk + 127) / 128);
  switch (norb) {
#define QA_CASE(NO) \
    case NO: omega_hf_kernel<NO><<<g, 128, 0, st>>>(E, U, SigHF, nk_in, beta, mu, nk, part, nhf, scale); break;
    QA_CASE(1) QA_CASE(2) QA_CASE(3) QA_CASE(4) QA_CASE(5)
#undef QA_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_omega_g(const double2* Hk, const double2* SigHF, double2* S, double2* G, int n0,
                           int rows, int norb, int nk, double beta, double mu, double* part,
                           double2* abar, double cs, double ca, int* err, cudaStream_t st) {
  const long long n = static_cast<long long>(rows) * nk;
  if (n <= 0) return cudaSuccess;
  const unsigned g = static_cast<unsigned>((n + 63) / 64);
  switch (norb) {
#define QA_CASE(NO)                                                                              \
    case NO: omega_g_kernel<NO><<<g, 64, 0, st>>>(Hk, SigHF, S, G, n0, rows, beta, mu, nk, part, \
                                                 abar, cs, ca, err); break;
    QA_CASE(1) QA_CASE(2) QA_CASE(3) QA_CASE(4) QA_CASE(5)
#undef QA_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

size_t omega_w_smem(int nb) {
  return static_cast<size_t>(kOwWarps) * 4 * nb * (nb + 1) * sizeof(double2);
}

cudaError_t launch_omega_w(double2* P, const double2* Vq, int nb, int nk, int rows, double* part,
                           double2* vbar, double cw, int* err, cudaStream_t st) {
  if (nb < 1 || nb > 32) return cudaErrorInvalidValue;
  const long long n = static_cast<long long>(rows) * nk;
  if (n <= 0) return cudaSuccess;
  const size_t smem = omega_w_smem(nb);
  cudaError_t e = set_smem(reinterpret_cast<const void*>(&omega_w_kernel), smem);
  if (e != cudaSuccess) return e;
  const unsigned g = static_cast<unsigned>((n + kOwWarps - 1) / kOwWarps);
  omega_w_kernel<<<g, kOwWarps * 32, smem, st>>>(P, Vq, nb, nk, rows, part, vbar, cw, err);
  return cudaGetLastError();
}

cudaError_t launch_sum_rows(const double2* buf, int rows, long long n, double2* out, int accumulate,
                            cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  sum_rows_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(buf, rows, n, out, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_sum_scalar(const double* part, long long n, double scale, double* acc, int slot,
                              cudaStream_t st) {
  sum_scalar_kernel<<<1, kSumThreads, 0, st>>>(part, n, scale, acc, slot);
  return cudaGetLastError();
}

cudaError_t launch_herm_scale(const double2* in, int kmajor, int norb, int nk, double coef, double2* out,
                              cudaStream_t st) {
  const long long n = static_cast<long long>(norb) * norb * nk;
  if (n <= 0) return cudaSuccess;
  herm_scale_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(in, kmajor, norb, nk, coef, out);
  return cudaGetLastError();
}

}  // namespace qa
