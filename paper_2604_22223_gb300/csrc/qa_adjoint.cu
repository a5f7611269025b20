// Hand-written adjoint of one GW iteration (FP64), stage by stage in reverse.
//
// Convention: for a real loss L and a complex quantity X the gradient is
// Xbar = dL/dRe X + i dL/dIm X, so a linear map Y = A X pulls back as
// Xbar = A^H Ybar, a product y = a b as abar += conj(b) ybar, and an inverse
// Y = X^-1 as Xbar = -Y^H Ybar Y^H.  Forward stages and their adjoints:
//   G(k,i w) = M^-1, M = i w + mu - H - Sigma^HF - Sigma^C      (Dyson for G)
//       Mbar = -G^H Gbar G^H;  Sigma^C bar = -Mbar;  (H, Sigma^HF) bar = -sum_n Mbar
//   Sigma^C_ad = -sum_bc G_bc W^C_(ab),(cd)                      (GW self-energy)
//       Gbar_bc = -sum_ad conj(W^C_(ab),(cd)) Sigmabar_ad;  W^C bar = -Sigmabar_ad conj(G_bc)
//   W = (1 - V P)^-1 V, W^C = W - V                             (screened interaction)
//       Pbar = W^H Wbar W^H;  Vbar = (1 - VP)^-H Wbar (1 + P W)^H - Wbar,
//       with the LU factors of 1 - VP kept by the forward recompute
//   P_(ab),(cd) = -s G_bc(R) G_da(-R, beta - tau)                (polarizability)
//       Gbar_bc(R) = -s sum_ad conj(G_da(-R)) Pbar;  Gbar_da(-R) = -s sum_bc conj(G_bc(R)) Pbar
// The mu of the forward step is held fixed.
#include "qa_common.cuh"

namespace qa {
namespace {

// ------------------------------------------------------------- Dyson G
// one thread per k, loop over the r Matsubara nodes
template <int NO>
__global__ void __launch_bounds__(128) dyson_g_bwd_kernel(
    const double2* __restrict__ Hk, const double2* __restrict__ SigHF,
    const double2* __restrict__ SigIw, const double* __restrict__ iw, double mu, int r, int nk,
    const double2* __restrict__ Gbar_iw, double2* SigCbar_iw, double2* Sbar) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nk) return;
  constexpr int NP = NO * NO;
  double2 S[NO][NO];
#pragma unroll
  for (int i = 0; i < NO; ++i)
#pragma unroll
    for (int j = 0; j < NO; ++j) S[i][j] = make_double2(0, 0);
  for (int n = 0; n < r; ++n) {
    double2 a[NO][NO], g[NO][NO];
#pragma unroll
    for (int i = 0; i < NO; ++i)
#pragma unroll
      for (int j = 0; j < NO; ++j) {
        double2 h = Hk[static_cast<size_t>(k) * NP + i * NO + j];
        double2 s = SigHF[static_cast<size_t>(k) * NP + i * NO + j];
        double2 sc = SigIw[(static_cast<size_t>(n) * NP + i * NO + j) * nk + k];
        double2 m = make_double2(-h.x - s.x - sc.x, -h.y - s.y - sc.y);
        if (i == j) { m.x += mu; m.y += iw[n]; }
        a[i][j] = m;
        g[i][j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
      }
#pragma unroll
    for (int c = 0; c < NO; ++c) {
      int p = c;
      double best = cabs2(a[c][c]);
#pragma unroll
      for (int i = c + 1; i < NO; ++i) {
        double v = cabs2(a[i][c]);
        if (v > best) { best = v; p = i; }
      }
#pragma unroll
      for (int i = c + 1; i < NO; ++i)
        if (i == p) {
#pragma unroll
          for (int j = 0; j < NO; ++j) {
            double2 t1 = a[c][j]; a[c][j] = a[i][j]; a[i][j] = t1;
            double2 t2 = g[c][j]; g[c][j] = g[i][j]; g[i][j] = t2;
          }
        }
      double2 inv = cinv(a[c][c]);
#pragma unroll
      for (int j = 0; j < NO; ++j) { a[c][j] = cmul(a[c][j], inv); g[c][j] = cmul(g[c][j], inv); }
#pragma unroll
      for (int i = 0; i < NO; ++i) {
        if (i == c) continue;
        double2 f = a[i][c];
#pragma unroll
        for (int j = 0; j < NO; ++j) {
          a[i][j] = cfms(f, a[c][j], a[i][j]);
          g[i][j] = cfms(f, g[c][j], g[i][j]);
        }
      }
    }
    // a <- X = G^H Gbar
#pragma unroll
    for (int j = 0; j < NO; ++j) {
      double2 gb[NO];
#pragma unroll
      for (int m = 0; m < NO; ++m) gb[m] = Gbar_iw[(static_cast<size_t>(n) * NP + m * NO + j) * nk + k];
#pragma unroll
      for (int i = 0; i < NO; ++i) {
        double2 acc = make_double2(0, 0);
#pragma unroll
        for (int m = 0; m < NO; ++m) acc = cfma(cconj(g[m][i]), gb[m], acc);
        a[i][j] = acc;
      }
    }
    // Sigma^C bar = -Mbar = X G^H ; S += X G^H
#pragma unroll
    for (int i = 0; i < NO; ++i)
#pragma unroll
      for (int j = 0; j < NO; ++j) {
        double2 acc = make_double2(0, 0);
#pragma unroll
        for (int m = 0; m < NO; ++m) acc = cfma(a[i][m], cconj(g[j][m]), acc);
        SigCbar_iw[(static_cast<size_t>(n) * NP + i * NO + j) * nk + k] = acc;
        S[i][j] = cadd(S[i][j], acc);
      }
  }
  // (H, Sigma^HF) bar = -sum_n Mbar = sum_n X G^H, stored [e][k]
#pragma unroll
  for (int i = 0; i < NO; ++i)
#pragma unroll
    for (int j = 0; j < NO; ++j) Sbar[static_cast<size_t>(i * NO + j) * nk + k] = S[i][j];
}

// -------------------------------------------------------- Sigma contraction
// one thread per (tau_j, R); W holds W^C(R, tau) on entry and Wbar on exit
template <int NO>
__global__ void __launch_bounds__(128) sigma_bwd_kernel(const double2* __restrict__ GR,
                                                        const double2* __restrict__ SigbarR,
                                                        double2* W, double2* GRbar, int nk) {
  constexpr int NP = NO * NO;
  const int t = blockIdx.x;
  const int R = blockIdx.y * blockDim.x + threadIdx.x;
  if (R >= nk) return;
  double2 g[NO][NO], sb[NO][NO], gb[NO][NO];
#pragma unroll
  for (int b = 0; b < NO; ++b)
#pragma unroll
    for (int c = 0; c < NO; ++c) {
      g[b][c] = GR[(static_cast<size_t>(t) * NP + b * NO + c) * nk + R];
      sb[b][c] = SigbarR[(static_cast<size_t>(t) * NP + b * NO + c) * nk + R];
      gb[b][c] = make_double2(0, 0);
    }
  double2* Wt = W + static_cast<size_t>(t) * NP * NP * nk + R;
#pragma unroll 1
  for (int a = 0; a < NO; ++a)
#pragma unroll
    for (int b = 0; b < NO; ++b)
#pragma unroll
      for (int c = 0; c < NO; ++c)
#pragma unroll
        for (int d = 0; d < NO; ++d) {
          const size_t idx = (static_cast<size_t>(a * NO + b) * NP + (c * NO + d)) * nk;
          double2 w = Wt[idx];
          gb[b][c] = cfms(cconj(w), sb[a][d], gb[b][c]);
          double2 wb = cmul(sb[a][d], cconj(g[b][c]));
          Wt[idx] = make_double2(-wb.x, -wb.y);
        }
#pragma unroll
  for (int b = 0; b < NO; ++b)
#pragma unroll
    for (int c = 0; c < NO; ++c) GRbar[(static_cast<size_t>(t) * NP + b * NO + c) * nk + R] = gb[b][c];
}

// ------------------------------------------------------------------ bubble
// one thread per (tau_j, R): GRbar(R) += ..., GLbar(-R) = ...
template <int NO>
__global__ void __launch_bounds__(128) bubble_bwd_kernel(const double2* __restrict__ GR,
                                                         const double2* __restrict__ GL,
                                                         const int* __restrict__ mR,
                                                         const double2* __restrict__ Pbar,
                                                         double2* GRbar, double2* GLbar, int nk,
                                                         double s) {
  constexpr int NP = NO * NO;
  const int t = blockIdx.x;
  const int R = blockIdx.y * blockDim.x + threadIdx.x;
  if (R >= nk) return;
  const int mr = mR[R];
  double2 gr[NO][NO], gl[NO][NO], grb[NO][NO], glb[NO][NO];
#pragma unroll
  for (int x = 0; x < NO; ++x)
#pragma unroll
    for (int y = 0; y < NO; ++y) {
      gr[x][y] = GR[(static_cast<size_t>(t) * NP + x * NO + y) * nk + R];
      gl[x][y] = GL[(static_cast<size_t>(t) * NP + x * NO + y) * nk + mr];
      grb[x][y] = GRbar[(static_cast<size_t>(t) * NP + x * NO + y) * nk + R];
      glb[x][y] = make_double2(0, 0);
    }
  const double2* Pt = Pbar + static_cast<size_t>(t) * NP * NP * nk + R;
#pragma unroll 1
  for (int a = 0; a < NO; ++a)
#pragma unroll
    for (int b = 0; b < NO; ++b)
#pragma unroll
      for (int c = 0; c < NO; ++c)
#pragma unroll
        for (int d = 0; d < NO; ++d) {
          double2 pb = Pt[(static_cast<size_t>(a * NO + b) * NP + (c * NO + d)) * nk];
          pb.x *= -s;
          pb.y *= -s;
          grb[b][c] = cfma(cconj(gl[d][a]), pb, grb[b][c]);
          glb[d][a] = cfma(cconj(gr[b][c]), pb, glb[d][a]);
        }
#pragma unroll
  for (int x = 0; x < NO; ++x)
#pragma unroll
    for (int y = 0; y < NO; ++y) {
      GRbar[(static_cast<size_t>(t) * NP + x * NO + y) * nk + R] = grb[x][y];
      GLbar[(static_cast<size_t>(t) * NP + x * NO + y) * nk + mr] = glb[x][y];
    }
}

// ------------------------------------------ reduced pair basis (term lists)
// The reduced basis replaces the explicit (ab),(cd) sums by the host term
// lists of the forward kernels: per reduced entry o = (i, j) the terms
// (coefficient c, indices) with
//   Pt_o(R)      += c G_g1(R, tau) G^refl_g2(-R, beta - tau)   (bubble, idx = g1 | g2 << 8)
//   Sigma_t(R)   += c G_g(R, tau) Wt^C_o(R, tau)                 (self-energy, idx = g | t << 8)
// and their adjoints  x_bar += conj(c y) z_bar  for every product z = c x y.
// One thread per (tau_j, R); the per-thread vectors of norb^2 values sit in
// shared memory (indexed at run time by the term lists).
constexpr int kTermThreads = 64;

__global__ void __launch_bounds__(kTermThreads) sigma_bwd_terms_kernel(
    const double2* __restrict__ GR, const double2* __restrict__ SigbarR, double2* W, double2* GRbar,
    const int* __restrict__ terms, const double2* __restrict__ coef, int nb2, int no2, int nk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* sg = reinterpret_cast<double2*>(smem_raw);          // [no2][threads]
  double2* ssb = sg + no2 * kTermThreads;
  double2* sgb = ssb + no2 * kTermThreads;
  const int t = blockIdx.x;
  const int R = blockIdx.y * kTermThreads + threadIdx.x;
  const int th = threadIdx.x;
  const bool ok = R < nk;
  for (int e = 0; e < no2; ++e) {
    const size_t at = (static_cast<size_t>(t) * no2 + e) * nk + R;
    sg[e * kTermThreads + th] = ok ? GR[at] : make_double2(0, 0);
    ssb[e * kTermThreads + th] = ok ? SigbarR[at] : make_double2(0, 0);
    sgb[e * kTermThreads + th] = make_double2(0, 0);
  }
  if (ok) {
    const int* idx = terms + nb2 + 1;
    double2* Wt = W + static_cast<size_t>(t) * nb2 * nk + R;
    for (int o = 0; o < nb2; ++o) {
      const double2 w = Wt[static_cast<size_t>(o) * nk];
      double2 wb = make_double2(0, 0);
      for (int e = terms[o]; e < terms[o + 1]; ++e) {
        const int g = idx[e] & 255, tg = idx[e] >> 8;
        const double2 c = coef[e], sb = ssb[tg * kTermThreads + th];
        wb = cfma(cconj(cmul(c, sg[g * kTermThreads + th])), sb, wb);
        sgb[g * kTermThreads + th] = cfma(cconj(cmul(c, w)), sb, sgb[g * kTermThreads + th]);
      }
      Wt[static_cast<size_t>(o) * nk] = wb;
    }
    for (int e = 0; e < no2; ++e)
      GRbar[(static_cast<size_t>(t) * no2 + e) * nk + R] = sgb[e * kTermThreads + th];
  }
}

__global__ void __launch_bounds__(kTermThreads) bubble_bwd_terms_kernel(
    const double2* __restrict__ GR, const double2* __restrict__ GL, const int* __restrict__ mR,
    const double2* __restrict__ Pbar, double2* GRbar, double2* GLbar, const int* __restrict__ terms,
    const double2* __restrict__ coef, int nb2, int no2, int nk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* sgr = reinterpret_cast<double2*>(smem_raw);         // [no2][threads]
  double2* sgl = sgr + no2 * kTermThreads;
  double2* sgrb = sgl + no2 * kTermThreads;
  double2* sglb = sgrb + no2 * kTermThreads;
  const int t = blockIdx.x;
  const int R = blockIdx.y * kTermThreads + threadIdx.x;
  const int th = threadIdx.x;
  const bool ok = R < nk;
  const int mr = ok ? mR[R] : 0;
  for (int e = 0; e < no2; ++e) {
    const size_t row = (static_cast<size_t>(t) * no2 + e) * nk;
    sgr[e * kTermThreads + th] = ok ? GR[row + R] : make_double2(0, 0);
    sgl[e * kTermThreads + th] = ok ? GL[row + mr] : make_double2(0, 0);
    sgrb[e * kTermThreads + th] = ok ? GRbar[row + R] : make_double2(0, 0);
    sglb[e * kTermThreads + th] = make_double2(0, 0);
  }
  if (ok) {
    const int* idx = terms + nb2 + 1;
    const double2* Pt = Pbar + static_cast<size_t>(t) * nb2 * nk + R;
    for (int o = 0; o < nb2; ++o) {
      const double2 pb = Pt[static_cast<size_t>(o) * nk];
      for (int e = terms[o]; e < terms[o + 1]; ++e) {
        const int g1 = idx[e] & 255, g2 = idx[e] >> 8;
        const double2 c = coef[e];
        sgrb[g1 * kTermThreads + th] =
            cfma(cconj(cmul(c, sgl[g2 * kTermThreads + th])), pb, sgrb[g1 * kTermThreads + th]);
        sglb[g2 * kTermThreads + th] =
            cfma(cconj(cmul(c, sgr[g1 * kTermThreads + th])), pb, sglb[g2 * kTermThreads + th]);
      }
    }
    for (int e = 0; e < no2; ++e) {
      const size_t row = (static_cast<size_t>(t) * no2 + e) * nk;
      GRbar[row + R] = sgrb[e * kTermThreads + th];
      GLbar[row + mr] = sglb[e * kTermThreads + th];
    }
  }
}

// --------------------------------------------------------------- Dyson W
constexpr int kWarpsB = 4;
constexpr int kMaxN = 25;

// C = op(A) op(B) row per lane; C may alias A or B.
template <bool HA, bool HB>
__device__ void wmm(const double2* A, const double2* B, double2* C, int n, int ld, int lane) {
  double2 row[kMaxN];
  if (lane < n) {
#pragma unroll
    for (int j = 0; j < kMaxN; ++j) {
      if (j < n) {
        double2 acc = make_double2(0, 0);
        for (int m = 0; m < n; ++m) {
          double2 a = HA ? cconj(A[m * ld + lane]) : A[lane * ld + m];
          double2 b = HB ? cconj(B[j * ld + m]) : B[m * ld + j];
          acc = cfma(a, b, acc);
        }
        row[j] = acc;
      }
    }
  }
  __syncwarp();
  if (lane < n) {
#pragma unroll
    for (int j = 0; j < kMaxN; ++j)
      if (j < n) C[lane * ld + j] = row[j];
  }
  __syncwarp();
}

// in-place LU with partial pivoting (L below the diagonal, unit); perm[c] = swapped row
__device__ bool wlu(double2* A, int* perm, int n, int ld, int lane) {
  bool singular = false;
  for (int c = 0; c < n; ++c) {
    double val = (lane >= c && lane < n) ? cabs2(A[lane * ld + c]) : -1.0;
    int idx = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double ov = __shfl_xor_sync(0xffffffffu, val, o);
      int oi = __shfl_xor_sync(0xffffffffu, idx, o);
      if (ov > val || (ov == val && oi < idx)) { val = ov; idx = oi; }
    }
    const int p = idx;
    if (!(val > 1e-26)) singular = true;
    if (lane == 0) perm[c] = p;
    if (p != c && lane < n) {
      double2 t = A[c * ld + lane]; A[c * ld + lane] = A[p * ld + lane]; A[p * ld + lane] = t;
    }
    __syncwarp();
    if (lane > c && lane < n) {
      double2 l = cmul(A[lane * ld + c], cinv(A[c * ld + c]));
      A[lane * ld + c] = l;
      for (int j = c + 1; j < n; ++j) A[lane * ld + j] = cfms(l, A[c * ld + j], A[lane * ld + j]);
    }
    __syncwarp();
  }
  return singular;
}

// solve A X = B (B overwritten), column per lane, with the factors of wlu
__device__ void wsolve(const double2* LU, const int* perm, double2* B, int n, int ld, int lane) {
  if (lane < n) {
    const int j = lane;
    for (int c = 0; c < n; ++c) {
      int p = perm[c];
      if (p != c) { double2 t = B[c * ld + j]; B[c * ld + j] = B[p * ld + j]; B[p * ld + j] = t; }
    }
    for (int c = 0; c < n; ++c)
      for (int i = c + 1; i < n; ++i) B[i * ld + j] = cfms(LU[i * ld + c], B[c * ld + j], B[i * ld + j]);
    for (int c = n - 1; c >= 0; --c) {
      double2 x = B[c * ld + j];
      for (int m = c + 1; m < n; ++m) x = cfms(LU[c * ld + m], B[m * ld + j], x);
      B[c * ld + j] = cmul(x, cinv(LU[c * ld + c]));
    }
  }
  __syncwarp();
}

// solve A^H X = B with P A = L U: A^H = U^H L^H P
__device__ void wsolve_h(const double2* LU, const int* perm, double2* B, int n, int ld, int lane) {
  if (lane < n) {
    const int j = lane;
    for (int c = 0; c < n; ++c) {
      double2 x = B[c * ld + j];
      for (int m = 0; m < c; ++m) x = cfms(cconj(LU[m * ld + c]), B[m * ld + j], x);
      B[c * ld + j] = cmul(x, cinv(cconj(LU[c * ld + c])));
    }
    for (int c = n - 1; c >= 0; --c) {
      double2 x = B[c * ld + j];
      for (int m = c + 1; m < n; ++m) x = cfms(cconj(LU[m * ld + c]), B[m * ld + j], x);
      B[c * ld + j] = x;
    }
    for (int c = n - 1; c >= 0; --c) {
      int p = perm[c];
      if (p != c) { double2 t = B[c * ld + j]; B[c * ld + j] = B[p * ld + j]; B[p * ld + j] = t; }
    }
  }
  __syncwarp();
}

// warp per (q, nu): reads P(q, i nu), V(q), Wbar(q, i nu) (in place -> Pbar),
// accumulates Vbar(q) with atomics into Vqbar [npair^2][N_k]
__global__ void __launch_bounds__(kWarpsB * 32) dyson_w_bwd_kernel(const double2* __restrict__ P,
                                                                  const double2* __restrict__ Vq,
                                                                  double2* Wb, double* Vqbar,
                                                                  int n, int nk, int* err,
                                                                  const double2* __restrict__ lu,
                                                                  const unsigned char* __restrict__ piv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int q = blockIdx.x * kWarpsB + w;
  const int nu = blockIdx.y;
  if (q >= nk) return;                     // whole warp; no block barriers
  const int ld = n + 1;
  const int msz = n * ld;
  double2* S0 = reinterpret_cast<double2*>(smem_raw) + static_cast<size_t>(w) * 5 * msz;
  double2* S1 = S0 + msz;
  double2* S2 = S1 + msz;
  double2* S3 = S2 + msz;
  double2* S4 = S3 + msz;
  int* perm = reinterpret_cast<int*>(reinterpret_cast<double2*>(smem_raw) + kWarpsB * 5 * msz) +
              w * kMaxN;
  const size_t nn = static_cast<size_t>(n) * n;
  const size_t base = static_cast<size_t>(nu) * nn * nk + q;
  for (int e = lane; e < n * n; e += 32) {
    int i = e / n, j = e - i * n;
    S0[i * ld + j] = P[base + static_cast<size_t>(e) * nk];
    S1[i * ld + j] = Vq[static_cast<size_t>(q) * nn + e];
    S2[i * ld + j] = Wb[base + static_cast<size_t>(e) * nk];
  }
  __syncwarp();
  bool singular = false;
  if (lu) {
    // the forward step's factors of A = 1 - V P (its singular pivots were reported there)
    for (int e = lane; e < n * n; e += 32) {
      int i = e / n, j = e - i * n;
      S3[i * ld + j] = lu[base + static_cast<size_t>(e) * nk];
    }
    for (int c = lane; c < n; c += 32) perm[c] = piv[(static_cast<size_t>(nu) * n + c) * nk + q];
    __syncwarp();
  } else {
    wmm<false, false>(S1, S0, S3, n, ld, lane);           // S3 = V P
    for (int e = lane; e < n * n; e += 32) {
      int i = e / n, j = e - i * n;
      double2 v = S3[i * ld + j];
      S3[i * ld + j] = make_double2((i == j ? 1.0 : 0.0) - v.x, -v.y);   // A = 1 - V P
    }
    __syncwarp();
    singular = wlu(S3, perm, n, ld, lane);
  }
  for (int e = lane; e < n * n; e += 32) {
    int i = e / n, j = e - i * n;
    S4[i * ld + j] = S1[i * ld + j];
  }
  __syncwarp();
  wsolve(S3, perm, S4, n, ld, lane);                     // S4 = W = A^-1 V
  for (int e = lane; e < n * n; e += 32) {
    int i = e / n, j = e - i * n;
    S1[i * ld + j] = S2[i * ld + j];
  }
  __syncwarp();
  wsolve_h(S3, perm, S1, n, ld, lane);                   // S1 = X = A^-H Wbar
  wmm<false, false>(S0, S4, S3, n, ld, lane);            // S3 = P W
  // Vbar = X + X (P W)^H - Wbar
  if (lane < n) {
    for (int j = 0; j < n; ++j) {
      double2 acc = S1[lane * ld + j];
      for (int m = 0; m < n; ++m) acc = cfma(S1[lane * ld + m], cconj(S3[j * ld + m]), acc);
      acc = csub(acc, S2[lane * ld + j]);
      double* dst = Vqbar + 2 * (static_cast<size_t>(lane * n + j) * nk + q);
      atomicAdd(dst, acc.x);
      atomicAdd(dst + 1, acc.y);
    }
  }
  __syncwarp();
  wmm<true, false>(S4, S2, S0, n, ld, lane);             // S0 = W^H Wbar
  wmm<false, true>(S0, S4, S2, n, ld, lane);             // S2 = Pbar = W^H Wbar W^H
  for (int e = lane; e < n * n; e += 32) {
    int i = e / n, j = e - i * n;
    Wb[base + static_cast<size_t>(e) * nk] = S2[i * ld + j];
  }
  if (singular && lane == 0) atomicCAS(err, 0, QA_ESINGULAR_CODE);
}

// ------------------------------------------------------------- small pieces

// Hartree/Fock adjoint, one block.  X[v][e] = (1/N_k) sum_k e^{+ik.R_v} Sbar_e(k)
// for v <= nV (v = nV: R = 0).  Writes VbarHF [nV][np^2] and nbarR [nV+1][no^2].
__global__ void hf_bwd_kernel(const double2* __restrict__ VR, const double2* __restrict__ nR,
                              const double2* __restrict__ X, int nV, int no, double s, int nk,
                              double2* VbarHF, double2* nbarR) {
  const int np = no * no, np2 = np * np;
  const double2* n0 = nR + static_cast<size_t>(nV) * np;
  const double2* sH = X + static_cast<size_t>(nV) * np;      // Sigma^H bar / N_k
  for (int o = threadIdx.x; o < nV * np2; o += blockDim.x) {
    const int v = o / np2, e = o % np2;
    const int A = e / np, B = e % np;
    const int a = A / no, b = A % no, c = B / no, d = B % no;
    const double2 sF = X[static_cast<size_t>(v) * np + a * no + d];   // Sigma^F bar(R_v) / N_k
    double2 acc = cscale(cmul(sH[a * no + b], cconj(n0[d * no + c])), s);
    acc = cfms(sF, cconj(nR[static_cast<size_t>(v) * np + b * no + c]), acc);
    VbarHF[o] = cscale(acc, static_cast<double>(nk));
  }
  for (int o = threadIdx.x; o < (nV + 1) * np; o += blockDim.x) {
    const int v = o / np, e = o % np;
    double2 acc = make_double2(0, 0);
    if (v < nV) {
      const int b = e / no, c = e % no;        // nbar_bc(R_v)
      const double2* Vv = VR + static_cast<size_t>(v) * np2;
      for (int a = 0; a < no; ++a)
        for (int d = 0; d < no; ++d)
          acc = cfms(cconj(Vv[(a * no + b) * np + c * no + d]), X[static_cast<size_t>(v) * np + a * no + d], acc);
    } else {
      const int d = e / no, c = e % no;        // nbar0_dc
      for (int w = 0; w < nV; ++w) {
        const double2* Vw = VR + static_cast<size_t>(w) * np2;
        for (int a = 0; a < no; ++a)
          for (int b = 0; b < no; ++b)
            acc = cfma(cconj(Vw[(a * no + b) * np + c * no + d]), sH[a * no + b], acc);
      }
      acc = cscale(acc, s);
    }
    nbarR[o] = cscale(acc, static_cast<double>(nk));
  }
}

// nbar(k)[e][k] = (1/N_k) sum_{v <= nV} e^{-ik.R_v} nbarR[v][e]
__global__ void nbar_k_kernel(const double2* __restrict__ nbarR, const int* __restrict__ R, int nV1,
                              int np, int nk, int n1, int n2, int n3, double2* nbk) {
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<long long>(nk) * np) return;
  const int e = static_cast<int>(idx / nk), k = static_cast<int>(idx % nk);
  double2 acc = make_double2(0, 0);
  for (int v = 0; v < nV1; ++v)
    acc = cfma(nbarR[static_cast<size_t>(v) * np + e], lattice_phase(k, n1, n2, n3, R + 3 * v, -1), acc);
  nbk[idx] = cscale(acc, 1.0 / nk);
}

// Gbar(k, i w_n)[n][e][k] += conj(dw_n) nbar_e / N_k
__global__ void add_dw_nbar_kernel(double2* Gbar_iw, const double2* __restrict__ dw,
                                   const double2* __restrict__ nbar, int r, int np, int nk) {
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<long long>(r) * np * nk) return;
  const int n = static_cast<int>(idx / (static_cast<long long>(np) * nk));
  const int e = static_cast<int>((idx / nk) % np);
  Gbar_iw[idx] = cfma(cconj(dw[n]), cscale(nbar[e], 1.0 / nk), Gbar_iw[idx]);
}

__global__ void axpy_kernel(double2* y, const double2* __restrict__ x, double a, long long n) {
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    y[i] = make_double2(y[i].x + a * x[i].x, y[i].y + a * x[i].y);
}

__global__ void scale_kernel(double2* y, double a, long long n) {
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    y[i] = cscale(y[i], a);
}

unsigned gsz(long long n) {
  long long b = (n + 255) / 256;
  return static_cast<unsigned>(b > 4864 ? 4864 : (b < 1 ? 1 : b));
}

}  // namespace

cudaError_t launch_dyson_g_bwd(const double2* Hk, const double2* SigHF, const double2* SigIw,
                               const double* iw, double mu, int r, int norb, int nk,
                               const double2* Gbar_iw, double2* SigCbar_iw, double2* Sbar,
                               cudaStream_t st) {
  const unsigned g = (nk + 127) / 128;
  switch (norb) {
#define QA_CASE(NO) case NO: dyson_g_bwd_kernel<NO><<<g, 128, 0, st>>>(Hk, SigHF, SigIw, iw, mu, r, nk, Gbar_iw, SigCbar_iw, Sbar); break;
    QA_CASE(1) QA_CASE(2) QA_CASE(3) QA_CASE(4) QA_CASE(5)
#undef QA_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_sigma_bwd(const double2* GR, const double2* SigbarR, double2* W, double2* GRbar,
                             int r, int norb, int nk, cudaStream_t st) {
  dim3 grid(r, (nk + 127) / 128);
  switch (norb) {
#define QA_CASE(NO) case NO: sigma_bwd_kernel<NO><<<grid, 128, 0, st>>>(GR, SigbarR, W, GRbar, nk); break;
    QA_CASE(1) QA_CASE(2) QA_CASE(3) QA_CASE(4) QA_CASE(5)
#undef QA_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_bubble_bwd(const double2* GR, const double2* GL, const int* mR,
                              const double2* Pbar, double2* GRbar, double2* GLbar, int r, int norb,
                              int nk, double s, cudaStream_t st) {
  dim3 grid(r, (nk + 127) / 128);
  switch (norb) {
#define QA_CASE(NO) case NO: bubble_bwd_kernel<NO><<<grid, 128, 0, st>>>(GR, GL, mR, Pbar, GRbar, GLbar, nk, s); break;
    QA_CASE(1) QA_CASE(2) QA_CASE(3) QA_CASE(4) QA_CASE(5)
#undef QA_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_sigma_bwd_terms(const double2* GR, const double2* SigbarR, double2* W, double2* GRbar,
                                   const int* terms, const double2* coef, int r, int nb2, int norb, int nk,
                                   cudaStream_t st) {
  const int no2 = norb * norb;
  if (no2 > 256) return cudaErrorInvalidValue;
  const size_t smem = static_cast<size_t>(3) * no2 * kTermThreads * sizeof(double2);
  cudaError_t e = set_smem(reinterpret_cast<const void*>(&sigma_bwd_terms_kernel), smem);
  if (e != cudaSuccess) return e;
  dim3 grid(r, (nk + kTermThreads - 1) / kTermThreads);
  sigma_bwd_terms_kernel<<<grid, kTermThreads, smem, st>>>(GR, SigbarR, W, GRbar, terms, coef, nb2, no2, nk);
  return cudaGetLastError();
}

cudaError_t launch_bubble_bwd_terms(const double2* GR, const double2* GL, const int* mR, const double2* Pbar,
                                    double2* GRbar, double2* GLbar, const int* terms, const double2* coef,
                                    int r, int nb2, int norb, int nk, cudaStream_t st) {
  const int no2 = norb * norb;
  if (no2 > 256) return cudaErrorInvalidValue;
  const size_t smem = static_cast<size_t>(4) * no2 * kTermThreads * sizeof(double2);
  cudaError_t e = set_smem(reinterpret_cast<const void*>(&bubble_bwd_terms_kernel), smem);
  if (e != cudaSuccess) return e;
  dim3 grid(r, (nk + kTermThreads - 1) / kTermThreads);
  bubble_bwd_terms_kernel<<<grid, kTermThreads, smem, st>>>(GR, GL, mR, Pbar, GRbar, GLbar, terms, coef, nb2,
                                                            no2, nk);
  return cudaGetLastError();
}

cudaError_t launch_dyson_w_bwd(const double2* P, const double2* Vq, double2* Wb, double* Vqbar,
                               int r, int npair, int nk, int* err, cudaStream_t st,
                               const double2* lu, const unsigned char* piv) {
  if (lu && !piv) return cudaErrorInvalidValue;
  if (npair > kMaxN) return cudaErrorInvalidValue;
  const size_t smem = static_cast<size_t>(kWarpsB) * 5 * npair * (npair + 1) * sizeof(double2) +
                      kWarpsB * kMaxN * sizeof(int);
  cudaError_t e = set_smem(reinterpret_cast<const void*>(&dyson_w_bwd_kernel), smem);
  if (e != cudaSuccess) return e;
  dim3 grid((nk + kWarpsB - 1) / kWarpsB, r);
  dyson_w_bwd_kernel<<<grid, kWarpsB * 32, smem, st>>>(P, Vq, Wb, Vqbar, npair, nk, err, lu, piv);
  return cudaGetLastError();
}

cudaError_t launch_hf_bwd(const double2* VR, const double2* nR, const double2* X, int nV, int norb,
                          double s, int nk, double2* VbarHF, double2* nbarR, cudaStream_t st) {
  hf_bwd_kernel<<<1, 256, 0, st>>>(VR, nR, X, nV, norb, s, nk, VbarHF, nbarR);
  return cudaGetLastError();
}

cudaError_t launch_nbar_k(const double2* nbarR, const int* R, int nV1, int np, int nk, int n1,
                          int n2, int n3, double2* nbk, cudaStream_t st) {
  long long n = static_cast<long long>(nk) * np;
  nbar_k_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(nbarR, R, nV1, np, nk, n1,
                                                                       n2, n3, nbk);
  return cudaGetLastError();
}

cudaError_t launch_add_dw_nbar(double2* Gbar_iw, const double2* dw, const double2* nbar, int r,
                               int np, int nk, cudaStream_t st) {
  long long n = static_cast<long long>(r) * np * nk;
  add_dw_nbar_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(Gbar_iw, dw, nbar, r,
                                                                             np, nk);
  return cudaGetLastError();
}

cudaError_t launch_axpy(double2* y, const double2* x, double a, long long n, cudaStream_t st) {
  axpy_kernel<<<gsz(n), 256, 0, st>>>(y, x, a, n);
  return cudaGetLastError();
}

cudaError_t launch_scale(double2* y, double a, long long n, cudaStream_t st) {
  scale_kernel<<<gsz(n), 256, 0, st>>>(y, a, n);
  return cudaGetLastError();
}

}  // namespace qa
