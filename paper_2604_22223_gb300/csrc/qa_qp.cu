// Hartree-Fock self-consistency and quasiparticle quantities (FP64).
//
// Hartree-Fock (paper Sec. "Hartree-Fock self-consistency", Fig. 3(a)):
// H(k) = H0(k) + Sigma^H + Sigma^F(k), mu from the filling, and the density
// matrix n(k) = 1 / (exp(beta (H(k) - mu)) + 1) through the eigendecomposition
// of each Hermitian H(k) (one thread per k, Jacobi rotations in registers).
//
// Quasiparticles (paper Secs. on the Z and SigStc classes; quasiparticle
// Hamiltonian of the graphene results): from Sigma^C(k, i w) at the DLR
// nodes, Sigma(+-i w0) at the lowest fermionic frequencies w0 = pi / beta
// (weights of the DLR expansion, built on the host), then
//   Sigma(0) = (Sigma(i w0) + Sigma(-i w0)) / 2 + Sigma^HF,
//   Z^-1 = 1 - (Sigma(i w0) - Sigma(-i w0)) / (2 i w0),
//   H_QP = sqrt(Z) (H0 + Sigma(0)) sqrt(Z)   and its eigenvalues,
// Hermitian parts taken; sqrt(Z) from the eigendecomposition of Z^-1.
#include "qa_common.cuh"

namespace qa {
namespace {

// Eigen-decomposition of a Hermitian NO x NO matrix held in registers
// (cyclic complex Jacobi rotations): on return the diagonal of a holds the
// eigenvalues in ascending order and the columns of v the eigenvectors.
template <int NO>
__device__ __forceinline__ void herm_eig(double2 (&a)[NO][NO], double2 (&v)[NO][NO], double (&ev)[NO]) {
#pragma unroll
  for (int i = 0; i < NO; ++i)
#pragma unroll
    for (int j = 0; j < NO; ++j) v[i][j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0, tot = 0.0;
#pragma unroll
    for (int i = 0; i < NO; ++i)
#pragma unroll
      for (int j = 0; j < NO; ++j) {
        const double x = cabs2(a[i][j]);
        tot += x;
        if (i != j) off += x;
      }
    if (!(off > 1e-30 * tot)) break;     // off-diagonal norm <= 1e-15 of the norm
#pragma unroll
    for (int p = 0; p < NO - 1; ++p)
#pragma unroll
      for (int q = p + 1; q < NO; ++q) {
        const double m = sqrt(cabs2(a[p][q]));
        if (m > 0.0) {
          const double2 e = make_double2(a[p][q].x / m, a[p][q].y / m);    // phase of a_pq
          const double zeta = (a[q][q].x - a[p][p].x) / (2.0 * m);
          const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
          const double2 se = cscale(e, s), sec = cscale(cconj(e), s);
#pragma unroll
          for (int k = 0; k < NO; ++k) {                               // columns p, q
            const double2 kp = a[k][p], kq = a[k][q];
            a[k][p] = csub(cscale(kp, c), cmul(sec, kq));
            a[k][q] = cadd(cmul(se, kp), cscale(kq, c));
          }
#pragma unroll
          for (int k = 0; k < NO; ++k) {                               // rows p, q
            const double2 pk = a[p][k], qk = a[q][k];
            a[p][k] = csub(cscale(pk, c), cmul(se, qk));
            a[q][k] = cadd(cmul(sec, pk), cscale(qk, c));
          }
#pragma unroll
          for (int k = 0; k < NO; ++k) {
            const double2 vp = v[k][p], vq = v[k][q];
            v[k][p] = csub(cscale(vp, c), cmul(sec, vq));
            v[k][q] = cadd(cmul(se, vp), cscale(vq, c));
          }
        }
      }
  }
#pragma unroll
  for (int i = 0; i < NO; ++i) ev[i] = a[i][i].x;
  // ascending order (selection by predicated swaps: indices stay compile-time)
#pragma unroll
  for (int i = 0; i < NO - 1; ++i)
#pragma unroll
    for (int j = i + 1; j < NO; ++j) {
      const bool sw = ev[j] < ev[i];
      const double ei = ev[i], ej = ev[j];
      ev[i] = sw ? ej : ei;
      ev[j] = sw ? ei : ej;
#pragma unroll
      for (int k = 0; k < NO; ++k) {
        const double2 vi = v[k][i], vj = v[k][j];
        v[k][i].x = sw ? vj.x : vi.x; v[k][i].y = sw ? vj.y : vi.y;
        v[k][j].x = sw ? vi.x : vj.x; v[k][j].y = sw ? vi.y : vj.y;
      }
    }
}

template <int NO>
__device__ __forceinline__ void load_herm(const double2* __restrict__ X, const double2* __restrict__ Y,
                                          double2 (&a)[NO][NO]) {
#pragma unroll
  for (int i = 0; i < NO; ++i)
#pragma unroll
    for (int j = 0; j < NO; ++j) {
      double2 x = X[i * NO + j], y = X[j * NO + i];
      if (Y) {
        const double2 u = Y[i * NO + j], w = Y[j * NO + i];
        x.x += u.x; x.y += u.y; y.x += w.x; y.y += w.y;
      }
      a[i][j] = make_double2(0.5 * (x.x + y.x), 0.5 * (x.y - y.y));        // Hermitian part
    }
}

__device__ __forceinline__ double fermi_fn(double x) {                    // 1 / (e^x + 1)
  if (x > 0.0) {
    const double e = exp(-x);
    return e / (1.0 + e);
  }
  return 1.0 / (1.0 + exp(x));
}

// E[k][i], U[k][a][i] of H(k) (+ SigHF(k))
template <int NO>
__global__ void hf_eig_kernel(const double2* __restrict__ Hk, const double2* __restrict__ SigHF,
                              int nk, double* __restrict__ E, double2* __restrict__ U) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nk) return;
  double2 a[NO][NO], v[NO][NO];
  double ev[NO];
  load_herm<NO>(Hk + static_cast<size_t>(k) * NO * NO,
                SigHF ? SigHF + static_cast<size_t>(k) * NO * NO : nullptr, a);
  herm_eig<NO>(a, v, ev);
#pragma unroll
  for (int i = 0; i < NO; ++i) E[static_cast<size_t>(k) * NO + i] = ev[i];
#pragma unroll
  for (int i = 0; i < NO; ++i)
#pragma unroll
    for (int j = 0; j < NO; ++j) U[static_cast<size_t>(k) * NO * NO + i * NO + j] = v[i][j];
}

// partial sums of f(beta (E - mu)) and beta f (1 - f) over all (k, i)
__global__ void fd_sum_kernel(const double* __restrict__ E, long long n, double beta, double mu,
                              double* part) {
  __shared__ double sh[64];
  double s1 = 0.0, s2 = 0.0;
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const double f = fermi_fn(beta * (E[i] - mu));
    s1 += f;
    s2 += beta * f * (1.0 - f);
  }
  block_sum2(s1, s2, sh);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s1;
    part[2 * blockIdx.x + 1] = s2;
  }
}

// n(k)_ab = sum_i U_ai f_i conj(U_bi), stored [a*NO+b][k]
template <int NO>
__global__ void fd_density_kernel(const double* __restrict__ E, const double2* __restrict__ U,
                                  int nk, double beta, double mu, double2* __restrict__ nk_out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nk) return;
  double f[NO];
#pragma unroll
  for (int i = 0; i < NO; ++i) f[i] = fermi_fn(beta * (E[static_cast<size_t>(k) * NO + i] - mu));
  const double2* u = U + static_cast<size_t>(k) * NO * NO;
#pragma unroll
  for (int a = 0; a < NO; ++a)
#pragma unroll
    for (int b = 0; b < NO; ++b) {
      double2 acc = make_double2(0.0, 0.0);
#pragma unroll
      for (int i = 0; i < NO; ++i) acc = cfma(cscale(u[a * NO + i], f[i]), cconj(u[b * NO + i]), acc);
      nk_out[static_cast<size_t>(a * NO + b) * nk + k] = acc;
    }
}

// resid = max |new - old|; new <- old + mix (new - old); old <- new
__global__ void mix_kernel(double2* __restrict__ cur, double2* __restrict__ old, double mix,
                           long long n, double* part) {
  __shared__ double sh[32];
  double best = 0.0;
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const double2 nw = cur[i], od = old[i];
    const double dx = nw.x - od.x, dy = nw.y - od.y;
    best = fmax(best, sqrt(dx * dx + dy * dy));
    const double2 m = make_double2(od.x + mix * dx, od.y + mix * dy);
    cur[i] = m;
    old[i] = m;
  }
  best = block_max(best, sh);
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = best; part[2 * blockIdx.x + 1] = 0.0; }
}

// part[2b] >= max E, part[2b+1] >= max(-E) over this block's share (upper
// bounds: the block reduction pads idle lanes with 0; enough for a bracket)
__global__ void fd_range_kernel(const double* __restrict__ E, long long n, double* part) {
  __shared__ double sh[32];
  double hi = -INFINITY, lo = -INFINITY;
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    hi = fmax(hi, E[i]);
    lo = fmax(lo, -E[i]);
  }
  hi = block_max(hi, sh);
  __syncthreads();
  lo = block_max(lo, sh);
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = hi; part[2 * blockIdx.x + 1] = lo; }
}

// Sigma(+-i w0) = sum_n w+-[n] Sigma^C(i w_n) for every (element, k): one
// thread per column, FP64 accumulation; S[0][c] = Sigma(+i w0), S[1][c] = Sigma(-i w0)
template <typename TS>
__global__ void qp_sums_kernel(const cplx<TS>* __restrict__ SigIw, const double2* __restrict__ wp,
                               const double2* __restrict__ wm, int r, long long m,
                               double2* __restrict__ S) {
  const long long c = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c >= m) return;
  double2 sp = make_double2(0, 0), sm = make_double2(0, 0);
  int n = 0;
  for (; n + 4 <= r; n += 4) {               // four independent loads in flight
    double2 x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = to_c64d(SigIw[static_cast<size_t>(n + u) * m + c]);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      sp = cfma(wp[n + u], x[u], sp);
      sm = cfma(wm[n + u], x[u], sm);
    }
  }
  for (; n < r; ++n) {
    const double2 x = to_c64d(SigIw[static_cast<size_t>(n) * m + c]);
    sp = cfma(wp[n], x, sp);
    sm = cfma(wm[n], x, sm);
  }
  S[c] = sp;
  S[m + c] = sm;
}

// quasiparticle quantities per k from S (qp_sums_kernel; null: no Sigma^C)
template <int NO>
__global__ void qp_kernel(const double2* __restrict__ Hk, const double2* __restrict__ SigHF,
                          const double2* __restrict__ S, int nk, double w0,
                          double2* __restrict__ Zo, double2* __restrict__ S0o,
                          double2* __restrict__ Hqo, double* __restrict__ epso, int* err) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nk) return;
  double2 sp[NO][NO], sm[NO][NO];
  const size_t m = static_cast<size_t>(NO) * NO * nk;
#pragma unroll
  for (int i = 0; i < NO; ++i)
#pragma unroll
    for (int j = 0; j < NO; ++j) {
      const size_t c = static_cast<size_t>(i * NO + j) * nk + k;
      sp[i][j] = S ? S[c] : make_double2(0, 0);
      sm[i][j] = S ? S[m + c] : make_double2(0, 0);
    }
  // Zi = 1 - (sp - sm) / (2 i w0); S0 = (sp + sm) / 2 + SigHF (raw, then Hermitian parts)
  double2 zi[NO][NO], s0[NO][NO];
  const double h = 0.5 / w0;
#pragma unroll
  for (int i = 0; i < NO; ++i)
#pragma unroll
    for (int j = 0; j < NO; ++j) {
      const double2 d = csub(sp[i][j], sm[i][j]);                // d / (2 i w0) = (d.y, -d.x) h
      zi[i][j] = make_double2((i == j ? 1.0 : 0.0) - d.y * h, d.x * h);
      s0[i][j] = make_double2(0.5 * (sp[i][j].x + sm[i][j].x), 0.5 * (sp[i][j].y + sm[i][j].y));
      if (SigHF) {
        const double2 f = SigHF[static_cast<size_t>(k) * NO * NO + i * NO + j];
        s0[i][j].x += f.x; s0[i][j].y += f.y;
      }
    }
  double2 a[NO][NO], v[NO][NO];
  double lam[NO];
#pragma unroll
  for (int i = 0; i < NO; ++i)
#pragma unroll
    for (int j = 0; j < NO; ++j)
      a[i][j] = make_double2(0.5 * (zi[i][j].x + zi[j][i].x), 0.5 * (zi[i][j].y - zi[j][i].y));
  herm_eig<NO>(a, v, lam);
  bool bad = false;
#pragma unroll
  for (int i = 0; i < NO; ++i) bad |= !(lam[i] > 0.0);
  // Z = V diag(1/lam) V^H, sqrt(Z) = V diag(lam^-1/2) V^H
  double2 z[NO][NO], sq[NO][NO];
#pragma unroll
  for (int i = 0; i < NO; ++i)
#pragma unroll
    for (int j = 0; j < NO; ++j) {
      double2 zz = make_double2(0, 0), ss = make_double2(0, 0);
#pragma unroll
      for (int l = 0; l < NO; ++l) {
        const double2 t = cmul(v[i][l], cconj(v[j][l]));
        const double il = bad ? 0.0 : 1.0 / lam[l];
        zz = cadd(zz, cscale(t, il));
        ss = cadd(ss, cscale(t, sqrt(il)));
      }
      z[i][j] = zz;
      sq[i][j] = ss;
    }
  // Hs = Hermitian part of H0 + S0; H_QP = sq Hs sq
  double2 hs[NO][NO], t1[NO][NO];
  const double2* H = Hk + static_cast<size_t>(k) * NO * NO;
#pragma unroll
  for (int i = 0; i < NO; ++i)
#pragma unroll
    for (int j = 0; j < NO; ++j) {
      const double2 x = cadd(H[i * NO + j], s0[i][j]), y = cadd(H[j * NO + i], s0[j][i]);
      hs[i][j] = make_double2(0.5 * (x.x + y.x), 0.5 * (x.y - y.y));
    }
#pragma unroll
  for (int i = 0; i < NO; ++i)
#pragma unroll
    for (int j = 0; j < NO; ++j) {
      double2 acc = make_double2(0, 0);
#pragma unroll
      for (int l = 0; l < NO; ++l) acc = cfma(hs[i][l], sq[l][j], acc);
      t1[i][j] = acc;
    }
#pragma unroll
  for (int i = 0; i < NO; ++i)
#pragma unroll
    for (int j = 0; j < NO; ++j) {
      double2 acc = make_double2(0, 0);
#pragma unroll
      for (int l = 0; l < NO; ++l) acc = cfma(sq[i][l], t1[l][j], acc);
      a[i][j] = acc;
    }
#pragma unroll
  for (int i = 0; i < NO; ++i)
#pragma unroll
    for (int j = 0; j < NO; ++j) {
      const double2 x = a[i][j], y = a[j][i];
      hs[i][j] = make_double2(0.5 * (x.x + y.x), 0.5 * (x.y - y.y));   // Hermitian H_QP
    }
  const size_t o = static_cast<size_t>(k) * NO * NO;
#pragma unroll
  for (int i = 0; i < NO; ++i)
#pragma unroll
    for (int j = 0; j < NO; ++j) {
      if (Zo) Zo[o + i * NO + j] = z[i][j];
      if (S0o) S0o[o + i * NO + j] = s0[i][j];
      if (Hqo) Hqo[o + i * NO + j] = hs[i][j];
    }
  if (epso) {
    double ev[NO];
    herm_eig<NO>(hs, v, ev);
#pragma unroll
    for (int i = 0; i < NO; ++i) epso[static_cast<size_t>(k) * NO + i] = ev[i];
  }
  if (bad) atomicCAS(err, 0, 5);                              // QA_ERANGE: Z not positive definite
}

}  // namespace

cudaError_t launch_hf_eig(const double2* Hk, const double2* SigHF, int norb, int nk, double* E,
                          double2* U, cudaStream_t st) {
  const unsigned g = static_cast<unsigned>((nk + 63) / 64);
  switch (norb) {
#define QA_CASE(NO) \
    case NO: hf_eig_kernel<NO><<<g, 64, 0, st>>>(Hk, SigHF, nk, E, U); break;
    QA_CASE(1) QA_CASE(2) QA_CASE(3) QA_CASE(4) QA_CASE(5)
#undef QA_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_fd_sum(const double* E, long long n, double beta, double mu, double* part,
                          int nblocks, cudaStream_t st) {
  fd_sum_kernel<<<nblocks, 256, 0, st>>>(E, n, beta, mu, part);
  return cudaGetLastError();
}

cudaError_t launch_fd_density(const double* E, const double2* U, int norb, int nk, double beta,
                              double mu, double2* nk_out, cudaStream_t st) {
  const unsigned g = static_cast<unsigned>((nk + 127) / 128);
  switch (norb) {
#define QA_CASE(NO) \
    case NO: fd_density_kernel<NO><<<g, 128, 0, st>>>(E, U, nk, beta, mu, nk_out); break;
    QA_CASE(1) QA_CASE(2) QA_CASE(3) QA_CASE(4) QA_CASE(5)
#undef QA_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_fd_range(const double* E, long long n, double* part, int nblocks,
                            cudaStream_t st) {
  fd_range_kernel<<<nblocks, 256, 0, st>>>(E, n, part);
  return cudaGetLastError();
}

cudaError_t launch_mix(double2* cur, double2* old, double mix, long long n, double* part,
                       int nblocks, cudaStream_t st) {
  mix_kernel<<<nblocks, 256, 0, st>>>(cur, old, mix, n, part);
  return cudaGetLastError();
}

template <typename TS>
cudaError_t launch_qp(const double2* Hk, const double2* SigHF, const void* SigIw,
                      const double2* wp, const double2* wm, int r, int norb, int nk, double w0,
                      double2* S, double2* Z, double2* S0, double2* Hqp, double* eps, int* err,
                      cudaStream_t st) {
  if (norb < 1 || norb > 5) return cudaErrorInvalidValue;
  const double2* Sp = nullptr;
  if (r > 0) {
    const long long m = static_cast<long long>(norb) * norb * nk;
    qp_sums_kernel<TS><<<static_cast<unsigned>((m + 255) / 256), 256, 0, st>>>(
        reinterpret_cast<const cplx<TS>*>(SigIw), wp, wm, r, m, S);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    Sp = S;
  }
  const unsigned g = static_cast<unsigned>((nk + 63) / 64);
  switch (norb) {
#define QA_CASE(NO) \
    case NO: qp_kernel<NO><<<g, 64, 0, st>>>(Hk, SigHF, Sp, nk, w0, Z, S0, Hqp, eps, err); break;
    QA_CASE(1) QA_CASE(2) QA_CASE(3) QA_CASE(4) QA_CASE(5)
#undef QA_CASE
  }
  return cudaGetLastError();
}

template cudaError_t launch_qp<double>(const double2*, const double2*, const void*, const double2*,
                                       const double2*, int, int, int, double, double2*, double2*,
                                       double2*, double2*, double*, int*, cudaStream_t);
template cudaError_t launch_qp<dfl>(const double2*, const double2*, const void*, const double2*,
                                    const double2*, int, int, int, double, double2*, double2*,
                                    double2*, double2*, double*, int*, cudaStream_t);
template cudaError_t launch_qp<float>(const double2*, const double2*, const void*, const double2*,
                                      const double2*, int, int, int, double, double2*, double2*,
                                      double2*, double2*, double*, int*, cudaStream_t);

}  // namespace qa
