// Small FP64 kernels: lattice Fourier tables, Hartree and Fock terms,
// k-averages and precision conversions.
//
// H(k) = sum_R H(R) e^{-i k.R} and V(q) = sum_R V(R) e^{-i q.R} (paper Eq. for
// the k<->R transform, cell gauge).  Hartree (paper Eq. for Sigma^H):
// Sigma^H_{ab} = s sum_{cd} V_{(ab),(cd)}(q=0) n_{dc}(R=0).  Fock (paper Eq. for
// Sigma^F): Sigma^F_{ad}(R) = -sum_{bc} V_{(ab),(cd)}(R) n_{bc}(R), summed back
// to k with e^{-i k.R}; n(R) = (1/N_k) sum_k e^{+i k.R} n(k).
#include "qa_common.cuh"

namespace qa {
namespace {

__global__ void ft_table_kernel(const int* __restrict__ R, const double2* __restrict__ XR, int nR,
                                int msize, int nk, int n1, int n2, int n3, double2* out) {
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<long long>(nk) * msize) return;
  const int k = static_cast<int>(idx / msize);
  const int e = static_cast<int>(idx - static_cast<long long>(k) * msize);
  double2 acc = make_double2(0, 0);
  for (int v = 0; v < nR; ++v) {
    double2 ph = lattice_phase(k, n1, n2, n3, R + 3 * v, -1);
    acc = cfma(XR[static_cast<size_t>(v) * msize + e], ph, acc);
  }
  out[idx] = acc;
}

// exp(+i k.R_v) for every listed R_v and k: [nR][N_k]
__global__ void phase_table_kernel(const int* __restrict__ R, int nR, int nk, int n1, int n2, int n3,
                                   double2* ph) {
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<long long>(nR) * nk) return;
  const int v = static_cast<int>(idx / nk), k = static_cast<int>(idx - static_cast<long long>(v) * nk);
  ph[idx] = lattice_phase(k, n1, n2, n3, R + 3 * v, +1);
}

// block per (v, e); phases from the table ph (exp(+i k.R_v)) when given
__global__ void density_R_kernel(const double2* __restrict__ nk_, const int* __restrict__ R,
                                 const double2* __restrict__ ptab, int norb2, int nk, int n1,
                                 int n2, int n3, double2* nR) {
  __shared__ double sh[64];
  const int v = blockIdx.x / norb2, e = blockIdx.x % norb2;
  double re = 0.0, im = 0.0;
  for (int k = threadIdx.x; k < nk; k += blockDim.x) {
    double2 ph = ptab ? ptab[static_cast<size_t>(v) * nk + k] : lattice_phase(k, n1, n2, n3, R + 3 * v, +1);
    double2 x = nk_[static_cast<size_t>(e) * nk + k];
    re += x.x * ph.x - x.y * ph.y;
    im += x.x * ph.y + x.y * ph.x;
  }
  block_sum2(re, im, sh);
  if (threadIdx.x == 0) nR[blockIdx.x] = make_double2(re / nk, im / nk);
}

// one block: Sigma^F(R_v) for every v and Sigma^H (stored after them).
// nR_in holds n(R_v) for v < nRv and n(R=0) at v = nRv.
__global__ void hf_real_kernel(const double2* __restrict__ VR, const double2* __restrict__ nR,
                               int nRv, int no, double s, double2* sigF_R) {
  const int np = no * no;
  const double2* n0 = nR + static_cast<size_t>(nRv) * np;
  for (int o = threadIdx.x; o < (nRv + 1) * np; o += blockDim.x) {
    const int v = o / np, e = o % np;
    const int a = e / no, d = e % no;
    double2 acc = make_double2(0, 0);
    if (v < nRv) {
      const double2* Vv = VR + static_cast<size_t>(v) * np * np;
      const double2* nv = nR + static_cast<size_t>(v) * np;
      for (int b = 0; b < no; ++b)
        for (int c = 0; c < no; ++c)
          acc = cfms(Vv[(a * no + b) * np + c * no + d], nv[b * no + c], acc);
    } else {
      // Hartree: (a, d) here play (a, b) of Sigma^H_ab
      for (int w = 0; w < nRv; ++w) {
        const double2* Vw = VR + static_cast<size_t>(w) * np * np;
        for (int c = 0; c < no; ++c)
          for (int dd = 0; dd < no; ++dd)
            acc = cfma(Vw[(a * no + d) * np + c * no + dd], n0[dd * no + c], acc);
      }
      acc.x *= s;
      acc.y *= s;
    }
    sigF_R[o] = acc;
  }
}

__global__ void hf_k_kernel(const double2* __restrict__ sigF_R, const int* __restrict__ R,
                            const double2* __restrict__ ptab, int nRv, int no, int nk, int n1,
                            int n2, int n3, double2* SigHF) {
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int np = no * no;
  if (idx >= static_cast<long long>(nk) * np) return;
  const int k = static_cast<int>(idx / np), e = static_cast<int>(idx % np);
  double2 acc = sigF_R[static_cast<size_t>(nRv) * np + e];   // Sigma^H
  for (int v = 0; v < nRv; ++v) {
    double2 ph = ptab ? cconj(ptab[static_cast<size_t>(v) * nk + k]) : lattice_phase(k, n1, n2, n3, R + 3 * v, -1);
    acc = cfma(sigF_R[static_cast<size_t>(v) * np + e], ph, acc);
  }
  SigHF[idx] = acc;
}

template <typename T>
__global__ void k_average_kernel(const cplx<T>* __restrict__ x, int nk, double2* out) {
  __shared__ double sh[64];
  const int e = blockIdx.x;
  double re = 0.0, im = 0.0;
  for (int k = threadIdx.x; k < nk; k += blockDim.x) {
    double2 v = to_c64d(x[static_cast<size_t>(e) * nk + k]);
    re += v.x;
    im += v.y;
  }
  block_sum2(re, im, sh);
  if (threadIdx.x == 0) out[e] = make_double2(re / nk, im / nk);
}

// n(k) = sum_j dtau_j G(k, tau_j) for every column of a complex128 G (FP64),
// and the complex64 copy of G when G32 is given: one pass over G, one thread
// per column, coalesced along the columns.  The FP64 multiply-adds bound it
// (GB300 runs FP64 at a small fraction of its FP32 rate), so REALW (real
// weights) takes the two FMAs a real weight needs instead of the complex four.
// DF: the copy is double-float (dfc) instead of complex64.
template <bool REALW, bool DF>
__global__ void __launch_bounds__(256) g_input_kernel(const double2* __restrict__ G,
                                                      const double2* __restrict__ dtau, int r,
                                                      long long ncol, void* __restrict__ Gc,
                                                      double2* __restrict__ nk_out) {
  __shared__ double2 d[128];
  for (int l = threadIdx.x; l < r; l += blockDim.x) d[l] = dtau[l];
  __syncthreads();
  for (long long col = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; col < ncol;
       col += static_cast<long long>(gridDim.x) * blockDim.x) {
    double2 acc[4] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
    for (int l0 = 0; l0 < r; l0 += 8) {       // eight loads in flight per thread
      double2 x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        x[u] = l0 + u < r ? G[static_cast<long long>(l0 + u) * ncol + col] : make_double2(0, 0);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (l0 + u < r) {
          if (Gc) {
            const long long o = static_cast<long long>(l0 + u) * ncol + col;
            if (DF) static_cast<dfc*>(Gc)[o] = from_d2<dfc>(x[u]);
            else static_cast<float2*>(Gc)[o] = make_float2(static_cast<float>(x[u].x), static_cast<float>(x[u].y));
          }
          if (REALW) {
            acc[u & 3].x = fma(d[l0 + u].x, x[u].x, acc[u & 3].x);
            acc[u & 3].y = fma(d[l0 + u].x, x[u].y, acc[u & 3].y);
          } else {
            acc[u & 3] = cfma(d[l0 + u], x[u], acc[u & 3]);
          }
        }
      }
    }
    nk_out[col] = cadd(cadd(acc[0], acc[1]), cadd(acc[2], acc[3]));
  }
}

__global__ void c128_to_c64_kernel(const double2* in, float2* out, long long n) {
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    out[i] = make_float2(static_cast<float>(in[i].x), static_cast<float>(in[i].y));
}

__global__ void c128_to_df_kernel(const double2* in, dfc* out, long long n) {
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    out[i] = from_d2<dfc>(in[i]);
}

__global__ void df_to_c128_kernel(const dfc* in, double2* out, long long n) {
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    out[i] = to_c64d(in[i]);
}

__global__ void c64_to_c128_kernel(const float2* in, double2* out, long long n) {
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    out[i] = make_double2(in[i].x, in[i].y);
}

unsigned grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  return static_cast<unsigned>(b > 4864 ? 4864 : (b < 1 ? 1 : b));
}

}  // namespace

cudaError_t launch_ft_table(const int* R, const double2* XR, int nR, int msize, const int*, int nk,
                            int n1, int n2, int n3, double2* out, cudaStream_t st) {
  long long n = static_cast<long long>(nk) * msize;
  ft_table_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(R, XR, nR, msize, nk, n1,
                                                                         n2, n3, out);
  return cudaGetLastError();
}

cudaError_t launch_phase_table(const int* R, int nR, int nk, int n1, int n2, int n3, double2* ph,
                               cudaStream_t st) {
  long long n = static_cast<long long>(nR) * nk;
  if (n <= 0) return cudaSuccess;
  phase_table_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(R, nR, nk, n1, n2, n3, ph);
  return cudaGetLastError();
}

cudaError_t launch_density_R(const double2* nk_, const int* R, int nRv, int norb2, const int*,
                             int nk, int n1, int n2, int n3, double2* nR_out, cudaStream_t st,
                             const double2* ph) {
  density_R_kernel<<<nRv * norb2, 256, 0, st>>>(nk_, R, ph, norb2, nk, n1, n2, n3, nR_out);
  return cudaGetLastError();
}

cudaError_t launch_hf(const double2* VR, const double2* nR_in, const int* R, int nRv, int norb,
                      double s, const int*, int nk, int n1, int n2, int n3, double2* sigF_R,
                      double2* SigHF, cudaStream_t st, const double2* ph) {
  hf_real_kernel<<<1, 256, 0, st>>>(VR, nR_in, nRv, norb, s, sigF_R);
  long long n = static_cast<long long>(nk) * norb * norb;
  hf_k_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(sigF_R, R, ph, nRv, norb, nk,
                                                                     n1, n2, n3, SigHF);
  return cudaGetLastError();
}

cudaError_t launch_g_input(const double2* G, const double2* dtau, int r, long long ncol,
                           float2* G32, double2* nk_out, cudaStream_t st, bool real_w) {
  if (r > 128) return cudaErrorInvalidValue;
  if (real_w)
    g_input_kernel<true, false><<<grid_for(ncol, 256), 256, 0, st>>>(G, dtau, r, ncol, G32, nk_out);
  else
    g_input_kernel<false, false><<<grid_for(ncol, 256), 256, 0, st>>>(G, dtau, r, ncol, G32, nk_out);
  return cudaGetLastError();
}

cudaError_t launch_g_input_df(const double2* G, const double2* dtau, int r, long long ncol,
                              void* Gdf, double2* nk_out, cudaStream_t st, bool real_w) {
  if (r > 128) return cudaErrorInvalidValue;
  if (real_w)
    g_input_kernel<true, true><<<grid_for(ncol, 256), 256, 0, st>>>(G, dtau, r, ncol, Gdf, nk_out);
  else
    g_input_kernel<false, true><<<grid_for(ncol, 256), 256, 0, st>>>(G, dtau, r, ncol, Gdf, nk_out);
  return cudaGetLastError();
}

cudaError_t launch_c128_to_df(const double2* in, void* out, long long n, cudaStream_t st) {
  c128_to_df_kernel<<<grid_for(n, 256), 256, 0, st>>>(in, static_cast<dfc*>(out), n);
  return cudaGetLastError();
}

cudaError_t launch_df_to_c128(const void* in, double2* out, long long n, cudaStream_t st) {
  df_to_c128_kernel<<<grid_for(n, 256), 256, 0, st>>>(static_cast<const dfc*>(in), out, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_k_average(const void* x, int m, int nk, double2* out, cudaStream_t st) {
  k_average_kernel<T><<<m, 256, 0, st>>>(reinterpret_cast<const cplx<T>*>(x), nk, out);
  return cudaGetLastError();
}

cudaError_t launch_c128_to_c64(const double2* in, float2* out, long long n, cudaStream_t st) {
  c128_to_c64_kernel<<<grid_for(n, 256), 256, 0, st>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_c64_to_c128(const float2* in, double2* out, long long n, cudaStream_t st) {
  c64_to_c128_kernel<<<grid_for(n, 256), 256, 0, st>>>(in, out, n);
  return cudaGetLastError();
}

template cudaError_t launch_k_average<double>(const void*, int, int, double2*, cudaStream_t);
template cudaError_t launch_k_average<float>(const void*, int, int, double2*, cudaStream_t);
template cudaError_t launch_k_average<dfl>(const void*, int, int, double2*, cudaStream_t);

}  // namespace qa
