// Pointwise real-space products of the GW iteration.
//
// Bubble (paper Eq. for the polarizability; per spin G(R,tau) G(-R,-tau) with
// G(-tau) = -G(beta - tau), times the spin factor s of W's Dyson equation):
//   P_{(ab),(cd)}(R, tau_j) = -s G_{bc}(R, tau_j) G_{da}(-R, beta - tau_j)
// Self-energy (paper Eq. for the GW self-energy, Wick contraction):
//   Sigma^C_{ad}(R, tau_j) = - sum_{bc} G_{bc}(R, tau_j) W^C_{(ab),(cd)}(R, tau_j)
// Both are streamed with R (the fastest index) across the threads of a warp,
// so every global access is a coalesced run along R.
#include "qa_common.cuh"

namespace qa {
namespace {

// grid.x = r * npair * npair slices (t, A, B); grid.y = R tiles
template <typename T>
__global__ void __launch_bounds__(256) bubble_kernel(const cplx<T>* __restrict__ GR,
                                                     const cplx<T>* __restrict__ GreflR,
                                                     const int* __restrict__ mR, cplx<T>* P, int norb,
                                                     int nk, T s) {
  using V = cplx<T>;
  const int npair = norb * norb;
  const long long slice = blockIdx.x;
  const int B = static_cast<int>(slice % npair);
  const int A = static_cast<int>((slice / npair) % npair);
  const int t = static_cast<int>(slice / (static_cast<long long>(npair) * npair));
  const int a = A / norb, b = A - a * norb, c = B / norb, d = B - c * norb;
  const int R = blockIdx.y * blockDim.x + threadIdx.x;
  if (R >= nk) return;
  const V g1 = GR[(static_cast<size_t>(t) * npair + b * norb + c) * nk + R];
  const V g2 = GreflR[(static_cast<size_t>(t) * npair + d * norb + a) * nk + mR[R]];
  V v = cmul(g1, g2);
  v.x *= -s;
  v.y *= -s;
  P[slice * nk + R] = v;
}

// one thread per (tau_j, R)
template <typename T, int NO>
__global__ void __launch_bounds__(128) sigma_kernel(const cplx<T>* __restrict__ GR,
                                                    const cplx<T>* __restrict__ WC, cplx<T>* Sig,
                                                    int nk) {
  using V = cplx<T>;
  constexpr int NP = NO * NO;
  const int t = blockIdx.x;
  const int R = blockIdx.y * blockDim.x + threadIdx.x;
  if (R >= nk) return;
  V g[NO][NO];
#pragma unroll
  for (int b = 0; b < NO; ++b)
#pragma unroll
    for (int c = 0; c < NO; ++c) g[b][c] = GR[(static_cast<size_t>(t) * NP + b * NO + c) * nk + R];
  const V* W = WC + static_cast<size_t>(t) * NP * NP * nk + R;
#pragma unroll 1
  for (int a = 0; a < NO; ++a) {
#pragma unroll
    for (int d = 0; d < NO; ++d) {
      V acc = cmk<V>(0, 0);
#pragma unroll
      for (int b = 0; b < NO; ++b)
#pragma unroll
        for (int c = 0; c < NO; ++c)
          acc = cfma(g[b][c], W[(static_cast<size_t>(a * NO + b) * NP + (c * NO + d)) * nk], acc);
      acc.x = -acc.x;
      acc.y = -acc.y;
      Sig[(static_cast<size_t>(t) * NP + a * NO + d) * nk + R] = acc;
    }
  }
}

}  // namespace

template <typename T>
cudaError_t launch_bubble(const void* GR, const void* GreflR, const int* mR, void* P, int r,
                          int norb, int nk, double s, cudaStream_t st) {
  const int npair = norb * norb;
  dim3 grid(static_cast<unsigned>(static_cast<long long>(r) * npair * npair), (nk + 255) / 256);
  bubble_kernel<T><<<grid, 256, 0, st>>>(reinterpret_cast<const cplx<T>*>(GR),
                                         reinterpret_cast<const cplx<T>*>(GreflR), mR,
                                         reinterpret_cast<cplx<T>*>(P), norb, nk, static_cast<T>(s));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sigma(const void* GR, const void* WC, void* Sig, int r, int norb, int nk,
                         cudaStream_t st) {
  dim3 grid(r, (nk + 127) / 128);
  auto g = reinterpret_cast<const cplx<T>*>(GR);
  auto w = reinterpret_cast<const cplx<T>*>(WC);
  auto s = reinterpret_cast<cplx<T>*>(Sig);
  switch (norb) {
    case 1: sigma_kernel<T, 1><<<grid, 128, 0, st>>>(g, w, s, nk); break;
    case 2: sigma_kernel<T, 2><<<grid, 128, 0, st>>>(g, w, s, nk); break;
    case 3: sigma_kernel<T, 3><<<grid, 128, 0, st>>>(g, w, s, nk); break;
    case 4: sigma_kernel<T, 4><<<grid, 128, 0, st>>>(g, w, s, nk); break;
    case 5: sigma_kernel<T, 5><<<grid, 128, 0, st>>>(g, w, s, nk); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template cudaError_t launch_bubble<double>(const void*, const void*, const int*, void*, int, int,
                                           int, double, cudaStream_t);
template cudaError_t launch_bubble<float>(const void*, const void*, const int*, void*, int, int,
                                          int, double, cudaStream_t);
template cudaError_t launch_sigma<double>(const void*, const void*, void*, int, int, int,
                                          cudaStream_t);
template cudaError_t launch_sigma<dfl>(const void*, const void*, void*, int, int, int, cudaStream_t);
template cudaError_t launch_bubble<dfl>(const void*, const void*, const int*, void*, int, int, int,
                                        double, cudaStream_t);
template cudaError_t launch_sigma<float>(const void*, const void*, void*, int, int, int,
                                         cudaStream_t);

}  // namespace qa
