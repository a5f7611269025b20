// DLR node-to-node transforms (Kaye, Chen & Parcollet 2022; the imaginary-time
// <-> Matsubara maps of the paper's dynamic lattice classes, Sec. on the code
// structure): out[j][c] = sum_l T[j][l] in[l][c] for every column c of a
// node-major array (c runs over orbital pairs and lattice points).
//
// Each block stages TILE columns x r nodes in shared memory (one HBM read),
// then every thread produces RB output rows of one column from registers.
// The tile is fully loaded before any write, so in == out is allowed.
#include <algorithm>

#include "qa_common.cuh"

namespace qa {
namespace {

template <typename T, int TILE, int RB>
__global__ void __launch_bounds__(256) dlr_apply_kernel(const cplx<T>* __restrict__ Tm, int rows_out,
                                                        int r, const cplx<T>* in, cplx<T>* out,
                                                        long long ncol, int accumulate) {
  using V = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* xs = reinterpret_cast<V*>(smem_raw);  // [r][TILE]
  const long long c0 = static_cast<long long>(blockIdx.x) * TILE;
  const int tid = threadIdx.x;
  for (int i = tid; i < r * TILE; i += blockDim.x) {
    int l = i / TILE, c = i - l * TILE;
    long long col = c0 + c;
    xs[i] = col < ncol ? in[static_cast<long long>(l) * ncol + col] : cmk<V>(0, 0);
  }
  __syncthreads();
  const int c = tid % TILE;
  const int g = tid / TILE;
  const int G = blockDim.x / TILE;
  const long long col = c0 + c;
  for (int j0 = g * RB; j0 < rows_out; j0 += G * RB) {
    V acc[RB];
#pragma unroll
    for (int b = 0; b < RB; ++b) acc[b] = cmk<V>(0, 0);
    for (int l = 0; l < r; ++l) {
      V x = xs[l * TILE + c];
#pragma unroll
      for (int b = 0; b < RB; ++b) {
        int j = j0 + b;
        V t = j < rows_out ? ldg_c(&Tm[static_cast<size_t>(j) * r + l]) : cmk<V>(0, 0);
        acc[b] = cfma(t, x, acc[b]);
      }
    }
    if (col < ncol) {
#pragma unroll
      for (int b = 0; b < RB; ++b)
        if (j0 + b < rows_out) {
          const long long o = static_cast<long long>(j0 + b) * ncol + col;
          out[o] = accumulate ? cadd(out[o], acc[b]) : acc[b];
        }
    }
  }
}

}  // namespace

// One output row (a weighted sum over the nodes, e.g. the density weights):
// one thread per column, the weights broadcast from L1.
template <typename T>
__global__ void __launch_bounds__(256) node_sum_kernel(const cplx<T>* __restrict__ w, int r,
                                                       const cplx<T>* __restrict__ in, cplx<T>* out,
                                                       long long ncol, int accumulate) {
  for (long long c = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; c < ncol;
       c += static_cast<long long>(gridDim.x) * blockDim.x) {
    cplx<T> acc = cmk<cplx<T>>(0, 0);
    for (int l = 0; l < r; ++l) acc = cfma(ldg_c(w + l), ldg_c(in + static_cast<long long>(l) * ncol + c), acc);
    out[c] = accumulate ? cadd(out[c], acc) : acc;
  }
}

template <typename T>
cudaError_t launch_dlr_apply(const void* Tm, int rows_out, int r, const void* in, void* out,
                             long long ncol, cudaStream_t st, int accumulate) {
  if (ncol <= 0 || rows_out <= 0) return cudaSuccess;
  if (rows_out == 1) {
    const long long nb = std::min<long long>((ncol + 255) / 256, 152LL * 16);
    node_sum_kernel<T><<<static_cast<unsigned>(nb), 256, 0, st>>>(
        reinterpret_cast<const cplx<T>*>(Tm), r, reinterpret_cast<const cplx<T>*>(in),
        reinterpret_cast<cplx<T>*>(out), ncol, accumulate);
    return cudaGetLastError();
  }
  constexpr int TILE = sizeof(cplx<T>) >= 16 ? 32 : 64;
  constexpr int RB = 4;
  size_t smem = static_cast<size_t>(r) * TILE * sizeof(cplx<T>);
  auto fn = &dlr_apply_kernel<T, TILE, RB>;
  cudaError_t e = set_smem(reinterpret_cast<const void*>(fn), smem);
  if (e != cudaSuccess) return e;
  long long nblk = (ncol + TILE - 1) / TILE;
  fn<<<static_cast<unsigned>(nblk), 256, smem, st>>>(reinterpret_cast<const cplx<T>*>(Tm), rows_out,
                                                     r, reinterpret_cast<const cplx<T>*>(in),
                                                     reinterpret_cast<cplx<T>*>(out), ncol, accumulate);
  return cudaGetLastError();
}

template cudaError_t launch_dlr_apply<double>(const void*, int, int, const void*, void*, long long,
                                              cudaStream_t, int);
template cudaError_t launch_dlr_apply<float>(const void*, int, int, const void*, void*, long long,
                                             cudaStream_t, int);
template cudaError_t launch_dlr_apply<dfl>(const void*, int, int, const void*, void*, long long,
                                           cudaStream_t, int);

}  // namespace qa
