// Arithmetic-rate probe (a measurement utility; the paper has no counterpart):
// every thread runs eight independent chains of fused multiply-adds, so the
// FMA pipes, not latency, bound the kernel.  The benchmark times it with CUDA
// events to obtain the FP32 and FP64 FMA rates of the GPU it runs on, the
// peaks of the iteration's ALU-bound (double-float and FP64) kernels.
#include "../../include/qa.h"
#include "qa_common.cuh"

namespace qa {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) fma_chain_kernel(int iters, T* out) {
  T a[kProbeChains];
#pragma unroll
  for (int j = 0; j < kProbeChains; ++j) a[j] = static_cast<T>(threadIdx.x + j) * static_cast<T>(1e-7);
  const T b = static_cast<T>(0.9999999), c = static_cast<T>(1e-9);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) a[j] = fma(a[j], b, c);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < kProbeChains; ++j) s += a[j];
  out[static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace qa

extern "C" int qa_fma_probe(int precision, int iters, void* out, long long* out_elems,
                            double* flops, void* stream) {
  if (iters < 1 || (precision != QA_FP64 && precision != QA_FP32)) return QA_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return QA_ECUDA;
  const long long blocks = 8ll * sms;
  const long long elems = blocks * qa::kProbeThreads;
  if (out_elems) *out_elems = elems;
  if (flops) *flops = 2.0 * elems * qa::kProbeChains * static_cast<double>(iters);
  if (!out) return QA_OK;                       // size query
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (precision == QA_FP64)
    qa::fma_chain_kernel<double><<<static_cast<unsigned>(blocks), qa::kProbeThreads, 0, st>>>(
        iters, static_cast<double*>(out));
  else
    qa::fma_chain_kernel<float><<<static_cast<unsigned>(blocks), qa::kProbeThreads, 0, st>>>(
        iters, static_cast<float*>(out));
  return cudaGetLastError() == cudaSuccess ? QA_OK : QA_ECUDA;
}
