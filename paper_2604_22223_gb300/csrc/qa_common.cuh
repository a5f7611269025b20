// Complex helpers and small device utilities shared by the qa kernels.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "qa_df.cuh"
#include "qa_internal.h"

namespace qa {

// Bounds checks of the index-map gathers (the -R map and the pair-basis term
// lists), compiled in only with QA_CHECK_BOUNDS: an index outside [0, n)
// records QA_EBOUNDS in the error word and the gather reads index 0 instead.
#ifdef QA_CHECK_BOUNDS
__device__ __forceinline__ int qa_index(int i, int n, int* err) {
  if (i >= 0 && i < n) return i;
  if (err) atomicCAS(err, 0, QA_EBOUNDS_CODE);
  return 0;
}
#else
__device__ __forceinline__ int qa_index(int i, int, int*) { return i; }
#endif

template <typename T> struct CplxOf;
template <> struct CplxOf<double> { using type = double2; };
template <> struct CplxOf<float> { using type = float2; };
template <> struct CplxOf<dfl> { using type = dfc; };
template <typename T> using cplx = typename CplxOf<T>::type;

template <typename V> __device__ __forceinline__ V cmk(double re, double im) {
  V v;
  v.x = static_cast<decltype(v.x)>(re);
  v.y = static_cast<decltype(v.y)>(im);
  return v;
}
// (re, im) from double-float components
template <typename V> __device__ __forceinline__ V cmk(dfl re, dfl im);
template <> __device__ __forceinline__ dfc cmk<dfc>(dfl re, dfl im) { return dfc{re, im}; }
// read-only cached load of one complex value
__device__ __forceinline__ double2 ldg_c(const double2* p) { return __ldg(p); }
__device__ __forceinline__ float2 ldg_c(const float2* p) { return __ldg(p); }
__device__ __forceinline__ dfc ldg_c(const dfc* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return dfc{dfl(v.x, v.y), dfl(v.z, v.w)};
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// c + a*b
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
  c.x = fma(a.x, b.x, c.x); c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y); c.y = fma(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
  c.x = fmaf(a.x, b.x, c.x); c.x = fmaf(-a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y); c.y = fmaf(a.y, b.x, c.y);
  return c;
}
// c - a*b
__device__ __forceinline__ double2 cfms(double2 a, double2 b, double2 c) {
  c.x = fma(-a.x, b.x, c.x); c.x = fma(a.y, b.y, c.x);
  c.y = fma(-a.x, b.y, c.y); c.y = fma(-a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ float2 cfms(float2 a, float2 b, float2 c) {
  c.x = fmaf(-a.x, b.x, c.x); c.x = fmaf(a.y, b.y, c.x);
  c.y = fmaf(-a.x, b.y, c.y); c.y = fmaf(-a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// 1/a
__device__ __forceinline__ double2 cinv(double2 a) {
  double d = 1.0 / cabs2(a);
  return make_double2(a.x * d, -a.y * d);
}
__device__ __forceinline__ float2 cinv(float2 a) {
  float d = __frcp_rn(cabs2(a));
  return make_float2(a.x * d, -a.y * d);
}
__device__ __forceinline__ double2 to_c64d(double2 a) { return a; }
__device__ __forceinline__ double2 to_c64d(float2 a) { return make_double2(a.x, a.y); }
template <typename V> __device__ __forceinline__ V from_d2(double2 a);
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 a) {
  return make_float2(static_cast<float>(a.x), static_cast<float>(a.y));
}
template <> __device__ __forceinline__ dfc from_d2<dfc>(double2 a) {
  return dfc{df_from_bits(a.x), df_from_bits(a.y)};
}

// exp(sign * 2 pi i * (sum_d (i_d R_d mod N_d) / N_d)) in FP64; the integer
// reduction keeps the phase argument exact for any R.
__device__ __forceinline__ double2 lattice_phase(int k, int n1, int n2, int n3, const int* R,
                                                 int sign) {
  int i3 = k % n3, i2 = (k / n3) % n2, i1 = k / (n3 * n2);
  long long m1 = ((static_cast<long long>(i1) * R[0]) % n1 + n1) % n1;
  long long m2 = ((static_cast<long long>(i2) * R[1]) % n2 + n2) % n2;
  long long m3 = ((static_cast<long long>(i3) * R[2]) % n3 + n3) % n3;
  double frac = static_cast<double>(m1) / n1 + static_cast<double>(m2) / n2 +
                static_cast<double>(m3) / n3;
  double s, c;
  sincospi(2.0 * sign * frac, &s, &c);
  return make_double2(c, s);
}

// Block-wide sum of two doubles (blockDim.x multiple of 32, <= 1024).
__device__ __forceinline__ void block_sum2(double& a, double& b, double* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sh[2 * w] = a; sh[2 * w + 1] = b; }
  __syncthreads();
  int nw = blockDim.x >> 5;
  if (w == 0) {
    a = l < nw ? sh[2 * l] : 0.0;
    b = l < nw ? sh[2 * l + 1] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
  }
}

__device__ __forceinline__ double block_max(double a, double* sh) {
  for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_down_sync(0xffffffffu, a, o));
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = a;
  __syncthreads();
  int nw = blockDim.x >> 5;
  if (w == 0) {
    a = l < nw ? sh[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_down_sync(0xffffffffu, a, o));
  }
  return a;
}

// Allow `bytes` of dynamic shared memory; max_carveout asks for the largest
// shared-memory carveout (for kernels that rely on shared memory, not L1).
inline cudaError_t set_smem(const void* fn, size_t bytes, bool max_carveout = false) {
  if (max_carveout) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(bytes));
}

}  // namespace qa
