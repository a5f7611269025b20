// Bubble and self-energy contractions in the reduced pair basis.
//
// With W^C = B Wt^C B^H and Pt = B^H P B (B: orthonormal basis of the
// subspace the interaction acts in, qa_basis.cpp) the two pointwise products
// of the iteration become, per (R, tau_j),
//   Pt_ij  = sum_{(ab) in i, (cd) in j} conj(B_(ab)i) B_(cd)j (-s) G_bc(R) G_da(-R, beta - tau)
//   Sigma_ad = - sum_ij Wt^C_ij sum_{(ab) in i, (cd) in j} B_(ab)i conj(B_(cd)j) G_bc(R)
// i.e. the paper's bubble and GW self-energy equations projected on the
// subspace.  The coefficient/index lists come from the host (one list per
// reduced entry, uniform across threads), so each thread owns one R at one
// tau, keeps its G (and G^refl, or its Sigma accumulators) as columns of
// shared memory [element][thread], and reads the term lists from shared
// memory as broadcasts.  Global traffic: the rho^2 reduced entries plus
// the small tensors, all coalesced along R.
#include "qa_common.cuh"

namespace qa {
namespace {

template <typename T> struct RedTpb { static constexpr int v = 256; };
template <> struct RedTpb<double> { static constexpr int v = 64; };

// one term as a single shared-memory record (one 16- or 32-byte load)
template <typename T> struct __align__(2 * sizeof(T) < 16 ? 16 : 32) TermRec {
  cplx<T> c;
  int idx;
};

template <typename T>
__device__ __forceinline__ void stage_terms(const int* __restrict__ terms,
                                            const cplx<T>* __restrict__ coef, int nout, int nterm,
                                            int* s_off, TermRec<T>* s_rec) {
  for (int e = threadIdx.x; e <= nout; e += blockDim.x) s_off[e] = terms[e];
  for (int e = threadIdx.x; e < nterm; e += blockDim.x) {
    TermRec<T> t;
    t.c = coef[e];
    t.idx = terms[nout + 1 + e];
    s_rec[e] = t;
  }
}

template <typename T>
__global__ void __launch_bounds__(RedTpb<T>::v) bubble_reduced_kernel(
    const cplx<T>* __restrict__ GR, const cplx<T>* __restrict__ GL, const int* __restrict__ mR,
    const int* __restrict__ terms, const cplx<T>* __restrict__ coef, int nterm,
    cplx<T>* __restrict__ Pt, int no2, int nout, int nk) {
  using V = cplx<T>;
  constexpr int TPB = RedTpb<T>::v;
  extern __shared__ __align__(32) unsigned char smem_raw[];
  TermRec<T>* s_rec = reinterpret_cast<TermRec<T>*>(smem_raw);
  V* g = reinterpret_cast<V*>(s_rec + nterm);   // [no2][TPB]
  V* gl = g + no2 * TPB;                        // [no2][TPB]
  int* s_off = reinterpret_cast<int*>(gl + no2 * TPB);
  const int tid = threadIdx.x;
  const int t = blockIdx.y;
  const int R = blockIdx.x * TPB + tid;
  stage_terms<T>(terms, coef, nout, nterm, s_off, s_rec);
  if (R < nk) {
    const int mr = mR[R];
    const V* gt = GR + static_cast<size_t>(t) * no2 * nk;
    const V* lt = GL + static_cast<size_t>(t) * no2 * nk;
#pragma unroll
    for (int e = 0; e < 25; ++e) {        // no2 <= 25: all loads in flight together
      if (e < no2) {
        g[e * TPB + tid] = gt[static_cast<size_t>(e) * nk + R];
        gl[e * TPB + tid] = lt[static_cast<size_t>(e) * nk + mr];
      }
    }
  }
  __syncthreads();
  if (R >= nk) return;                        // no barriers below
  V* out = Pt + static_cast<size_t>(t) * nout * nk + R;
  int e0 = s_off[0];
  for (int o = 0; o < nout; ++o) {
    const int e1 = s_off[o + 1];
    V acc0 = cmk<V>(0, 0), acc1 = cmk<V>(0, 0);
    int e = e0;
    for (; e + 1 < e1; e += 2) {
      const TermRec<T> r0 = s_rec[e], r1 = s_rec[e + 1];
      acc0 = cfma(r0.c, cmul(g[(r0.idx & 255) * TPB + tid], gl[(r0.idx >> 8) * TPB + tid]), acc0);
      acc1 = cfma(r1.c, cmul(g[(r1.idx & 255) * TPB + tid], gl[(r1.idx >> 8) * TPB + tid]), acc1);
    }
    if (e < e1) {
      const TermRec<T> r0 = s_rec[e];
      acc0 = cfma(r0.c, cmul(g[(r0.idx & 255) * TPB + tid], gl[(r0.idx >> 8) * TPB + tid]), acc0);
    }
    out[static_cast<size_t>(o) * nk] = cadd(acc0, acc1);
    e0 = e1;
  }
}

// W^C entries are read in batches of kWb (independent loads in flight per
// thread) before their terms are applied.
constexpr int kWb = 16;

template <typename T, bool DISTINCT>
__global__ void __launch_bounds__(RedTpb<T>::v) sigma_reduced_kernel(
    const cplx<T>* __restrict__ GR, const cplx<T>* __restrict__ Wt, const int* __restrict__ terms,
    const cplx<T>* __restrict__ coef, int nterm, cplx<T>* __restrict__ Sig, int no2, int nout,
    int nk) {
  using V = cplx<T>;
  constexpr int TPB = RedTpb<T>::v;
  extern __shared__ __align__(32) unsigned char smem_raw[];
  TermRec<T>* s_rec = reinterpret_cast<TermRec<T>*>(smem_raw);
  V* g = reinterpret_cast<V*>(s_rec + nterm);   // [no2][TPB]
  V* sg = g + no2 * TPB;                        // [no2][TPB] accumulators
  int* s_off = reinterpret_cast<int*>(sg + no2 * TPB);
  const int tid = threadIdx.x;
  const int t = blockIdx.y;
  const int R = blockIdx.x * TPB + tid;
  stage_terms<T>(terms, coef, nout, nterm, s_off, s_rec);
  if (R < nk) {
    const V* gt = GR + static_cast<size_t>(t) * no2 * nk;
#pragma unroll
    for (int e = 0; e < 25; ++e) {        // no2 <= 25: all loads in flight together
      if (e < no2) {
        g[e * TPB + tid] = gt[static_cast<size_t>(e) * nk + R];
        sg[e * TPB + tid] = cmk<V>(0, 0);
      }
    }
  }
  __syncthreads();
  if (R >= nk) return;                        // no barriers below
  const V* w = Wt + static_cast<size_t>(t) * nout * nk + R;
  for (int o0 = 0; o0 < nout; o0 += kWb) {
    V wb[kWb];
#pragma unroll
    for (int u = 0; u < kWb; ++u)
      wb[u] = o0 + u < nout ? w[static_cast<size_t>(o0 + u) * nk] : cmk<V>(0, 0);
#pragma unroll
    for (int u = 0; u < kWb; ++u) {
      if (o0 + u < nout) {
        const int e1 = s_off[o0 + u + 1];
        int e = s_off[o0 + u];
        if (DISTINCT) {
          // the terms of one output entry update distinct accumulators: four at a
          // time, all loads before the stores
          for (; e + 4 <= e1; e += 4) {
            TermRec<T> rr[4];
            V* sp[4];
            V acc[4], gv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              rr[q] = s_rec[e + q];
              sp[q] = sg + (rr[q].idx >> 8) * TPB + tid;
              acc[q] = *sp[q];
              gv[q] = g[(rr[q].idx & 255) * TPB + tid];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) *sp[q] = cfma(cmul(rr[q].c, wb[u]), gv[q], acc[q]);
          }
        }
        for (; e < e1; ++e) {
          const TermRec<T> r0 = s_rec[e];
          V* sp = sg + (r0.idx >> 8) * TPB + tid;
          *sp = cfma(cmul(r0.c, wb[u]), g[(r0.idx & 255) * TPB + tid], *sp);
        }
      }
    }
  }
  V* out = Sig + static_cast<size_t>(t) * no2 * nk + R;
  for (int e = 0; e < no2; ++e) out[static_cast<size_t>(e) * nk] = sg[e * TPB + tid];
}

template <typename T>
size_t reduced_smem(int no2, int nout, int nterm) {
  return static_cast<size_t>(nterm) * sizeof(TermRec<T>) +
         static_cast<size_t>(2) * no2 * RedTpb<T>::v * sizeof(cplx<T>) +
         static_cast<size_t>(nout + 1) * sizeof(int);
}

}  // namespace

template <typename T>
cudaError_t launch_bubble_reduced(const void* GR, const void* GreflR, const int* mR,
                                  const int* terms, const void* coef, int nterm, void* Pt, int r,
                                  int norb, int rho, int nk, cudaStream_t st) {
  if (nterm < 0 || nterm > kMaxPairTerms || norb > 5 || rho < 1) return cudaErrorInvalidValue;
  const int no2 = norb * norb, nout = rho * rho;
  const size_t smem = reduced_smem<T>(no2, nout, nterm);
  cudaError_t e = set_smem(reinterpret_cast<const void*>(&bubble_reduced_kernel<T>), smem);
  if (e != cudaSuccess) return e;
  constexpr int TPB = RedTpb<T>::v;
  dim3 grid((nk + TPB - 1) / TPB, r);
  bubble_reduced_kernel<T><<<grid, TPB, smem, st>>>(
      reinterpret_cast<const cplx<T>*>(GR), reinterpret_cast<const cplx<T>*>(GreflR), mR, terms,
      reinterpret_cast<const cplx<T>*>(coef), nterm, reinterpret_cast<cplx<T>*>(Pt), no2, nout, nk);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sigma_reduced(const void* GR, const void* Wt, const int* terms, const void* coef,
                                 int nterm, void* Sig, int r, int norb, int rho, int nk,
                                 cudaStream_t st, int distinct) {
  if (nterm < 0 || nterm > kMaxPairTerms || norb > 5 || rho < 1) return cudaErrorInvalidValue;
  const int no2 = norb * norb, nout = rho * rho;
  const size_t smem = reduced_smem<T>(no2, nout, nterm);
  auto fn = distinct ? &sigma_reduced_kernel<T, true> : &sigma_reduced_kernel<T, false>;
  cudaError_t e = set_smem(reinterpret_cast<const void*>(fn), smem);
  if (e != cudaSuccess) return e;
  constexpr int TPB = RedTpb<T>::v;
  dim3 grid((nk + TPB - 1) / TPB, r);
  fn<<<grid, TPB, smem, st>>>(
      reinterpret_cast<const cplx<T>*>(GR), reinterpret_cast<const cplx<T>*>(Wt), terms,
      reinterpret_cast<const cplx<T>*>(coef), nterm, reinterpret_cast<cplx<T>*>(Sig), no2, nout, nk);
  return cudaGetLastError();
}

template cudaError_t launch_bubble_reduced<double>(const void*, const void*, const int*, const int*,
                                                   const void*, int, void*, int, int, int, int,
                                                   cudaStream_t);
template cudaError_t launch_bubble_reduced<float>(const void*, const void*, const int*, const int*,
                                                  const void*, int, void*, int, int, int, int,
                                                  cudaStream_t);
template cudaError_t launch_sigma_reduced<double>(const void*, const void*, const int*, const void*,
                                                  int, void*, int, int, int, int, cudaStream_t, int);
template cudaError_t launch_sigma_reduced<float>(const void*, const void*, const int*, const void*,
                                                 int, void*, int, int, int, int, cudaStream_t, int);

}  // namespace qa
