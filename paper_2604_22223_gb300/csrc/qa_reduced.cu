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
#include <utility>

#include "qa_common.cuh"

namespace qa {
namespace {

template <typename T> struct RedTpb { static constexpr int v = 256; };
template <> struct RedTpb<double> { static constexpr int v = 64; };
template <> struct RedTpb<dfl> { static constexpr int v = 64; };

// one term as a single shared-memory record (one 16- or 32-byte load)
template <typename T> struct __align__(sizeof(cplx<T>) < 16 ? 16 : 32) TermRec {
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

// ------------------------------------------- Sigma on the canonical basis
// Kanamori-type interactions give the reduced basis a fixed shape: the N
// diagonal pairs (a,a) as unit vectors, then one vector on {(a,b), (b,a)} for
// each a < b in lexicographic order (the components of the pair graph, taken
// in the order of their first pair).  Then the term list of the Sigma
// contraction is a fixed pattern, N^4 terms with the entry of Wt, the source
// G_bc and the target Sigma_ad of each known at compile time; only the
// coefficients -B_(ab)i conj(B_(cd)j) depend on the interaction.  The kernel
// keeps G and the N^2 accumulators in registers, reads each Wt entry once
// (coalesced along R) and takes the coefficients from its parameter space, so
// it moves the tensors' bytes and nothing else.  Its terms run in the order
// of the generic list, so both kernels give the same bits.
template <int N> struct CanonBasis {
  static constexpr int RHO = N + N * (N - 1) / 2;
  static constexpr int NO2 = N * N;
  static constexpr int NT = NO2 * NO2;
  // number of pairs of basis vector i, and of vectors 0 .. i-1
  __host__ __device__ static constexpr int npairs(int i) { return i < N ? 1 : 2; }
  __host__ __device__ static constexpr int before(int i) { return i < N ? i : N + 2 * (i - N); }
  // first term of the output entry (i, j)
  __host__ __device__ static constexpr int first_term(int i, int j) {
    return before(i) * NO2 + npairs(i) * before(j);
  }
  // pair index a * N + b of the k-th pair of basis vector i
  __host__ __device__ static constexpr int pair(int i, int k) {
    if (i < N) return i * N + i;
    int m = i - N, a = 0;
    while (m >= N - 1 - a) { m -= N - 1 - a; ++a; }
    const int b = a + 1 + m;
    return k == 0 ? a * N + b : b * N + a;
  }
};

template <int N> struct CanonCoefs { float2 c[CanonBasis<N>::NT]; };

// one term: pair KA of vector i and pair KB of vector j of the entry O = i * rho + j
template <int N, int O, int KA, int KB>
__device__ __forceinline__ void canon_term(float2 w, const float2 (&g)[N * N], float2 (&acc)[N * N],
                                           const CanonCoefs<N>& cf) {
  using C = CanonBasis<N>;
  constexpr int i = O / C::RHO, j = O % C::RHO;
  if constexpr (KA < C::npairs(i) && KB < C::npairs(j)) {
    constexpr int A = C::pair(i, KA), B = C::pair(j, KB);
    constexpr int tgt = (A / N) * N + B % N;     // Sigma_ad with (ab) = A, (cd) = B
    constexpr int src = (A % N) * N + B / N;     // G_bc
    constexpr int e = C::first_term(i, j) + KA * C::npairs(j) + KB;
    acc[tgt] = cfma(cmul(cf.c[e], w), g[src], acc[tgt]);
  }
}

template <int N, int O>
__device__ __forceinline__ void canon_entry(const float2* __restrict__ w, int nk, const float2 (&g)[N * N],
                                            float2 (&acc)[N * N], const CanonCoefs<N>& cf) {
  const float2 wv = __ldg(w + static_cast<size_t>(O) * nk);
  canon_term<N, O, 0, 0>(wv, g, acc, cf);
  canon_term<N, O, 0, 1>(wv, g, acc, cf);
  canon_term<N, O, 1, 0>(wv, g, acc, cf);
  canon_term<N, O, 1, 1>(wv, g, acc, cf);
}

template <int N, int... Os>
__device__ __forceinline__ void canon_entries(const float2* __restrict__ w, int nk, const float2 (&g)[N * N],
                                              float2 (&acc)[N * N], const CanonCoefs<N>& cf,
                                              std::integer_sequence<int, Os...>) {
  (canon_entry<N, Os>(w, nk, g, acc, cf), ...);
}

// 64 threads per block, one R each; 168 registers (N = 5) leave 12 warps per SM
constexpr int kCanonTpb = 64;

template <int N>
__global__ void __launch_bounds__(kCanonTpb, 6) sigma_canonical_kernel(
    const float2* __restrict__ GR, const float2* __restrict__ Wt, const __grid_constant__ CanonCoefs<N> cf,
    float2* __restrict__ Sig, int nk) {
  using C = CanonBasis<N>;
  const int t = blockIdx.y, R = blockIdx.x * kCanonTpb + threadIdx.x;
  if (R >= nk) return;
  float2 g[C::NO2], acc[C::NO2];
  const float2* gt = GR + static_cast<size_t>(t) * C::NO2 * nk + R;
#pragma unroll
  for (int e = 0; e < C::NO2; ++e) {
    g[e] = __ldg(gt + static_cast<size_t>(e) * nk);
    acc[e] = make_float2(0.f, 0.f);
  }
  const float2* w = Wt + static_cast<size_t>(t) * C::RHO * C::RHO * nk + R;
  canon_entries<N>(w, nk, g, acc, cf, std::make_integer_sequence<int, C::RHO * C::RHO>{});
  float2* out = Sig + static_cast<size_t>(t) * C::NO2 * nk + R;
#pragma unroll
  for (int e = 0; e < C::NO2; ++e) out[static_cast<size_t>(e) * nk] = acc[e];
}

template <int N>
bool canon_matches(const int* off, const int* idx, int nout, int nterm) {
  using C = CanonBasis<N>;
  if (nout != C::RHO * C::RHO || nterm != C::NT || off[0] != 0) return false;
  for (int i = 0; i < C::RHO; ++i)
    for (int j = 0; j < C::RHO; ++j) {
      const int o = i * C::RHO + j, e0 = C::first_term(i, j);
      if (off[o] != e0 || off[o + 1] != e0 + C::npairs(i) * C::npairs(j)) return false;
      for (int ka = 0; ka < C::npairs(i); ++ka)
        for (int kb = 0; kb < C::npairs(j); ++kb) {
          const int A = C::pair(i, ka), B = C::pair(j, kb);
          const int want = ((A % N) * N + B / N) | (((A / N) * N + B % N) << 8);
          if (idx[e0 + ka * C::npairs(j) + kb] != want) return false;
        }
    }
  return true;
}

template <int N>
cudaError_t launch_canon(const void* GR, const void* Wt, const std::complex<double>* coef, void* Sig,
                         int r, int nk, cudaStream_t st) {
  CanonCoefs<N> cf;
  for (int e = 0; e < CanonBasis<N>::NT; ++e)
    cf.c[e] = make_float2(static_cast<float>(coef[e].real()), static_cast<float>(coef[e].imag()));
  dim3 grid((nk + kCanonTpb - 1) / kCanonTpb, r);
  sigma_canonical_kernel<N><<<grid, kCanonTpb, 0, st>>>(reinterpret_cast<const float2*>(GR),
                                                        reinterpret_cast<const float2*>(Wt), cf,
                                                        reinterpret_cast<float2*>(Sig), nk);
  return cudaGetLastError();
}

}  // namespace

int sigma_canonical_norb(const int* off, const int* idx, int nout, int nterm, int norb) {
  switch (norb) {
    case 2: return canon_matches<2>(off, idx, nout, nterm) ? 2 : 0;
    case 3: return canon_matches<3>(off, idx, nout, nterm) ? 3 : 0;
    case 4: return canon_matches<4>(off, idx, nout, nterm) ? 4 : 0;
    case 5: return canon_matches<5>(off, idx, nout, nterm) ? 5 : 0;
    default: return 0;
  }
}

cudaError_t launch_sigma_canonical(const void* GR, const void* Wt, const std::complex<double>* coef,
                                   int norb, void* Sig, int r, int nk, cudaStream_t st) {
  if (r < 1 || nk < 1 || r > 65535) return cudaErrorInvalidValue;
  switch (norb) {
    case 2: return launch_canon<2>(GR, Wt, coef, Sig, r, nk, st);
    case 3: return launch_canon<3>(GR, Wt, coef, Sig, r, nk, st);
    case 4: return launch_canon<4>(GR, Wt, coef, Sig, r, nk, st);
    case 5: return launch_canon<5>(GR, Wt, coef, Sig, r, nk, st);
    default: return cudaErrorInvalidValue;
  }
}

// ---- Sigma in double-float (accurate mixed path), any pair basis.
// One thread per (R, target entry Sigma_ad) walks the target's terms
// Sigma_ad += coef * Wt_o(R) * G_g(R) from a per-target list (the sigma term
// lists regrouped by target on the host); the block is 32 consecutive R x all
// targets, so each load is a coalesced run along R and the Wt entries shared by
// several targets of one R are re-read from L1.  The sum is compensated: every
// leading FP32 product split exactly by an FMA, the high parts added with
// TwoSum.  A short loop instead of an unrolled term pattern keeps the code in
// the instruction cache.
constexpr int kSigDfR = 16;

__device__ __forceinline__ void df_acc_prod(float& s, float& e, dfl u, dfl v) {
  const float p = __fmul_rn(u.hi, v.hi);
  float q = __fmaf_rn(u.hi, v.hi, -p);
  q = __fmaf_rn(u.hi, v.lo, q);
  q = __fmaf_rn(u.lo, v.hi, q);
  float t;
  two_sum(s, p, s, t);
  e = __fadd_rn(e, __fadd_rn(t, q));
}

// RC: every term coefficient is real (a real pair basis), so c Wt takes two
// double-float products instead of a complex one.
template <bool RC>
__global__ void __launch_bounds__(kSigDfR * 25) sigma_target_df_kernel(
    const dfc* __restrict__ GR, const dfc* __restrict__ Wt, const int* __restrict__ toff,
    const int2* __restrict__ tidx, const dfc* __restrict__ tcoef, dfc* __restrict__ Sig, int no2,
    int nout, int nk, int* err) {
  const int R = blockIdx.x * kSigDfR + threadIdx.x;
  const int tg = threadIdx.y;                 // target entry a * norb + d
  const int t = blockIdx.y;
  if (R >= nk || tg >= no2) return;
  const dfc* g = GR + static_cast<size_t>(t) * no2 * nk + R;
  const dfc* w = Wt + static_cast<size_t>(t) * nout * nk + R;
  float rs = 0.f, re = 0.f, is = 0.f, ie = 0.f;
  const int e1 = toff[tg + 1];
  for (int e = toff[tg]; e < e1; ++e) {
    const int2 ix = __ldg(tidx + e);          // (Wt entry, G entry)
    const dfc cf = ldg_c(tcoef + e), wv = ldg_c(w + static_cast<size_t>(qa_index(ix.x, nout, err)) * nk);
    const dfc cw = RC ? dfc{cf.x * wv.x, cf.x * wv.y} : cmul(cf, wv);
    const dfc gv = ldg_c(g + static_cast<size_t>(qa_index(ix.y, no2, err)) * nk);
    df_acc_prod(rs, re, cw.x, gv.x);
    df_acc_prod(rs, re, -cw.y, gv.y);
    df_acc_prod(is, ie, cw.x, gv.y);
    df_acc_prod(is, ie, cw.y, gv.x);
  }
  const dfl vr = df_norm(rs, re), vi = df_norm(is, ie);
  reinterpret_cast<float4*>(Sig)[(static_cast<size_t>(t) * no2 + tg) * nk + R] =
      make_float4(vr.hi, vr.lo, vi.hi, vi.lo);
}

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
template cudaError_t launch_bubble_reduced<dfl>(const void*, const void*, const int*, const int*,
                                                const void*, int, void*, int, int, int, int,
                                                cudaStream_t);
template cudaError_t launch_sigma_reduced<dfl>(const void*, const void*, const int*, const void*,
                                               int, void*, int, int, int, int, cudaStream_t, int);

cudaError_t launch_sigma_target_df(const void* GR, const void* Wt, const int* toff, const void* tidx,
                                   const void* tcoef, void* Sig, int r, int norb, int nout, int nk,
                                   cudaStream_t st, int* err, bool real_coef) {
  const int no2 = norb * norb;
  if (no2 > 25 || r < 1 || r > 65535) return cudaErrorInvalidValue;
  dim3 block(kSigDfR, no2), grid((nk + kSigDfR - 1) / kSigDfR, r);
  auto fn = real_coef ? &sigma_target_df_kernel<true> : &sigma_target_df_kernel<false>;
  fn<<<grid, block, 0, st>>>(static_cast<const dfc*>(GR), static_cast<const dfc*>(Wt),
                                                 toff, static_cast<const int2*>(tidx),
                                                 static_cast<const dfc*>(tcoef), static_cast<dfc*>(Sig),
                                                 no2, nout, nk, err);
  return cudaGetLastError();
}

}  // namespace qa
