// Batched Dyson solves.
//
// Screened interaction (paper Eq. for W): W = V + V P W per (q, i nu_m) in the
// pair basis, so (1 - V P) W = V and W^C = W - V.  One warp owns one
// npair x npair system: the matrices sit in shared memory, lane i owns row i
// during the elimination, the pivot is chosen with warp shuffles (largest
// |a_ic|, ties to the lowest row), and lane j owns column j of the
// right-hand side during back substitution.  The FP32 variant solves for
// W^C directly with the right-hand side V P V, which avoids the cancellation
// of W - V when the screening is weak.
//
// Green's function (paper Eq. for the full Green's function):
// G(k, i w_n) = (i w_n + mu - H(k) - Sigma^HF(k) - Sigma^C(k, i w_n))^-1 per
// (n, k), one thread per system, Gauss-Jordan with partial pivoting in
// registers, from a per-step table of the mu-independent part.  The density
// N(mu) = (s/N_k) sum_{k,n} Re(dw_n Tr G) and its derivative
// -(s/N_k) sum Re(dw_n Tr G^2) are accumulated in FP64.
#include <type_traits>

#include "qa_common.cuh"

namespace qa {
namespace {

constexpr int kMaxPair = 25;
constexpr int kWarpsW = 4;

template <typename T> struct Tiny;
template <> struct Tiny<double> { static constexpr double v = 1e-26; };   // |pivot|^2
template <> struct Tiny<float> { static constexpr float v = 1e-12f; };
template <> struct Tiny<dfl> { static constexpr double v = 1e-26; };

__device__ void report(int* err, long long* first_bad, int code, long long idx) {
  atomicCAS(err, 0, code);
  if (first_bad) atomicMin(reinterpret_cast<unsigned long long*>(first_bad),
                           static_cast<unsigned long long>(idx));
}

template <typename T, bool VPV>
__global__ void __launch_bounds__(kWarpsW * 32) dyson_w_kernel(const cplx<T>* __restrict__ P,
                                                               const cplx<T>* __restrict__ Vq,
                                                               cplx<T>* WC, int n, int nk,
                                                               int* err, long long* first_bad,
                                                               cplx<T>* lu, unsigned char* piv) {
  using V = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int q = blockIdx.x * kWarpsW + w;
  const int nu = blockIdx.y;
  if (q >= nk) return;                  // whole warp leaves; no block barriers below
  const int ld = n + 1;
  V* A = reinterpret_cast<V*>(smem_raw) + static_cast<size_t>(w) * 2 * n * ld;
  V* Bm = A + n * ld;
  const size_t nn = static_cast<size_t>(n) * n;
  const V* Pq = P + static_cast<size_t>(nu) * nn * nk + q;
  const V* Vqq = Vq + static_cast<size_t>(q) * nn;
  for (int e = lane; e < n * n; e += 32) {
    int i = e / n, j = e - i * n;
    A[i * ld + j] = Pq[static_cast<size_t>(e) * nk];
    Bm[i * ld + j] = Vqq[e];
  }
  __syncwarp();
  // row `lane` of V P (and of V P V)
  V vp[kMaxPair];
  V rhs[VPV ? kMaxPair : 1];
  if (lane < n) {
#pragma unroll
    for (int j = 0; j < kMaxPair; ++j) {
      if (j < n) {
        V acc = cmk<V>(0, 0);
        for (int m = 0; m < n; ++m) acc = cfma(Bm[lane * ld + m], A[m * ld + j], acc);
        vp[j] = acc;
      }
    }
    if (VPV) {
#pragma unroll
      for (int j = 0; j < kMaxPair; ++j) {
        if (j < n) {
          V acc = cmk<V>(0, 0);
#pragma unroll
          for (int m = 0; m < kMaxPair; ++m)
            if (m < n) acc = cfma(vp[m], Bm[m * ld + j], acc);
          rhs[VPV ? j : 0] = acc;
        }
      }
    }
  }
  __syncwarp();
  if (lane < n) {
#pragma unroll
    for (int j = 0; j < kMaxPair; ++j) {
      if (j < n) {
        V a = cmk<V>(j == lane ? 1.0 : 0.0, 0.0);
        A[lane * ld + j] = csub(a, vp[j]);
        if (VPV) Bm[lane * ld + j] = rhs[VPV ? j : 0];
      }
    }
  }
  __syncwarp();
  bool singular = false;
  for (int c = 0; c < n; ++c) {
    T val = (lane >= c && lane < n) ? cabs2(A[lane * ld + c]) : static_cast<T>(-1);
    int idx = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      T ov = __shfl_xor_sync(0xffffffffu, val, o);
      int oi = __shfl_xor_sync(0xffffffffu, idx, o);
      if (ov > val || (ov == val && oi < idx)) { val = ov; idx = oi; }
    }
    const int p = idx;
    if (val < Tiny<T>::v || !(val == val)) singular = true;
    if (lu && lane == 0) piv[(static_cast<size_t>(nu) * n + c) * nk + q] = static_cast<unsigned char>(p);
    if (p != c && lane < n) {
      // whole rows when the factors are kept (columns < c then hold multipliers)
      if (lane >= c || lu) {
        V tmp = A[c * ld + lane]; A[c * ld + lane] = A[p * ld + lane]; A[p * ld + lane] = tmp;
      }
      V tmp = Bm[c * ld + lane]; Bm[c * ld + lane] = Bm[p * ld + lane]; Bm[p * ld + lane] = tmp;
    }
    __syncwarp();
    if (lane > c && lane < n) {
      V l = cmul(A[lane * ld + c], cinv(A[c * ld + c]));
      if (lu) A[lane * ld + c] = l;
      for (int j = c + 1; j < n; ++j) A[lane * ld + j] = cfms(l, A[c * ld + j], A[lane * ld + j]);
      for (int j = 0; j < n; ++j) Bm[lane * ld + j] = cfms(l, Bm[c * ld + j], Bm[lane * ld + j]);
    }
    __syncwarp();
  }
  if (lane < n) {
    for (int c = n - 1; c >= 0; --c) {
      V x = Bm[c * ld + lane];
      for (int m = c + 1; m < n; ++m) x = cfms(A[c * ld + m], Bm[m * ld + lane], x);
      Bm[c * ld + lane] = cmul(x, cinv(A[c * ld + c]));
    }
  }
  __syncwarp();
  V* out = WC + static_cast<size_t>(nu) * nn * nk + q;
  for (int e = lane; e < n * n; e += 32) {
    int i = e / n, j = e - i * n;
    V x = Bm[i * ld + j];
    if (!VPV) x = csub(x, Vqq[e]);
    out[static_cast<size_t>(e) * nk] = x;
    if (lu) lu[(static_cast<size_t>(nu) * nn + e) * nk + q] = A[i * ld + j];
  }
  if (singular && lane == 0) report(err, first_bad, QA_ESINGULAR_CODE, static_cast<long long>(nu) * nk + q);
}

// ------------------------------------------------- Dyson W, register rows
// FP32 variant with the rows in registers.  W lanes (W = next power of two
// >= n) own one system, so a warp solves 32/W systems side by side, and a
// block of 8 warps takes 8*32/W consecutive q at one nu: the P / W^C tiles
// move through shared memory with coalesced runs along q.  Lane i of a
// system owns row i of A = 1 - V P and of the right-hand side V P V;
// elimination tracks the pivot lanes instead of swapping rows (the pivot row
// is broadcast with width-W warp shuffles), and the triangular solve runs
// column-parallel from shared memory.

constexpr int kWarpsR = 8;

template <int MAXN, int W>
__global__ void __launch_bounds__(kWarpsR * 32) dyson_w_reg_kernel(const float2* __restrict__ P,
                                                                  const float2* __restrict__ Vq,
                                                                  float2* WC, int n, int nk,
                                                                  int* err, long long* first_bad) {
  static_assert(MAXN <= W && W <= 32 && (W & (W - 1)) == 0, "system width");
  constexpr int SPW = 32 / W;                 // systems per warp
  constexpr int NSYS = kWarpsR * SPW;         // systems per block
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nn = n * n;
  float2* Ps = reinterpret_cast<float2*>(smem_raw);        // [NSYS][nn]
  float2* Vs = Ps + NSYS * nn;                              // [NSYS][nn]
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int l = lane % W;                                   // row owned in the system
  const int sys = w * SPW + lane / W;                       // system within the block
  const int q0 = blockIdx.x * NSYS;
  const int nu = blockIdx.y;
  const size_t slab = static_cast<size_t>(nu) * nn * nk;
  // batches of 8 loads per thread in flight (the trip count depends on n)
  for (int idx0 = tid; idx0 < NSYS * nn; idx0 += 8 * kWarpsR * 32) {
    float2 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = idx0 + u * kWarpsR * 32;
      const int e = idx / NSYS, ss = idx - e * NSYS;
      const int q = q0 + ss;
      v[u] = (idx < NSYS * nn && q < nk) ? P[slab + static_cast<size_t>(e) * nk + q] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = idx0 + u * kWarpsR * 32;
      const int e = idx / NSYS, ss = idx - e * NSYS;
      if (idx < NSYS * nn) Ps[ss * nn + e] = v[u];
    }
  }
  for (int idx0 = tid; idx0 < NSYS * nn; idx0 += 8 * kWarpsR * 32) {
    float2 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = idx0 + u * kWarpsR * 32;
      const int ss = idx / nn;
      const int q = q0 + ss;
      v[u] = (idx < NSYS * nn && q < nk) ? Vq[static_cast<size_t>(q0) * nn + idx] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = idx0 + u * kWarpsR * 32;
      if (idx < NSYS * nn) Vs[idx] = v[u];
    }
  }
  __syncthreads();
  const int q = q0 + sys;
  float2* Pw = Ps + sys * nn;
  float2* Vw = Vs + sys * nn;
  float2 a[MAXN], b[MAXN];
  const bool row = l < n;
  // a = row l of V P
#pragma unroll
  for (int j = 0; j < MAXN; ++j) a[j] = make_float2(0.f, 0.f);
  if (row) {
    for (int m = 0; m < n; ++m) {
      float2 v = Vw[l * n + m];
#pragma unroll
      for (int j = 0; j < MAXN; ++j)
        if (j < n) a[j] = cfma(v, Pw[m * n + j], a[j]);
    }
  }
  // b = row l of (V P) V
#pragma unroll
  for (int j = 0; j < MAXN; ++j) b[j] = make_float2(0.f, 0.f);
  if (row) {
#pragma unroll
    for (int m = 0; m < MAXN; ++m) {
      if (m < n) {
#pragma unroll
        for (int j = 0; j < MAXN; ++j)
          if (j < n) b[j] = cfma(a[m], Vw[m * n + j], b[j]);
      }
    }
  }
  // a = 1 - V P
#pragma unroll
  for (int j = 0; j < MAXN; ++j) {
    a[j].x = (row && j == l ? 1.f : 0.f) - a[j].x;
    a[j].y = -a[j].y;
  }
  bool used = !row;
  int mypos = -1;
  bool singular = false;
#pragma unroll
  for (int c = 0; c < MAXN; ++c) {
    if (c < n) {
      float val = used ? -1.f : cabs2(a[c]);
      int idx = l;
#pragma unroll
      for (int o = W / 2; o > 0; o >>= 1) {
        float ov = __shfl_xor_sync(0xffffffffu, val, o);
        int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ov > val || (ov == val && oi < idx)) { val = ov; idx = oi; }
      }
      const int p = idx;                      // pivot row within the system
      if (!(val >= 1e-12f)) singular = true;
      if (l == p) { used = true; mypos = c; }
      float2 apc = make_float2(__shfl_sync(0xffffffffu, a[c].x, p, W),
                               __shfl_sync(0xffffffffu, a[c].y, p, W));
      float2 f = used ? make_float2(0.f, 0.f) : cmul(a[c], cinv(apc));
      // Up to 16 rows, a fixed range with a predicate (not j = c + 1 ..) keeps
      // a[] in registers.  The 25-row systems keep the shorter loop: their
      // register-resident form needs 162 registers (one block per SM) and
      // measured slower than the variant that holds a[] in local memory.
#pragma unroll
      for (int j = (W < 32 ? 1 : c + 1); j < MAXN; ++j) {
        if ((W == 32 || j > c) && j < n) {
          float2 apj = make_float2(__shfl_sync(0xffffffffu, a[j].x, p, W),
                                   __shfl_sync(0xffffffffu, a[j].y, p, W));
          a[j] = cfms(f, apj, a[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < MAXN; ++j) {
        if (j < n) {
          float2 bpj = make_float2(__shfl_sync(0xffffffffu, b[j].x, p, W),
                                   __shfl_sync(0xffffffffu, b[j].y, p, W));
          b[j] = cfms(f, bpj, b[j]);
        }
      }
    }
  }
  // rows of the triangular factor to shared memory, in pivot order
  __syncwarp();
  if (mypos >= 0) {
#pragma unroll
    for (int j = 0; j < MAXN; ++j)
      if (j < n) { Pw[mypos * n + j] = a[j]; Vw[mypos * n + j] = b[j]; }
  }
  __syncwarp();
  if (row) {
    for (int c = n - 1; c >= 0; --c) {
      float2 x = Vw[c * n + l];
      for (int m = c + 1; m < n; ++m) x = cfms(Pw[c * n + m], Vw[m * n + l], x);
      Vw[c * n + l] = cmul(x, cinv(Pw[c * n + c]));
    }
  }
  if (singular && l == 0 && q < nk)
    report(err, first_bad, QA_ESINGULAR_CODE, static_cast<long long>(nu) * nk + q);
  __syncthreads();
  for (int idx = tid; idx < NSYS * nn; idx += blockDim.x) {
    int e = idx / NSYS, ss = idx - e * NSYS;
    int qq = q0 + ss;
    if (qq < nk) WC[slab + static_cast<size_t>(e) * nk + qq] = Vs[ss * nn + e];
  }
}

template <int MAXN, int W>
cudaError_t launch_dyson_w_reg(const void* P, const void* Vq, void* WC, int r, int n, int nk,
                               int* err, long long* first_bad, cudaStream_t st) {
  constexpr int NSYS = kWarpsR * (32 / W);
  const size_t smem = static_cast<size_t>(2) * NSYS * n * n * sizeof(float2);
  auto fn = &dyson_w_reg_kernel<MAXN, W>;
  cudaError_t e = set_smem(reinterpret_cast<const void*>(fn), smem);
  if (e != cudaSuccess) return e;
  dim3 grid((nk + NSYS - 1) / NSYS, r);
  fn<<<grid, kWarpsR * 32, smem, st>>>(reinterpret_cast<const float2*>(P),
                                       reinterpret_cast<const float2*>(Vq),
                                       reinterpret_cast<float2*>(WC), n, nk, err, first_bad);
  return cudaGetLastError();
}

// ------------------------------------------- Dyson W, swizzled tiles
// FP32 kernel for systems of n <= 16 (the reduced pair basis): MAXN lanes
// own one system (lane i = row i of A = 1 - V P and of the right-hand side
// V P V), 32/MAXN systems per warp, 8 warps per block over consecutive q.
// P and V sit in shared memory as MAXN x MAXN tiles whose rows hold pairs of
// complex values, the pair index XOR-swizzled by the row: a lane reading its
// own row and all lanes reading one row (a broadcast) both move 16 bytes per
// load without bank conflicts.  The pivot of each column is found with a
// packed (|a|^2 | row) key, and the pivot row reaches the other lanes
// through shared memory (one 16-byte store and load per two values instead
// of two shuffles per value).  Gauss-Jordan elimination leaves each lane with
// one row of the solution (no back-substitution phase).

template <int MAXN>
__device__ __forceinline__ int swz(int row, int col) {
  return row * MAXN + 2 * ((col >> 1) ^ (row & (MAXN / 2 - 1))) + (col & 1);
}

template <int MAXN>
__device__ __forceinline__ float4 lds_pair(const float2* tile, int row, int pair) {
  return *reinterpret_cast<const float4*>(tile + row * MAXN + 2 * (pair ^ (row & (MAXN / 2 - 1))));
}

// NFIX > 0: the system size is the compile-time constant NFIX (n is ignored), so
// every size test below folds away; NFIX = 0: runtime n <= MAXN.
// BLK: V(q) is block diagonal (blk.lo / blk.hi per index); the products V P and
// V P V skip its zero blocks (the skipped terms are exact zeros).
template <int MAXN, int NFIX, bool BLK>
__global__ void __launch_bounds__(kWarpsR * 32, NFIX > 0 ? 2 : 3) dyson_w_tile_kernel(const float2* __restrict__ P,
                                                                   const float2* __restrict__ Vq,
                                                                   float2* WC, int n_arg, int nk,
                                                                   int* err, long long* first_bad,
                                                                   DysonBlocks blk) {
  const int n = NFIX > 0 ? NFIX : n_arg;
  static_assert(MAXN == 4 || MAXN == 8 || MAXN == 16, "tile width");
  constexpr int W = MAXN;                      // lanes per system
  constexpr int SPW = 32 / W;
  constexpr int NSYS = kWarpsR * SPW;
  constexpr int TT = MAXN * MAXN;              // tile entries
  constexpr int TS = TT + 2;                   // tile stride: 16 bytes of padding per system
                                               // spread the per-q loads and stores over the banks
  constexpr int NPAIR = MAXN / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* Ps = reinterpret_cast<float2*>(smem_raw);        // [NSYS][TS]
  float2* Vs = Ps + NSYS * TS;                              // [NSYS][TS]
  float2* Rs = Vs + NSYS * TS;                              // [NSYS][2][2 * MAXN] pivot rows
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int l = lane & (W - 1);
  const int sys = w * SPW + lane / W;
  const int q0 = blockIdx.x * NSYS;
  const int nu = blockIdx.y;
  const int nn = n * n;
  const size_t slab = static_cast<size_t>(nu) * nn * nk;
  // tile loads: compile-time trip counts, so all of a thread's loads are in
  // flight together (NSYS * TT is a multiple of the block size)
  constexpr int kThr = kWarpsR * 32, kIt = NSYS * TT / kThr;
  static_assert(NSYS * TT % kThr == 0, "tile / block size");
  {
    float2 v[kIt];
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
      const int idx = tid + it * kThr;
      const int pos = idx / NSYS, ss = idx - pos * NSYS;
      const int row = pos / MAXN, col = pos - row * MAXN;
      const int q = q0 + ss;
      v[it] = (row < n && col < n && q < nk) ? P[slab + static_cast<size_t>(row * n + col) * nk + q]
                                             : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
      const int idx = tid + it * kThr;
      const int pos = idx / NSYS, ss = idx - pos * NSYS;
      Ps[ss * TS + swz<MAXN>(pos / MAXN, pos % MAXN)] = v[it];
    }
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
      const int idx = tid + it * kThr;
      const int ss = idx / TT, pos = idx - ss * TT;
      const int row = pos / MAXN, col = pos - row * MAXN;
      const int q = q0 + ss;
      v[it] = (row < n && col < n && q < nk) ? Vq[static_cast<size_t>(q) * nn + row * n + col]
                                             : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
      const int idx = tid + it * kThr;
      const int ss = idx / TT, pos = idx - ss * TT;
      Vs[ss * TS + swz<MAXN>(pos / MAXN, pos % MAXN)] = v[it];
    }
  }
  __syncthreads();
  const int q = q0 + sys;
  float2* Pw = Ps + sys * TS;
  float2* Vw = Vs + sys * TS;
  float2* Ra = Rs + sys * 4 * MAXN;             // two buffers: pivot row of A, then of B
  float2 a[MAXN], b[MAXN];
  const bool row = l < n;
  // a = row l of V P (padding rows and columns of the tiles are zero)
#pragma unroll
  for (int j = 0; j < MAXN; ++j) a[j] = make_float2(0.f, 0.f);
  if (BLK) {
    // row l of V is non-zero only on its block [lo, hi)
    const int lo = row ? blk.lo[l] : 0, hi = row ? blk.hi[l] : 0;
    for (int m = lo; m < hi; ++m) {
      const float2 vlm = Vw[swz<MAXN>(l, m)];
#pragma unroll
      for (int jp = 0; jp < NPAIR; ++jp) {
        if (2 * jp < n) {
          const float4 p0 = lds_pair<MAXN>(Pw, m, jp);
          a[2 * jp] = cfma(vlm, make_float2(p0.x, p0.y), a[2 * jp]);
          a[2 * jp + 1] = cfma(vlm, make_float2(p0.z, p0.w), a[2 * jp + 1]);
        }
      }
    }
  } else {
#pragma unroll
    for (int mp = 0; mp < NPAIR; ++mp) {
      if (2 * mp < n) {
        const float4 vv = lds_pair<MAXN>(Vw, l, mp);
        const float2 v0 = make_float2(vv.x, vv.y), v1 = make_float2(vv.z, vv.w);
#pragma unroll
        for (int jp = 0; jp < NPAIR; ++jp) {
          if (2 * jp < n) {
            const float4 p0 = lds_pair<MAXN>(Pw, 2 * mp, jp);
            const float4 p1 = lds_pair<MAXN>(Pw, 2 * mp + 1, jp);
            a[2 * jp] = cfma(v0, make_float2(p0.x, p0.y), a[2 * jp]);
            a[2 * jp] = cfma(v1, make_float2(p1.x, p1.y), a[2 * jp]);
            a[2 * jp + 1] = cfma(v0, make_float2(p0.z, p0.w), a[2 * jp + 1]);
            a[2 * jp + 1] = cfma(v1, make_float2(p1.z, p1.w), a[2 * jp + 1]);
          }
        }
      }
    }
  }
  // b = row l of (V P) V
#pragma unroll
  for (int j = 0; j < MAXN; ++j) b[j] = make_float2(0.f, 0.f);
#pragma unroll
  for (int m = 0; m < MAXN; ++m) {
    if (m < n) {
      const int mlo = BLK ? blk.lo[m] : 0, mhi = BLK ? blk.hi[m] : MAXN;
#pragma unroll
      for (int jp = 0; jp < NPAIR; ++jp) {
        // (uniform test: the columns 2 jp, 2 jp + 1 meet row m's block)
        if (2 * jp < n && 2 * jp + 1 >= mlo && 2 * jp < mhi) {
          const float4 vr = lds_pair<MAXN>(Vw, m, jp);
          b[2 * jp] = cfma(a[m], make_float2(vr.x, vr.y), b[2 * jp]);
          b[2 * jp + 1] = cfma(a[m], make_float2(vr.z, vr.w), b[2 * jp + 1]);
        }
      }
    }
  }
  // a = 1 - V P
#pragma unroll
  for (int j = 0; j < MAXN; ++j) {
    a[j].x = (row && j == l ? 1.f : 0.f) - a[j].x;
    a[j].y = -a[j].y;
  }
  // Gauss-Jordan elimination of [A | B] with partial pivoting: at column c the
  // pivot row (largest |a_ic| among the rows not yet used) reaches the other
  // lanes through shared memory and every other row, used or not, eliminates
  // column c.  A ends diagonal in pivot order, so the lane that pivoted column
  // c holds row c of the solution as b / a_c: no back substitution.  The pivot
  // rows alternate between two buffers, one warp barrier per column.
  bool used = !row;
  int mypos = -1;
  float2 dval = make_float2(1.f, 0.f);
  bool singular = false;
#pragma unroll
  for (int c = 0; c < MAXN; ++c) {
    if (c < n) {
      float2* Ra_c = Ra + (c & 1) * 2 * MAXN;
      float2* Rb_c = Ra_c + MAXN;
      // pivot: largest |a_ic|^2 over the unused rows, near-ties (low 4 mantissa
      // bits) to the lowest row; used rows carry key 0
      const float v2 = cabs2(a[c]);
      unsigned key = used ? 0u : (max(__float_as_uint(v2) & ~0xFu, 0x10u) | (W - 1 - l));
#pragma unroll
      for (int o = W / 2; o > 0; o >>= 1) key = max(key, __shfl_xor_sync(0xffffffffu, key, o));
      const int p = W - 1 - static_cast<int>(key & (W - 1));
      if (!(__uint_as_float(key & ~0xFu) >= 1e-12f)) singular = true;
      const bool me = (l == p);
      if (me) {
        used = true;
        mypos = c;
        dval = a[c];
#pragma unroll
        for (int jp = c / 2; jp < NPAIR; ++jp)
          *reinterpret_cast<float4*>(Ra_c + 2 * jp) = make_float4(a[2 * jp].x, a[2 * jp].y, a[2 * jp + 1].x, a[2 * jp + 1].y);
#pragma unroll
        for (int jp = 0; jp < NPAIR; ++jp)
          *reinterpret_cast<float4*>(Rb_c + 2 * jp) = make_float4(b[2 * jp].x, b[2 * jp].y, b[2 * jp + 1].x, b[2 * jp + 1].y);
      }
      __syncwarp();
      const float2 apc = Ra_c[c];
      const float2 f = me ? make_float2(0.f, 0.f) : cmul(a[c], cinv(apc));
#pragma unroll
      for (int jp = (c + 1) / 2; jp < NPAIR; ++jp) {
        if (2 * jp < n) {
          const float4 pr = *reinterpret_cast<const float4*>(Ra_c + 2 * jp);
          if (2 * jp > c) a[2 * jp] = cfms(f, make_float2(pr.x, pr.y), a[2 * jp]);
          a[2 * jp + 1] = cfms(f, make_float2(pr.z, pr.w), a[2 * jp + 1]);
        }
      }
#pragma unroll
      for (int jp = 0; jp < NPAIR; ++jp) {
        if (2 * jp < n) {
          const float4 br = *reinterpret_cast<const float4*>(Rb_c + 2 * jp);
          b[2 * jp] = cfms(f, make_float2(br.x, br.y), b[2 * jp]);
          b[2 * jp + 1] = cfms(f, make_float2(br.z, br.w), b[2 * jp + 1]);
        }
      }
    }
  }
  // row `mypos` of the solution into the V tile (rows of other systems untouched)
  if (mypos >= 0) {
    const float2 inv = cinv(dval);
#pragma unroll
    for (int jp = 0; jp < NPAIR; ++jp) {
      const float2 x0 = cmul(b[2 * jp], inv), x1 = cmul(b[2 * jp + 1], inv);
      *reinterpret_cast<float4*>(Vw + mypos * MAXN + 2 * (jp ^ (mypos & (NPAIR - 1)))) =
          make_float4(x0.x, x0.y, x1.x, x1.y);
    }
  }
  if (singular && l == 0 && q < nk)
    report(err, first_bad, QA_ESINGULAR_CODE, static_cast<long long>(nu) * nk + q);
  __syncthreads();
  for (int idx = tid; idx < NSYS * nn; idx += blockDim.x) {
    const int e = idx / NSYS, ss = idx - e * NSYS;
    const int rr = e / n, cc = e - rr * n;
    const int qq = q0 + ss;
    if (qq < nk) WC[slab + static_cast<size_t>(e) * nk + qq] = Vs[ss * TS + swz<MAXN>(rr, cc)];
  }
}

template <int MAXN, int NFIX = 0>
cudaError_t launch_dyson_w_tile(const void* P, const void* Vq, void* WC, int r, int n, int nk,
                                int* err, long long* first_bad, cudaStream_t st,
                                const DysonBlocks* blk) {
  constexpr int NSYS = kWarpsR * (32 / MAXN);
  const size_t smem = (static_cast<size_t>(2) * NSYS * (MAXN * MAXN + 2) + NSYS * 4 * MAXN) * sizeof(float2);
  const bool use_blk = blk && blk->nblk > 1;
  auto fn = use_blk ? &dyson_w_tile_kernel<MAXN, NFIX, true> : &dyson_w_tile_kernel<MAXN, NFIX, false>;
  cudaError_t e = set_smem(reinterpret_cast<const void*>(fn), smem);
  if (e != cudaSuccess) return e;
  dim3 grid((nk + NSYS - 1) / NSYS, r);
  fn<<<grid, kWarpsR * 32, smem, st>>>(reinterpret_cast<const float2*>(P),
                                       reinterpret_cast<const float2*>(Vq),
                                       reinterpret_cast<float2*>(WC), n, nk, err, first_bad,
                                       use_blk ? *blk : DysonBlocks{});
  return cudaGetLastError();
}

// ------------------------------------------------------------------ Dyson G

// In-place Gauss-Jordan inverse with partial pivoting (row swaps recorded,
// undone as column swaps at the end); every index is a compile-time constant.
template <typename V, int NO>
__device__ __forceinline__ bool gj_inverse(V (&a)[NO][NO]) {
  bool bad = false;
  int piv[NO];
#pragma unroll
  for (int c = 0; c < NO; ++c) {
    int p = c;
    auto best = cabs2(a[c][c]);
#pragma unroll
    for (int i = c + 1; i < NO; ++i) {
      auto v = cabs2(a[i][c]);
      if (v > best) { best = v; p = i; }
    }
    if (!(best > 0)) bad = true;
    piv[c] = p;
    // row swap c <-> p as branch-free selects (keeps the matrix in registers)
#pragma unroll
    for (int i = c + 1; i < NO; ++i) {
      const bool sw = (i == p);
#pragma unroll
      for (int j = 0; j < NO; ++j) {
        const V ti = a[i][j], tc = a[c][j];
        a[c][j].x = sw ? ti.x : tc.x; a[c][j].y = sw ? ti.y : tc.y;
        a[i][j].x = sw ? tc.x : ti.x; a[i][j].y = sw ? tc.y : ti.y;
      }
    }
    const V inv = cinv(a[c][c]);
    a[c][c] = cmk<V>(1.0, 0.0);
#pragma unroll
    for (int j = 0; j < NO; ++j) a[c][j] = cmul(a[c][j], inv);
#pragma unroll
    for (int i = 0; i < NO; ++i) {
      if (i == c) continue;
      const V f = a[i][c];
      a[i][c] = cmk<V>(0.0, 0.0);
#pragma unroll
      for (int j = 0; j < NO; ++j) a[i][j] = cfms(f, a[c][j], a[i][j]);
    }
  }
#pragma unroll
  for (int c = NO - 1; c >= 0; --c) {
#pragma unroll
    for (int k = c + 1; k < NO; ++k) {
      const bool sw = (piv[c] == k);
#pragma unroll
      for (int i = 0; i < NO; ++i) {
        const V tk = a[i][k], tc = a[i][c];
        a[i][c].x = sw ? tk.x : tc.x; a[i][c].y = sw ? tk.y : tc.y;
        a[i][k].x = sw ? tc.x : tk.x; a[i][k].y = sw ? tc.y : tk.y;
      }
    }
  }
  return bad;
}


// ---- FP64-accurate density from FP32 arithmetic (mixed path)
// A = i w_n + mu - H(k) - Sigma^HF(k) - Sigma^C(k, i w_n) with Sigma^C given
// in complex64.  G32 = FP32 inverse of A rounded to FP32; one refinement
// step G = G32 + G32 R with the residual R = I - A G32 evaluated in
// double-float arithmetic (each FP32 product split exactly by an FMA,
// compensated sums, Dekker/Knuth), so that Tr G carries FP64-level accuracy
// although no FP64 multiply runs per matrix entry.  The mu-dependent part
// mu - H - Sigma^HF comes from a per-k double-float table (hi, lo).

// x = hi + lo exactly as FP32 pair (hi = rn(x))
__device__ __forceinline__ float2 df_split(double x) {
  const float hi = static_cast<float>(x);
  return make_float2(hi, static_cast<float>(x - static_cast<double>(hi)));
}

// TwoSum: s = rn(a + b), e = (a + b) - s exactly.  The _rn intrinsics keep
// the compiler from contracting or reassociating these steps.
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
  return s;
}

// s + c += a * b exactly up to the final rounding of c (TwoProd + TwoSum)
__device__ __forceinline__ void df_madd(float a, float b, float& s, float& c) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  float es;
  s = two_sum(s, p, es);
  c = __fadd_rn(c, __fadd_rn(es, e));
}

__global__ void hs_table_kernel(const double2* __restrict__ Hk, const double2* __restrict__ SigHF,
                                double mu, int no, int nk, float4* __restrict__ hs) {
  const int no2 = no * no;
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<long long>(nk) * no2) return;
  const int e = static_cast<int>(idx % no2);
  double2 h = Hk[idx];
  if (SigHF) { h.x += SigHF[idx].x; h.y += SigHF[idx].y; }
  double re = -h.x, im = -h.y;
  if (e / no == e % no) re += mu;
  const float2 a = df_split(re), b = df_split(im);
  hs[idx] = make_float4(a.x, b.x, a.y, b.y);      // (hi.re, hi.im, lo.re, lo.im)
}

// A_ij = hs - SigIw (+ i w_n on the diagonal) as hi + lo pairs
template <int NO>
__device__ __forceinline__ void df_entry(const float4* __restrict__ hs_k, const float2* __restrict__ SigIw,
                                         const float2 wdf, int n, int k, int nk, int i, int j,
                                         float2& hi, float2& lo) {
  const float4 t = hs_k[i * NO + j];
  const float2 sc = SigIw[(static_cast<size_t>(n) * NO * NO + i * NO + j) * nk + k];
  // re: t.x + t.z - sc.x ; im: t.y + t.w - sc.y (+ w on the diagonal)
  float er, ei;
  const float sr = two_sum(t.x, -sc.x, er);
  float si = two_sum(t.y, -sc.y, ei);
  const float lr = __fadd_rn(t.z, er);
  float li = __fadd_rn(t.w, ei);
  if (i == j) {
    float ew;
    si = two_sum(si, wdf.x, ew);
    li = __fadd_rn(li, __fadd_rn(ew, wdf.y));
  }
  hi = make_float2(sr, si);
  lo = make_float2(lr, li);
}

template <int NO>
__global__ void __launch_bounds__(256) dyson_g_refine_kernel(const float4* __restrict__ hs,
                                                             const float2* __restrict__ SigIw,
                                                             const double2* __restrict__ dw,
                                                             const double* __restrict__ iw, int r,
                                                             int nk, double* part, int* err) {
  __shared__ double sh[64];
  const long long total = static_cast<long long>(r) * nk;
  double s1 = 0.0, s2 = 0.0;
  bool bad = false;
  for (long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
       idx += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int n = static_cast<int>(idx / nk);
    const int k = static_cast<int>(idx - static_cast<long long>(n) * nk);
    const float4* hk = hs + static_cast<size_t>(k) * NO * NO;
    const float2 wdf = df_split(iw[n]);
    float2 g[NO][NO];
#pragma unroll
    for (int i = 0; i < NO; ++i)
#pragma unroll
      for (int j = 0; j < NO; ++j) {
        float2 hi, lo;
        df_entry<NO>(hk, SigIw, wdf, n, k, nk, i, j, hi, lo);
        g[i][j] = hi;
      }
    bad |= gj_inverse<float2, NO>(g);
    // Tr G = Tr G32 + sum_ij G32_ij R_ji,  R = I - A G32 (double-float)
    float2 corr = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < NO; ++i) {
      float2 ahi[NO], alo[NO];
#pragma unroll
      for (int m = 0; m < NO; ++m) df_entry<NO>(hk, SigIw, wdf, n, k, nk, i, m, ahi[m], alo[m]);
#pragma unroll
      for (int j = 0; j < NO; ++j) {
        float sr = (i == j) ? -1.f : 0.f, cr = 0.f, si = 0.f, ci = 0.f;   // (A G32 - I)_ij
#pragma unroll
        for (int m = 0; m < NO; ++m) {
          df_madd(ahi[m].x, g[m][j].x, sr, cr);
          df_madd(-ahi[m].y, g[m][j].y, sr, cr);
          df_madd(ahi[m].x, g[m][j].y, si, ci);
          df_madd(ahi[m].y, g[m][j].x, si, ci);
          cr = fmaf(alo[m].x, g[m][j].x, cr);
          cr = fmaf(-alo[m].y, g[m][j].y, cr);
          ci = fmaf(alo[m].x, g[m][j].y, ci);
          ci = fmaf(alo[m].y, g[m][j].x, ci);
        }
        const float2 Rij = make_float2(-(sr + cr), -(si + ci));
        corr = cfma(g[j][i], Rij, corr);        // sum_ij G32_ji R_ij
      }
    }
    double trr = corr.x, tri = corr.y;
    float2 tr2 = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < NO; ++i) {
      trr += static_cast<double>(g[i][i].x);
      tri += static_cast<double>(g[i][i].y);
#pragma unroll
      for (int j = 0; j < NO; ++j) tr2 = cfma(g[i][j], g[j][i], tr2);
    }
    const double2 wn = dw[n];
    s1 += wn.x * trr - wn.y * tri;
    s2 += wn.x * static_cast<double>(tr2.x) - wn.y * static_cast<double>(tr2.y);
  }
  if (bad) atomicCAS(err, 0, QA_ESINGULAR_CODE);
  block_sum2(s1, s2, sh);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s1;
    part[2 * blockIdx.x + 1] = s2;
  }
}

// Bm(k, i w_n) = (mu_ref - H(k) - Sigma^HF(k)) - Sigma^C(k, i w_n), the
// mu-independent part of the inverse's argument, with a reference chemical
// potential folded into the diagonal in FP64 (the search then adds the small
// difference mu - mu_ref).  One thread per (k, matrix entry) walks the r
// frequencies.  part[2 b] receives norb * max (|mu_ref - H - Sigma^HF|_entry +
// |Sigma^C|_entry), an upper bound of the row-sum norm of H + Sigma^HF +
// Sigma^C - mu_ref (the window of the chemical-potential search).
template <typename T>
__global__ void __launch_bounds__(256) dyson_g_prep_kernel(const double2* __restrict__ Hk,
                                                           const double2* __restrict__ SigHF,
                                                           const cplx<T>* __restrict__ SigIw,
                                                           double mu_ref, int r, int no, int nk,
                                                           cplx<T>* __restrict__ Bm, double* part) {
  using V = cplx<T>;
  __shared__ double sh[32];
  const int no2 = no * no;
  const long long total = static_cast<long long>(nk) * no2;
  double best = 0.0;
  for (long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
       idx += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int e = static_cast<int>(idx / nk);
    const int k = static_cast<int>(idx - static_cast<long long>(e) * nk);
    double2 h = Hk[static_cast<size_t>(k) * no2 + e];
    if (SigHF) {
      const double2 s = SigHF[static_cast<size_t>(k) * no2 + e];
      h.x += s.x; h.y += s.y;
    }
    h.x = -h.x; h.y = -h.y;
    if (e / no == e % no) h.x += mu_ref;
    const V hb = from_d2<V>(h);
    T smax = 0;
    for (int n = 0; n < r; ++n) {
      const size_t o = (static_cast<size_t>(n) * no2 + e) * nk + k;
      V b = hb;
      if (SigIw) {
        const V s = SigIw[o];
        b = csub(hb, s);
        smax = fmax(smax, sqrt(cabs2(s)));
      }
      Bm[o] = b;
    }
    best = fmax(best, sqrt(h.x * h.x + h.y * h.y) + static_cast<double>(smax));
  }
  best = block_max(best, sh);
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = best * no; part[2 * blockIdx.x + 1] = 0.0; }
}

// G(k, i w_n) = (i w_n + dmu + Bm(k, i w_n))^-1, dmu = mu - mu_ref (with mus:
// mus[0] - mus[1], the device-side search's current point and reference).
// mode 0: per-block partial sums of Re(dw_n Tr G) and Re(dw_n Tr G^2) (FP64
// accumulation of the per-system traces); mode 1: also store G.
template <typename T, int NO>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 || std::is_same<T, dfl>::value) ? 2 : 1) dyson_g_kernel(const cplx<T>* __restrict__ Bm,
                                                      const cplx<T>* __restrict__ dw,
                                                      const double* __restrict__ iw, double dmu,
                                                      const double* mus, int r, int nk, cplx<T>* Giw,
                                                      double* part, int mode, int* err) {
  using V = cplx<T>;
  __shared__ double sh[64];
  const long long total = static_cast<long long>(r) * nk;
  double s1 = 0.0, s2 = 0.0;
  bool bad = false;
  const T dm = static_cast<T>(mus ? mus[0] - mus[1] : dmu);
  for (long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
       idx += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int n = static_cast<int>(idx / nk);
    const int k = static_cast<int>(idx - static_cast<long long>(n) * nk);
    const T wv = static_cast<T>(iw[n]);
    V a[NO][NO];
#pragma unroll
    for (int i = 0; i < NO; ++i)
#pragma unroll
      for (int j = 0; j < NO; ++j) {
        V m = Bm[(static_cast<size_t>(n) * NO * NO + i * NO + j) * nk + k];
        if (i == j) { m.x += dm; m.y += wv; }
        a[i][j] = m;
      }
    bad |= gj_inverse<V, NO>(a);
    // a = G(k, i w_n)
    V tr = cmk<V>(0, 0), tr2 = cmk<V>(0, 0);
#pragma unroll
    for (int i = 0; i < NO; ++i) {
      tr = cadd(tr, a[i][i]);
#pragma unroll
      for (int j = 0; j < NO; ++j) tr2 = cfma(a[i][j], a[j][i], tr2);
    }
    const V wn = dw[n];
    s1 += static_cast<double>(wn.x * tr.x - wn.y * tr.y);
    s2 += static_cast<double>(wn.x * tr2.x - wn.y * tr2.y);
    if (mode == 1) {
#pragma unroll
      for (int i = 0; i < NO; ++i)
#pragma unroll
        for (int j = 0; j < NO; ++j) Giw[(static_cast<size_t>(n) * NO * NO + i * NO + j) * nk + k] = a[i][j];
    }
  }
  if (bad) atomicCAS(err, 0, QA_ESINGULAR_CODE);
  block_sum2(s1, s2, sh);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s1;
    part[2 * blockIdx.x + 1] = s2;
  }
}

__global__ void reduce_pairs_kernel(const double* part, int n, int op_max, double* out) {
  __shared__ double sh[64];
  double a = op_max ? 0.0 : 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if (op_max) { a = fmax(a, part[2 * i]); b = fmax(b, part[2 * i + 1]); }
    else { a += part[2 * i]; b += part[2 * i + 1]; }
  }
  if (op_max) {
    a = block_max(a, sh);
    __syncthreads();
    b = block_max(b, sh);
  } else {
    block_sum2(a, b, sh);
  }
  if (threadIdx.x == 0) { out[0] = a; out[1] = b; }
}

}  // namespace

int dyson_g_blocks(int r, int nk) {
  long long total = static_cast<long long>(r) * nk;
  long long b = (total + 255) / 256;
  return static_cast<int>(b < 1216 ? (b < 1 ? 1 : b) : 1216);   // 8 per SM on 152 SMs
}

template <typename T>
cudaError_t launch_dyson_w(const void* P, const void* Vq, void* WC, int r, int npair, int nk,
                           int* err, long long* first_bad, cudaStream_t st,
                           const DysonBlocks* blk, void* lu, unsigned char* piv) {
  if (npair > kMaxPair) return cudaErrorInvalidValue;
  if (lu && (sizeof(T) != 8 || !piv)) return cudaErrorInvalidValue;
  if (sizeof(T) == 4) {
    // register-row kernel: W^C = (1 - V P)^-1 V P V directly
    if (npair <= 4) return launch_dyson_w_tile<4>(P, Vq, WC, r, npair, nk, err, first_bad, st, blk);
    if (npair <= 8) return launch_dyson_w_tile<8>(P, Vq, WC, r, npair, nk, err, first_bad, st, blk);
    if (npair == 15) return launch_dyson_w_tile<16, 15>(P, Vq, WC, r, npair, nk, err, first_bad, st, blk);
    if (npair == 16) return launch_dyson_w_tile<16, 16>(P, Vq, WC, r, npair, nk, err, first_bad, st, blk);
    if (npair <= 16) return launch_dyson_w_tile<16>(P, Vq, WC, r, npair, nk, err, first_bad, st, blk);
    return launch_dyson_w_reg<25, 32>(P, Vq, WC, r, npair, nk, err, first_bad, st);
  }
  size_t smem = static_cast<size_t>(kWarpsW) * 2 * npair * (npair + 1) * sizeof(cplx<T>);
  auto fn = &dyson_w_kernel<T, false>;
  cudaError_t e = set_smem(reinterpret_cast<const void*>(fn), smem);
  if (e != cudaSuccess) return e;
  dim3 grid((nk + kWarpsW - 1) / kWarpsW, r);
  fn<<<grid, kWarpsW * 32, smem, st>>>(reinterpret_cast<const cplx<T>*>(P),
                                       reinterpret_cast<const cplx<T>*>(Vq),
                                       reinterpret_cast<cplx<T>*>(WC), npair, nk, err, first_bad,
                                       reinterpret_cast<cplx<T>*>(lu), piv);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dyson_g_prep(const double2* Hk, const double2* SigHF, const void* SigIw,
                                double mu_ref, int r, int norb, int nk, void* Bm, double* part,
                                int nblocks, cudaStream_t st) {
  dyson_g_prep_kernel<T><<<nblocks, 256, 0, st>>>(Hk, SigHF, reinterpret_cast<const cplx<T>*>(SigIw),
                                                  mu_ref, r, norb, nk, reinterpret_cast<cplx<T>*>(Bm),
                                                  part);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dyson_g(const void* Bm, const void* dw, const double* iw, double dmu, int r,
                           int norb, int nk, void* Giw, double* part, int nblocks, int mode,
                           int* err, cudaStream_t st, const double* mus) {
  auto b = reinterpret_cast<const cplx<T>*>(Bm);
  auto d = reinterpret_cast<const cplx<T>*>(dw);
  auto g = reinterpret_cast<cplx<T>*>(Giw);
  switch (norb) {
#define QA_CASE(NO) \
    case NO: dyson_g_kernel<T, NO><<<nblocks, 256, 0, st>>>(b, d, iw, dmu, mus, r, nk, g, part, mode, err); break;
    QA_CASE(1) QA_CASE(2) QA_CASE(3) QA_CASE(4) QA_CASE(5)
#undef QA_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_dyson_g_refine(const double2* Hk, const double2* SigHF, const void* SigIw,
                                  const void* dw, const double* iw, double mu, int r, int norb,
                                  int nk, void* hs, double* part, int nblocks, int* err,
                                  cudaStream_t st) {
  const long long ne = static_cast<long long>(nk) * norb * norb;
  hs_table_kernel<<<static_cast<unsigned>((ne + 255) / 256), 256, 0, st>>>(
      Hk, SigHF, mu, norb, nk, reinterpret_cast<float4*>(hs));
  auto h = reinterpret_cast<const float4*>(hs);
  auto s = reinterpret_cast<const float2*>(SigIw);
  auto d = reinterpret_cast<const double2*>(dw);
  switch (norb) {
#define QA_CASE(NO)     case NO: dyson_g_refine_kernel<NO><<<nblocks, 256, 0, st>>>(h, s, d, iw, r, nk, part, err); break;
    QA_CASE(1) QA_CASE(2) QA_CASE(3) QA_CASE(4) QA_CASE(5)
#undef QA_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_reduce_pairs(const double* part, int n, int op_max, double* out,
                                cudaStream_t st) {
  reduce_pairs_kernel<<<1, 256, 0, st>>>(part, n, op_max, out);
  return cudaGetLastError();
}

template cudaError_t launch_dyson_w<double>(const void*, const void*, void*, int, int, int, int*,
                                            long long*, cudaStream_t, const DysonBlocks*, void*, unsigned char*);
template cudaError_t launch_dyson_w<float>(const void*, const void*, void*, int, int, int, int*,
                                           long long*, cudaStream_t, const DysonBlocks*, void*, unsigned char*);
template cudaError_t launch_dyson_g<double>(const void*, const void*, const double*, double, int,
                                            int, int, void*, double*, int, int, int*, cudaStream_t, const double*);
template cudaError_t launch_dyson_g<float>(const void*, const void*, const double*, double, int, int,
                                           int, void*, double*, int, int, int*, cudaStream_t, const double*);
template cudaError_t launch_dyson_g_prep<double>(const double2*, const double2*, const void*, double,
                                                 int, int, int, void*, double*, int, cudaStream_t);
template cudaError_t launch_dyson_g_prep<float>(const double2*, const double2*, const void*, double,
                                                int, int, int, void*, double*, int, cudaStream_t);
template cudaError_t launch_dyson_w<dfl>(const void*, const void*, void*, int, int, int, int*,
                                         long long*, cudaStream_t, const DysonBlocks*, void*, unsigned char*);
template cudaError_t launch_dyson_g<dfl>(const void*, const void*, const double*, double, int, int,
                                         int, void*, double*, int, int, int*, cudaStream_t, const double*);
template cudaError_t launch_dyson_g_prep<dfl>(const double2*, const double2*, const void*, double,
                                              int, int, int, void*, double*, int, cudaStream_t);

}  // namespace qa
