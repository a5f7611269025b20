// DLR node transforms of double-float data on the 5th-generation tensor cores
// (tcgen05, sm_103a) with fixed-point bf16 slices: the accurate mixed path's
// form of the imaginary-time <-> Matsubara maps (Kaye, Chen & Parcollet 2022,
// cited by the paper for its DLR grids).
//
// The complex map out[j][c] = sum_l T[j][l] in[l][c] of every column c is one
// real GEMM Y (cols x 2r) = X (cols x 2r) Tt^T with Tt the real embedding
// [[Re T, -Im T], [Im T, Re T]] of T.  Both operands are cut into five bf16
// slices on a fixed-point grid (the scheme of Ozaki, Ogita, Oishi & Rump for
// accurate matrix products from low-precision units):
//   row n of Tt:   Tt[n][k] = 2^(a_n - 8) sum_i tau_i[n][k] 256^-i
//   column c of X: X[c][k]  = 2^(b_c - 8) sum_j sig_j[c][k] 256^-j
// with integer slices |tau_i|, |sig_j| <= 129 and one exponent per row of Tt
// (a_n, host) and per column of X (b_c, from the column's largest entry).
// Every product of two slices is then an integer, and the products of one
// level l = i + j share the unit 2^(a_n + b_c - 16 - 8 l): the level sums
//   A_l[c][n] = sum_{i+j=l} sum_k tau_i[n][k] sig_j[c][k]
// stay below 5 * 192 * 129 * 128 < 2^24 for 2r <= 192, so the tensor core's
// FP32 accumulation is exact whatever its rounding.  Levels 0..4 are kept (15
// slice products); the first dropped level weighs 2^-40 against sum |T||X|.
//   Y[c][n] = 2^(a_n + b_c - 16) sum_l A_l 256^-l   (combined in double-float)
//
// TMEM holds the five level accumulators side by side (5 x Nw columns of 32
// bits, Nw <= 96), so the 2r output columns are split into parts of at most
// 96 that separate CTAs compute from the same input tile (out must not alias
// in).  One persistent CTA per SM, warp-specialised: 16 worker warps load
// and slice 128-column tiles of X in K-chunks of 16 (8 nodes x re/im) into
// double-buffered shared memory, one issuer thread issues the 15 MMAs of a
// chunk (M = 128, N = Nw, K = 16) and commits them to an mbarrier; at the end
// of a tile the workers read the five accumulators back (tcgen05.ld), combine
// them and store Y.  Every wait is bounded; on time-out the kernel records
// QA_ETIMEOUT, waits (bounded) for its own MMAs, frees TMEM and returns.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "qa_common.cuh"
#include "qa_tc.cuh"

namespace qa {
namespace {

constexpr int kOzSlices = 5;
constexpr int kOzMaxNw = 96;
constexpr int kTileM = 128;
constexpr int kChunkK = 16;
constexpr int kWorkers = 512;                   // 16 worker warps; warp 16 issues the MMAs
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAChunk = kTileM * kChunkK * 2;   // bytes of one slice of one chunk

struct OzArgs {
  const uint8_t* pack;     // per part: [5][Nw][Kp] bf16 slices (canonical layout); then int a_n[2r]
  int r, Kp, nparts;
  int Nw[2], n0[2];
  long long off[2];        // byte offset of each part's slices in pack
  long long rexp_off;      // byte offset of the row exponents
  const dfc* in;
  void* out;               // dfc, or double2 when OUT64
  long long ncol;
  int* err;
  long long wait_limit;    // polls of each pipeline wait before the time-out path
  const float* colscale;   // 2^(8 - b_c) per column (col_scale_kernel or col_scale_code_kernel)
};

__device__ __forceinline__ uint32_t pack_hi16(float a, float b) {
  // integers of at most 8 significant bits: the bf16 value is the float's top half
  return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);
}

// five fixed-point slices of x * 2^(8 - b) (|value| <= 128): s_j = rint of the
// running remainder's high part, the remainder kept exactly as a double-float
__device__ __forceinline__ void slice5(dfl x, float scale, float* s) {
  float h = x.hi * scale, l = x.lo * scale;
#pragma unroll
  for (int j = 0; j < kOzSlices; ++j) {
    s[j] = rintf(h);
    const float t = __fsub_rn(h, s[j]);           // exact
    const dfl nx = df_norm(t, l);                  // exact: t is 0 or a multiple of ulp(h) >= 2|l|
    h = nx.hi * 256.0f;
    l = nx.lo * 256.0f;
  }
}

// sum_l A_l 256^-l as a double-float (A_l exact integers below 2^24)
__device__ __forceinline__ dfl combine5(const float* A) {
  float s, e, s2, e2;
  two_sum(A[0], A[1] * 0x1p-8f, s, e);
  two_sum(s, A[2] * 0x1p-16f, s2, e2);
  const float t = fmaf(A[4], 0x1p-32f, A[3] * 0x1p-24f);
  return df_norm(s2, __fadd_rn(__fadd_rn(e, e2), t));
}

template <bool OUT64>
__global__ void __launch_bounds__(kWorkers + 32, 1) dlr_oz_kernel(OzArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int part = blockIdx.x % a.nparts;
  const int Nw = a.Nw[part], n0 = a.n0[part];
  const uint32_t bslice = static_cast<uint32_t>(Nw) * a.Kp * 2;
  uint8_t* Bs = smem;                                         // [5][Nw][Kp]
  uint8_t* As = smem + kOzSlices * bslice;                    // [2][5][kAChunk]
  uint64_t* bars = reinterpret_cast<uint64_t*>(As + 2 * kOzSlices * kAChunk);
  uint64_t* done = bars;          // [2] MMAs of the chunk in buffer b finished
  uint64_t* full = bars + 2;      // [2] buffer b staged by all worker warps
  uint64_t* prep = bars + 4;      // [2] column exponents of a tile written
  uint64_t* drained = bars + 6;   // accumulators read back
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 8);
  float* s_b = reinterpret_cast<float*>(tslot + 4);           // [2][128] 2^(8 - b_c) per tile row
  int* s_rexp = reinterpret_cast<int*>(s_b + 2 * kTileM);     // [Nw] a_n of this part
  __shared__ int s_abort;
  __shared__ long long s_issued;

  {
    const uint4* src = reinterpret_cast<const uint4*>(a.pack + a.off[part]);
    for (uint32_t i = tid; i < kOzSlices * bslice / 16; i += blockDim.x)
      reinterpret_cast<uint4*>(Bs)[i] = src[i];
    const int* rx = reinterpret_cast<const int*>(a.pack + a.rexp_off);
    for (int i = tid; i < Nw; i += blockDim.x) s_rexp[i] = (n0 + i < 2 * a.r) ? rx[n0 + i] : 0;
  }
  if (tid == 0) {
    tc::mbar_init(&done[0], 1);
    tc::mbar_init(&done[1], 1);
    tc::mbar_init(&full[0], kWorkers / 32);
    tc::mbar_init(&full[1], kWorkers / 32);
    tc::mbar_init(&prep[0], kWorkers / 32);
    tc::mbar_init(&prep[1], kWorkers / 32);
    tc::mbar_init(drained, kWorkers / 32);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
    s_issued = 0;
  }
  if (warp == 0) tc::tmem_alloc(tslot, kTmemCols);
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  volatile int* abort_flag = &s_abort;
  const uint32_t taddr = *tslot;
  const int nchunk = a.Kp / kChunkK;
  const long long ntiles = (a.ncol + kTileM - 1) / kTileM;
  const int cpp = gridDim.x / a.nparts;                        // CTAs per part
  const int cp = blockIdx.x / a.nparts;

  if (warp == kWorkers / 32) {
    // ---- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = tc::instr_desc(kTileM, Nw);
      const uint32_t bsbo = static_cast<uint32_t>(a.Kp / 8) * 128;
      long long g = 0, tl = 0;
      bool ok = true;
      for (long long tile = cp; tile < ntiles && ok; tile += cpp, ++tl) {
        if (tl > 0) {
          if (!tc::mbar_wait(drained, static_cast<uint32_t>((tl - 1) & 1), abort_flag, a.wait_limit)) { ok = false; break; }
          tc::fence_after();
        }
        for (int ch = 0; ch < nchunk; ++ch, ++g) {
          const int b = static_cast<int>(g & 1);
          if (!tc::mbar_wait(&full[b], static_cast<uint32_t>((g >> 1) & 1), abort_flag, a.wait_limit)) { ok = false; break; }
          tc::fence_after();
#pragma unroll
          for (int lvl = 0; lvl < kOzSlices; ++lvl) {
#pragma unroll
            for (int i = 0; i <= lvl; ++i) {
              const int j = lvl - i;                // tau_i x sig_j
              const uint32_t aaddr = tc::smem_u32(As + (b * kOzSlices + j) * kAChunk);
              const uint32_t baddr = tc::smem_u32(Bs + i * bslice) + static_cast<uint32_t>(ch) * 256;
              tc::mma_bf16(taddr + static_cast<uint32_t>(lvl * Nw), tc::smem_desc(aaddr, 128, 256),
                           tc::smem_desc(baddr, 128, bsbo), idesc, (ch > 0 || i > 0) ? 1u : 0u);
            }
          }
          tc::mma_commit(&done[b]);
        }
      }
      if (!ok) *abort_flag = 1;
      s_issued = g;
    }
    __syncwarp();
  } else {
    // ---- workers: tile row m (TMEM lane), quarter qt of each chunk's nodes
    // and of the accumulator columns
    const int m = 32 * (warp & 3) + lane;
    const int qt = warp >> 2;
    const uint32_t lane_base = static_cast<uint32_t>(32 * (warp & 3)) << 16;
    const uint32_t roff = static_cast<uint32_t>(m >> 3) * 256 + static_cast<uint32_t>(m & 7) * 16 +
                          static_cast<uint32_t>(qt >> 1) * 128 + static_cast<uint32_t>(qt & 1) * 8;
    const int cq = Nw / 4;                                     // accumulator columns per thread
    long long g = 0, tl = 0;
    bool ok = true;
    // this thread's two values of chunk ch of the column cl
    auto load2 = [&](int ch, long long cl, bool cok, dfc* v) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int l = ch * 8 + qt * 2 + e;
        v[e] = dfc{dfl(0.0f, 0.0f), dfl(0.0f, 0.0f)};
        if (cok && ch < nchunk && l < a.r) v[e] = ldg_c(a.in + static_cast<long long>(l) * a.ncol + cl);
      }
    };
    // the column, its slice grid 2^(8 - b_c) (col_scale_kernel) and the first chunk of
    // a tile are fetched before the previous tile's accumulators are drained, so
    // these loads fly during the drain
    long long col = static_cast<long long>(cp) * kTileM + m;
    bool colok = cp < ntiles && col < a.ncol;
    float scale = colok ? __ldg(a.colscale + col) : 1.0f;
    dfc cur[2], nxt[2];
    load2(0, col, colok, cur);
    for (long long tile = cp; tile < ntiles && ok; tile += cpp, ++tl) {
      // the next chunk's values are loaded before the current one is sliced
      for (int ch = 0; ch < nchunk; ++ch, ++g) {
        const int b = static_cast<int>(g & 1);
        load2(ch + 1, col, colok, nxt);
        if (g >= 2) {
          const bool w = tc::mbar_wait(&done[b], static_cast<uint32_t>(((g - 2) >> 1) & 1), abort_flag, a.wait_limit);
          if (__any_sync(0xffffffffu, !w)) { ok = false; break; }
        }
        float s[4][kOzSlices];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          slice5(cur[e].x, scale, s[2 * e]);
          slice5(cur[e].y, scale, s[2 * e + 1]);
          cur[e] = nxt[e];
        }
#pragma unroll
        for (int j = 0; j < kOzSlices; ++j) {
          uint2 v;
          v.x = pack_hi16(s[0][j], s[1][j]);
          v.y = pack_hi16(s[2][j], s[3][j]);
          *reinterpret_cast<uint2*>(As + (b * kOzSlices + j) * kAChunk + roff) = v;
        }
        tc::fence_async_smem();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&full[b]);
      }
      if (!ok) break;
      // the tile's MMAs are done once its last chunk's commit has arrived
      {
        const bool w = tc::mbar_wait(&done[(g - 1) & 1], static_cast<uint32_t>(((g - 1) >> 1) & 1), abort_flag, a.wait_limit);
        if (__any_sync(0xffffffffu, !w)) { ok = false; break; }
      }
      // the next tile's column, grid and first chunk
      const long long ntile = tile + cpp;
      const long long col_n = ntile * kTileM + m;
      const bool colok_n = ntile < ntiles && col_n < a.ncol;
      const float scale_n = colok_n ? __ldg(a.colscale + col_n) : 1.0f;
      load2(0, col_n, colok_n, cur);
      tc::fence_after();
      const float oscale = 0x1p-16f / scale * 256.0f;          // 2^(b_c - 16)
      for (int c4 = qt * cq; c4 < (qt + 1) * cq; c4 += 4) {
        float A[kOzSlices][4];
#pragma unroll
        for (int lvl = 0; lvl < kOzSlices; ++lvl)
          tc::tmem_ld4(taddr + lane_base + static_cast<uint32_t>(lvl * Nw + c4), A[lvl]);
        tc::tmem_wait_ld();
        dfl y[4];
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          float L[kOzSlices];
#pragma unroll
          for (int lvl = 0; lvl < kOzSlices; ++lvl) L[lvl] = A[lvl][cc];
          const dfl v = combine5(L);
          const float sc = ldexpf(oscale, s_rexp[c4 + cc]);
          y[cc] = dfl(v.hi * sc, v.lo * sc);
        }
        if (colok) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int j = (n0 + c4) / 2 + h;                   // output node (re, im in columns 2j, 2j+1)
            if (j < a.r) {
              const long long o = static_cast<long long>(j) * a.ncol + col;
              if (OUT64)
                static_cast<double2*>(a.out)[o] =
                    make_double2(static_cast<double>(y[2 * h].hi) + static_cast<double>(y[2 * h].lo),
                                 static_cast<double>(y[2 * h + 1].hi) + static_cast<double>(y[2 * h + 1].lo));
              else
                reinterpret_cast<float4*>(a.out)[o] =
                    make_float4(y[2 * h].hi, y[2 * h].lo, y[2 * h + 1].hi, y[2 * h + 1].lo);
            }
          }
        }
      }
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(drained);
      col = col_n;
      colok = colok_n;
      scale = scale_n;
    }
    if (!ok) *abort_flag = 1;
  }
  __syncthreads();
  if (tid == 0 && *abort_flag) {
    atomicCAS(a.err, 0, QA_ETIMEOUT_CODE);
    // let this CTA's own MMAs finish (bounded) before TMEM is released
    const long long gl = s_issued - 1;
    if (gl >= 0) tc::mbar_wait(&done[gl & 1], static_cast<uint32_t>((gl >> 1) & 1), nullptr);
  }
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(taddr, kTmemCols);
}

// 2^(8 - b_c) per column c of in [r][ncol] (double-float complex), with 2^(b_c) > 2 max over
// the column's 2r real values of |high part| (1 + 2^-19), b_c >= -100: the fixed-point grid of
// the column's slices.  Consecutive threads read consecutive columns (coalesced).
__global__ void __launch_bounds__(256) col_scale_kernel(const dfc* __restrict__ in, int r, long long ncol,
                                                        float* __restrict__ scale) {
  for (long long c = blockIdx.x * 256LL + threadIdx.x; c < ncol; c += static_cast<long long>(gridDim.x) * 256) {
    float mx = 0.0f;
#pragma unroll 8
    for (int l = 0; l < r; ++l) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(in + static_cast<long long>(l) * ncol + c));
      mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.z)));
    }
    int e = 0;
    if (mx > 0.0f) frexpf(mx * 2.000004f, &e);
    e = max(e, -100);
    scale[c] = ldexpf(1.0f, 8 - e);
  }
}

// 2^(8 - b_c) from a column's largest grid code b (0: an all-zero column, b_c = 0)
__device__ __forceinline__ float code_scale(unsigned b) {
  const int e = b == 0 ? 0 : static_cast<int>(b) - 101;
  return ldexpf(1.0f, 8 - e);
}

// The same grids from the one-byte codes that the producing kernel stored beside
// each value (oz_grid_code; code [r][ncol]): the largest code of a column decodes
// to the exponent col_scale_kernel would find, so the two give identical scales
// while this pass reads one byte per value instead of sixteen.
__global__ void __launch_bounds__(256) col_scale_code_kernel(const uint8_t* __restrict__ code, int r,
                                                             long long ncol, float* __restrict__ scale) {
  for (long long c = blockIdx.x * 256LL + threadIdx.x; c < ncol; c += static_cast<long long>(gridDim.x) * 256) {
    unsigned mx = 0;
#pragma unroll 8
    for (int l = 0; l < r; ++l) mx = max(mx, static_cast<unsigned>(__ldg(code + static_cast<long long>(l) * ncol + c)));
    scale[c] = code_scale(mx);
  }
}

// col_scale_code_kernel for ncol a multiple of 4 (code and scale 16-byte aligned):
// four columns per thread, one 32-bit load per node and a bytewise maximum
__global__ void __launch_bounds__(256) col_scale_code4_kernel(const uint8_t* __restrict__ code, int r,
                                                              long long ncol, float* __restrict__ scale) {
  const long long nc4 = ncol >> 2;
  const unsigned* __restrict__ c4 = reinterpret_cast<const unsigned*>(code);
  for (long long c = blockIdx.x * 256LL + threadIdx.x; c < nc4; c += static_cast<long long>(gridDim.x) * 256) {
    unsigned mx = 0;
#pragma unroll 8
    for (int l = 0; l < r; ++l) mx = __vmaxu4(mx, __ldg(c4 + static_cast<long long>(l) * nc4 + c));
    reinterpret_cast<float4*>(scale)[c] = make_float4(code_scale(mx & 0xffu), code_scale((mx >> 8) & 0xffu),
                                                      code_scale((mx >> 16) & 0xffu), code_scale(mx >> 24));
  }
}

uint16_t bf16_of_int(long double v) {
  const float f = static_cast<float>(v);           // an integer of at most 8 significant bits
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return static_cast<uint16_t>(u >> 16);
}

}  // namespace

DlrOzLayout dlr_oz_layout(int r) {
  DlrOzLayout L;
  L.Kp = ((2 * r + 15) / 16) * 16;
  L.nparts = (2 * r + kOzMaxNw - 1) / kOzMaxNw;
  long long off = 0;
  for (int p = 0; p < L.nparts && p < 2; ++p) {
    L.n0[p] = p * kOzMaxNw;
    const int w = std::min(kOzMaxNw, 2 * r - L.n0[p]);
    L.Nw[p] = ((w + 15) / 16) * 16;
    L.off[p] = off;
    off += static_cast<long long>(kOzSlices) * L.Nw[p] * L.Kp * 2;
  }
  L.rexp_off = off;
  L.bytes = off + static_cast<long long>(2 * r) * 4;
  L.smem = static_cast<size_t>(kOzSlices) * kOzMaxNw * L.Kp * 2 + 2ull * kOzSlices * kAChunk + 8 * 8 +
           16 + 2 * kTileM * 4 + kOzMaxNw * 4;
  return L;
}

bool dlr_oz_supported(int r) {
  if (r < 1) return false;
  const DlrOzLayout L = dlr_oz_layout(r);
  return L.Kp <= 192 && L.nparts <= 2 && L.smem <= 227 * 1024;
}

// Real embedding of the complex r x r matrix T cut into five fixed-point bf16
// slices per row (row exponent a_n: 2^a_n >= 2 max_k |Tt[n][k]|), laid out per
// part of output rows in the canonical K-major no-swizzle core-matrix order;
// the row exponents follow the slices.
void pack_dlr_oz(const std::complex<double>* T, int r, std::vector<uint8_t>* dst) {
  const DlrOzLayout L = dlr_oz_layout(r);
  dst->assign(static_cast<size_t>(L.bytes), 0);
  const int K = 2 * r;
  std::vector<long double> row(K);
  std::vector<int> rexp(K, 0);
  for (int n = 0; n < K; ++n) {
    const int j = n >> 1, cp = n & 1;
    long double mx = 0;
    for (int k = 0; k < K; ++k) {
      const int l = k >> 1, c = k & 1;
      const std::complex<double> t = T[static_cast<size_t>(j) * r + l];
      long double x;
      if (cp == 0) x = c == 0 ? t.real() : -t.imag();
      else x = c == 0 ? t.imag() : t.real();
      row[k] = x;
      mx = std::max(mx, std::fabs(x));
    }
    int e = 0;
    if (mx > 0) std::frexp(2.0L * mx, &e);                    // 2^e > 2 mx
    rexp[n] = e;
    const int p = n / kOzMaxNw, nl = n - L.n0[p];
    uint16_t* base = reinterpret_cast<uint16_t*>(dst->data() + L.off[p]);
    const size_t slice_elems = static_cast<size_t>(L.Nw[p]) * L.Kp;
    for (int k = 0; k < K; ++k) {
      long double u = std::ldexp(row[k], 8 - e);              // |u| <= 128
      const size_t off = static_cast<size_t>(nl / 8) * (L.Kp / 8) * 64 + static_cast<size_t>(k / 8) * 64 +
                         static_cast<size_t>(nl % 8) * 8 + (k % 8);
      for (int s = 0; s < kOzSlices; ++s) {
        const long double q = std::nearbyint(u);
        base[static_cast<size_t>(s) * slice_elems + off] = bf16_of_int(q);
        u = (u - q) * 256.0L;
      }
    }
  }
  std::memcpy(dst->data() + L.rexp_off, rexp.data(), rexp.size() * 4);
}

cudaError_t launch_dlr_oz(const void* pack, int r, const void* in, void* out, long long ncol, int* err,
                          cudaStream_t st, bool out_c128, long long wait_limit, float* colscale,
                          const uint8_t* code) {
  if (!dlr_oz_supported(r) || in == out || !colscale) return cudaErrorInvalidValue;
  if (ncol <= 0) return cudaSuccess;
  {
    const long long nb = std::min<long long>((ncol + 255) / 256, 152LL * 8);
    const bool v4 = (ncol & 3) == 0 && (reinterpret_cast<uintptr_t>(code) & 15) == 0 &&
                    (reinterpret_cast<uintptr_t>(colscale) & 15) == 0;
    if (code && v4)
      col_scale_code4_kernel<<<static_cast<unsigned>(std::min<long long>((ncol / 4 + 255) / 256, 152LL * 8)), 256,
                               0, st>>>(code, r, ncol, colscale);
    else if (code)
      col_scale_code_kernel<<<static_cast<unsigned>(nb), 256, 0, st>>>(code, r, ncol, colscale);
    else
      col_scale_kernel<<<static_cast<unsigned>(nb), 256, 0, st>>>(static_cast<const dfc*>(in), r, ncol, colscale);
    cudaError_t e0 = cudaGetLastError();
    if (e0 != cudaSuccess) return e0;
  }
  const DlrOzLayout L = dlr_oz_layout(r);
  auto fn = out_c128 ? &dlr_oz_kernel<true> : &dlr_oz_kernel<false>;
  cudaError_t e = set_smem(reinterpret_cast<const void*>(fn), L.smem, true);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long ntiles = (ncol + kTileM - 1) / kTileM;
  long long cpp = std::min<long long>(ntiles, sms / L.nparts);
  if (cpp < 1) cpp = 1;
  OzArgs a;
  a.pack = static_cast<const uint8_t*>(pack);
  a.r = r;
  a.Kp = L.Kp;
  a.nparts = L.nparts;
  for (int p = 0; p < 2; ++p) {
    a.Nw[p] = p < L.nparts ? L.Nw[p] : 0;
    a.n0[p] = p < L.nparts ? L.n0[p] : 0;
    a.off[p] = p < L.nparts ? L.off[p] : 0;
  }
  a.rexp_off = L.rexp_off;
  a.in = static_cast<const dfc*>(in);
  a.out = out;
  a.ncol = ncol;
  a.err = err;
  a.wait_limit = wait_limit >= 0 ? wait_limit : tc::kWaitLimit;
  a.colscale = colscale;
  fn<<<static_cast<unsigned>(cpp * L.nparts), kWorkers + 32, L.smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace qa
