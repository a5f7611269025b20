// DLR node transforms of the big tensors on the 5th-generation tensor cores
// (tcgen05, sm_103a), FP32 data with split-bf16 operands and FP32 accumulation.
//
// The complex transform out[j][c] = sum_l T[j][l] in[l][c] of every column c
// is one real GEMM  Y (cols x 2r) = X (cols x 2r) * Tt^T (2r x 2r), where
// X[c][(l,re/im)] are the interleaved input values and Tt is the real
// embedding [[Re T, -Im T], [Im T, Re T]] of T.  Every operand is split into
// three bf16 pieces (x = x0 + x1 + x2, ~24 significant bits) and the six
// leading cross products x_i t_j (i + j <= 2) accumulate in FP32 in tensor
// memory, which keeps the FP32-level accuracy of the SIMT kernel.
//
// One persistent CTA per SM, warp-specialised (16 worker warps and one MMA
// issuer warp, synchronised only through mbarriers): the three Tt pieces stay
// resident in shared memory (K-major canonical layout, no swizzle); each
// 128-column tile of X streams through double-buffered K-chunks of 16 (8 nodes
// x re/im) that the workers convert to bf16 pieces while the previous chunk's
// six MMAs run; one thread issues tcgen05.mma (M = 128, N = 2r padded to 16,
// K = 16) into a 128 x N FP32 accumulator in TMEM; the workers read it back
// with tcgen05.ld (warps w, w+4, w+8, w+12 <-> TMEM lanes 32w..32w+31, thread
// <-> column, each warp a quarter of the accumulator columns) and store Y in
// place of X.  The input is read through a register ring several chunks deep.
// Every mbarrier wait is bounded; on time-out the kernel records QA_ETIMEOUT,
// waits (bounded) for its own MMAs, frees TMEM and returns.
#include <cuda_bf16.h>

#include <cstring>
#include <vector>

#include "qa_common.cuh"

namespace qa {
namespace {

constexpr int kTcThreads = 128;
constexpr int kTileM = 128;
constexpr int kChunkK = 16;
constexpr uint32_t kTmemCols = 256;
constexpr long long kWaitLimit = 1ll << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait; returns false on time-out
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long long i = 0; i < kWaitLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// shared-memory matrix descriptor: K-major, no swizzle; LBO = byte stride of
// core matrices along K, SBO = byte stride along M/N (core = 8 rows x 16 B)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((addr >> 4) & 0x3FFF);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFF) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFF) << 32;
  d |= 1ull << 46;                                  // descriptor version for tcgen05
  return d;                                         // base offset 0, swizzle none
}

// instruction descriptor: kind::f16 with BF16 A/B, FP32 D, both K-major
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t taddr, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(taddr),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void split3(float x, uint16_t& h0, uint16_t& h1, uint16_t& h2) {
  __nv_bfloat16 b0 = __float2bfloat16_rn(x);
  float r1 = x - __bfloat162float(b0);
  __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
  float r2 = r1 - __bfloat162float(b1);
  __nv_bfloat16 b2 = __float2bfloat16_rn(r2);
  h0 = __bfloat16_as_ushort(b0);
  h1 = __bfloat16_as_ushort(b1);
  h2 = __bfloat16_as_ushort(b2);
}

struct TcArgs {
  const uint4* Bsplit;   // 3 pieces x Np x Kp bf16 in the canonical layout
  int Np, Kp, r;
  const float2* in;
  float2* out;
  double2* out64;          // when set, the result is stored here as complex128 instead
  long long ncol;
  int* err;
  long long wait_limit;    // polls of each pipeline wait before the time-out path
};

// acc[0..23] += the 24 TMEM columns at taddr (this thread's lane), rounded to
// nearest: three x8 loads (column offsets multiples of 8), one wait and the
// adds in one block (only 24 temporaries live beside the accumulators)
__device__ __forceinline__ void tmem_acc24(uint32_t taddr, float* acc) {
  asm volatile(
      "{\n\t.reg .b32 t0, t1, t2, t3, t4, t5, t6, t7, t8, t9, t10, t11, t12, t13, t14, t15, t16, t17, t18, t19, t20, t21, t22, t23;\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {t0, t1, t2, t3, t4, t5, t6, t7}, [%24];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {t8, t9, t10, t11, t12, t13, t14, t15}, [%25];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {t16, t17, t18, t19, t20, t21, t22, t23}, [%26];\n\t"
      "tcgen05.wait::ld.sync.aligned;\n\t"
      "add.rn.f32 %0, %0, t0;\n\tadd.rn.f32 %1, %1, t1;\n\tadd.rn.f32 %2, %2, t2;\n\tadd.rn.f32 %3, %3, t3;\n\tadd.rn.f32 %4, %4, t4;\n\tadd.rn.f32 %5, %5, t5;\n\tadd.rn.f32 %6, %6, t6;\n\tadd.rn.f32 %7, %7, t7;\n\tadd.rn.f32 %8, %8, t8;\n\tadd.rn.f32 %9, %9, t9;\n\tadd.rn.f32 %10, %10, t10;\n\tadd.rn.f32 %11, %11, t11;\n\tadd.rn.f32 %12, %12, t12;\n\tadd.rn.f32 %13, %13, t13;\n\tadd.rn.f32 %14, %14, t14;\n\tadd.rn.f32 %15, %15, t15;\n\tadd.rn.f32 %16, %16, t16;\n\tadd.rn.f32 %17, %17, t17;\n\tadd.rn.f32 %18, %18, t18;\n\tadd.rn.f32 %19, %19, t19;\n\tadd.rn.f32 %20, %20, t20;\n\tadd.rn.f32 %21, %21, t21;\n\tadd.rn.f32 %22, %22, t22;\n\tadd.rn.f32 %23, %23, t23;\n\t}"
      : "+f"(acc[0]), "+f"(acc[1]), "+f"(acc[2]), "+f"(acc[3]), "+f"(acc[4]), "+f"(acc[5]), "+f"(acc[6]), "+f"(acc[7]), "+f"(acc[8]), "+f"(acc[9]), "+f"(acc[10]), "+f"(acc[11]), "+f"(acc[12]), "+f"(acc[13]), "+f"(acc[14]), "+f"(acc[15]), "+f"(acc[16]), "+f"(acc[17]), "+f"(acc[18]), "+f"(acc[19]), "+f"(acc[20]), "+f"(acc[21]), "+f"(acc[22]), "+f"(acc[23])
      : "r"(taddr), "r"(taddr + 8u), "r"(taddr + 16u)
      : "memory");
}

constexpr int kQMax = 48;               // accumulator columns per worker thread (Np <= 192)
constexpr int kDepth = 2;               // K-chunks of input in flight per worker (registers)
constexpr int kPrefetch = 16;            // further K-chunks requested into L2 ahead of the ring
constexpr int kWorkers = 4 * kTcThreads;   // 16 worker warps; warp 16 issues the MMAs

// bounded wait (lim polls) that also gives up once another thread has flagged an abort
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity,
                                                   volatile int* abort_flag, long long lim) {
  for (long long i = 0; i < lim; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 1023) == 1023 && *abort_flag) return false;
  }
  return false;
}

// Warp-specialised: worker thread (w < 16, lane) owns TMEM lane / tile row
// m = 32 (w % 4) + lane and quarter qt = w / 4 of the work of that row:
// accumulator columns [48 qt, 48 qt + 48) and nodes 2 qt, 2 qt + 1 of each
// chunk's 8.  For chunk g (this CTA's chunks numbered across its tiles) the
// workers stage the bf16 pieces of X into buffer g % 2 and arrive on full[g % 2];
// the issuer (one thread of warp 16) waits for it, issues the six MMAs into the
// fresh accumulator g % 2 and commits to done[g % 2]; the workers wait on
// done[(g-1) % 2] and drain chunk g-1 into FP32 registers with round-to-nearest
// adds while chunk g runs, so the tensor core never sums more than 96 products.
// No block-wide barrier inside the stream: the issuer never waits on the
// drains of other chunks, and the workers never wait on the MMA issue.
// Buffer and accumulator reuse: chunk g is staged only after each worker has
// waited for chunk g-2's MMAs and drained it, and full[g % 2] completes only
// when every worker warp has arrived for chunk g.
template <bool OUT64>
__global__ void __launch_bounds__(kWorkers + 32, 1) dlr_tc_kernel(TcArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bpiece = static_cast<uint32_t>(a.Np) * a.Kp * 2;    // bytes of one Tt piece
  uint8_t* Bs = smem;
  uint8_t* As = smem + 3 * bpiece;                                    // [2 buffers][3 pieces][4096 B]
  uint64_t* done = reinterpret_cast<uint64_t*>(As + 2 * 3 * kTileM * kChunkK * 2);
  uint64_t* full = done + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(full + 2);
  __shared__ int s_abort;
  __shared__ long long s_issued;

  for (uint32_t i = tid; i < 3 * bpiece / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(Bs)[i] = a.Bsplit[i];
  if (tid == 0) {
    mbar_init(&done[0], 1);
    mbar_init(&done[1], 1);
    mbar_init(&full[0], kWorkers / 32);
    mbar_init(&full[1], kWorkers / 32);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
    s_issued = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(2 * kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  volatile int* abort_flag = &s_abort;
  const uint32_t taddr = *tslot;
  const int nchunk = a.Kp / kChunkK;
  const long long ntiles = (a.ncol + kTileM - 1) / kTileM;
  const long long my_tiles = blockIdx.x < ntiles ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const long long nstream = my_tiles * nchunk;       // this CTA's chunks, tile after tile

  if (warp == kWorkers / 32) {
    // ---- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = instr_desc(kTileM, a.Np);
      const uint32_t bsbo = static_cast<uint32_t>(a.Kp / 8) * 128;
      const int pa[6] = {0, 0, 1, 0, 1, 2};
      const int pb[6] = {0, 1, 0, 2, 1, 0};
      int ch = 0;
      long long g = 0;
      for (; g < nstream; ++g) {
        const int b = static_cast<int>(g & 1);
        if (!mbar_wait_or_abort(&full[b], static_cast<uint32_t>((g >> 1) & 1), abort_flag, a.wait_limit)) {
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t dcol = static_cast<uint32_t>(b) * kTmemCols;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const uint32_t aaddr = smem_u32(As + (b * 3 + pa[q]) * (kTileM * kChunkK * 2));
          const uint32_t baddr = smem_u32(Bs + pb[q] * bpiece) + static_cast<uint32_t>(ch) * 256;
          mma_bf16(taddr + dcol, smem_desc(aaddr, 128, 256), smem_desc(baddr, 128, bsbo), idesc,
                   q > 0 ? 1u : 0u);
        }
        mma_commit(&done[b]);
        if (++ch == nchunk) ch = 0;
      }
      s_issued = g;
    }
    __syncwarp();
  } else {
    // ---- workers
    const int m = 32 * (warp & 3) + lane;
    const int qt = warp >> 2;
    const int nodes = a.r;
    const int cb = kQMax * qt;                       // first accumulator column of this thread
    const int nq = a.Np - cb < kQMax ? a.Np - cb : kQMax;   // its column count (may be <= 0)
    const uint32_t lane_base = static_cast<uint32_t>(32 * (warp & 3)) << 16;
    const uint32_t roff = static_cast<uint32_t>(m >> 3) * 256 + static_cast<uint32_t>(m & 7) * 16 +
                          static_cast<uint32_t>(qt >> 1) * 128 + static_cast<uint32_t>(qt & 1) * 8;
    // prefetch stream position (tile, chunk), advanced once per load
    long long pf_tile = blockIdx.x, pf_s = 0;
    int pf_ch = 0;
    auto load_next = [&](float2* dst) {
      const long long col = pf_tile * kTileM + m;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int l = pf_ch * 8 + qt * 2 + e;
        dst[e] = (pf_s < nstream && col < a.ncol && l < nodes)
                     ? a.in[static_cast<long long>(l) * a.ncol + col] : make_float2(0.f, 0.f);
      }
      ++pf_s;
      if (++pf_ch == nchunk) { pf_ch = 0; pf_tile += gridDim.x; }
    };
    // L2 prefetch cursor kPrefetch chunks ahead of the register ring (no
    // registers held): deepens the loads in flight from HBM
    long long pp_tile = blockIdx.x, pp_s = 0;
    int pp_ch = 0;
    auto prefetch_next = [&]() {
      const long long col = pp_tile * kTileM + m;
      if (pp_s < nstream && col < a.ncol) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int l = pp_ch * 8 + qt * 2 + e;
          if (l < nodes)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(a.in + static_cast<long long>(l) * a.ncol + col));
        }
      }
      ++pp_s;
      if (++pp_ch == nchunk) { pp_ch = 0; pp_tile += gridDim.x; }
    };
    for (int d = 0; d < kDepth + kPrefetch; ++d) prefetch_next();
    float2 ring[kDepth][2];
#pragma unroll
    for (int d = 0; d < kDepth; ++d) load_next(ring[d]);
    auto drain = [&](long long gd, float* acc) {
      const uint32_t dcol = static_cast<uint32_t>((gd & 1) * kTmemCols + cb);
#pragma unroll
      for (int c24 = 0; c24 < kQMax / 24; ++c24)
        if (c24 * 24 < nq) tmem_acc24(taddr + lane_base + dcol + static_cast<uint32_t>(c24 * 24), acc + c24 * 24);
      tc_fence_before();
    };
    long long g = 0;
    bool ok = true;
    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      const long long col = tile * kTileM + m;
      const bool colok = col < a.ncol;
      float acc[kQMax];
#pragma unroll
      for (int i = 0; i < kQMax; ++i) acc[i] = 0.f;
      for (int ch = 0; ch < nchunk; ++ch, ++g) {
        const int b = static_cast<int>(g & 1);
        const float2 c0 = ring[0][0], c1 = ring[0][1];
#pragma unroll
        for (int d = 0; d + 1 < kDepth; ++d) { ring[d][0] = ring[d + 1][0]; ring[d][1] = ring[d + 1][1]; }
        load_next(ring[kDepth - 1]);
        prefetch_next();
        uint16_t h[3][4];
        split3(c0.x, h[0][0], h[1][0], h[2][0]);
        split3(c0.y, h[0][1], h[1][1], h[2][1]);
        split3(c1.x, h[0][2], h[1][2], h[2][2]);
        split3(c1.y, h[0][3], h[1][3], h[2][3]);
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          uint2 v;
          v.x = h[p][0] | (static_cast<uint32_t>(h[p][1]) << 16);
          v.y = h[p][2] | (static_cast<uint32_t>(h[p][3]) << 16);
          *reinterpret_cast<uint2*>(As + (b * 3 + p) * (kTileM * kChunkK * 2) + roff) = v;
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full[b])) : "memory");
        if (ch > 0) {
          const bool w = mbar_wait_or_abort(&done[(g - 1) & 1], static_cast<uint32_t>(((g - 1) >> 1) & 1), abort_flag, a.wait_limit);
          if (__any_sync(0xffffffffu, !w)) {          // warp-uniform exit
            *abort_flag = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          if (nq > 0) drain(g - 1, acc);
        }
      }
      if (!ok) break;
      const bool w = mbar_wait_or_abort(&done[(g - 1) & 1], static_cast<uint32_t>(((g - 1) >> 1) & 1), abort_flag, a.wait_limit);
      if (__any_sync(0xffffffffu, !w)) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      if (nq > 0) drain(g - 1, acc);                   // the tile's last chunk
      if (colok) {
#pragma unroll
        for (int i = 0; i < kQMax; i += 2) {
          const int j = (cb + i) >> 1;
          if (i < nq && j < nodes)
          {
            const long long o = static_cast<long long>(j) * a.ncol + col;
            if (OUT64) a.out64[o] = make_double2(acc[i], acc[i + 1]);
            else a.out[o] = make_float2(acc[i], acc[i + 1]);
          }
        }
      }
    }
  }
  __syncthreads();
  if (tid == 0 && *abort_flag) {
    atomicCAS(a.err, 0, QA_ETIMEOUT_CODE);
    // let this CTA's own MMAs finish (bounded) before TMEM is released
    const long long gl = s_issued - 1;
    if (gl >= 0) mbar_wait(&done[gl & 1], static_cast<uint32_t>((gl >> 1) & 1));
  }
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                 "r"(2 * kTmemCols)
                 : "memory");
}

uint16_t bf16_rn(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7F800000u) == 0x7F800000u) return static_cast<uint16_t>(u >> 16);   // inf / nan
  uint32_t rounding = 0x7FFFu + ((u >> 16) & 1u);
  return static_cast<uint16_t>((u + rounding) >> 16);
}
double bf16_val(uint16_t h) {
  uint32_t u = static_cast<uint32_t>(h) << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

}  // namespace

bool dlr_tc_supported(int r, size_t* smem_bytes) {
  const int Kp = ((2 * r + 15) / 16) * 16;
  const size_t bytes = 3ull * Kp * Kp * 2 + 2ull * 3 * kTileM * kChunkK * 2 + 4 * 8 + 16;
  if (smem_bytes) *smem_bytes = bytes;
  return Kp <= 192 && bytes <= 227 * 1024;
}

// Real embedding of the complex r x r matrix T, split into three bf16 pieces,
// laid out K-major (n = output index 2j + c', k = input index 2l + c) in the
// canonical no-swizzle core-matrix order.  dst has 3 * Kp * Kp uint16 entries.
void pack_dlr_tc(const std::complex<double>* T, int r, std::vector<uint16_t>* dst) {
  const int Kp = ((2 * r + 15) / 16) * 16, Np = Kp;
  dst->assign(3ull * Np * Kp, 0);
  for (int n = 0; n < 2 * r; ++n)
    for (int k = 0; k < 2 * r; ++k) {
      const int j = n >> 1, cp = n & 1, l = k >> 1, c = k & 1;
      const std::complex<double> t = T[static_cast<size_t>(j) * r + l];
      double x;
      if (cp == 0) x = c == 0 ? t.real() : -t.imag();
      else x = c == 0 ? t.imag() : t.real();
      const size_t off = static_cast<size_t>(n / 8) * (Kp / 8) * 64 + static_cast<size_t>(k / 8) * 64 +
                         static_cast<size_t>(n % 8) * 8 + (k % 8);
      double rem = x;
      for (int p = 0; p < 3; ++p) {
        uint16_t h = bf16_rn(static_cast<float>(rem));
        (*dst)[static_cast<size_t>(p) * Np * Kp + off] = h;
        rem -= bf16_val(h);
      }
    }
}

cudaError_t launch_dlr_tc(const void* Bsplit, int r, const void* in, void* out, long long ncol,
                          int* err, cudaStream_t st, bool out_c128, long long wait_limit) {
  size_t smem = 0;
  if (!dlr_tc_supported(r, &smem)) return cudaErrorInvalidValue;
  if (ncol <= 0) return cudaSuccess;
  auto fn = out_c128 ? &dlr_tc_kernel<true> : &dlr_tc_kernel<false>;
  cudaError_t e = set_smem(reinterpret_cast<const void*>(fn), smem, true);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long ntiles = (ncol + kTileM - 1) / kTileM;
  const int grid = static_cast<int>(ntiles < sms ? ntiles : sms);
  TcArgs a;
  a.Bsplit = reinterpret_cast<const uint4*>(Bsplit);
  a.Kp = ((2 * r + 15) / 16) * 16;
  a.Np = a.Kp;
  a.r = r;
  a.in = reinterpret_cast<const float2*>(in);
  a.out = out_c128 ? nullptr : reinterpret_cast<float2*>(out);
  a.out64 = out_c128 ? reinterpret_cast<double2*>(out) : nullptr;
  a.ncol = ncol;
  a.err = err;
  a.wait_limit = wait_limit >= 0 ? wait_limit : kWaitLimit;
  fn<<<grid, kWorkers + 32, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace qa
