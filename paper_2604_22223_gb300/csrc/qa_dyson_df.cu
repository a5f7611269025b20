// Screened interaction on the accurate mixed path (paper Eq. for W):
// W^C = (1 - S P)^-1 S P S per (q, i nu) with P and S(q) given in double-float,
// as an FP32 solve refined by one double-float residual step (mixed-precision
// iterative refinement):
//   1. A = 1 - S P and B = S P S from the FP32 high parts; Gauss-Jordan
//      elimination of [A | B] with partial pivoting in FP32 gives X0 and
//      leaves each lane its elimination multipliers;
//   2. R = B - A X0 = M Y - X0 with M = S P (double-float) and Y = S + X0,
//      the n^3 product M Y on the tensor cores from exact fixed-point bf16
//      slices (warp-level MMA), its levels added in double-float;
//   3. delta = A^-1 R by replaying the recorded elimination on R in FP32;
//   4. X1 = X0 + delta as a double-float.
// One step takes the FP32 error cond(A) u to (cond(A) u)^2.  S is block
// diagonal on the reduced pair basis (the interaction's connected pair
// components); its rows are kept compactly (BW entries from lo[i]).
//
// Layout: 16 lanes per system (lane i = row i), two systems per warp, four
// warps per block over 8 consecutive q at one nu; the tiles sit in shared
// memory and move to and from HBM in coalesced runs along q.
#include "qa_common.cuh"

namespace qa {
namespace {

constexpr int kDfLanes = 16;
constexpr int kDfWarps = 4;
constexpr int kDfSys = kDfWarps * 32 / kDfLanes;      // systems per block
constexpr int kPS = 17;                               // padded row stride of the 16-wide tiles
// per-system strides of the shared tiles, padded so that the same entry of
// consecutive systems (the coalesced tile loads and stores, and the two
// systems of a warp) falls in different banks
constexpr int kSysP = kDfLanes * kPS + 1;             // P / Z / X1 tile, dfc
constexpr int kSysX = kDfLanes * kPS + 2;             // X0 tile, float2
constexpr int kSysR = 4 * kDfLanes + 2;               // pivot rows, float2

__device__ void report_df(int* err, long long* first_bad, int code, long long idx) {
  atomicCAS(err, 0, code);
  if (first_bad) atomicMin(reinterpret_cast<unsigned long long*>(first_bad),
                           static_cast<unsigned long long>(idx));
}

// double-float accumulator with an unnormalised low part: value = s + e
struct DfAcc {
  float s, e;
};
__device__ __forceinline__ void acc_add(DfAcc& a, float p) {
  float t;
  two_sum(a.s, p, a.s, t);
  a.e = __fadd_rn(a.e, t);
}
// a += x * y (both double-float)
__device__ __forceinline__ void acc_fma(DfAcc& a, dfl x, dfl y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float q = __fmaf_rn(x.hi, y.hi, -p);
  q = __fmaf_rn(x.hi, y.lo, q);
  q = __fmaf_rn(x.lo, y.hi, q);
  acc_add(a, p);
  a.e = __fadd_rn(a.e, q);
}
__device__ __forceinline__ dfl acc_val(const DfAcc& a) { return df_norm(a.s, a.e); }

// re/im accumulators of a complex sum
struct CAcc {
  DfAcc re, im;
};
__device__ __forceinline__ void cacc_fma(CAcc& a, dfc x, dfc y) {
  acc_fma(a.re, x.x, y.x);
  acc_fma(a.re, -x.y, y.y);
  acc_fma(a.im, x.x, y.y);
  acc_fma(a.im, x.y, y.x);
}

// a += x * y with x real (a double-float), y complex
__device__ __forceinline__ void cacc_fma(CAcc& a, dfl x, dfc y) {
  acc_fma(a.re, x, y.x);
  acc_fma(a.im, x, y.y);
}

__device__ __forceinline__ float2 hi2(dfc v) { return make_float2(v.x.hi, v.y.hi); }
// c + s b, s real
__device__ __forceinline__ float2 rfma(float s, float2 b, float2 c) {
  return make_float2(fmaf(s, b.x, c.x), fmaf(s, b.y, c.y));
}

// ---- fixed-point bf16 slices for the residual's tensor-core product
constexpr int kSl = 5;                                // slices per operand (levels 0..4)

// e with max < 2^e for a row (or column) maximum, clamped so that every grid
// constant below stays a normal float
__device__ __forceinline__ int grid_exp(float mx) {
  const int e = static_cast<int>((__float_as_uint(mx) >> 23) & 0xffu) - 126;
  return max(-60, min(e, 100));
}
// v = hi + lo cut into kSl slices: slice t is the remainder rounded to a
// multiple of 2^(e-7-8t) (adding and subtracting 1.5 * 2^(e+16-8t) rounds to
// that grid), an integer of at most 8 bits times the grid, so exact in bf16.
// The remainder stays exact as the pair (r, lo): r - s is exact because s is
// a grid multiple no coarser than r's own spacing at the scale of r.
__device__ __forceinline__ void slice_df(dfl v, int e, float (&s)[kSl]) {
  float r = v.hi;
#pragma unroll
  for (int t = 0; t < kSl; ++t) {
    const float C = __uint_as_float((static_cast<unsigned>(e + 143 - 8 * t) << 23) | 0x400000u);
    const float x = __fadd_rn(r, v.lo);
    const float c = __fsub_rn(__fadd_rn(x, C), C);
    s[t] = c;
    r = __fsub_rn(r, c);
  }
}
// two values of at most 8 significant bits as bf16x2 (exact): lo in the low half
__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  unsigned d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
// c += a b on a 16x8x16 tile (a row-major 16x16, b column-major 16x8), FP32 accumulation
__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// NFIX > 0: system size fixed at compile time.  BW: bound of the block width of S.
// RS: S(q) is real (real S(R) with S(-R) = S(R)): its products take half the work.
template <int NFIX, int BW, bool RS>
__global__ void __launch_bounds__(kDfWarps * 32, 3) dyson_w_df_kernel(
    const dfc* __restrict__ P, const dfc* __restrict__ Vq, dfc* __restrict__ WC, int n_arg, int nk,
    int* err, long long* first_bad, DysonBlocks blk, unsigned char* __restrict__ code) {
  const int n = NFIX > 0 ? NFIX : n_arg;
  constexpr int M = kDfLanes;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int kSysS = M * BW + 1;
  dfc* Pt = reinterpret_cast<dfc*>(smem_raw);                 // [sys][M][kPS]: P, then R, then X1
  dfc* Sc = Pt + kDfSys * kSysP;                               // [sys][M][BW] rows of S in their block
  float2* X0 = reinterpret_cast<float2*>(Sc + kDfSys * kSysS);   // [sys][M][kPS]
  float2* Rb = X0 + kDfSys * kSysX;                            // [sys][2][2 M] pivot rows
  const int tid = threadIdx.x, lane = tid & 31;
  const int l = lane & (M - 1);
  const int sys = tid / M;
  const int q0 = blockIdx.x * kDfSys;
  const int nu = blockIdx.y;
  const int nn = n * n;
  const size_t slab = static_cast<size_t>(nu) * nn * nk;
  // block bounds of row i of S (the whole row when no block structure is known)
  auto blo = [&](int i) { return blk.nblk > 0 ? static_cast<int>(blk.lo[i]) : 0; };
  auto bhi = [&](int i) { return blk.nblk > 0 ? static_cast<int>(blk.hi[i]) : n; };
  // ---- tiles: P (coalesced along q), rows of S
  for (int idx = tid; idx < kDfSys * M * M; idx += blockDim.x) {
    const int ss = idx % kDfSys, e = idx / kDfSys;
    const int i = e / M, j = e - i * M;
    const int q = q0 + ss;
    dfc v = dfc{dfl(0.f, 0.f), dfl(0.f, 0.f)};
    if (i < n && j < n && q < nk) v = ldg_c(P + slab + static_cast<size_t>(i * n + j) * nk + q);
    Pt[ss * kSysP + i * kPS + j] = v;
  }
  for (int idx = tid; idx < kDfSys * M * BW; idx += blockDim.x) {
    const int ss = idx / (M * BW), e = idx - ss * (M * BW);
    const int i = e / BW, t = e - i * BW;
    const int q = q0 + ss;
    dfc v = dfc{dfl(0.f, 0.f), dfl(0.f, 0.f)};
    if (i < n && q < nk) {
      const int m = blo(i) + t;
      if (m < bhi(i)) v = ldg_c(Vq + static_cast<size_t>(q) * nn + i * n + m);
    }
    Sc[ss * kSysS + i * BW + t] = v;
  }
  __syncthreads();
  const int q = q0 + sys;
  dfc* Pw = Pt + sys * kSysP;
  const dfc* Sw = Sc + sys * kSysS;
  float2* Xw = X0 + sys * kSysX;
  float2* Rw = Rb + sys * kSysR;
  const bool row = l < n;
  const int lo_l = row ? blo(l) : 0, hi_l = row ? bhi(l) : 0;

  // ---- 1. a = row l of S P, b = row l of (S P) S, from the FP32 high parts
  float2 a[M], b[M];
#pragma unroll
  for (int j = 0; j < M; ++j) a[j] = make_float2(0.f, 0.f);
  for (int m = lo_l; m < hi_l; ++m) {
    const float2 slm = hi2(Sw[l * BW + (m - lo_l)]);
#pragma unroll
    for (int j = 0; j < M; ++j)
      if (j < n) a[j] = RS ? rfma(slm.x, hi2(Pw[m * kPS + j]), a[j]) : cfma(slm, hi2(Pw[m * kPS + j]), a[j]);
  }
#pragma unroll
  for (int j = 0; j < M; ++j) b[j] = make_float2(0.f, 0.f);
#pragma unroll
  for (int m = 0; m < M; ++m) {
    if (m < n) {
      const int lo_m = blo(m), hi_m = bhi(m);
#pragma unroll
      for (int k = 0; k < M; ++k)
        if (k >= lo_m && k < hi_m)
          b[k] = RS ? rfma(Sw[m * BW + (k - lo_m)].x.hi, a[m], b[k]) : cfma(a[m], hi2(Sw[m * BW + (k - lo_m)]), b[k]);
    }
  }
#pragma unroll
  for (int j = 0; j < M; ++j) {
    a[j].x = (row && j == l ? 1.f : 0.f) - a[j].x;
    a[j].y = -a[j].y;
  }

  // ---- Gauss-Jordan on [A | B] in FP32, recording each lane's multipliers
  bool used = !row;
  int mypos = -1;
  float2 dval = make_float2(1.f, 0.f);
  bool singular = false;
  float2 frec[M];
#pragma unroll
  for (int j = 0; j < M; ++j) frec[j] = make_float2(0.f, 0.f);
  // with a compile-time size the column loop is unrolled (every register index
  // and predicate a constant); otherwise it stays rolled and the register arrays
  // are indexed by c through compile-time selects
#pragma unroll(NFIX > 0 ? NFIX : 1)
  for (int c = 0; c < n; ++c) {
    float2* Ra_c = Rw + (c & 1) * 2 * M;
    float2* Rb_c = Ra_c + M;
    float2 ac = a[0];
#pragma unroll
    for (int j = 1; j < M; ++j)
      if (j == c) ac = a[j];
    const float v2 = cabs2(ac);
    unsigned key = used ? 0u : (max(__float_as_uint(v2) & ~0xFu, 0x10u) | (M - 1 - l));
#pragma unroll
    for (int o = M / 2; o > 0; o >>= 1) key = max(key, __shfl_xor_sync(0xffffffffu, key, o));
    const int p = M - 1 - static_cast<int>(key & (M - 1));
    if (!(__uint_as_float(key & ~0xFu) >= 1e-12f)) singular = true;
    const bool me = (l == p);
    if (me) {
      used = true;
      mypos = c;
      dval = ac;
#pragma unroll
      for (int j = 0; j < M; ++j) {
        if (j >= c) Ra_c[j] = a[j];
        Rb_c[j] = b[j];
      }
    }
    __syncwarp();
    const float2 apc = Ra_c[c];
    const float2 f = me ? make_float2(0.f, 0.f) : cmul(ac, cinv(apc));
#pragma unroll
    for (int j = 0; j < M; ++j)
      if (j == c) frec[j] = f;
#pragma unroll
    for (int j = 0; j < M; ++j) {
      if (j > c && j < n) a[j] = cfms(f, Ra_c[j], a[j]);
      if (j < n) b[j] = cfms(f, Rb_c[j], b[j]);
    }
  }
  // X0: row mypos of the FP32 solution
  if (mypos >= 0) {
    const float2 inv = cinv(dval);
#pragma unroll
    for (int j = 0; j < M; ++j) Xw[mypos * kPS + j] = j < n ? cmul(b[j], inv) : make_float2(0.f, 0.f);
  }
  __syncwarp();

  // ---- 2. residual R = B - A X0 = M Y - X0 with M = S P and Y = S + X0, on the
  // tensor cores.  M and Y are formed in double-float straight into the
  // register layout of the warp-level MMA (m16n8k16: bf16 operands, FP32
  // accumulation) and cut into kSl bf16 slices on a fixed-point grid per row of
  // M and per column of Y (slice t of a row with |M| < 2^e is a multiple of
  // 2^(e-7-8t) with at most 8 significant bits; Ozaki, Ogita, Oishi & Rump 2012).
  // Each slice product is exact and every level sum (slice indices t + u = L)
  // stays below 2^22 units of its grid, so the tensor core's FP32
  // accumulation of a level is exact; the levels are added in double-float.
  // The warp's two systems go through this one after the other on all 32
  // lanes; R lands in the system's P tile (P is not needed after M).
  __syncwarp();
  {
    const int g = lane >> 2, t4 = lane & 3;
    const int wsys = (tid >> 5) * 2;
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      const int ss = wsys + h;
      const dfc* Ps = Pt + ss * kSysP;
      const dfc* Ss = Sc + ss * kSysS;
      const float2* Xs = X0 + ss * kSysX;
      float2* Rt = reinterpret_cast<float2*>(Pt + ss * kSysP);
      // A operand: M at rows g, g + 8 and columns 2 t4 + {0, 1}, 2 t4 + {8, 9}
      unsigned ar[kSl][4], ai[kSl][4];
      {
        dfc me[2][4];
        float mx[2] = {0.f, 0.f};
#pragma unroll
        for (int rh = 0; rh < 2; ++rh) {
          const int row = g + 8 * rh;
          const int lo_r = row < n ? blo(row) : 0, hi_r = row < n ? bhi(row) : 0;
#pragma unroll
          for (int ci = 0; ci < 4; ++ci) {
            const int col = 2 * t4 + (ci & 1) + 8 * (ci >> 1);
            CAcc z = CAcc{{0.f, 0.f}, {0.f, 0.f}};
            if (col < n)
              for (int m = lo_r; m < hi_r; ++m) {
                if (RS)
                  cacc_fma(z, Ss[row * BW + (m - lo_r)].x, Ps[m * kPS + col]);
                else
                  cacc_fma(z, Ss[row * BW + (m - lo_r)], Ps[m * kPS + col]);
              }
            me[rh][ci] = dfc{acc_val(z.re), acc_val(z.im)};
            mx[rh] = fmaxf(mx[rh], fmaxf(fabsf(me[rh][ci].x.hi), fabsf(me[rh][ci].y.hi)));
          }
        }
        int er[2];
#pragma unroll
        for (int rh = 0; rh < 2; ++rh) {
          mx[rh] = fmaxf(mx[rh], __shfl_xor_sync(0xffffffffu, mx[rh], 1));
          mx[rh] = fmaxf(mx[rh], __shfl_xor_sync(0xffffffffu, mx[rh], 2));
          er[rh] = grid_exp(mx[rh]);
        }
#pragma unroll
        for (int qr = 0; qr < 4; ++qr) {
          const int rh = qr & 1, c0 = (qr >> 1) * 2;
          float s0[kSl], s1[kSl];
          slice_df(me[rh][c0].x, er[rh], s0);
          slice_df(me[rh][c0 + 1].x, er[rh], s1);
#pragma unroll
          for (int t = 0; t < kSl; ++t) ar[t][qr] = pack_bf16(s0[t], s1[t]);
          slice_df(me[rh][c0].y, er[rh], s0);
          slice_df(me[rh][c0 + 1].y, er[rh], s1);
#pragma unroll
          for (int t = 0; t < kSl; ++t) ai[t][qr] = pack_bf16(s0[t], s1[t]);
        }
      }
      __syncwarp();                       // every lane has read P: R may overwrite it
#pragma unroll 1
      for (int nt = 0; nt < 2; ++nt) {
        // B operand: Y at rows 2 t4 + {0, 1}, 2 t4 + {8, 9} and column g + 8 nt
        const int col = g + 8 * nt;
        unsigned br[kSl][2], bi[kSl][2];
        {
          dfc ye[4];
          float my = 0.f;
#pragma unroll
          for (int ri = 0; ri < 4; ++ri) {
            const int j = 2 * t4 + (ri & 1) + 8 * (ri >> 1);
            dfc y = dfc{dfl(0.f, 0.f), dfl(0.f, 0.f)};
            if (j < n && col < n) {
              const float2 x0 = Xs[j * kPS + col];
              const int lo_j = blo(j), hi_j = bhi(j);
              dfc sv = dfc{dfl(0.f, 0.f), dfl(0.f, 0.f)};
              if (col >= lo_j && col < hi_j) sv = Ss[j * BW + (col - lo_j)];
              float s, e;
              two_sum(x0.x, sv.x.hi, s, e);
              y.x = df_norm(s, __fadd_rn(e, sv.x.lo));
              two_sum(x0.y, sv.y.hi, s, e);
              y.y = df_norm(s, __fadd_rn(e, sv.y.lo));
            }
            ye[ri] = y;
            my = fmaxf(my, fmaxf(fabsf(y.x.hi), fabsf(y.y.hi)));
          }
          my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, 1));
          my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, 2));
          const int ey = grid_exp(my);
#pragma unroll
          for (int qr = 0; qr < 2; ++qr) {
            float s0[kSl], s1[kSl];
            slice_df(ye[2 * qr].x, ey, s0);
            slice_df(ye[2 * qr + 1].x, ey, s1);
#pragma unroll
            for (int t = 0; t < kSl; ++t) br[t][qr] = pack_bf16(s0[t], s1[t]);
            slice_df(ye[2 * qr].y, ey, s0);
            slice_df(ye[2 * qr + 1].y, ey, s1);
#pragma unroll
            for (int t = 0; t < kSl; ++t) bi[t][qr] = pack_bf16(s0[t], s1[t]);
          }
        }
        // level sums: re = Mr Yr - Mi Yi, im = Mr Yi + Mi Yr
        float acc[kSl][2][4];
#pragma unroll
        for (int L = 0; L < kSl; ++L)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[L][0][c] = acc[L][1][c] = 0.f;
#pragma unroll
        for (int t = 0; t < kSl; ++t) {
          unsigned nai[4];
#pragma unroll
          for (int qr = 0; qr < 4; ++qr) nai[qr] = ai[t][qr] ^ 0x80008000u;
#pragma unroll
          for (int u = 0; u + t < kSl; ++u) {
            mma_bf16(acc[t + u][0], ar[t], br[u][0], br[u][1]);
            mma_bf16(acc[t + u][0], nai, bi[u][0], bi[u][1]);
            mma_bf16(acc[t + u][1], ar[t], bi[u][0], bi[u][1]);
            mma_bf16(acc[t + u][1], ai[t], br[u][0], br[u][1]);
          }
        }
        // R = (sum of the levels) - X0 at rows g, g + 8 and columns 2 t4 + {0, 1} + 8 nt
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int row = g + 8 * (c >> 1), k = 2 * t4 + (c & 1) + 8 * nt;
          float2 rv = make_float2(0.f, 0.f);
          if (row < n && k < n) {
            const float2 x0 = Xs[row * kPS + k];
            float v[2];
#pragma unroll
            for (int p = 0; p < 2; ++p) {
              float s = acc[0][p][c], e = 0.f, tt;
#pragma unroll
              for (int L = 1; L < kSl; ++L) {
                two_sum(s, acc[L][p][c], s, tt);
                e = __fadd_rn(e, tt);
              }
              const dfl z = df_norm(s, e);
              v[p] = __fadd_rn(__fsub_rn(z.hi, p ? x0.y : x0.x), z.lo);
            }
            rv = make_float2(v[0], v[1]);
          }
          Rt[row * kPS + k] = rv;
        }
      }
    }
  }
  __syncwarp();
  float2 rres[M];
  {
    const float2* Rt = reinterpret_cast<const float2*>(Pw);
#pragma unroll
    for (int k = 0; k < M; ++k) rres[k] = (row && k < n) ? Rt[l * kPS + k] : make_float2(0.f, 0.f);
  }
  __syncwarp();

  // ---- 3. delta = A^-1 R: the recorded elimination replayed on R (rolled: the
  // instruction cache holds the unrolled elimination above)
#pragma unroll 1
  for (int c = 0; c < n; ++c) {
    float2* Rr = Rw + (c & 1) * 2 * M;
    if (mypos == c) {
#pragma unroll
      for (int j = 0; j < M; ++j) Rr[j] = rres[j];
    }
    __syncwarp();
    float2 f = frec[0];
#pragma unroll
    for (int j = 1; j < M; ++j)
      if (j == c) f = frec[j];
#pragma unroll
    for (int j = 0; j < M; ++j)
      if (j < n) rres[j] = cfms(f, Rr[j], rres[j]);
  }
  __syncwarp();
  // ---- 4. X1 = X0 + delta (row mypos), into the P/Z tile
  if (mypos >= 0) {
    const float2 inv = cinv(dval);
#pragma unroll
    for (int j = 0; j < M; ++j) {
      if (j < n) {
        const float2 d = cmul(rres[j], inv);
        const float2 x0 = Xw[mypos * kPS + j];
        float s, e;
        two_sum(x0.x, d.x, s, e);
        const dfl re = df_norm(s, e);
        two_sum(x0.y, d.y, s, e);
        const dfl im = df_norm(s, e);
        Pw[mypos * kPS + j] = dfc{re, im};
      }
    }
  }
  if (singular && l == 0 && q < nk)
    report_df(err, first_bad, QA_ESINGULAR_CODE, static_cast<long long>(nu) * nk + q);
  __syncthreads();
  for (int idx = tid; idx < kDfSys * nn; idx += blockDim.x) {
    const int ss = idx % kDfSys, e = idx / kDfSys;
    const int i = e / n, j = e - i * n;
    const int qq = q0 + ss;
    if (qq < nk) {
      const dfc v = Pt[ss * kSysP + i * kPS + j];
      const size_t o = slab + static_cast<size_t>(e) * nk + qq;
      reinterpret_cast<float4*>(WC)[o] = make_float4(v.x.hi, v.x.lo, v.y.hi, v.y.lo);
      if (code) code[o] = static_cast<unsigned char>(oz_grid_code(v));
    }
  }
}

template <int NFIX, int BW, bool RS>
cudaError_t launch_df(const void* P, const void* Vq, void* WC, int r, int n, int nk, int* err,
                      long long* first_bad, cudaStream_t st, const DysonBlocks& blk, unsigned char* code) {
  constexpr int M = kDfLanes;
  const size_t smem = static_cast<size_t>(kDfSys) * kSysP * sizeof(dfc) +
                      static_cast<size_t>(kDfSys) * (M * BW + 1) * sizeof(dfc) +
                      static_cast<size_t>(kDfSys) * kSysX * sizeof(float2) +
                      static_cast<size_t>(kDfSys) * kSysR * sizeof(float2);
  auto fn = &dyson_w_df_kernel<NFIX, BW, RS>;
  cudaError_t e = set_smem(reinterpret_cast<const void*>(fn), smem, true);
  if (e != cudaSuccess) return e;
  dim3 grid((nk + kDfSys - 1) / kDfSys, r);
  fn<<<grid, kDfWarps * 32, smem, st>>>(static_cast<const dfc*>(P), static_cast<const dfc*>(Vq),
                                        static_cast<dfc*>(WC), n, nk, err, first_bad, blk, code);
  return cudaGetLastError();
}

}  // namespace

bool dyson_w_df_supported(int n) { return n >= 1 && n <= kDfLanes; }

cudaError_t launch_dyson_w_df(const void* P, const void* Vq, void* WC, int r, int n, int nk,
                              int* err, long long* first_bad, cudaStream_t st,
                              const DysonBlocks* blk, bool real_s, unsigned char* code) {
  if (!dyson_w_df_supported(n) || P == WC) return cudaErrorInvalidValue;
  DysonBlocks b = blk ? *blk : DysonBlocks{};
  int bw = 0;
  for (int i = 0; i < n && b.nblk > 0; ++i) bw = max(bw, static_cast<int>(b.hi[i]) - static_cast<int>(b.lo[i]));
  if (b.nblk > 0 && bw <= 5) {
    if (n == 15)
      return real_s ? launch_df<15, 5, true>(P, Vq, WC, r, n, nk, err, first_bad, st, b, code)
                    : launch_df<15, 5, false>(P, Vq, WC, r, n, nk, err, first_bad, st, b, code);
    return launch_df<0, 5, false>(P, Vq, WC, r, n, nk, err, first_bad, st, b, code);
  }
  b.nblk = 0;
  return launch_df<0, kDfLanes, false>(P, Vq, WC, r, n, nk, err, first_bad, st, b, code);
}

}  // namespace qa
