// Batched 3-D lattice FFT in shared memory (paper Eq. for the k <-> R
// transform, which the paper evaluates with FFTs).
//
// One block owns `lpb` whole lines of N_k = N1*N2*N3 points (k fastest,
// C order over (i1, i2, i3)).  The line is staged in shared memory once,
// transformed axis by axis with in-place mixed-radix decimation-in-frequency
// stages (radices 4, 2, 3, 5, 7, ... from the host plan), and written back
// through the plan's digit-reversal tables, so each line costs one HBM read
// and one HBM write.
#include "qa_common.cuh"

namespace qa {
namespace {

constexpr int kMaxRadix = 13;
constexpr int kMaxLineTerms = 640;      // terms of one bubble output (<= npair^2 = 625)
constexpr int kFftThreads = 256;        // block size of the register-FFT kernel

// term lists of the bubble for the fused bubble + FFT lines (may be empty)
struct BubbleSrc {
  const void* GR;
  const void* GL;
  const int* mR;
  const int* terms;       // off[nout + 1] then idx[]
  const void* coef;
  int nout;
  int no2;
  int mt;                 // term capacity of the shared-memory lists (multiple of 4)
  int* err;               // error word (bounds-checked builds)
  int real_coef;          // every coefficient is real: c x y as x (c y), c y a real scaling
  unsigned char* code;    // grid codes of the stored values, like out (double-float line kernel)
};

template <typename V>
__device__ __forceinline__ V tw_get(const V* tw, int idx, int sign) {
  V w = tw[idx];
  if (sign > 0) w.y = -w.y;
  return w;
}

template <typename T>
__global__ void __launch_bounds__(512) fft3d_kernel(FftDev p, int sign, const cplx<T>* in,
                                                    cplx<T>* out, int nk, int lpb, long long nlines,
                                                    T scale) {
  using V = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* buf = reinterpret_cast<V*>(smem_raw);
  V* tws = buf + static_cast<size_t>(lpb) * nk;
  const int tid = threadIdx.x, bd = blockDim.x;
  const long long line0 = static_cast<long long>(blockIdx.x) * lpb;
  const int nl = static_cast<int>(min(static_cast<long long>(lpb), nlines - line0));
  const int ntw = p.n[0] + p.n[1] + p.n[2];
  const V* twg = reinterpret_cast<const V*>(p.tw);
  for (int i = tid; i < ntw; i += bd) tws[i] = twg[i];
  const V* src = in + line0 * nk;
  for (int i = tid; i < nl * nk; i += bd) buf[i] = src[i];
  __syncthreads();

  const int stride[3] = {p.n[1] * p.n[2], p.n[2], 1};
  for (int d = 0; d < 3; ++d) {
    const int L = p.n[d];
    if (L == 1) continue;
    const int S = stride[d];
    const V* tw = tws + p.tw_off[d];
    int Ls = L;
    for (int s = 0; s < p.nfac[d]; ++s) {
      const int rad = p.fac[d][s];
      const int Lp = Ls / rad;
      const int per_line = nk / rad;
      const int nbf = nl * per_line;
      const int nblk = L / Ls;
      const int tstep = L / Ls;        // twiddle stride for w_Ls
      const int pstep = L / rad;       // twiddle stride for w_rad
      for (int b = tid; b < nbf; b += bd) {
        int line = b / per_line;
        int rem = b - line * per_line;
        int o_lo = rem % S; rem /= S;
        int jp = rem % Lp; rem /= Lp;
        int blk = rem % nblk;
        int o_hi = rem / nblk;
        V* base = buf + static_cast<size_t>(line) * nk + static_cast<size_t>(o_hi) * L * S +
                  static_cast<size_t>(blk * Ls + jp) * S + o_lo;
        const int es = Lp * S;
        if (rad == 2) {
          V x0 = base[0], x1 = base[es];
          V y0 = cadd(x0, x1), y1 = csub(x0, x1);
          base[0] = y0;
          base[es] = cmul(y1, tw_get(tw, (jp * tstep) % L, sign));
        } else if (rad == 4) {
          V x0 = base[0], x1 = base[es], x2 = base[2 * es], x3 = base[3 * es];
          V a0 = cadd(x0, x2), a1 = csub(x0, x2), b0 = cadd(x1, x3), b1 = csub(x1, x3);
          // -i*b1 for the forward sign, +i*b1 for the inverse
          V jb1 = sign < 0 ? cmk<V>(b1.y, -b1.x) : cmk<V>(-b1.y, b1.x);
          V y0 = cadd(a0, b0), y1 = cadd(a1, jb1), y2 = csub(a0, b0), y3 = csub(a1, jb1);
          base[0] = y0;
          base[es] = cmul(y1, tw_get(tw, (jp * tstep) % L, sign));
          base[2 * es] = cmul(y2, tw_get(tw, (2 * jp * tstep) % L, sign));
          base[3 * es] = cmul(y3, tw_get(tw, (3 * jp * tstep) % L, sign));
        } else {
          V x[kMaxRadix];
#pragma unroll
          for (int j = 0; j < kMaxRadix; ++j)
            if (j < rad) x[j] = base[j * es];
          for (int k1 = 0; k1 < rad; ++k1) {
            V acc = x[0];
            for (int j1 = 1; j1 < rad; ++j1)
              acc = cfma(x[j1], tw_get(tw, ((j1 * k1) % rad) * pstep, sign), acc);
            base[k1 * es] = k1 == 0 ? acc : cmul(acc, tw_get(tw, (jp * k1 * tstep) % L, sign));
          }
        }
      }
      __syncthreads();
      Ls = Lp;
    }
  }
  const int* pos0 = p.pos + p.pos_off[0];
  const int* pos1 = p.pos + p.pos_off[1];
  const int* pos2 = p.pos + p.pos_off[2];
  V* dst = out + line0 * nk;
  for (int i = tid; i < nl * nk; i += bd) {
    int line = i / nk, k = i - line * nk;
    int k3 = k % p.n[2], k2 = (k / p.n[2]) % p.n[1], k1 = k / (p.n[2] * p.n[1]);
    int s_idx = (pos0[k1] * p.n[1] + pos1[k2]) * p.n[2] + pos2[k3];
    V v = buf[static_cast<size_t>(line) * nk + s_idx];
    v.x *= scale;
    v.y *= scale;
    dst[i] = v;
  }
}

// ---------------------------------------------------------------------------
// Register path for power-of-two axes (L <= 32): each thread
// owns one whole line along the current axis, loads it in bit-reversed
// order, runs the radix-2 stages in registers with compile-time indices and
// stores it back in natural order, so no digit-reversal pass is needed.
// The staged line is padded by one element after every `pad` elements (pad =
// innermost non-trivial axis length) so that threads walking the innermost
// axis hit distinct shared-memory banks.

__host__ __device__ constexpr int brev_bits(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}
__host__ __device__ constexpr int ilog2(int L) { return L <= 1 ? 0 : 1 + ilog2(L / 2); }

// cos(2 pi j / 64): the first-octant values (j = 0..16, rounded to double) and
// the symmetries of the cosine; after unrolling every call has a constant
// argument and folds to a literal.
__host__ __device__ constexpr double cos64(int j) {
  constexpr double c[17] = {1.0,
                            0.99518472667219693, 0.98078528040323043, 0.95694033573220882,
                            0.92387953251128674, 0.88192126434835505, 0.83146961230254524,
                            0.77301045336273699, 0.70710678118654757, 0.63439328416364549,
                            0.55557023301960229, 0.47139673682599781, 0.38268343236508984,
                            0.29028467725446233, 0.19509032201612833, 0.09801714032956077,
                            0.0};
  j &= 63;
  if (j > 32) j = 64 - j;
  return j > 16 ? -c[32 - j] : c[j];
}
__host__ __device__ constexpr double sin64(int j) { return cos64((j + 48) & 63); }

// v * exp(SIGN 2 pi i j / 64); j = 0 and j = 16 (a quarter turn) without multiplications
template <typename V, int SIGN>
__device__ __forceinline__ V tw_mul(int j, V v) {
  if (j == 0) return v;
  if (j == 16) return SIGN < 0 ? cmk<V>(v.y, -v.x) : cmk<V>(-v.y, v.x);
  return cmul(cmk<V>(cos64(j), SIGN * sin64(j)), v);
}

// Butterfly sums.  For double-float values the sum is left unnormalised: the
// exact sum of the high parts (TwoSum) with the low parts and its error added
// into the low word, which keeps hi + lo exact up to the low word's rounding
// (~2^-48 of the operands) and saves the renormalisation (3 of 11 instructions
// per add); products (the twiddles) read both words and renormalise, and the
// kernels renormalise every value they store to global memory.
template <typename V>
__device__ __forceinline__ V bf_add(V a, V b) { return cadd(a, b); }
template <typename V>
__device__ __forceinline__ V bf_sub(V a, V b) { return csub(a, b); }
__device__ __forceinline__ dfl add_unnorm(dfl a, dfl b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return dfl(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
template <>
__device__ __forceinline__ dfc bf_add<dfc>(dfc a, dfc b) {
  return dfc{add_unnorm(a.x, b.x), add_unnorm(a.y, b.y)};
}
template <>
__device__ __forceinline__ dfc bf_sub<dfc>(dfc a, dfc b) {
  return dfc{add_unnorm(a.x, -b.x), add_unnorm(a.y, -b.y)};
}

// In-register radix-2 transform of length L (input in bit-reversed order,
// output in natural order): X_f = sum_j x_j exp(SIGN 2 pi i f j / L).
template <typename V, int L, int SIGN>
__device__ __forceinline__ void fft_regs(V (&x)[L]) {
#pragma unroll
  for (int m = 2; m <= L; m <<= 1) {
#pragma unroll
    for (int k = 0; k < m / 2; ++k) {
#pragma unroll
      for (int s0 = 0; s0 < L; s0 += m) {
        const V u = x[s0 + k];
        const V t = tw_mul<V, SIGN>(k * (64 / m), x[s0 + k + m / 2]);
        x[s0 + k] = bf_add(u, t);
        x[s0 + k + m / 2] = bf_sub(u, t);
      }
    }
  }
}

// L contiguous values at p into x in bit-reversed order (16-byte loads when vec)
template <typename V, int L>
__device__ __forceinline__ void ld_seg_brev(const V* __restrict__ p, V (&x)[L], bool vec) {
  constexpr int B = ilog2(L);
  if (sizeof(V) == 8 && vec) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int i = 0; i < L / 2; ++i) {
      const float4 v = q[i];
      x[brev_bits(2 * i, B)] = cmk<V>(v.x, v.y);
      x[brev_bits(2 * i + 1, B)] = cmk<V>(v.z, v.w);
    }
  } else {
#pragma unroll
    for (int j = 0; j < L; ++j) x[brev_bits(j, B)] = p[j];
  }
}

// Lines of N1 x N2 x N3 points with every N_d a power of two <= 32.  The axes
// are transformed innermost first, one length-L transform per thread and task,
// in registers.  The first pass reads its contiguous segments straight from
// global memory (16-byte loads); with BUB the lines are instead formed in
// shared memory from the bubble term lists: line (tau, o) holds
// sum_terms coef G[tau][g1](R) G^refl[tau][g2](-R), so P(R, tau) never goes
// through HBM before its transform to q.  Middle passes work in shared memory
// (one padding element per 2^lp points spreads the strided passes over the
// banks); the last pass writes global memory directly (consecutive threads own
// consecutive columns, so each of its stores is coalesced).
// L1C, L2C, L3C >= 0: the log2 axis lengths as compile-time constants (every
// pass compiles to its one transform length, which lowers the register need
// enough for three blocks per SM in FP32); -1: runtime lengths.
template <typename T, bool BUB, int SIGN, int L1C, int L2C, int L3C>
__global__ void __launch_bounds__(kFftThreads, sizeof(T) == 4 ? (L1C >= 0 ? 3 : 2) : 1)
    fft3d_reg_kernel(int l1_arg, int l2_arg, int l3_arg, const cplx<T>* in, cplx<T>* out, int lpb,
                     long long nlines, int lp, T scale, int vec, BubbleSrc bs) {
  const int l1 = L1C >= 0 ? L1C : l1_arg, l2 = L2C >= 0 ? L2C : l2_arg, l3 = L3C >= 0 ? L3C : l3_arg;
  using V = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tc = reinterpret_cast<V*>(smem_raw);                 // [bs.mt] term coefficients (BUB)
  int* ti = reinterpret_cast<int*>(tc + (BUB ? bs.mt : 0));
  V* buf = reinterpret_cast<V*>(ti + (BUB ? bs.mt : 0));
  const int tid = threadIdx.x, bd = blockDim.x;
  const int lnk = l1 + l2 + l3, nk = 1 << lnk;
  const int line_sz = nk + (nk >> lp);
  const long long line0 = static_cast<long long>(blockIdx.x) * lpb;
  const int nl = static_cast<int>(min(static_cast<long long>(lpb), nlines - line0));
  if (BUB) {
    const V* GR = reinterpret_cast<const V*>(bs.GR);
    const V* GL = reinterpret_cast<const V*>(bs.GL);
    const V* cf = reinterpret_cast<const V*>(bs.coef);
    for (int line = 0; line < nl; ++line) {
      const long long gline = line0 + line;
      const int tau = static_cast<int>(gline / bs.nout), o = static_cast<int>(gline - static_cast<long long>(tau) * bs.nout);
      const int e0 = bs.terms[o], nt = bs.terms[o + 1] - e0;
      __syncthreads();                                  // the previous line's terms are consumed
      for (int e = tid; e < nt; e += bd) {
        tc[e] = cf[e0 + e];
        ti[e] = bs.terms[bs.nout + 1 + e0 + e];
      }
      __syncthreads();
      const V* gt = GR + static_cast<size_t>(tau) * bs.no2 * nk;
      const V* lt = GL + static_cast<size_t>(tau) * bs.no2 * nk;
      // eight points per thread at a time: sixteen loads in flight per term
      for (int e0 = tid; e0 < nk; e0 += 8 * kFftThreads) {
        int mr[8];
        V acc[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = e0 + u * kFftThreads;
          mr[u] = e < nk ? qa_index(bs.mR[e], nk, bs.err) : 0;
          acc[u] = cmk<V>(0, 0);
        }
        for (int v = 0; v < nt; ++v) {
          const int id = ti[v];
          const V c = tc[v];
          const V* g1 = gt + static_cast<size_t>(qa_index(id & 255, bs.no2, bs.err)) * nk;
          const V* g2 = lt + static_cast<size_t>(qa_index(id >> 8, bs.no2, bs.err)) * nk;
          V x[8], y[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * kFftThreads;
            x[u] = e < nk ? g1[e] : cmk<V>(0, 0);
            y[u] = e < nk ? g2[mr[u]] : cmk<V>(0, 0);
          }
#pragma unroll
          for (int u = 0; u < 8; ++u)
            acc[u] = bs.real_coef ? cfma(x[u], cscale(y[u], c.x), acc[u]) : cfma(c, cmul(x[u], y[u]), acc[u]);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = e0 + u * kFftThreads;
          if (e < nk) buf[line * line_sz + e + (e >> lp)] = acc[u];
        }
      }
    }
    __syncthreads();
  }
  const int na = (l1 > 0) + (l2 > 0) + (l3 > 0);       // non-trivial axes, innermost first
#pragma unroll
  for (int pass = 0; pass < 3; ++pass) {
    if (pass >= na) break;
    const bool first = pass == 0, last = pass == na - 1;
    int lL = 0, lS = 0;                                 // log2 length and log2 stride of the axis
    {
      int k = pass;
      if (l3) { if (k == 0) { lL = l3; lS = 0; } --k; }
      if (l2) { if (k == 0) { lL = l2; lS = l3; } --k; }
      if (l1) { if (k == 0) { lL = l1; lS = l2 + l3; } }
    }
    const int lper = lnk - lL;                          // transforms per line = 2^lper
    for (int task = tid; task < (nl << lper); task += bd) {
      const int line = task >> lper, rem = task & ((1 << lper) - 1);
      const int o_lo = rem & ((1 << lS) - 1), o_hi = rem >> lS;
      const int base = (o_hi << (lL + lS)) + o_lo;
      const int S = 1 << lS;
      const long long gl = line0 + line;
      V* lb = buf + static_cast<size_t>(line) * line_sz;
      const int pb = base + (base >> lp), ps = S + (S >> lp);
      switch (lL) {
#define QA_FFT_PASS(LL)                                                                          \
  case LL: {                                                                                     \
    constexpr int L = 1 << LL;                                                                   \
    V x[L];                                                                                      \
    if (first && !BUB) {                                                                         \
      ld_seg_brev<V, L>(in + gl * nk + base, x, vec != 0);                                       \
    } else {                                                                                     \
      _Pragma("unroll") for (int j = 0; j < L; ++j) x[brev_bits(j, LL)] = lb[pb + j * ps];       \
    }                                                                                            \
    fft_regs<V, L, SIGN>(x);                                                                     \
    if (last) {                                                                                  \
      V* dst = out + gl * nk + base;                                                             \
      _Pragma("unroll") for (int j = 0; j < L; ++j) dst[static_cast<size_t>(j) * S] =            \
          cscale(x[j], scale);                                                \
    } else {                                                                                     \
      _Pragma("unroll") for (int j = 0; j < L; ++j) lb[pb + j * ps] = x[j];                      \
    }                                                                                            \
  } break;
        QA_FFT_PASS(1)
        QA_FFT_PASS(2)
        QA_FFT_PASS(3)
        QA_FFT_PASS(4)
        QA_FFT_PASS(5)
#undef QA_FFT_PASS
        default: break;
      }
    }
    if (!last) __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Line-per-block path for 16-byte elements (FP64 and double-float) on the
// 32x32x8 and 16x16x8 grids.  A whole line of N_k points stays in shared
// memory (at 32x32x8 that is one line per SM), so the block runs up to 512
// threads and each task holds one transform of at most 8 points: an axis of
// 16 or 32 points is split as L = A * 8 by decimation in frequency (8-point
// transforms over elements A apart, the twiddles w_L^(n1 k2) from the plan's
// table, then A-point transforms over adjacent elements), which leaves the
// axis in digit order, frequency 8 k1 + k2 at position k1 + A k2; the final
// store maps positions to frequencies.  The code is one small codelet per
// radix instead of whole 32-point transforms in registers, and the
// occupancy is 16 warps per SM instead of 8.
constexpr int kLineMaxThreads = 512;

__host__ __device__ constexpr int pad8(int e) { return e + (e >> 3); }

template <int LL>                      // log2 of an axis length
struct AxisSplit {
  static constexpr int steps = LL == 0 ? 0 : (LL <= 3 ? 1 : 2);
  static constexpr int A = LL <= 3 ? 1 : (1 << (LL - 3));
};

// frequency held at position p of an axis after its transform
template <int LL>
__device__ __forceinline__ int axis_freq(int p) {
  if constexpr (LL <= 3) {
    return p;
  } else {
    constexpr int A = 1 << (LL - 3);
    return 8 * (p & (A - 1)) + (p >> (LL - 3));
  }
}

// One step along the axis of log2 length LL and log2 stride LS.
// STEP 0: the whole axis (LL <= 3); 1: 8-point transforms over elements A
// apart, then the twiddles; 2: A-point transforms over adjacent elements.
// SRC_G: read the input line in natural order; DST_G: write the output line
// in natural order (scaled), otherwise in place in shared memory; cd (double-float
// only, optional): the line's grid codes, one byte per stored value.
template <typename T, int SIGN, int NTH, int L1, int L2, int L3, int LL, int LS, int STEP, bool SRC_G,
          bool DST_G>
__device__ __forceinline__ void line_step(const cplx<T>* __restrict__ src, cplx<T>* __restrict__ dst,
                                          cplx<T>* buf, const cplx<T>* __restrict__ tw, T scale,
                                          unsigned char* __restrict__ cd) {
  using V = cplx<T>;
  constexpr int NK = 1 << (L1 + L2 + L3);
  constexpr int L = 1 << LL, S = 1 << LS;
  constexpr int A = AxisSplit<LL>::A;
  constexpr int LR = STEP == 0 ? LL : (STEP == 1 ? 3 : LL - 3);
  constexpr int R = 1 << LR;
  constexpr int NT = NK / R;
  for (int task = threadIdx.x; task < NT; task += NTH) {
    const int o_lo = task & (S - 1);
    const int rest = task >> LS;
    int base, n1 = 0;
    if constexpr (STEP == 0) {
      base = (rest << (LL + LS)) + o_lo;
    } else if constexpr (STEP == 1) {
      n1 = rest & (A - 1);
      base = ((rest >> (LL - 3)) << (LL + LS)) + (n1 << LS) + o_lo;
    } else {
      base = ((rest >> 3) << (LL + LS)) + ((A * (rest & 7)) << LS) + o_lo;
    }
    constexpr int st = STEP == 1 ? A * S : S;
    V x[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int e = base + j * st;
      x[brev_bits(j, LR)] = SRC_G ? src[e] : buf[pad8(e)];
    }
    fft_regs<V, R, SIGN>(x);
    if constexpr (STEP == 1) {
#pragma unroll
      for (int j = 1; j < R; ++j) x[j] = cmul(x[j], tw_get(tw, (n1 * j) & (L - 1), SIGN));
    }
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int e = base + j * st;
      if constexpr (DST_G) {
        const int p3 = e & ((1 << L3) - 1), p2 = (e >> L3) & ((1 << L2) - 1), p1 = e >> (L2 + L3);
        const int f = (axis_freq<L1>(p1) << (L2 + L3)) + (axis_freq<L2>(p2) << L3) + axis_freq<L3>(p3);
        const V v = cscale(x[j], scale);
        dst[f] = v;
        if constexpr (std::is_same<T, dfl>::value) {
          if (cd) cd[f] = static_cast<unsigned char>(oz_grid_code(v));
        }
      } else {
        buf[pad8(e)] = x[j];
      }
    }
  }
}

template <typename T, int SIGN, int NTH, int L1, int L2, int L3, int LL, int LS, bool SRC_G, bool DST_G>
__device__ __forceinline__ void line_axis(const cplx<T>* src, cplx<T>* dst, cplx<T>* buf,
                                          const cplx<T>* tw, T scale, unsigned char* cd) {
  if constexpr (AxisSplit<LL>::steps == 1) {
    line_step<T, SIGN, NTH, L1, L2, L3, LL, LS, 0, SRC_G, DST_G>(src, dst, buf, tw, scale, cd);
  } else if constexpr (AxisSplit<LL>::steps == 2) {
    line_step<T, SIGN, NTH, L1, L2, L3, LL, LS, 1, SRC_G, false>(src, dst, buf, tw, scale, cd);
    __syncthreads();
    line_step<T, SIGN, NTH, L1, L2, L3, LL, LS, 2, false, DST_G>(src, dst, buf, tw, scale, cd);
  }
}

template <typename T, bool BUB, int SIGN, int L1, int L2, int L3>
__global__ void __launch_bounds__(((1 << (L1 + L2 + L3)) / 8 < kLineMaxThreads ? (1 << (L1 + L2 + L3)) / 8
                                                                                 : kLineMaxThreads),
                                  1)
    fft3d_line_kernel(FftDev p, const cplx<T>* in, cplx<T>* out, T scale, BubbleSrc bs) {
  using V = cplx<T>;
  constexpr int NK = 1 << (L1 + L2 + L3);
  constexpr int NTH = NK / 8 < kLineMaxThreads ? NK / 8 : kLineMaxThreads;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tc = reinterpret_cast<V*>(smem_raw);                 // [bs.mt] term coefficients (BUB)
  int* ti = reinterpret_cast<int*>(tc + (BUB ? bs.mt : 0));
  V* buf = reinterpret_cast<V*>(ti + (BUB ? bs.mt : 0));
  const int tid = threadIdx.x;
  const long long gl = blockIdx.x;
  const V* twg = reinterpret_cast<const V*>(p.tw);
  if (BUB) {
    const V* GR = reinterpret_cast<const V*>(bs.GR);
    const V* GL = reinterpret_cast<const V*>(bs.GL);
    const V* cf = reinterpret_cast<const V*>(bs.coef);
    const int tau = static_cast<int>(gl / bs.nout), o = static_cast<int>(gl - static_cast<long long>(tau) * bs.nout);
    const int e0 = bs.terms[o], nt = bs.terms[o + 1] - e0;
    for (int e = tid; e < nt; e += NTH) {
      tc[e] = cf[e0 + e];
      ti[e] = bs.terms[bs.nout + 1 + e0 + e];
    }
    __syncthreads();
    const V* gt = GR + static_cast<size_t>(tau) * bs.no2 * NK;
    const V* lt = GL + static_cast<size_t>(tau) * bs.no2 * NK;
    // four points per thread at a time: eight loads in flight per term
    for (int eb = tid; eb < NK; eb += 4 * NTH) {
      int mr[4];
      V acc[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = eb + u * NTH;
        mr[u] = e < NK ? qa_index(bs.mR[e], NK, bs.err) : 0;
        acc[u] = cmk<V>(0, 0);
      }
      for (int v = 0; v < nt; ++v) {
        const int id = ti[v];
        const V c = tc[v];
        const V* g1 = gt + static_cast<size_t>(qa_index(id & 255, bs.no2, bs.err)) * NK;
        const V* g2 = lt + static_cast<size_t>(qa_index(id >> 8, bs.no2, bs.err)) * NK;
        V xv[4], yv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = eb + u * NTH;
          xv[u] = e < NK ? g1[e] : cmk<V>(0, 0);
          yv[u] = e < NK ? g2[mr[u]] : cmk<V>(0, 0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          acc[u] = bs.real_coef ? cfma(xv[u], cscale(yv[u], c.x), acc[u]) : cfma(c, cmul(xv[u], yv[u]), acc[u]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = eb + u * NTH;
        if (e < NK) buf[pad8(e)] = acc[u];
      }
    }
    __syncthreads();
  }
  const V* src = in + gl * NK;
  V* dst = out + gl * NK;
  unsigned char* cd = BUB && bs.code ? bs.code + gl * NK : nullptr;
  constexpr bool h3 = L3 > 0, h2 = L2 > 0, h1 = L1 > 0;
  if constexpr (h3) {
    line_axis<T, SIGN, NTH, L1, L2, L3, L3, 0, !BUB, !h2 && !h1>(src, dst, buf, twg + p.tw_off[2], scale, cd);
    if constexpr (h2 || h1) __syncthreads();
  }
  if constexpr (h2) {
    line_axis<T, SIGN, NTH, L1, L2, L3, L2, L3, !BUB && !h3, !h1>(src, dst, buf, twg + p.tw_off[1], scale, cd);
    if constexpr (h1) __syncthreads();
  }
  if constexpr (h1) {
    line_axis<T, SIGN, NTH, L1, L2, L3, L1, L2 + L3, !BUB && !h3 && !h2, true>(src, dst, buf,
                                                                              twg + p.tw_off[0], scale, cd);
  }
}

template <typename T, bool BUB, int L1, int L2, int L3>
cudaError_t launch_fft3d_line(const FftDev& plan, int sign, const void* in, void* out, long long nlines,
                              cudaStream_t st, T sc, const BubbleSrc& bs) {
  constexpr int NK = 1 << (L1 + L2 + L3);
  constexpr int NTH = NK / 8 < kLineMaxThreads ? NK / 8 : kLineMaxThreads;
  const size_t extra = BUB ? static_cast<size_t>(bs.mt) * (sizeof(cplx<T>) + sizeof(int)) : 0;
  const size_t smem = static_cast<size_t>(pad8(NK)) * sizeof(cplx<T>) + extra;
  auto fn = sign > 0 ? &fft3d_line_kernel<T, BUB, 1, L1, L2, L3> : &fft3d_line_kernel<T, BUB, -1, L1, L2, L3>;
  cudaError_t e = set_smem(reinterpret_cast<const void*>(fn), smem, true);
  if (e != cudaSuccess) return e;
  if (nlines > 0x7fffffffLL) return cudaErrorInvalidValue;
  fn<<<static_cast<unsigned>(nlines), NTH, smem, st>>>(plan, reinterpret_cast<const cplx<T>*>(in),
                                                       reinterpret_cast<cplx<T>*>(out), sc, bs);
  return cudaGetLastError();
}

bool reg_axis_ok(int L, int maxL) {
  return L >= 1 && L <= maxL && (L & (L - 1)) == 0;
}

bool reg_plan_ok(const FftDev& plan) {
  const int nk = plan.n[0] * plan.n[1] * plan.n[2];
  return reg_axis_ok(plan.n[0], 32) && reg_axis_ok(plan.n[1], 32) && reg_axis_ok(plan.n[2], 32) &&
         nk >= 2;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

template <typename T, bool BUB>
cudaError_t launch_fft3d_reg(const FftDev& plan, int sign, const void* in, void* out,
                             long long nlines, cudaStream_t st, T sc, const BubbleSrc& bs) {
  const int nk = plan.n[0] * plan.n[1] * plan.n[2];
  const int pad = plan.n[2] > 1 ? plan.n[2] : (plan.n[1] > 1 ? plan.n[1] : plan.n[0]);
  const int lp = ilog2(pad);
  const int line_sz = nk + (nk >> lp);
  int lpb = 1;
  while (lpb * 2 * line_sz * static_cast<int>(sizeof(cplx<T>)) <= 32768 && lpb * 2 <= 64) lpb *= 2;
  const size_t extra = BUB ? static_cast<size_t>(bs.mt) * (sizeof(cplx<T>) + sizeof(int)) : 0;
  const size_t smem = static_cast<size_t>(lpb) * line_sz * sizeof(cplx<T>) + extra;
  const int vec = BUB ? 0 : aligned16(in);
  const int l1 = ilog2(plan.n[0]), l2 = ilog2(plan.n[1]), l3 = ilog2(plan.n[2]);
  if constexpr (sizeof(cplx<T>) == 16) {
    // one line per block (16-byte elements)
    if (l1 == 5 && l2 == 5 && l3 == 3) return launch_fft3d_line<T, BUB, 5, 5, 3>(plan, sign, in, out, nlines, st, sc, bs);
    if (l1 == 4 && l2 == 4 && l3 == 3) return launch_fft3d_line<T, BUB, 4, 4, 3>(plan, sign, in, out, nlines, st, sc, bs);
  }
  auto fn = sign > 0 ? &fft3d_reg_kernel<T, BUB, 1, -1, -1, -1> : &fft3d_reg_kernel<T, BUB, -1, -1, -1, -1>;
  if (l1 == 5 && l2 == 5 && l3 == 3)          // 32 x 32 x 8
    fn = sign > 0 ? &fft3d_reg_kernel<T, BUB, 1, 5, 5, 3> : &fft3d_reg_kernel<T, BUB, -1, 5, 5, 3>;
  else if (l1 == 4 && l2 == 4 && l3 == 3)     // 16 x 16 x 8
    fn = sign > 0 ? &fft3d_reg_kernel<T, BUB, 1, 4, 4, 3> : &fft3d_reg_kernel<T, BUB, -1, 4, 4, 3>;
  cudaError_t e = set_smem(reinterpret_cast<const void*>(fn), smem, true);
  if (e != cudaSuccess) return e;
  long long nblk = (nlines + lpb - 1) / lpb;
  fn<<<static_cast<unsigned>(nblk), kFftThreads, smem, st>>>(
      l1, l2, l3, reinterpret_cast<const cplx<T>*>(in),
      reinterpret_cast<cplx<T>*>(out), lpb, nlines, lp, sc, vec, bs);
  return cudaGetLastError();
}

}  // namespace

bool fft3d_bubble_supported(const FftDev& plan) { return reg_plan_ok(plan); }

// the grids on which 16-byte lines take fft3d_line_kernel (the kernel that writes codes)
bool fft3d_bubble_codes(const FftDev& plan) {
  if (!reg_plan_ok(plan)) return false;
  const int l1 = ilog2(plan.n[0]), l2 = ilog2(plan.n[1]), l3 = ilog2(plan.n[2]);
  return (l1 == 5 && l2 == 5 && l3 == 3) || (l1 == 4 && l2 == 4 && l3 == 3);
}

template <typename T>
cudaError_t launch_fft3d_bubble(const FftDev& plan, const void* GR, const void* GreflR,
                                const int* mR, const int* terms, const void* coef, int max_terms,
                                int nout, int norb, void* out, int r, cudaStream_t st, int* err,
                                bool real_coef, unsigned char* code) {
  if (!reg_plan_ok(plan) || max_terms > kMaxLineTerms || norb * norb > 256) return cudaErrorInvalidValue;
  const int mt = (max_terms + 3) / 4 * 4;            // keeps the line buffer aligned
  BubbleSrc bs{GR, GreflR, mR, terms, coef, nout, norb * norb, mt < 4 ? 4 : mt, err, real_coef ? 1 : 0,
               std::is_same<T, dfl>::value ? code : nullptr};
  return launch_fft3d_reg<T, true>(plan, -1, nullptr, out, static_cast<long long>(nout) * r, st,
                                   static_cast<T>(1), bs);
}

template <typename T>
cudaError_t launch_fft3d(const FftDev& plan, int sign, const void* in, void* out, long long nlines,
                         cudaStream_t st, double scale) {
  if (nlines <= 0) return cudaSuccess;
  const int nk = plan.n[0] * plan.n[1] * plan.n[2];
  const T sc = static_cast<T>(scale > 0 ? scale : (sign > 0 ? 1.0 / nk : 1.0));
  if (reg_plan_ok(plan)) return launch_fft3d_reg<T, false>(plan, sign, in, out, nlines, st, sc, BubbleSrc{});
  // lines per block: keep the tile near 16 KB for small grids
  int lpb = 1;
  while (lpb * 2 * nk * static_cast<int>(sizeof(cplx<T>)) <= 16384 && lpb * 2 <= 64) lpb *= 2;
  size_t smem = (static_cast<size_t>(lpb) * nk + plan.n[0] + plan.n[1] + plan.n[2]) * sizeof(cplx<T>);
  cudaError_t e = set_smem(reinterpret_cast<const void*>(&fft3d_kernel<T>), smem);
  if (e != cudaSuccess) return e;
  long long nblk = (nlines + lpb - 1) / lpb;
  int threads = nk * lpb >= 2048 ? 512 : 256;
  fft3d_kernel<T><<<static_cast<unsigned>(nblk), threads, smem, st>>>(
      plan, sign, reinterpret_cast<const cplx<T>*>(in), reinterpret_cast<cplx<T>*>(out), nk, lpb,
      nlines, sc);
  return cudaGetLastError();
}

template cudaError_t launch_fft3d_bubble<double>(const FftDev&, const void*, const void*, const int*,
                                                 const int*, const void*, int, int, int, void*, int,
                                                 cudaStream_t, int*, bool, unsigned char*);
template cudaError_t launch_fft3d_bubble<float>(const FftDev&, const void*, const void*, const int*,
                                                const int*, const void*, int, int, int, void*, int,
                                                cudaStream_t, int*, bool, unsigned char*);
template cudaError_t launch_fft3d<double>(const FftDev&, int, const void*, void*, long long,
                                          cudaStream_t, double);
template cudaError_t launch_fft3d<float>(const FftDev&, int, const void*, void*, long long,
                                         cudaStream_t, double);
template cudaError_t launch_fft3d<dfl>(const FftDev&, int, const void*, void*, long long,
                                       cudaStream_t, double);
template cudaError_t launch_fft3d_bubble<dfl>(const FftDev&, const void*, const void*, const int*,
                                              const int*, const void*, int, int, int, void*, int,
                                              cudaStream_t, int*, bool, unsigned char*);

}  // namespace qa
