// Chemical-potential search on the device (paper Sec. "GW self-consistency":
// mu is fixed by the filling, N(mu) = (s/N_k) sum_k Tr n(k) = N_target).
//
// The search is a safeguarded Newton iteration on N(mu) - N_target: Newton
// steps from the warm start while each at least quarters the residual, then
// (if needed) a march with growing steps toward the root
// until N - N_target changes sign (inside the window outside which N is empty
// or full), then bisection with Newton steps taken when they stay inside the
// bracket and at least halve the step before last.  Its state lives in device
// memory and is advanced by mu_update_kernel after every density evaluation;
// the host captures [density kernel, update kernel] once as the body of a
// CUDA-graph while-node, and the update kernel ends the loop through the
// node's condition when the search has converged or failed.  A step thus
// runs the whole search without host round trips and reads the result once.
#include "qa_common.cuh"

namespace qa {
namespace {

constexpr int kQaENOCONV = 4;
constexpr int kQaERANGE = 5;
constexpr int kMaxEvals = 300;

enum : int { kPhStart = 0, kPhNewton = 1, kPhMarch = 2, kPhSafe = 3, kPhFinal = 4, kPhDone = 5 };

__device__ __forceinline__ double tol_b(const MuState* s, double m) {
  return (s->fp64 ? 2e-13 : 2e-7) * fmax(1.0, fabs(m));
}

__device__ void finish(MuState* s, int status) {
  s->status = status;
  s->phase = kPhDone;
}

// Bisection / Newton step of the bracketed phase: sets the next point (and
// phase) or finishes.
__device__ void safe_step(MuState* s) {
  if (!(fabs(s->f) > s->tolN)) { finish(s, 0); return; }
  if (s->f < 0) s->lo = fmax(s->lo, s->mu); else s->hi = fmin(s->hi, s->mu);
  if (s->hi - s->lo <= tol_b(s, s->mu)) {
    s->mu = 0.5 * (s->lo + s->hi);
    s->phase = kPhFinal;
    return;
  }
  const double cand = s->mu - s->f / s->d;
  if (!(s->d > 0) || !isfinite(cand) || cand <= s->lo || cand >= s->hi ||
      fabs(2.0 * s->f) > fabs(s->dxold * s->d)) {
    s->dxold = s->dx;
    s->dx = 0.5 * (s->hi - s->lo);
    s->mu = s->lo + s->dx;
  } else {
    s->dxold = s->dx;
    s->dx = s->f / s->d;
    s->mu = cand;
    if (!s->fp64 && fabs(s->dx) <= tol_b(s, s->mu)) {     // converged to the density noise
      s->phase = kPhFinal;
      return;
    }
  }
  s->phase = kPhSafe;
}

// Newton step from the point just evaluated (kept as the fallback); on the
// FP32 path a step below the density noise ends the search after one more
// evaluation.
__device__ void newton_from(MuState* s, double fv, double dv) {
  s->mu0 = s->mu;
  s->f0 = fv;
  s->d0 = dv;
  s->nt += 1;
  const double dx = fv / dv;
  s->mu = s->mu - dx;
  s->phase = (!s->fp64 && fabs(dx) <= tol_b(s, s->mu)) ? kPhFinal : kPhNewton;
}

// From the current point: finish, or start the march toward the root.
__device__ void march_start(MuState* s) {
  if (!(fabs(s->f) > s->tolN)) { finish(s, 0); return; }
  double step = (s->d > 0 && isfinite(s->f / s->d)) ? 1.5 * fabs(s->f / s->d) : 1.0;
  s->step = fmin(fmax(step, 1e-6), s->wid);
  s->dir = s->f < 0 ? 1.0 : -1.0;
  s->a = s->mu;
  s->fa = s->f;
  s->m = 0;
  s->b = fmin(fmax(s->a + s->dir * s->step, s->wlo), s->whi);
  s->mu = s->b;
  s->phase = kPhMarch;
}

// Consume the density just evaluated at s->mu and decide the next point.
__device__ void mu_advance(MuState* s, double N, double dN) {
  s->count += 1;
  s->N = N;
  s->dN = dN;
  if (!isfinite(N)) { finish(s, kQaERANGE); return; }
  const double fv = N - s->target, dv = dN;
  switch (s->phase) {
    case kPhStart:
      s->f = fv;
      s->d = dv;
      s->nt = 0;
      if (fabs(fv) > s->tolN && dv > 0 && isfinite(fv / dv) && fabs(fv / dv) < 0.25 * s->wid) {
        newton_from(s, fv, dv);
        return;
      }
      march_start(s);
      return;
    case kPhNewton:
      if (fabs(fv) <= s->tolN) {
        s->f = fv;
        s->d = dv;
        finish(s, 0);
        return;
      }
      // converging (the residual at least quartered): another Newton step
      if (fabs(fv) < 0.25 * fabs(s->f0) && s->nt < 6 && dv > 0 && isfinite(fv / dv) &&
          fabs(fv / dv) < 0.25 * s->wid) {
        newton_from(s, fv, dv);
        return;
      }
      if (fabs(fv) < fabs(s->f0)) {
        s->f = fv;
        s->d = dv;
      } else {
        s->mu = s->mu0;
        s->f = s->f0;
        s->d = s->d0;
      }
      march_start(s);
      return;
    case kPhMarch: {
      s->fb = fv;
      s->db = dv;
      if ((s->fb < 0) != (s->fa < 0) || fabs(s->fb) <= s->tolN) {
        s->lo = fmin(s->a, s->b);
        s->hi = fmax(s->a, s->b);
        if (fabs(s->fb) < fabs(s->fa)) { s->mu = s->b; s->f = s->fb; s->d = s->db; }
        else { s->mu = s->a; s->f = s->fa; }
        s->dx = s->hi - s->lo;
        s->dxold = s->dx;
        s->it = 0;
        safe_step(s);
        return;
      }
      if (s->b == s->whi || s->b == s->wlo) { finish(s, kQaERANGE); return; }   // filling out of reach
      s->a = s->b;
      s->fa = s->fb;
      s->step *= 4.0;
      if (++s->m >= 64) { finish(s, kQaENOCONV); return; }
      s->b = fmin(fmax(s->a + s->dir * s->step, s->wlo), s->whi);
      s->mu = s->b;
      return;
    }
    case kPhSafe:
      s->f = fv;
      s->d = dv;
      if (s->it == 199 && fabs(s->f) > s->tolN) { finish(s, kQaENOCONV); return; }
      s->it += 1;
      safe_step(s);
      return;
    case kPhFinal:
      s->f = fv;
      s->d = dv;
      finish(s, 0);
      return;
    default:
      finish(s, kQaENOCONV);
  }
}

// Window from the bound of ||H + Sigma - mu_ref|| (bound[0]), start at mu_s.
__global__ void mu_init_kernel(MuState* s, const double* bound, double mu_s, double target, double beta,
                               int fp64) {
  const double b = bound[0];
  const double wid = b + 1.0 + 10.0 / beta;
  s->mu = mu_s;
  s->mu_ref = mu_s;
  s->target = target;
  s->fp64 = fp64;
  s->tolN = (fp64 ? 1e-12 : 2e-6) * fmax(1.0, target);
  s->wid = wid;
  s->wlo = mu_s - wid;
  s->whi = mu_s + wid;
  s->count = 0;
  s->status = 0;
  s->N = 0.0;
  s->phase = isfinite(b) ? kPhStart : kPhDone;
  if (!isfinite(b)) s->status = kQaERANGE;
}

// Reduce the density kernel's block sums (the same order as the host-side
// reduction), advance the search, and keep the while-node running until done.
__global__ void __launch_bounds__(256) mu_update_kernel(const double* __restrict__ part, int nblocks,
                                                        MuState* s, double nspin, int nk,
                                                        cudaGraphConditionalHandle cond) {
  __shared__ double sh[64];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
  block_sum2(a, b, sh);
  if (threadIdx.x == 0) {
    if (s->phase != kPhDone) {
      mu_advance(s, nspin * a / nk, -nspin * b / nk);
      if (s->count >= kMaxEvals && s->phase != kPhDone) finish(s, kQaENOCONV);
    }
    cudaGraphSetConditional(cond, s->phase == kPhDone ? 0u : 1u);
  }
}

}  // namespace

cudaError_t launch_mu_init(MuState* s, const double* bound, double mu_s, double target, double beta,
                           int fp64, cudaStream_t st) {
  mu_init_kernel<<<1, 1, 0, st>>>(s, bound, mu_s, target, beta, fp64);
  return cudaGetLastError();
}

cudaError_t launch_mu_update(const double* part, int nblocks, MuState* s, double nspin, int nk,
                             cudaGraphConditionalHandle cond, cudaStream_t st) {
  mu_update_kernel<<<1, 256, 0, st>>>(part, nblocks, s, nspin, nk, cond);
  return cudaGetLastError();
}

}  // namespace qa
