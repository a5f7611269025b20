// Host-side DLR builder and transform-matrix composition.
//
// Construction of the discrete Lehmann representation (Kaye, Chen &
// Parcollet, PRB 105, 235115 (2022)), which the paper uses for the
// imaginary-time / Matsubara sampling of every dynamic quantity (Sec.
// "Methods", after the bare Green's function equations; "DLR" class):
//   1. dimensionless kernel k(t, x) = e^{-t x} / (1 + e^{-x}), t in [0,1],
//      x in [-Lambda, Lambda];
//   2. composite Chebyshev fine grids, dyadically refined toward x = 0 and
//      toward t = 0 and t = 1 (p = 24 first-kind points per panel,
//      ceil(log2 Lambda) panels per half-line);
//   3. column-pivoted Gram-Schmidt on the discretised kernel selects the
//      real poles x_l (stop when the largest residual 2-norm is <= eps times
//      the largest initial column norm);
//   4. the same pivoted Gram-Schmidt on the rows of k(t, x_l) selects the r
//      imaginary-time nodes, and on the rows of the Matsubara kernels
//      1/(i(2n+1)pi - x) and tanh(x/2)/(i 2 pi m - x) (candidates
//      |n| <= ceil(Lambda)) selects r fermionic and r bosonic frequencies.
// Pivot ties go to the lowest index within a relative 1e-12 of the maximum.
// Times t > 1/2 are carried in relative format (t - 1), so nodes near beta
// keep full precision and the reflection beta - tau is exact.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "qa_internal.h"

namespace qa {
namespace {

constexpr int kCheb = 24;
constexpr double kTie = 1e-12;

int panel_count(double Lambda) {
  int n = static_cast<int>(std::ceil(std::log2(Lambda)));
  return n < 1 ? 1 : n;
}

void cheb_points(double a, double b, std::vector<double>* out) {
  for (int k = 0; k < kCheb; ++k)
    out->push_back(0.5 * (a + b) - 0.5 * (b - a) * std::cos(M_PI * (k + 0.5) / kCheb));
}

std::vector<double> x_candidates(double Lambda) {
  int np = panel_count(Lambda);
  std::vector<double> pos;
  double lo = 0.0;
  for (int i = 1; i <= np; ++i) {
    double hi = Lambda / std::ldexp(1.0, np - i);
    cheb_points(lo, hi, &pos);
    lo = hi;
  }
  std::vector<double> all;
  for (int i = static_cast<int>(pos.size()) - 1; i >= 0; --i) all.push_back(-pos[i]);
  for (double v : pos) all.push_back(v);
  return all;
}

std::vector<double> t_candidates(double Lambda) {
  int np = panel_count(Lambda);
  std::vector<double> left;
  double lo = 0.0;
  for (int i = 1; i <= np; ++i) {
    double hi = std::ldexp(1.0, i - np - 1);
    cheb_points(lo, hi, &left);
    lo = hi;
  }
  std::vector<double> all(left);
  for (int i = static_cast<int>(left.size()) - 1; i >= 0; --i) all.push_back(-left[i]);
  return all;
}

// k(t, x) with t in relative format; both exponents are <= 0.
template <typename R>
R kernel(R t_rel, R x) {
  R t_from0, one_minus_t;
  if (t_rel >= 0) { t_from0 = t_rel; one_minus_t = R(1) - t_rel; }
  else { t_from0 = R(1) + t_rel; one_minus_t = -t_rel; }
  if (x >= 0) return std::exp(-t_from0 * x) / (R(1) + std::exp(-x));
  return std::exp(one_minus_t * x) / (R(1) + std::exp(x));
}

template <typename R>
R fermi_fn(R x) {
  if (x >= 0) return std::exp(-x) / (R(1) + std::exp(-x));
  return R(1) / (R(1) + std::exp(x));
}

inline double cj(double v) { return v; }
inline std::complex<double> cj(std::complex<double> v) { return std::conj(v); }

// Column-pivoted Gram-Schmidt on a column-major matrix (rows x cols) of
// type S (double or complex<double>).  rank > 0: exactly `rank` columns;
// otherwise stop at tolerance eps.
template <typename S>
std::vector<int> pivoted_gs(std::vector<S> A, int rows, int cols, double eps, int rank) {
  auto col = [&](int j) { return A.data() + static_cast<size_t>(j) * rows; };
  std::vector<char> chosen(cols, 0);
  std::vector<double> nrm(cols);
  auto norms = [&]() {
    for (int j = 0; j < cols; ++j) {
      double s = 0;
      const S* c = col(j);
      for (int i = 0; i < rows; ++i) s += std::norm(c[i]);
      nrm[j] = std::sqrt(s);
    }
  };
  norms();
  double ref = *std::max_element(nrm.begin(), nrm.end());
  std::vector<int> sel;
  int limit = rank > 0 ? rank : std::min(rows, cols);
  std::vector<S> q(rows);
  while (static_cast<int>(sel.size()) < limit) {
    if (!sel.empty()) norms();
    double m = -1.0;
    for (int j = 0; j < cols; ++j)
      if (!chosen[j] && nrm[j] > m) m = nrm[j];
    if (rank <= 0 && m <= eps * ref) break;
    int piv = -1;
    for (int j = 0; j < cols; ++j)
      if (!chosen[j] && nrm[j] >= m * (1.0 - kTie)) { piv = j; break; }
    const S* pc = col(piv);
    for (int i = 0; i < rows; ++i) q[i] = pc[i] / nrm[piv];
    for (int pass = 0; pass < 2; ++pass) {
      for (int j = 0; j < cols; ++j) {
        S* c = col(j);
        S dot = S(0);
        for (int i = 0; i < rows; ++i) dot += cj(q[i]) * c[i];
        for (int i = 0; i < rows; ++i) c[i] -= q[i] * dot;
      }
    }
    chosen[piv] = 1;
    sel.push_back(piv);
  }
  return sel;
}

double abs_t(double t) { return t >= 0 ? t : 1.0 + t; }

using cld = std::complex<long double>;

// Inverse of an r x r complex matrix (row-major) by Gauss-Jordan elimination
// with partial pivoting, in long double.
std::vector<cld> invert(std::vector<cld> A, int r) {
  std::vector<cld> I(static_cast<size_t>(r) * r, cld(0));
  for (int i = 0; i < r; ++i) I[static_cast<size_t>(i) * r + i] = cld(1);
  for (int c = 0; c < r; ++c) {
    int p = c;
    long double best = std::abs(A[static_cast<size_t>(c) * r + c]);
    for (int i = c + 1; i < r; ++i) {
      long double v = std::abs(A[static_cast<size_t>(i) * r + c]);
      if (v > best) { best = v; p = i; }
    }
    if (p != c)
      for (int j = 0; j < r; ++j) {
        std::swap(A[static_cast<size_t>(c) * r + j], A[static_cast<size_t>(p) * r + j]);
        std::swap(I[static_cast<size_t>(c) * r + j], I[static_cast<size_t>(p) * r + j]);
      }
    cld inv = cld(1) / A[static_cast<size_t>(c) * r + c];
    for (int j = 0; j < r; ++j) {
      A[static_cast<size_t>(c) * r + j] *= inv;
      I[static_cast<size_t>(c) * r + j] *= inv;
    }
    for (int i = 0; i < r; ++i) {
      if (i == c) continue;
      cld f = A[static_cast<size_t>(i) * r + c];
      if (f == cld(0)) continue;
      for (int j = 0; j < r; ++j) {
        A[static_cast<size_t>(i) * r + j] -= f * A[static_cast<size_t>(c) * r + j];
        I[static_cast<size_t>(i) * r + j] -= f * I[static_cast<size_t>(c) * r + j];
      }
    }
  }
  return I;
}

// C = A (rows x r) * B (r x r), row-major, converted to double.
std::vector<std::complex<double>> matmul(const std::vector<cld>& A, const std::vector<cld>& B,
                                         int rows, int r) {
  std::vector<std::complex<double>> C(static_cast<size_t>(rows) * r);
  for (int i = 0; i < rows; ++i)
    for (int j = 0; j < r; ++j) {
      cld s(0);
      for (int l = 0; l < r; ++l) s += A[static_cast<size_t>(i) * r + l] * B[static_cast<size_t>(l) * r + j];
      C[static_cast<size_t>(i) * r + j] = std::complex<double>(static_cast<double>(s.real()),
                                                               static_cast<double>(s.imag()));
    }
  return C;
}

}  // namespace

int build_dlr(double Lambda, double eps, DlrGrid* out) {
  if (!(Lambda > 1.0) || !(eps > 0.0) || !(eps < 1.0)) return 1;
  std::vector<double> xf = x_candidates(Lambda);
  std::vector<double> tf = t_candidates(Lambda);
  const int nx = static_cast<int>(xf.size()), nt = static_cast<int>(tf.size());
  // kernel matrix, columns = x candidates
  std::vector<double> A(static_cast<size_t>(nt) * nx);
  for (int j = 0; j < nx; ++j)
    for (int i = 0; i < nt; ++i) A[static_cast<size_t>(j) * nt + i] = kernel<double>(tf[i], xf[j]);
  std::vector<int> ix = pivoted_gs<double>(A, nt, nx, eps, 0);
  const int r = static_cast<int>(ix.size());
  if (r < 1 || r > 128) return 1;
  std::vector<double> x;
  for (int j : ix) x.push_back(xf[j]);
  std::sort(x.begin(), x.end());
  // tau nodes: columns = t candidates, rows = selected x
  std::vector<double> B(static_cast<size_t>(r) * nt);
  for (int i = 0; i < nt; ++i)
    for (int l = 0; l < r; ++l) B[static_cast<size_t>(i) * r + l] = kernel<double>(tf[i], x[l]);
  std::vector<int> it = pivoted_gs<double>(B, r, nt, 0.0, r);
  std::vector<double> t;
  for (int i : it) t.push_back(tf[i]);
  std::sort(t.begin(), t.end(), [](double a, double b) { return abs_t(a) < abs_t(b); });
  // Matsubara nodes
  const int nmax = static_cast<int>(std::ceil(Lambda));
  using cd = std::complex<double>;
  {
    const int nc = 2 * nmax;
    std::vector<cd> C(static_cast<size_t>(r) * nc);
    for (int c = 0; c < nc; ++c) {
      double n = static_cast<double>(c - nmax);
      for (int l = 0; l < r; ++l)
        C[static_cast<size_t>(c) * r + l] = 1.0 / cd(-x[l], (2.0 * n + 1.0) * M_PI);
    }
    std::vector<int> jf = pivoted_gs<cd>(C, r, nc, 0.0, r);
    out->nf.clear();
    for (int c : jf) out->nf.push_back(c - nmax);
    std::sort(out->nf.begin(), out->nf.end());
  }
  {
    const int nc = 2 * nmax + 1;
    std::vector<cd> C(static_cast<size_t>(r) * nc);
    for (int c = 0; c < nc; ++c) {
      int m = c - nmax;
      for (int l = 0; l < r; ++l) {
        cd v;
        if (m == 0 && x[l] == 0.0) v = cd(-0.5, 0.0);
        else v = std::tanh(0.5 * x[l]) / cd(-x[l], 2.0 * M_PI * m);
        C[static_cast<size_t>(c) * r + l] = v;
      }
    }
    std::vector<int> jb = pivoted_gs<cd>(C, r, nc, 0.0, r);
    out->mb.clear();
    for (int c : jb) out->mb.push_back(c - nmax);
    std::sort(out->mb.begin(), out->mb.end());
  }
  out->r = r;
  out->x = x;
  out->t = t;
  return 0;
}

void build_dlr_matrices(const DlrGrid& g, double beta, DlrMatrices* m) {
  const int r = g.r;
  using ld = long double;
  const ld b = beta;
  const ld pi = 3.141592653589793238462643383279502884L;
  std::vector<cld> Kt(static_cast<size_t>(r) * r), Ktr(Kt.size()), KF(Kt.size()), KB(Kt.size());
  std::vector<cld> f(r);
  for (int l = 0; l < r; ++l) f[l] = cld(fermi_fn<ld>(static_cast<ld>(g.x[l])), 0);
  for (int j = 0; j < r; ++j)
    for (int l = 0; l < r; ++l) {
      ld x = g.x[l];
      Kt[static_cast<size_t>(j) * r + l] = cld(-kernel<ld>(static_cast<ld>(g.t[j]), x), 0);
      Ktr[static_cast<size_t>(j) * r + l] = cld(-kernel<ld>(static_cast<ld>(g.t[j]), -x), 0);
      KF[static_cast<size_t>(j) * r + l] = b / cld(-x, (2 * static_cast<ld>(g.nf[j]) + 1) * pi);
      if (g.mb[j] == 0 && g.x[l] == 0.0) KB[static_cast<size_t>(j) * r + l] = cld(-b / 2, 0);
      else KB[static_cast<size_t>(j) * r + l] = b * std::tanh(x / 2) / cld(-x, 2 * pi * g.mb[j]);
    }
  std::vector<cld> Kti = invert(Kt, r), KFi = invert(KF, r), KBi = invert(KB, r);
  m->Trefl = matmul(Ktr, Kti, r, r);
  m->Ttn = matmul(KB, Kti, r, r);
  m->Tnt = matmul(Kt, KBi, r, r);
  m->Ttw = matmul(KF, Kti, r, r);
  m->Twt = matmul(Kt, KFi, r, r);
  m->dtau = matmul(f, Kti, 1, r);
  m->dw = matmul(f, KFi, 1, r);
  // Sigma(+-i pi/beta) = sum_n wq_{+-}[n] Sigma(i w_n): K_F at the lowest
  // fermionic frequencies times K_F^-1 (the DLR fit at the Matsubara nodes)
  std::vector<cld> kp(r), km(r);
  for (int l = 0; l < r; ++l) {
    const ld x = g.x[l];
    kp[l] = b / cld(-x, pi);
    km[l] = b / cld(-x, -pi);
  }
  m->wq_p = matmul(kp, KFi, 1, r);
  m->wq_m = matmul(km, KFi, 1, r);
  m->iw.resize(r);
  for (int j = 0; j < r; ++j) m->iw[j] = (2.0 * g.nf[j] + 1.0) * M_PI / beta;
}

// Uniform Matsubara evaluation of the expansions: the fermionic kernel at
// i w_n times K_tau^-1 (from the tau-node values) and the bosonic kernel at
// i nu_m times K_B^-1 (from the bosonic-node values), composed in long double.
void build_uniform_maps(const DlrGrid& g, double beta, int M, std::vector<std::complex<double>>* EF,
                        std::vector<std::complex<double>>* EB) {
  const int r = g.r;
  using ld = long double;
  const ld b = beta;
  const ld pi = 3.141592653589793238462643383279502884L;
  std::vector<cld> Kt(static_cast<size_t>(r) * r), KB(Kt.size());
  for (int j = 0; j < r; ++j)
    for (int l = 0; l < r; ++l) {
      const ld x = g.x[l];
      Kt[static_cast<size_t>(j) * r + l] = cld(-kernel<ld>(static_cast<ld>(g.t[j]), x), 0);
      if (g.mb[j] == 0 && g.x[l] == 0.0) KB[static_cast<size_t>(j) * r + l] = cld(-b / 2, 0);
      else KB[static_cast<size_t>(j) * r + l] = b * std::tanh(x / 2) / cld(-x, 2 * pi * g.mb[j]);
    }
  const std::vector<cld> Kti = invert(Kt, r), KBi = invert(KB, r);
  std::vector<cld> F(static_cast<size_t>(2 * M) * r), B(static_cast<size_t>(2 * M + 1) * r);
  for (int n = -M; n < M; ++n)
    for (int l = 0; l < r; ++l)
      F[static_cast<size_t>(n + M) * r + l] = b / cld(-static_cast<ld>(g.x[l]), (2 * static_cast<ld>(n) + 1) * pi);
  for (int m = -M; m <= M; ++m)
    for (int l = 0; l < r; ++l) {
      const ld x = g.x[l];
      B[static_cast<size_t>(m + M) * r + l] =
          (m == 0 && g.x[l] == 0.0) ? cld(-b / 2, 0) : b * std::tanh(x / 2) / cld(-x, 2 * pi * m);
    }
  *EF = matmul(F, Kti, 2 * M, r);
  *EB = matmul(B, KBi, 2 * M + 1, r);
}

void plan_fft_axis(int L, FftAxisPlan* p, std::vector<int>* pos) {
  p->L = L;
  p->nfac = 0;
  int rem = L;
  while (rem % 4 == 0) { p->fac[p->nfac++] = 4; rem /= 4; }
  while (rem % 2 == 0) { p->fac[p->nfac++] = 2; rem /= 2; }
  for (int f = 3; rem > 1; f += 2)
    while (rem % f == 0) { p->fac[p->nfac++] = f; rem /= f; }
  // After the decimation-in-frequency stages, position
  //   i = k_1 (L/p_1) + k_2 (L/(p_1 p_2)) + ... + k_m
  // holds frequency f = k_1 + p_1 (k_2 + p_2 (k_3 + ...)).
  pos->assign(L, 0);
  for (int i = 0; i < L; ++i) {
    int rest = i, sub = L, f = 0, mult = 1;
    for (int s = 0; s < p->nfac; ++s) {
      sub /= p->fac[s];
      int k = rest / sub;
      rest %= sub;
      f += k * mult;
      mult *= p->fac[s];
    }
    (*pos)[f] = i;
  }
}

}  // namespace qa
