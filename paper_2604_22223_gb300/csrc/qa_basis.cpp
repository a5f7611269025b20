// Reduced pair basis for the screened interaction (host side).
//
// Every interaction matrix V(R) maps into, and is read from, the span of the
// columns of the matrices V(R) and V(R)^H over the listed R.  Let the columns
// of B (npair x rho, orthonormal) span that subspace.  Then
// V(q) = B S(q) B^H for every q with S(q) = B^H V(q) B, and the paper's Dyson
// equation for the screened interaction, W = V + V P W, closes inside the
// subspace (W = V + V P W puts both the range and the row space of W in it):
//   W = B Wt B^H,  Wt = S + S Pt Wt,  Pt = B^H P B,
//   W^C = B (1 - S Pt)^-1 S Pt S B^H.
// For Kanamori plus density-density interactions rho = norb + norb(norb-1)/2
// (15 of 25 pairs for five orbitals, 2 of 4 for a two-site density-density
// model).  It is an exact instance of the rank reduction of the orbital-index
// contraction that the paper proposes for the O(N_orb^4) polarizability
// (Sec. "Results", five-orbital benchmark).
//
// Construction, aimed at a sparse B: the pairs split into connected
// components (two pairs are connected when one column of some V(R) or V(R)^H
// is non-zero on both).  A component whose columns have full rank keeps its
// unit vectors e_A; a rank-deficient one gets the orthonormal vectors of a
// column-pivoted Gram-Schmidt with re-orthogonalisation (long double), stopping
// when the largest remaining column norm falls below 1e-13 of the largest
// column norm of all V(R).
#include <algorithm>
#include <cmath>
#include <complex>
#include <numeric>
#include <vector>

#include "qa_internal.h"

namespace qa {

namespace {

using cld = std::complex<long double>;

int find_root(std::vector<int>& parent, int x) {
  while (parent[x] != x) {
    parent[x] = parent[parent[x]];
    x = parent[x];
  }
  return x;
}

}  // namespace

int reduced_pair_basis(const std::vector<std::complex<double>>& VR, int nV, int npair,
                       std::vector<std::complex<double>>* B) {
  B->clear();
  const int n = npair;
  if (nV <= 0 || n <= 0) return 0;
  // columns of X = [V(R_1), V(R_1)^H, V(R_2), ...] as vectors of length n
  std::vector<std::vector<cld>> cols;
  for (int v = 0; v < nV; ++v) {
    const std::complex<double>* X = VR.data() + static_cast<size_t>(v) * n * n;
    for (int j = 0; j < n; ++j) {
      std::vector<cld> c1(n), c2(n);
      for (int i = 0; i < n; ++i) {
        const std::complex<double> a = X[static_cast<size_t>(i) * n + j];   // column j of V
        const std::complex<double> b = X[static_cast<size_t>(j) * n + i];   // column j of V^H
        c1[i] = cld(a.real(), a.imag());
        c2[i] = cld(b.real(), -b.imag());
      }
      cols.push_back(c1);
      cols.push_back(c2);
    }
  }
  long double cmax = 0;
  for (const auto& c : cols) {
    long double s = 0;
    for (const cld& x : c) s += std::norm(x);
    cmax = std::max(cmax, std::sqrt(s));
  }
  if (!(cmax > 0)) return 0;
  const long double tol = 1e-13L * cmax;
  // components of the pairs
  std::vector<int> parent(n);
  std::iota(parent.begin(), parent.end(), 0);
  std::vector<char> touched(n, 0);
  for (const auto& c : cols) {
    int first = -1;
    for (int i = 0; i < n; ++i) {
      if (c[i] == cld(0)) continue;
      touched[i] = 1;
      if (first < 0) first = i;
      else parent[find_root(parent, i)] = find_root(parent, first);
    }
  }
  std::vector<std::vector<cld>> basis;    // full-length columns
  std::vector<char> done(n, 0);
  for (int s = 0; s < n; ++s) {
    if (!touched[s] || done[s]) continue;
    const int root = find_root(parent, s);
    std::vector<int> comp;
    for (int i = 0; i < n; ++i)
      if (touched[i] && find_root(parent, i) == root) { comp.push_back(i); done[i] = 1; }
    const int m = static_cast<int>(comp.size());
    // this component's columns, restricted to its rows
    std::vector<std::vector<cld>> cc;
    for (const auto& c : cols) {
      if (c[comp[0]] == cld(0)) {
        bool any = false;
        for (int i : comp) any |= (c[i] != cld(0));
        if (!any) continue;
      }
      std::vector<cld> x(m);
      for (int k = 0; k < m; ++k) x[k] = c[comp[k]];
      cc.push_back(x);
    }
    // column-pivoted Gram-Schmidt with one re-orthogonalisation pass
    std::vector<std::vector<cld>> q;
    std::vector<char> taken(cc.size(), 0);
    while (static_cast<int>(q.size()) < m) {
      int best = -1;
      long double bn = 0;
      for (size_t k = 0; k < cc.size(); ++k) {
        if (taken[k]) continue;
        long double s2 = 0;
        for (const cld& x : cc[k]) s2 += std::norm(x);
        if (s2 > bn) { bn = s2; best = static_cast<int>(k); }
      }
      if (best < 0 || std::sqrt(bn) <= tol) break;
      taken[best] = 1;
      std::vector<cld> u = cc[best];
      for (int pass = 0; pass < 2; ++pass)
        for (const auto& e : q) {
          cld d(0);
          for (int k = 0; k < m; ++k) d += std::conj(e[k]) * u[k];
          for (int k = 0; k < m; ++k) u[k] -= d * e[k];
        }
      long double nu = 0;
      for (const cld& x : u) nu += std::norm(x);
      nu = std::sqrt(nu);
      if (!(nu > tol)) continue;
      for (cld& x : u) x /= nu;
      q.push_back(u);
      // remove the new direction from every remaining column
      for (size_t k = 0; k < cc.size(); ++k) {
        if (taken[k]) continue;
        cld d(0);
        for (int i = 0; i < m; ++i) d += std::conj(u[i]) * cc[k][i];
        for (int i = 0; i < m; ++i) cc[k][i] -= d * u[i];
      }
    }
    if (static_cast<int>(q.size()) == m) {
      for (int k = 0; k < m; ++k) {     // full rank: unit vectors keep B sparse
        std::vector<cld> e(n, cld(0));
        e[comp[k]] = cld(1);
        basis.push_back(e);
      }
    } else {
      for (const auto& u : q) {
        std::vector<cld> e(n, cld(0));
        for (int k = 0; k < m; ++k) e[comp[k]] = u[k];
        basis.push_back(e);
      }
    }
  }
  const int rho = static_cast<int>(basis.size());
  B->assign(static_cast<size_t>(n) * rho, std::complex<double>(0, 0));
  for (int j = 0; j < rho; ++j)
    for (int i = 0; i < n; ++i)
      (*B)[static_cast<size_t>(i) * rho + j] =
          std::complex<double>(static_cast<double>(basis[j][i].real()),
                               static_cast<double>(basis[j][i].imag()));
  return rho;
}

void pair_basis_terms(const std::vector<std::complex<double>>& B, int norb, int rho, double s,
                      PairTerms* bubble, PairTerms* sigma) {
  const int np = norb * norb;
  std::vector<std::vector<int>> supp(rho);
  for (int j = 0; j < rho; ++j)
    for (int A = 0; A < np; ++A)
      if (B[static_cast<size_t>(A) * rho + j] != std::complex<double>(0, 0)) supp[j].push_back(A);
  for (PairTerms* t : {bubble, sigma}) {
    t->off.assign(1, 0);
    t->idx.clear();
    t->coef.clear();
  }
  for (int i = 0; i < rho; ++i)
    for (int j = 0; j < rho; ++j) {
      for (int A : supp[i])
        for (int Bp : supp[j]) {
          const int a = A / norb, b = A % norb, c = Bp / norb, d = Bp % norb;
          const std::complex<double> bi = B[static_cast<size_t>(A) * rho + i];
          const std::complex<double> bj = B[static_cast<size_t>(Bp) * rho + j];
          // Pt_ij += conj(B_Ai) B_Bj P_AB,  P_(ab),(cd) = -s G_bc G^refl_da
          bubble->idx.push_back((b * norb + c) | ((d * norb + a) << 8));
          bubble->coef.push_back(-s * std::conj(bi) * bj);
          // Sigma_ad += -B_(ab)i conj(B_(cd)j) G_bc Wt_ij
          sigma->idx.push_back((b * norb + c) | ((a * norb + d) << 8));
          sigma->coef.push_back(-bi * std::conj(bj));
        }
      bubble->off.push_back(static_cast<int>(bubble->idx.size()));
      sigma->off.push_back(static_cast<int>(sigma->idx.size()));
    }
  for (PairTerms* t : {bubble, sigma}) {
    t->distinct_targets = true;
    for (size_t o = 0; o + 1 < t->off.size() && t->distinct_targets; ++o)
      for (int e = t->off[o]; e < t->off[o + 1] && t->distinct_targets; ++e)
        for (int f = e + 1; f < t->off[o + 1]; ++f)
          if ((t->idx[e] >> 8) == (t->idx[f] >> 8)) { t->distinct_targets = false; break; }
  }
}

}  // namespace qa
