// C ABI of libqa: problem validation, the host planner (DLR grid, FFT plans,
// index maps), device workspace layout, and the stage sequence of one GW
// iteration (paper Fig. 3(b)).  Every arithmetic step of the iteration runs
// in the CUDA kernels of qa_*.cu; the host only orders launches and runs the
// scalar chemical-potential search on device-computed densities.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "../../include/qa.h"
#include "qa_internal.h"

using cd = std::complex<double>;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// The three arithmetic modes: T = double (QA_FP64), qa::dfl (QA_MIXED,
// double-float storage of every tensor), float (QA_FP32).
template <typename T> constexpr bool is_f64() { return std::is_same<T, double>::value; }
template <typename T> constexpr bool is_df() { return std::is_same<T, qa::dfl>::value; }
template <typename T> constexpr bool is_f32() { return std::is_same<T, float>::value; }

struct DevTables {          // DLR matrices in one precision (complex)
  void* Trefl = nullptr;
  void* Ttn = nullptr;
  void* Tnt = nullptr;
  void* Ttw = nullptr;
  void* Twt = nullptr;
  void* dtau = nullptr;
  void* dw = nullptr;
};

}  // namespace

// Scalar results the host reads after every density evaluation and at the end
// of a call: pinned host memory that the kernels write through its device
// alias, so reading them needs a stream synchronisation but no copy (copies of
// large buffers on other streams, which share the copy engines, never delay them).
struct QaMailbox {
  double red[2];            // reduction results
  long long bad;            // first failing (nu, q) or (n, k) index
  int err;                  // device error word
  int pad;
  double2 nloc[25];         // local density matrix
  qa::MuState mus;          // final state of the device-side chemical-potential search
};

struct qa_ctx {
  // problem
  int n[3] = {1, 1, 1};
  int nk = 1, norb = 1, npair = 1, nspin = 2, r = 0, precision = QA_FP64;
  double beta = 1, Lambda = 1, eps = 1e-10, filling = 1;
  std::vector<int> hopR;          // [nH][3]
  std::vector<cd> hopH;           // [nH][norb][norb], H(R)
  std::vector<int> vR;            // [nV + 1][3], last = R 0 (for the Hartree density)
  std::vector<cd> vV;             // [nV][npair][npair]
  int nH = 0, nV = 0;
  qa::DlrGrid grid;
  qa::DlrMatrices mats;
  qa::FftAxisPlan ax[3];
  std::vector<int> pos[3];
  std::vector<int> mR;            // -R map
  // device
  bool bound = false;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  DevTables t64, t32, tdf;
  double* d_iw = nullptr;
  void* d_tw64 = nullptr;
  void* d_tw32 = nullptr;
  void* d_twdf = nullptr;
  int* d_pos = nullptr;
  int* d_mR = nullptr;
  int* d_hR = nullptr;
  double2* d_hH = nullptr;
  int* d_vR = nullptr;
  double2* d_vV = nullptr;
  double2* d_Hk = nullptr;
  void* d_Vq = nullptr;
  double2* d_G0 = nullptr;
  void* d_Gk = nullptr;       // G_in in the compute precision (QA_MIXED, QA_FP32)
  void* d_Grefl = nullptr;    // G(k, beta-tau) then G(-R..) in place
  void* d_GR = nullptr;
  double2* d_nk = nullptr;    // [norb^2][N_k] FP64 density of G_in
  double2* d_nR = nullptr;    // [nV+1][norb^2]
  double2* d_sigFR = nullptr; // [nV+1][norb^2]
  double2* d_SigHF = nullptr; // [N_k][norb^2]
  void* d_SigC = nullptr;     // Sigma^C(R,tau) -> (k,tau)
  void* d_SigIw = nullptr;    // Sigma^C(k, i w)
  void* d_Giw = nullptr;      // G(k, i w) (sized for FP64)
  void* d_Gt = nullptr;       // G(k, tau) / n(k) scratch (sized for FP64)
  void* d_P = nullptr;
  void* d_W = nullptr;
  float* d_colscale = nullptr;  // per-column slice grids of the tensor-core DLR maps (mixed)
  unsigned char* d_ozcode = nullptr;  // [r][nb^2 N_k] grid codes of a big-tensor map's input (mixed)
  double* d_part = nullptr;
  double* d_red = nullptr;
  int* d_err = nullptr;
  long long* d_bad = nullptr;
  double2* d_nloc = nullptr;
  qa::FftDev fft64{}, fft32{}, fftdf{};
  int nblocks_g = 1;
  double mu0 = 0.0, mu = 0.0;
  bool have_mu = false;
  bool timing = false;
  int launches = 0;           // kernels launched by the current call
  bool mu_fixed = false;      // qa_set_mu: use mu_value instead of the search
  long long wait_limit = -1;  // qa_set_wait_limit: polls of the tensor-core kernels' pipeline waits
  double mu_value = 0.0;
  // adjoint (FP64 contexts only)
  DevTables tH;               // conjugate transposes of the FP64 DLR matrices
  double2* d_GRbar = nullptr;
  double2* d_GLbar = nullptr;
  double2* d_Sbar = nullptr;  // [norb^2][N_k]
  double* d_Vqbar = nullptr;  // [npair^2][N_k] complex as doubles
  double2* d_X = nullptr;     // density_R outputs
  double2* d_VbarHF = nullptr;
  double2* d_nbarR = nullptr;
  double2* d_tbar = nullptr;
  double2* d_Vbar = nullptr;
  double2* d_nbar = nullptr;
  void* d_lu = nullptr;           // LU factors of 1 - V P (full-basis FP64 contexts)
  unsigned char* d_piv = nullptr; // their pivot rows [r][npair][N_k]
  bool keep_lu = false;           // the next FP64 forward keeps them (set by the adjoint)
  int nH_user = 0;
  // tensor-core DLR operands (QA_FP32 contexts)
  bool use_tc = false;
  std::vector<uint16_t> tc_Ttn, tc_Tnt, tc_Trefl, tc_Ttw, tc_Twt;
  void* d_tc_Ttn = nullptr;
  void* d_tc_Tnt = nullptr;
  void* d_tc_Trefl = nullptr;
  void* d_tc_Ttw = nullptr;
  void* d_tc_Twt = nullptr;
  // tensor-core DLR operands of the accurate mixed path (fixed-point bf16 slices)
  bool use_oz = false;
  std::vector<uint8_t> oz_Ttn, oz_Tnt, oz_Trefl, oz_Ttw, oz_Twt;
  void* d_oz_Ttn = nullptr;
  void* d_oz_Tnt = nullptr;
  void* d_oz_Trefl = nullptr;
  void* d_oz_Ttw = nullptr;
  void* d_oz_Twt = nullptr;
  void* d_Pnu = nullptr;          // third big tensor (QA_MIXED): P(q, i nu)
  int* d_tgo = nullptr;           // Sigma terms regrouped by target entry (QA_MIXED): offsets,
  void* d_tgi = nullptr;          // (Wt entry, G entry) pairs
  void* d_tgc = nullptr;          // and double-float coefficients
  // pair basis of the big tensors: full (npair) or reduced (rho, qa_basis.cpp)
  int pair_mode = QA_PAIRS_AUTO;
  bool reduced = false;
  int rho = 0;                    // rank of the interaction subspace
  int sig_canon = 0;              // norb when the Sigma terms follow the canonical pattern
  bool dtau_real = false;         // the density weights dtau are real (they are by construction)
  int nb = 1;                     // size of the big-tensor matrices (npair or rho)
  std::vector<cd> basis;          // [npair][rho]
  std::vector<cd> sV;             // [nV][rho][rho] = B^H V(R) B
  bool s_real = false;            // S(q) real for all q: every S(R) real with S(-R) = S(R)
  bool tsig_real = false;         // every Sigma term coefficient real
  bool tbub_real = false;         // every bubble term coefficient real
  qa::PairTerms tbub, tsig;
  int* d_tbub = nullptr;          // off + idx
  void* d_cbub = nullptr;         // coefficients (compute precision)
  int* d_tsig = nullptr;
  void* d_csig = nullptr;
  double2* d_sV = nullptr;        // [nV][rho][rho] FP64
  void* d_Bm = nullptr;           // mu-independent part of the G Dyson argument (sized for FP64)
  double2* d_phV = nullptr;       // [nV + 1][N_k] e^{+i k.R_v} of the interaction's R list
  void* d_hs = nullptr;           // [N_k][norb^2] double-float mu - H - Sigma^HF (mixed density check)
  double mu_ref = 0.0;            // reference chemical potential folded into d_Bm
  // Hartree-Fock loop and quasiparticle quantities
  double2* d_wq = nullptr;        // [2][r] weights of Sigma(+i w0), Sigma(-i w0)
  bool sighf_valid = false;       // d_SigHF holds the last step's (or the HF loop's) Sigma^HF
  bool sigc_valid = false;        // d_SigIw holds the last step's Sigma^C(k, i w)
  qa::DysonBlocks dblk;           // diagonal blocks of S(q) on the reduced basis (nblk = 0: none)
  QaMailbox* mb = nullptr;        // pinned host mailbox (qa_bind) and its device alias
  QaMailbox* mb_dev = nullptr;
  size_t ws_need = 0;             // workspace bytes of the bound layout
  // grand potential (qa_free_energy): uniform-frequency maps of cutoff om_M,
  // fermionic / bosonic chunk rows om_cf / om_cb, and the scratch they use
  int om_M = 0, om_cf = 0, om_cb = 0;
  double2* d_omEF = nullptr;      // [2M][r]
  double2* d_omEFH = nullptr;     // per fermionic chunk: [r][rows] conjugate transpose
  double2* d_omEB = nullptr;      // [2M+1][r]
  double2* d_omEBH = nullptr;     // per bosonic chunk: [r][rows]
  char* d_om = nullptr;           // scratch (allocated on the first qa_free_energy call)
  // device-side chemical-potential search: its state and one instantiated graph
  // (a while-node over [density, update]) per arithmetic, built on first use
  qa::MuState* d_mus = nullptr;
  cudaGraphExec_t mu_exec[3] = {nullptr, nullptr, nullptr};
  void drop_mu_graphs() {
    for (cudaGraphExec_t& g : mu_exec)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
  }
  ~qa_ctx() {
    drop_mu_graphs();
    if (d_mus) cudaFree(d_mus);
    if (mb) cudaFreeHost(mb);
    for (void* p : {static_cast<void*>(d_omEF), static_cast<void*>(d_omEFH), static_cast<void*>(d_omEB),
                    static_cast<void*>(d_omEBH), static_cast<void*>(d_om)})
      if (p) cudaFree(p);
  }
};

namespace {

#define QA_TRY(x)                                   \
  do {                                              \
    cudaError_t e__ = (x);                          \
    if (e__ != cudaSuccess) return QA_ECUDA;        \
  } while (0)

// a launcher call that enqueues `n` kernels
#define QA_LAUNCH(c, n, x)                          \
  do {                                              \
    QA_TRY(x);                                      \
    (c)->launches += (n);                           \
  } while (0)

bool small_primes_only(int L) {
  for (int p = 2; p <= L; ++p)
    while (L % p == 0) {
      if (p > 13) return false;
      L /= p;
    }
  return true;
}

int grid_index(const qa_ctx* c, int i1, int i2, int i3) {
  return (i1 * c->n[1] + i2) * c->n[2] + i3;
}

// Pair basis of the big tensors.  The interaction subspace (rank rho, basis
// B) is found on the host; the reduced basis is used when the mode asks for it
// (QA_PAIRS_AUTO: on the mixed path) and 0 < rho < npair with term lists that
// fit the reduced kernels.  Then S(R) = B^H V(R) B replaces V(R) in the Dyson
// equation for W.  With `bound` set (the workspace is laid out) the choice and
// rho must stay as they are.
int setup_pairs(qa_ctx* c, bool bound) {
  std::vector<cd> B;
  const int rho = qa::reduced_pair_basis(c->vV, c->nV, c->npair, &B);
  qa::PairTerms tb, ts;
  bool ok = rho > 0 && rho < c->npair;
  if (ok) {
    qa::pair_basis_terms(B, c->norb, rho, static_cast<double>(c->nspin), &tb, &ts);
    ok = static_cast<int>(tb.idx.size()) <= qa::kMaxPairTerms &&
         static_cast<int>(ts.idx.size()) <= qa::kMaxPairTerms;
  }
  const bool want = c->pair_mode == QA_PAIRS_REDUCED ||
                    (c->pair_mode == QA_PAIRS_AUTO && c->precision != QA_FP64);
  const bool red = want && ok;
  if (bound && (red != c->reduced || (red && rho != c->rho))) return QA_EINVAL;
  if (!red) {
    // the full product basis is the special case B = identity (one term per entry)
    std::vector<cd> I(static_cast<size_t>(c->npair) * c->npair, cd(0, 0));
    for (int A = 0; A < c->npair; ++A) I[static_cast<size_t>(A) * c->npair + A] = cd(1, 0);
    qa::pair_basis_terms(I, c->norb, c->npair, static_cast<double>(c->nspin), &tb, &ts);
  }
  c->rho = rho;
  c->basis = B;
  c->reduced = red;
  c->nb = red ? rho : c->npair;
  c->tbub = tb;
  c->tsig = ts;
  c->sig_canon = red ? qa::sigma_canonical_norb(ts.off.data(), ts.idx.data(),
                                                static_cast<int>(ts.off.size()) - 1,
                                                static_cast<int>(ts.idx.size()), c->norb)
                     : 0;
  c->sV.clear();
  if (red) {
    const int np = c->npair;
    c->sV.assign(static_cast<size_t>(c->nV) * rho * rho, cd(0, 0));
    for (int v = 0; v < c->nV; ++v) {
      const cd* X = c->vV.data() + static_cast<size_t>(v) * np * np;
      std::vector<cd> XB(static_cast<size_t>(np) * rho, cd(0, 0));      // V(R) B
      for (int A = 0; A < np; ++A)
        for (int Bp = 0; Bp < np; ++Bp) {
          const cd x = X[static_cast<size_t>(A) * np + Bp];
          if (x == cd(0, 0)) continue;
          for (int j = 0; j < rho; ++j) XB[static_cast<size_t>(A) * rho + j] += x * B[static_cast<size_t>(Bp) * rho + j];
        }
      cd* S = c->sV.data() + static_cast<size_t>(v) * rho * rho;
      for (int A = 0; A < np; ++A)
        for (int i = 0; i < rho; ++i) {
          const cd bi = std::conj(B[static_cast<size_t>(A) * rho + i]);
          if (bi == cd(0, 0)) continue;
          for (int j = 0; j < rho; ++j) S[static_cast<size_t>(i) * rho + j] += bi * XB[static_cast<size_t>(A) * rho + j];
        }
    }
  }
  // diagonal blocks of S: indices coupled by some S(R) entry, as contiguous ranges
  c->dblk = qa::DysonBlocks{};
  if (red && rho <= 16) {
    std::vector<int> comp(rho);
    for (int i = 0; i < rho; ++i) comp[i] = i;
    auto root = [&](int x) { while (comp[x] != x) x = comp[x] = comp[comp[x]]; return x; };
    for (int v = 0; v < c->nV; ++v)
      for (int i = 0; i < rho; ++i)
        for (int k = 0; k < rho; ++k)
          if (c->sV[(static_cast<size_t>(v) * rho + i) * rho + k] != cd(0, 0)) comp[root(i)] = root(k);
    bool contiguous = true;
    int nblk = 0;
    for (int i = 0; i < rho && contiguous;) {
      int k = i;
      while (k < rho && root(k) == root(i)) ++k;
      for (int t = k; t < rho; ++t)
        if (root(t) == root(i)) contiguous = false;
      for (int t = i; t < k; ++t) {
        c->dblk.lo[t] = static_cast<unsigned char>(i);
        c->dblk.hi[t] = static_cast<unsigned char>(k);
      }
      ++nblk;
      i = k;
    }
    c->dblk.nblk = contiguous ? nblk : 0;
  }
  return QA_OK;
}

// Room for the term lists: every list a later qa_set_params can make (rho^2
// outputs of at most npair^2 terms each, capped by the kernels' limit), or
// one term per entry on the full basis.
size_t term_capacity(const qa_ctx* c) {
  if (!c->reduced) return static_cast<size_t>(c->npair) * c->npair;
  const size_t bound = static_cast<size_t>(c->rho) * c->rho * c->npair * c->npair;
  return std::min(bound, static_cast<size_t>(qa::kMaxPairTerms));
}

// the largest term count of one output entry
int max_terms_per_entry(const qa::PairTerms& t) {
  int m = 0;
  for (size_t o = 0; o + 1 < t.off.size(); ++o) m = std::max(m, t.off[o + 1] - t.off[o]);
  return m;
}

// layout of the workspace; when `base` is null only sizes are accumulated
size_t layout(qa_ctx* c, char* base) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> void* {
    void* p = base ? base + off : nullptr;
    off += align_up(bytes);
    return p;
  };
  const size_t r = c->r, nk = c->nk, no2 = static_cast<size_t>(c->norb) * c->norb,
               np2 = static_cast<size_t>(c->npair) * c->npair,
               nb2 = static_cast<size_t>(c->nb) * c->nb;    // big-tensor matrix entries
  const size_t es = c->precision == QA_FP32 ? 8 : 16;   // big/compute element size
  const size_t rr = r * r;
  for (DevTables* t : {&c->t64, &c->t32, &c->tdf}) {
    const size_t e = (t == &c->t32) ? 8 : 16;
    t->Trefl = take(rr * e);
    t->Ttn = take(rr * e);
    t->Tnt = take(rr * e);
    t->Ttw = take(rr * e);
    t->Twt = take(rr * e);
    t->dtau = take(r * e);
    t->dw = take(r * e);
  }
  const size_t ntw = c->n[0] + c->n[1] + c->n[2];
  c->d_iw = static_cast<double*>(take(r * 8));
  c->d_tw64 = take(ntw * 16);
  c->d_tw32 = take(ntw * 8);
  c->d_twdf = take(ntw * 16);
  c->d_pos = static_cast<int*>(take(ntw * 4));
  c->d_mR = static_cast<int*>(take(nk * 4));
  c->d_hR = static_cast<int*>(take(std::max(1, c->nH) * 12));
  c->d_hH = static_cast<double2*>(take(std::max(1, c->nH) * no2 * 16));
  c->d_vR = static_cast<int*>(take((c->nV + 1) * 12));
  c->d_vV = static_cast<double2*>(take(std::max(1, c->nV) * np2 * 16));
  c->d_Hk = static_cast<double2*>(take(nk * no2 * 16));
  c->d_Vq = take(nk * nb2 * es);
  c->d_G0 = static_cast<double2*>(take(r * no2 * nk * 16));
  c->d_Gk = take(r * no2 * nk * es);
  c->d_Grefl = take(r * no2 * nk * es);
  c->d_GR = take(r * no2 * nk * es);
  c->d_nk = static_cast<double2*>(take(no2 * nk * 16));
  c->d_nR = static_cast<double2*>(take((c->nV + 1) * no2 * 16));
  c->d_sigFR = static_cast<double2*>(take((c->nV + 1) * no2 * 16));
  c->d_SigHF = static_cast<double2*>(take(nk * no2 * 16));
  c->d_SigC = take(r * no2 * nk * es);
  c->d_SigIw = take(r * no2 * nk * es);
  c->d_Giw = take(r * no2 * nk * 16);
  c->d_Gt = take(r * no2 * nk * 16);
  c->d_Bm = take(r * no2 * nk * 16);
  c->d_phV = static_cast<double2*>(take((c->nV + 1) * nk * 16));
  c->d_hs = take(nk * no2 * 16);
  // big tensors last; P must also hold the FP64 V(q) staging of qa_bind
  c->d_P = take(std::max(r * nb2 * nk * es, nk * nb2 * 16));
  c->d_W = take(r * nb2 * nk * es);
  if (c->precision == QA_MIXED && c->use_oz) {
    c->d_Pnu = take(r * nb2 * nk * es);
    c->d_colscale = static_cast<float*>(take(std::max(nb2, no2) * nk * 4));
    c->d_ozcode = static_cast<unsigned char*>(take(r * nb2 * nk));
  }
  if (c->precision == QA_MIXED) {
    const size_t cap = term_capacity(c);
    c->d_tgo = static_cast<int*>(take((no2 + 1) * 4));
    c->d_tgi = take(cap * 8);
    c->d_tgc = take(cap * 16);
  }
  c->nblocks_g = qa::dyson_g_blocks(c->r, c->nk);
  c->d_part = static_cast<double*>(take(2 * static_cast<size_t>(c->nblocks_g) * 8));
  c->d_red = static_cast<double*>(take(2 * 8));
  c->d_err = static_cast<int*>(take(4));
  c->d_bad = static_cast<long long*>(take(8));
  c->d_nloc = static_cast<double2*>(take(no2 * 16));
  c->d_wq = static_cast<double2*>(take(2 * r * 16));
  if (c->precision == QA_MIXED && c->use_oz) {
    c->d_oz_Ttn = take(c->oz_Ttn.size());
    c->d_oz_Tnt = take(c->oz_Tnt.size());
    c->d_oz_Trefl = take(c->oz_Trefl.size());
    c->d_oz_Ttw = take(c->oz_Ttw.size());
    c->d_oz_Twt = take(c->oz_Twt.size());
  }
  if (c->precision == QA_FP32 && c->use_tc) {
    c->d_tc_Ttn = take(c->tc_Ttn.size() * 2);
    c->d_tc_Tnt = take(c->tc_Tnt.size() * 2);
    c->d_tc_Trefl = take(c->tc_Trefl.size() * 2);
    c->d_tc_Ttw = take(c->tc_Ttw.size() * 2);
    c->d_tc_Twt = take(c->tc_Twt.size() * 2);
  }
  {
    if (c->reduced) c->d_sV = static_cast<double2*>(take(std::max(1, c->nV) * nb2 * 16));
    const size_t cap = term_capacity(c);
    c->d_tbub = static_cast<int*>(take((nb2 + 1 + cap) * 4));
    c->d_cbub = take(cap * es);
    c->d_tsig = static_cast<int*>(take((nb2 + 1 + cap) * 4));
    c->d_csig = take(cap * es);
  }
  if (c->precision == QA_FP64) {
    c->tH.Trefl = take(rr * 16);
    c->tH.Ttn = take(rr * 16);
    c->tH.Tnt = take(rr * 16);
    c->tH.Ttw = take(rr * 16);
    c->tH.Twt = take(rr * 16);
    c->tH.dtau = take(r * 16);
    c->d_GRbar = static_cast<double2*>(take(r * no2 * nk * 16));
    c->d_GLbar = static_cast<double2*>(take(r * no2 * nk * 16));
    c->d_Sbar = static_cast<double2*>(take(no2 * nk * 16));
    c->d_Vqbar = static_cast<double*>(take(np2 * nk * 16));
    const size_t nx = std::max({static_cast<size_t>(c->nV + 1) * no2, static_cast<size_t>(c->nH) * no2,
                                static_cast<size_t>(std::max(1, c->nV)) * np2});
    c->d_X = static_cast<double2*>(take(nx * 16));
    c->d_VbarHF = static_cast<double2*>(take(std::max(1, c->nV) * np2 * 16));
    c->d_nbarR = static_cast<double2*>(take((c->nV + 1) * no2 * 16));
    c->d_tbar = static_cast<double2*>(take(std::max(1, c->nH) * no2 * 16));
    c->d_Vbar = static_cast<double2*>(take(std::max(1, c->nV) * np2 * 16));
    c->d_nbar = static_cast<double2*>(take(no2 * 16));
    c->d_lu = take(r * nb2 * nk * 16);
    c->d_piv = static_cast<unsigned char*>(take(r * c->nb * nk));
  }
  return off;
}

template <typename T>
cudaError_t upload_c(void* dst, const std::vector<cd>& src, cudaStream_t st) {
  if (is_f64<T>()) {
    return cudaMemcpyAsync(dst, src.data(), src.size() * 16, cudaMemcpyHostToDevice, st);
  }
  std::vector<float> f;
  if (is_df<T>()) {
    // double-float: (re.hi, re.lo, im.hi, im.lo), hi = rn(x), lo = rn(x - hi)
    f.resize(4 * src.size());
    auto split = [](double x, float* o) {
      o[0] = static_cast<float>(x);
      o[1] = static_cast<float>(x - static_cast<double>(o[0]));
    };
    for (size_t i = 0; i < src.size(); ++i) {
      split(src[i].real(), &f[4 * i]);
      split(src[i].imag(), &f[4 * i + 2]);
    }
  } else {
    f.resize(2 * src.size());
    for (size_t i = 0; i < src.size(); ++i) {
      f[2 * i] = static_cast<float>(src[i].real());
      f[2 * i + 1] = static_cast<float>(src[i].imag());
    }
  }
  cudaError_t e = cudaMemcpyAsync(dst, f.data(), f.size() * 4, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);   // f goes out of scope
}

// The interaction tables of the Dyson equation for W: V(q) on the full pair
// basis, or the term lists, S(R) = B^H V(R) B and S(q) on the reduced one.
int upload_interaction(qa_ctx* c, cudaStream_t st) {
  const int nb2 = c->nb * c->nb;
  const double2* src = c->d_vV;
  {
    c->tbub_real = true;
    for (const cd& v : c->tbub.coef)
      if (v.imag() != 0.0) c->tbub_real = false;
    const qa::PairTerms* tl[2] = {&c->tbub, &c->tsig};
    int* di[2] = {c->d_tbub, c->d_tsig};
    void* dc[2] = {c->d_cbub, c->d_csig};
    for (int k = 0; k < 2; ++k) {
      std::vector<int> iv(tl[k]->off);
      iv.insert(iv.end(), tl[k]->idx.begin(), tl[k]->idx.end());
      QA_TRY(cudaMemcpyAsync(di[k], iv.data(), iv.size() * 4, cudaMemcpyHostToDevice, st));
      QA_TRY(cudaStreamSynchronize(st));
      if (c->precision == QA_FP64) QA_TRY(upload_c<double>(dc[k], tl[k]->coef, st));
      else if (c->precision == QA_MIXED) QA_TRY(upload_c<qa::dfl>(dc[k], tl[k]->coef, st));
      else QA_TRY(upload_c<float>(dc[k], tl[k]->coef, st));
    }
  }
  if (c->precision == QA_MIXED) {
    // the Sigma terms grouped by target entry Sigma_ad (idx >> 8), in list order
    const qa::PairTerms& ts = c->tsig;
    const int no2 = c->norb * c->norb, nout = static_cast<int>(ts.off.size()) - 1;
    std::vector<int> toff(no2 + 1, 0), tidx;
    std::vector<cd> tcoef;
    for (int tg = 0; tg < no2; ++tg) {
      toff[tg] = static_cast<int>(tcoef.size());
      for (int o = 0; o < nout; ++o)
        for (int e = ts.off[o]; e < ts.off[o + 1]; ++e)
          if ((ts.idx[e] >> 8) == tg) {
            tidx.push_back(o);
            tidx.push_back(ts.idx[e] & 255);
            tcoef.push_back(ts.coef[e]);
          }
    }
    toff[no2] = static_cast<int>(tcoef.size());
    c->tsig_real = true;
    for (const cd& v : tcoef)
      if (v.imag() != 0.0) c->tsig_real = false;
    QA_TRY(cudaMemcpyAsync(c->d_tgo, toff.data(), toff.size() * 4, cudaMemcpyHostToDevice, st));
    QA_TRY(cudaMemcpyAsync(c->d_tgi, tidx.data(), tidx.size() * 4, cudaMemcpyHostToDevice, st));
    QA_TRY(upload_c<qa::dfl>(c->d_tgc, tcoef, st));
  }
  if (c->reduced) {
    if (c->nV > 0) QA_TRY(upload_c<double>(c->d_sV, c->sV, st));
    src = c->d_sV;
    // S(q) = sum_R S(R) e^{-iq.R} is real when every S(R) is real and S(-R) = S(R)
    const size_t nb2s = static_cast<size_t>(nb2);
    bool real = c->nV > 0;
    for (int v = 0; v < c->nV && real; ++v) {
      int w = -1;
      for (int u = 0; u < c->nV && w < 0; ++u)
        if (c->vR[3 * u] == -c->vR[3 * v] && c->vR[3 * u + 1] == -c->vR[3 * v + 1] &&
            c->vR[3 * u + 2] == -c->vR[3 * v + 2])
          w = u;
      if (w < 0) { real = false; break; }
      for (size_t e = 0; e < nb2s && real; ++e) {
        const cd a = c->sV[v * nb2s + e], b = c->sV[w * nb2s + e];
        if (a.imag() != 0.0 || a != b) real = false;
      }
    }
    c->s_real = real;
  }
  if (c->precision == QA_FP64) {
    QA_LAUNCH(c, 1, qa::launch_ft_table(c->d_vR, src, c->nV, nb2, nullptr, c->nk, c->n[0], c->n[1],
                                        c->n[2], static_cast<double2*>(c->d_Vq), st));
  } else {
    QA_LAUNCH(c, 1, qa::launch_ft_table(c->d_vR, src, c->nV, nb2, nullptr, c->nk, c->n[0], c->n[1],
                                        c->n[2], static_cast<double2*>(c->d_P), st));
    if (c->precision == QA_MIXED)
      QA_LAUNCH(c, 1, qa::launch_c128_to_df(static_cast<const double2*>(c->d_P), c->d_Vq,
                                            static_cast<long long>(c->nk) * nb2, st));
    else
      QA_LAUNCH(c, 1, qa::launch_c128_to_c64(static_cast<const double2*>(c->d_P),
                                             static_cast<float2*>(c->d_Vq),
                                             static_cast<long long>(c->nk) * nb2, st));
  }
  QA_TRY(cudaStreamSynchronize(st));
  return QA_OK;
}

// The mu-independent part of the G Dyson argument, relative to mu_ref, and
// an upper bound of the norm of H + Sigma - mu_ref (all k, all DLR nodes).
template <typename T>
int prepare_g(qa_ctx* c, const double2* SigHF, const void* SigIw, double mu_ref, double* bound,
              cudaStream_t st) {
  c->mu_ref = mu_ref;
  QA_LAUNCH(c, 1, qa::launch_dyson_g_prep<T>(c->d_Hk, SigHF, SigIw, mu_ref, c->r, c->norb, c->nk,
                                             c->d_Bm, c->d_part, c->nblocks_g, st));
  QA_LAUNCH(c, 1, qa::launch_reduce_pairs(c->d_part, c->nblocks_g, 1, c->d_red, st));
  double h[2];
  QA_TRY(cudaStreamSynchronize(st));
  h[0] = c->mb->red[0];
  h[1] = c->mb->red[1];
  *bound = h[0];
  return QA_OK;
}

// Density and derivative at mu (after prepare_g).  Result: N(mu), dN/dmu.
template <typename T>
int eval_density(qa_ctx* c, const DevTables& tab, double mu, double* N, double* dN,
                 cudaStream_t st) {
  QA_LAUNCH(c, 1, qa::launch_dyson_g<T>(c->d_Bm, tab.dw, c->d_iw, mu - c->mu_ref, c->r, c->norb,
                                        c->nk, nullptr, c->d_part, c->nblocks_g, 0, c->d_err, st));
  QA_LAUNCH(c, 1, qa::launch_reduce_pairs(c->d_part, c->nblocks_g, 0, c->d_red, st));
  double h[2];
  QA_TRY(cudaStreamSynchronize(st));
  h[0] = c->mb->red[0];
  h[1] = c->mb->red[1];
  *N = c->nspin * h[0] / c->nk;
  *dN = -c->nspin * h[1] / c->nk;
  return QA_OK;
}

// The device-side search's graph for arithmetic T: a while-node whose body
// is [density at the state's mu, update of the state], captured once per
// context (the pointers it holds are fixed by qa_bind).
template <typename T>
int mu_graph(qa_ctx* c, const DevTables& tab, cudaGraphExec_t* out) {
  const int slot = is_f64<T>() ? 0 : (is_df<T>() ? 1 : 2);
  if (c->mu_exec[slot]) {
    *out = c->mu_exec[slot];
    return QA_OK;
  }
  if (!c->d_mus && cudaMalloc(reinterpret_cast<void**>(&c->d_mus), sizeof(qa::MuState)) != cudaSuccess)
    return QA_ENOMEM;
  cudaGraph_t g = nullptr;
  cudaStream_t cs = nullptr;
  cudaGraphExec_t ex = nullptr;
  auto fail = [&]() {
    if (cs) cudaStreamDestroy(cs);
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return QA_ECUDA;
  };
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return fail();
  cudaGraphConditionalHandle cond;
  if (cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) return fail();
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) != cudaSuccess) return fail();
  cudaGraph_t body = np.conditional.phGraph_out[0];
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return fail();
  if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
      cudaSuccess)
    return fail();
  cudaError_t e1 = qa::launch_dyson_g<T>(c->d_Bm, tab.dw, c->d_iw, 0.0, c->r, c->norb, c->nk, nullptr,
                                         c->d_part, c->nblocks_g, 0, c->d_err, cs,
                                         reinterpret_cast<const double*>(c->d_mus));
  cudaError_t e2 = qa::launch_mu_update(c->d_part, c->nblocks_g, c->d_mus, static_cast<double>(c->nspin),
                                        c->nk, cond, cs);
  cudaGraph_t captured = nullptr;
  cudaError_t e3 = cudaStreamEndCapture(cs, &captured);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) return fail();
  cudaStreamDestroy(cs);
  cs = nullptr;
  if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) return fail();
  cudaGraphDestroy(g);
  c->mu_exec[slot] = ex;
  *out = ex;
  return QA_OK;
}

// Chemical potential: the root of N(mu) = filling (N increases with mu),
// found on the device (qa_mu.cu): Newton steps from the warm start mu_s (the
// previous mu) while each at least quarters the residual; otherwise a bracket
// by marching from the better point toward the root with growing steps,
// clamped to the window
// |mu - mu_s| <= max ||H + Sigma - mu_s|| + 1 + 10/beta outside which N is
// empty or full; then bisection with Newton steps taken when they stay inside
// the bracket and at least halve the step before last (safeguarded Newton).
// Stop when |N - filling| <= tolN or the bracket (or, on the FP32 path whose
// density carries ~1e-6 noise, the Newton step) is below tolB.  The whole
// search is one graph launch; the host reads its final state once.
template <typename T>
int mu_search(qa_ctx* c, const double2* SigHF, const void* SigIw, const DevTables& tab,
              double mu_start, double* mu_out, double* N_out, int* evals, cudaStream_t st) {
  const double mu_s = std::isfinite(mu_start) ? mu_start : 0.0;
  const double target = c->filling;
  const bool fp64 = !is_f32<T>();     // FP64 or double-float densities
  cudaGraphExec_t ex = nullptr;
  if (int rc = mu_graph<T>(c, tab, &ex)) return rc;
  c->mu_ref = mu_s;
  QA_LAUNCH(c, 1, qa::launch_dyson_g_prep<T>(c->d_Hk, SigHF, SigIw, mu_s, c->r, c->norb, c->nk,
                                             c->d_Bm, c->d_part, c->nblocks_g, st));
  QA_LAUNCH(c, 1, qa::launch_reduce_pairs(c->d_part, c->nblocks_g, 1, c->d_red, st));
  QA_LAUNCH(c, 1, qa::launch_mu_init(c->d_mus, c->d_red, mu_s, target, c->beta, fp64 ? 1 : 0, st));
  QA_TRY(cudaGraphLaunch(ex, st));
  QA_TRY(cudaMemcpyAsync(&c->mb->mus, c->d_mus, sizeof(qa::MuState), cudaMemcpyDeviceToHost, st));
  QA_TRY(cudaStreamSynchronize(st));
  const qa::MuState& ms = c->mb->mus;
  int count = ms.count;
  c->launches += 2 * std::max(count, 1);
  if (ms.status != QA_OK) return ms.status;
  double mu = ms.mu;
  double N = ms.N;
  if (!fp64) {
    // one FP64-accurate evaluation at the FP32 root (FP32 inverse refined by a
    // double-float residual step) and a Newton correction: removes the bias
    // of FP32 densities (the DLR density weights amplify FP32 rounding) from mu
    QA_LAUNCH(c, 2, qa::launch_dyson_g_refine(c->d_Hk, SigHF, SigIw, c->t64.dw, c->d_iw, mu, c->r,
                                              c->norb, c->nk, c->d_hs, c->d_part, c->nblocks_g,
                                              c->d_err, st));
    QA_LAUNCH(c, 1, qa::launch_reduce_pairs(c->d_part, c->nblocks_g, 0, c->d_red, st));
    double h2[2];
    QA_TRY(cudaStreamSynchronize(st));
    h2[0] = c->mb->red[0];
    h2[1] = c->mb->red[1];
    ++count;
    const double N64 = c->nspin * h2[0] / c->nk;
    const double d64 = -c->nspin * h2[1] / c->nk;
    N = N64;
    if (std::isfinite(N64) && d64 > 0) {
      const double step = (N64 - target) / d64;
      if (std::fabs(step) < 1e-3 * std::max(1.0, std::fabs(mu))) {
        mu -= step;
        N = N64 - step * d64;     // FP64 density linearised over the correction
      }
    }
  }
  *evals = count;
  *mu_out = mu;
  *N_out = N;
  return QA_OK;
}

int check_err(qa_ctx* c, qa_step_stats* stats, cudaStream_t st) {
  QA_TRY(cudaStreamSynchronize(st));
  const int herr = c->mb->err;
  const long long hbad = c->mb->bad;
  if (stats) {
    stats->status = herr;
    stats->first_bad = herr ? hbad : -1;
  }
  return herr;
}

int reset_err(qa_ctx* c, cudaStream_t st) {
  // host writes, ordered after the stream's earlier work
  QA_TRY(cudaStreamSynchronize(st));
  c->mb->err = 0;
  c->mb->bad = 0x7f7f7f7f7f7f7f7fLL;
  return QA_OK;
}

// G(k,tau) = Twt G(k, i w) at mu (after prepare_g), and the local density matrix.
template <typename T>
int finish_g(qa_ctx* c, const DevTables& tab, double mu, void* G_out_c128, double* n_out,
             cudaStream_t st) {
  const long long ncol = static_cast<long long>(c->norb) * c->norb * c->nk;
  QA_LAUNCH(c, 1, qa::launch_dyson_g<T>(c->d_Bm, tab.dw, c->d_iw, mu - c->mu_ref, c->r, c->norb,
                                        c->nk, c->d_Giw, c->d_part, c->nblocks_g, 1, c->d_err, st));
  if (is_f64<T>()) {
    QA_LAUNCH(c, 1, qa::launch_dlr_apply<T>(tab.Twt, c->r, c->r, c->d_Giw, G_out_c128, ncol, st));
  } else if (is_df<T>()) {
    if (c->use_oz) {
      // the transform stores complex128 directly
      QA_LAUNCH(c, 2, qa::launch_dlr_oz(c->d_oz_Twt, c->r, c->d_Giw, G_out_c128, ncol, c->d_err, st, true, c->wait_limit, c->d_colscale));
    } else {
      QA_LAUNCH(c, 1, qa::launch_dlr_apply<T>(tab.Twt, c->r, c->r, c->d_Giw, c->d_Gt, ncol, st));
      QA_LAUNCH(c, 1, qa::launch_df_to_c128(c->d_Gt, static_cast<double2*>(G_out_c128), ncol * c->r, st));
    }
  } else {
    if (c->use_tc) {
      // the transform stores complex128 directly
      QA_LAUNCH(c, 1, qa::launch_dlr_tc(c->d_tc_Twt, c->r, c->d_Giw, G_out_c128, ncol, c->d_err, st,
                                        true, c->wait_limit));
    } else {
      QA_LAUNCH(c, 1, qa::launch_dlr_apply<T>(tab.Twt, c->r, c->r, c->d_Giw, c->d_Gt, ncol, st));
      QA_LAUNCH(c, 1, qa::launch_c64_to_c128(static_cast<const float2*>(c->d_Gt),
                                             static_cast<double2*>(G_out_c128), ncol * c->r, st));
    }
  }
  if (n_out) {
    // n(k) = sum_n dw_n G(k, i w_n), then its k-average (n(R = 0))
    QA_LAUNCH(c, 1, qa::launch_dlr_apply<T>(tab.dw, 1, c->r, c->d_Giw, c->d_Gt, ncol, st));
    QA_LAUNCH(c, 1, qa::launch_k_average<T>(c->d_Gt, c->norb * c->norb, c->nk, c->d_nloc, st));
    QA_TRY(cudaStreamSynchronize(st));
    std::memcpy(n_out, c->mb->nloc, static_cast<size_t>(c->norb) * c->norb * 16);
  }
  return QA_OK;
}

struct StageTimer {
  qa_ctx* c;
  cudaStream_t st;
  cudaEvent_t ev[17];
  int n = 0;
  bool on;
  StageTimer(qa_ctx* cc, cudaStream_t s) : c(cc), st(s), on(cc->timing) {
    if (on)
      for (auto& e : ev) cudaEventCreate(&e);
    mark();
  }
  void mark() {
    if (on && n < 17) cudaEventRecord(ev[n++], st);
  }
  void finish(qa_step_stats* stats) {
    if (!on) return;
    cudaEventSynchronize(ev[n - 1]);
    for (int i = 0; i + 1 < n && i < 16; ++i) {
      float ms = 0;
      cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
      if (stats) stats->stage_ms[i] = ms;
    }
  }
  ~StageTimer() {
    if (on)
      for (auto& e : ev) cudaEventDestroy(e);
  }
};

// Stages of one iteration up to Sigma^C(k, i w) and Sigma^HF(k) from G_in
// (device, G layout, complex128).  Leaves G(R,tau), G(-R,beta-tau) (small),
// P(q, i nu) (big tensor 1), W^C(R, tau) (big tensor 2), Sigma^C(k, tau),
// Sigma^C(k, i w), Sigma^HF(k) and n(R_v) in the workspace.
template <typename T>
int forward_sigma(qa_ctx* c, const double2* Gin, StageTimer& tm, cudaStream_t st) {
  const DevTables& tab = is_f64<T>() ? c->t64 : (is_df<T>() ? c->tdf : c->t32);
  const qa::FftDev& fft = is_f64<T>() ? c->fft64 : (is_df<T>() ? c->fftdf : c->fft32);
  constexpr bool f32 = is_f32<T>();
  const int r = c->r, no2 = c->norb * c->norb, nk = c->nk, nb2 = c->nb * c->nb;
  const long long ncs = static_cast<long long>(no2) * nk;     // small-tensor columns
  const long long ncb = static_cast<long long>(nb2) * nk;     // big-tensor columns
  // n(k) = -G(k, beta^-) of the input (FP64) with G in the compute precision,
  // then Hartree and Fock (FP64)
  const void* Gk = Gin;
  if (!is_f64<T>()) Gk = c->d_Gk;
  if (is_df<T>())
    QA_LAUNCH(c, 1, qa::launch_g_input_df(Gin, static_cast<const double2*>(c->t64.dtau), r, ncs,
                                          c->d_Gk, c->d_nk, st, c->dtau_real));
  else
    QA_LAUNCH(c, 1, qa::launch_g_input(Gin, static_cast<const double2*>(c->t64.dtau), r, ncs,
                                       f32 ? static_cast<float2*>(c->d_Gk) : nullptr,
                                       c->d_nk, st, c->dtau_real));
  QA_LAUNCH(c, 1, qa::launch_density_R(c->d_nk, c->d_vR, c->nV + 1, no2, nullptr, nk, c->n[0], c->n[1],
                              c->n[2], c->d_nR, st, c->d_phV));
  QA_LAUNCH(c, 2, qa::launch_hf(c->d_vV, c->d_nR, c->d_vR, c->nV, c->norb, c->nspin, nullptr, nk, c->n[0],
                       c->n[1], c->n[2], c->d_sigFR, c->d_SigHF, st, c->d_phV));
  tm.mark();  // 0: HF
  // G(k, beta - tau), real-space G
  const bool oz = is_df<T>() && c->use_oz;
  if (f32 && c->use_tc)
    QA_LAUNCH(c, 1, qa::launch_dlr_tc(c->d_tc_Trefl, r, Gk, c->d_Grefl, ncs, c->d_err, st, false, c->wait_limit));
  else if (oz)
    QA_LAUNCH(c, 2, qa::launch_dlr_oz(c->d_oz_Trefl, r, Gk, c->d_Grefl, ncs, c->d_err, st, false, c->wait_limit, c->d_colscale));
  else
    QA_LAUNCH(c, 1, qa::launch_dlr_apply<T>(tab.Trefl, r, r, Gk, c->d_Grefl, ncs, st));
  QA_LAUNCH(c, 1, qa::launch_fft3d<T>(fft, +1, Gk, c->d_GR, ncs / nk * r, st));
  QA_LAUNCH(c, 1, qa::launch_fft3d<T>(fft, +1, c->d_Grefl, c->d_Grefl, ncs / nk * r, st));
  tm.mark();  // 1: G -> R
  bool p_codes = false;   // the bubble stage stored the grid codes of P(q, tau)
  if (qa::fft3d_bubble_supported(fft) && max_terms_per_entry(c->tbub) <= 640) {
    // bubble and R -> q transform in one pass (the bubble stage reads as 0)
    tm.mark();  // 2: bubble
    QA_LAUNCH(c, 1, qa::launch_fft3d_bubble<T>(fft, c->d_GR, c->d_Grefl, c->d_mR, c->d_tbub, c->d_cbub,
                                               max_terms_per_entry(c->tbub), nb2, c->norb, c->d_P, r, st,
                                               c->d_err, c->tbub_real, oz ? c->d_ozcode : nullptr));
    p_codes = oz && qa::fft3d_bubble_codes(fft);
  } else {
    if (c->reduced)
      QA_LAUNCH(c, 1, qa::launch_bubble_reduced<T>(c->d_GR, c->d_Grefl, c->d_mR, c->d_tbub, c->d_cbub,
                                                   static_cast<int>(c->tbub.idx.size()), c->d_P, r,
                                                   c->norb, c->rho, nk, st));
    else
      QA_LAUNCH(c, 1, qa::launch_bubble<T>(c->d_GR, c->d_Grefl, c->d_mR, c->d_P, r, c->norb, nk, c->nspin, st));
    tm.mark();  // 2: bubble
    QA_LAUNCH(c, 1, qa::launch_fft3d<T>(fft, -1, c->d_P, c->d_P, ncb / nk * r, st));
  }
  tm.mark();  // 3: FFT R -> q
  if (oz) {
    // out-of-place tensor-core maps: P(q, tau) [P] -> P(q, i nu) [Pnu] -> W^C(q, i nu) [P]
    // -> W^C(q, tau) [W]
    // (the slice grids of both maps come from the grid codes their producers store,
    // where those producers write them)
    QA_LAUNCH(c, 2, qa::launch_dlr_oz(c->d_oz_Ttn, r, c->d_P, c->d_Pnu, ncb, c->d_err, st, false, c->wait_limit,
                                      c->d_colscale, p_codes ? c->d_ozcode : nullptr));
    tm.mark();  // 4: DLR tau -> nu
    const bool w_codes = qa::dyson_w_df_supported(c->nb);
    if (w_codes)
      QA_LAUNCH(c, 1, qa::launch_dyson_w_df(c->d_Pnu, c->d_Vq, c->d_P, r, c->nb, nk, c->d_err, c->d_bad,
                                            st, &c->dblk, c->s_real, c->d_ozcode));
    else
      QA_LAUNCH(c, 1, qa::launch_dyson_w<T>(c->d_Pnu, c->d_Vq, c->d_P, r, c->nb, nk, c->d_err, c->d_bad,
                                            st, &c->dblk));
    tm.mark();  // 5: Dyson W
    QA_LAUNCH(c, 2, qa::launch_dlr_oz(c->d_oz_Tnt, r, c->d_P, c->d_W, ncb, c->d_err, st, false, c->wait_limit,
                                      c->d_colscale, w_codes ? c->d_ozcode : nullptr));
  } else {
    if (f32 && c->use_tc)
      QA_LAUNCH(c, 1, qa::launch_dlr_tc(c->d_tc_Ttn, r, c->d_P, c->d_P, ncb, c->d_err, st, false, c->wait_limit));
    else
      QA_LAUNCH(c, 1, qa::launch_dlr_apply<T>(tab.Ttn, r, r, c->d_P, c->d_P, ncb, st));
    tm.mark();  // 4: DLR tau -> nu
    const bool keep = is_f64<T>() && c->keep_lu && c->d_lu;
    QA_LAUNCH(c, 1, qa::launch_dyson_w<T>(c->d_P, c->d_Vq, c->d_W, r, c->nb, nk, c->d_err, c->d_bad, st,
                                          &c->dblk, keep ? c->d_lu : nullptr, keep ? c->d_piv : nullptr));
    tm.mark();  // 5: Dyson W
    if (f32 && c->use_tc)
      QA_LAUNCH(c, 1, qa::launch_dlr_tc(c->d_tc_Tnt, r, c->d_W, c->d_W, ncb, c->d_err, st, false, c->wait_limit));
    else
      QA_LAUNCH(c, 1, qa::launch_dlr_apply<T>(tab.Tnt, r, r, c->d_W, c->d_W, ncb, st));
  }
  tm.mark();  // 6: DLR nu -> tau
  QA_LAUNCH(c, 1, qa::launch_fft3d<T>(fft, +1, c->d_W, c->d_W, ncb / nk * r, st));
  tm.mark();  // 7: FFT q -> R
  if (c->reduced && f32 && c->sig_canon)
    QA_LAUNCH(c, 1, qa::launch_sigma_canonical(c->d_GR, c->d_W, c->tsig.coef.data(), c->sig_canon,
                                               c->d_SigC, r, nk, st));
  else if (is_df<T>())
    QA_LAUNCH(c, 1, qa::launch_sigma_target_df(c->d_GR, c->d_W, c->d_tgo, c->d_tgi, c->d_tgc, c->d_SigC,
                                               r, c->norb, nb2, nk, st, c->d_err, c->tsig_real));
  else if (c->reduced)
    QA_LAUNCH(c, 1, qa::launch_sigma_reduced<T>(c->d_GR, c->d_W, c->d_tsig, c->d_csig,
                                                static_cast<int>(c->tsig.idx.size()), c->d_SigC, r,
                                                c->norb, c->rho, nk, st, c->tsig.distinct_targets));
  else
    QA_LAUNCH(c, 1, qa::launch_sigma<T>(c->d_GR, c->d_W, c->d_SigC, r, c->norb, nk, st));
  tm.mark();  // 8: Sigma contraction
  QA_LAUNCH(c, 1, qa::launch_fft3d<T>(fft, -1, c->d_SigC, c->d_SigC, ncs / nk * r, st));
  if (f32 && c->use_tc)
    QA_LAUNCH(c, 1, qa::launch_dlr_tc(c->d_tc_Ttw, r, c->d_SigC, c->d_SigIw, ncs, c->d_err, st, false, c->wait_limit));
  else if (oz)
    QA_LAUNCH(c, 2, qa::launch_dlr_oz(c->d_oz_Ttw, r, c->d_SigC, c->d_SigIw, ncs, c->d_err, st, false, c->wait_limit, c->d_colscale));
  else
    QA_LAUNCH(c, 1, qa::launch_dlr_apply<T>(tab.Ttw, r, r, c->d_SigC, c->d_SigIw, ncs, st));
  tm.mark();  // 9: Sigma -> (k, i w)
  c->sighf_valid = c->sigc_valid = true;
  return QA_OK;
}

template <typename T>
int gw_step_impl(qa_ctx* c, const void* G_in, void* G_out, double* mu_out, double* n_out,
                 qa_step_stats* stats, cudaStream_t st) {
  const DevTables& tab = is_f64<T>() ? c->t64 : (is_df<T>() ? c->tdf : c->t32);
  const double2* Gin = static_cast<const double2*>(G_in ? G_in : c->d_G0);
  c->launches = 0;
  if (int rc = reset_err(c, st)) return rc;
  StageTimer tm(c, st);
  if (int rc = forward_sigma<T>(c, Gin, tm, st)) return rc;
  double mu = 0, N = 0;
  int evals = 0;
  int rc = QA_OK;
  if (c->mu_fixed) {
    double dN = 0, bound = 0;
    mu = c->mu_value;
    rc = prepare_g<T>(c, c->d_SigHF, c->d_SigIw, mu, &bound, st);
    if (rc == QA_OK) rc = eval_density<T>(c, tab, mu, &N, &dN, st);
    evals = 1;
  } else {
    rc = mu_search<T>(c, c->d_SigHF, c->d_SigIw, tab, c->have_mu ? c->mu : c->mu0, &mu, &N,
                      &evals, st);
  }
  if (rc != QA_OK) {
    // a device-side failure earlier in the step (a singular Dyson pivot, a
    // timed-out wait) is the cause of what the search saw: report it first
    const int herr = check_err(c, stats, st);
    return herr ? herr : rc;
  }
  tm.mark();  // 10: mu search
  rc = finish_g<T>(c, tab, mu, G_out, n_out, st);
  if (rc != QA_OK) {
    const int herr = check_err(c, stats, st);
    return herr ? herr : rc;
  }
  tm.mark();  // 11: Dyson G + G(tau)
  tm.finish(stats);
  c->mu = mu;
  c->have_mu = true;
  if (mu_out) *mu_out = mu;
  if (stats) {
    stats->mu = mu;
    stats->N = N;
    stats->mu_evals = evals;
    stats->launches = c->launches;
  }
  int herr = check_err(c, stats, st);
  return herr;
}

// ------------------------------------------------ grand potential (FP64)

// Scratch of the grand potential (d_om): eigen-decomposition of H + Sigma^HF,
// the cotangents collected before the adjoint chain runs, frequency chunks,
// per-point terms and the four accumulated terms.
struct OmScratch {
  double* E;
  double2* U;
  double2* abar;      // [norb^2][N_k] cotangent of H + Sigma^HF
  double2* sig_x;     // [norb^2][N_k] cotangent of Sigma^HF alone
  double2* nbar_x;    // [norb^2][N_k] cotangent of n(k)
  double2* sbar_tau;  // [r][norb^2][N_k] cotangent of Sigma^C(k, tau)
  double2* gbar_tau;  // [r][norb^2][N_k] cotangent of G_in
  double2* bufS;
  double2* bufG;
  double2* bufA;
  double2* bufP;
  double2* bufV;
  double* part;
  double* acc;        // [4]: Omega_HF, Omega_dc, Omega_G, Omega_W
};

size_t om_layout(const qa_ctx* c, int cf, int cb, OmScratch* o) {
  const size_t nk = c->nk, no = c->norb, no2 = no * no, r = c->r;
  const size_t ncs = no2 * nk, ncb = static_cast<size_t>(c->nb) * c->nb * nk;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t a = off;
    off += align_up(bytes);
    return a;
  };
  const size_t oE = take(nk * no * 8), oU = take(nk * no2 * 16), oA = take(ncs * 16), oSx = take(ncs * 16),
               oNx = take(ncs * 16), oSt = take(r * ncs * 16), oGt = take(r * ncs * 16),
               oBS = take(cf * ncs * 16), oBG = take(cf * ncs * 16), oBA = take(cf * ncs * 16),
               oBP = take(cb * ncb * 16), oBV = take(cb * ncb * 16),
               oPart = take(std::max({2 * nk, static_cast<size_t>(cf) * nk, static_cast<size_t>(cb) * nk}) * 8),
               oAcc = take(4 * 8);
  if (o) {
    char* b = c->d_om;
    o->E = reinterpret_cast<double*>(b + oE);
    o->U = reinterpret_cast<double2*>(b + oU);
    o->abar = reinterpret_cast<double2*>(b + oA);
    o->sig_x = reinterpret_cast<double2*>(b + oSx);
    o->nbar_x = reinterpret_cast<double2*>(b + oNx);
    o->sbar_tau = reinterpret_cast<double2*>(b + oSt);
    o->gbar_tau = reinterpret_cast<double2*>(b + oGt);
    o->bufS = reinterpret_cast<double2*>(b + oBS);
    o->bufG = reinterpret_cast<double2*>(b + oBG);
    o->bufA = reinterpret_cast<double2*>(b + oBA);
    o->bufP = reinterpret_cast<double2*>(b + oBP);
    o->bufV = reinterpret_cast<double2*>(b + oBV);
    o->part = reinterpret_cast<double*>(b + oPart);
    o->acc = reinterpret_cast<double*>(b + oAcc);
  }
  return off;
}

void om_free(qa_ctx* c) {
  for (double2** p : {&c->d_omEF, &c->d_omEFH, &c->d_omEB, &c->d_omEBH}) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  if (c->d_om) cudaFree(c->d_om);
  c->d_om = nullptr;
  c->om_M = 0;
}

// Uniform-frequency maps of cutoff M (and their per-chunk conjugate
// transposes) and the scratch, allocated on first use and kept.
int ensure_omega(qa_ctx* c, int M) {
  if (c->om_M == M && c->d_om) return QA_OK;
  om_free(c);
  std::vector<cd> EF, EB;
  qa::build_uniform_maps(c->grid, c->beta, M, &EF, &EB);
  const int r = c->r;
  const size_t ncs = static_cast<size_t>(c->norb) * c->norb * c->nk;
  const size_t ncb = static_cast<size_t>(c->nb) * c->nb * c->nk;
  const size_t cap = static_cast<size_t>(512) << 20;     // bytes of one chunk buffer at most
  const int cf = static_cast<int>(std::min<size_t>({static_cast<size_t>(2 * M), 256,
                                                    std::max<size_t>(1, cap / (ncs * 16))}));
  const int cb = static_cast<int>(std::min<size_t>({static_cast<size_t>(2 * M + 1), 256,
                                                    std::max<size_t>(1, cap / (ncb * 16))}));
  auto chunked_h = [r](const std::vector<cd>& A, int rows_all, int ch) {
    std::vector<cd> H(A.size());
    for (int j0 = 0; j0 < rows_all; j0 += ch) {
      const int rows = std::min(ch, rows_all - j0);
      for (int j = 0; j < r; ++j)
        for (int i = 0; i < rows; ++i)
          H[static_cast<size_t>(j0) * r + static_cast<size_t>(j) * rows + i] =
              std::conj(A[static_cast<size_t>(j0 + i) * r + j]);
    }
    return H;
  };
  const std::vector<cd> EFH = chunked_h(EF, 2 * M, cf), EBH = chunked_h(EB, 2 * M + 1, cb);
  struct Up {
    double2** dst;
    const std::vector<cd>* src;
  } ups[4] = {{&c->d_omEF, &EF}, {&c->d_omEFH, &EFH}, {&c->d_omEB, &EB}, {&c->d_omEBH, &EBH}};
  for (const Up& u : ups) {
    if (cudaMalloc(reinterpret_cast<void**>(u.dst), u.src->size() * 16) != cudaSuccess) {
      om_free(c);
      return QA_ENOMEM;
    }
    QA_TRY(cudaMemcpy(*u.dst, u.src->data(), u.src->size() * 16, cudaMemcpyHostToDevice));
  }
  if (cudaMalloc(reinterpret_cast<void**>(&c->d_om), om_layout(c, cf, cb, nullptr)) != cudaSuccess) {
    om_free(c);
    return QA_ENOMEM;
  }
  c->om_M = M;
  c->om_cf = cf;
  c->om_cb = cb;
  return QA_OK;
}

// The four terms of the grand potential for the G_in whose stages
// forward_sigma<double> has just computed (Sigma^HF, n, Sigma^C(k, tau),
// P(q, i nu) in place), into parts[4] on the host.
int omega_value(qa_ctx* c, const double2* Gin, double mu, double* parts, cudaStream_t st) {
  OmScratch o;
  om_layout(c, c->om_cf, c->om_cb, &o);
  const int r = c->r, no = c->norb, nk = c->nk, nb = c->nb, M = c->om_M;
  const long long ncs = static_cast<long long>(no) * no * nk, ncb = static_cast<long long>(nb) * nb * nk;
  const double s = c->nspin, beta = c->beta;
  QA_TRY(cudaMemsetAsync(o.acc, 0, 4 * sizeof(double), st));
  QA_LAUNCH(c, 1, qa::launch_hf_eig(c->d_Hk, c->d_SigHF, no, nk, o.E, o.U, st));
  QA_LAUNCH(c, 1, qa::launch_omega_hf(o.E, o.U, c->d_SigHF, c->d_nk, no, nk, beta, mu, o.part, nullptr, 0.0, st));
  QA_LAUNCH(c, 1, qa::launch_sum_scalar(o.part, nk, -s / (beta * nk), o.acc, 0, st));
  QA_LAUNCH(c, 1, qa::launch_sum_scalar(o.part + nk, nk, -0.5 * s / nk, o.acc, 1, st));
  for (int j0 = 0; j0 < 2 * M; j0 += c->om_cf) {
    const int rows = std::min(c->om_cf, 2 * M - j0);
    const double2* E = c->d_omEF + static_cast<size_t>(j0) * r;
    QA_LAUNCH(c, 1, qa::launch_dlr_apply<double>(E, rows, r, c->d_SigC, o.bufS, ncs, st));
    QA_LAUNCH(c, 1, qa::launch_dlr_apply<double>(E, rows, r, Gin, o.bufG, ncs, st));
    QA_LAUNCH(c, 1, qa::launch_omega_g(c->d_Hk, c->d_SigHF, o.bufS, o.bufG, j0 - M, rows, no, nk, beta, mu,
                                       o.part, nullptr, 0.0, 0.0, c->d_err, st));
    QA_LAUNCH(c, 1, qa::launch_sum_scalar(o.part, static_cast<long long>(rows) * nk, -s / (beta * nk), o.acc, 2, st));
  }
  for (int j0 = 0; j0 < 2 * M + 1; j0 += c->om_cb) {
    const int rows = std::min(c->om_cb, 2 * M + 1 - j0);
    QA_LAUNCH(c, 1, qa::launch_dlr_apply<double>(c->d_omEB + static_cast<size_t>(j0) * r, rows, r, c->d_P,
                                                 o.bufP, ncb, st));
    QA_LAUNCH(c, 1, qa::launch_omega_w(o.bufP, static_cast<const double2*>(c->d_Vq), nb, nk, rows, o.part,
                                       nullptr, 0.0, c->d_err, st));
    QA_LAUNCH(c, 1, qa::launch_sum_scalar(o.part, static_cast<long long>(rows) * nk, 1.0 / (2.0 * beta * nk),
                                          o.acc, 3, st));
  }
  QA_TRY(cudaMemcpyAsync(parts, o.acc, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  QA_TRY(cudaStreamSynchronize(st));
  return QA_OK;
}

// Cotangents of the grand potential's explicit dependences, taken before the
// adjoint chain reuses the forward buffers: abar (H + Sigma^HF), sig_x
// (Sigma^HF alone), nbar_x (n(k)), sbar_tau (Sigma^C(k, tau)), gbar_tau (G_in).
int omega_bwd_pre(qa_ctx* c, const double2* Gin, double mu, double wbar, cudaStream_t st) {
  OmScratch o;
  om_layout(c, c->om_cf, c->om_cb, &o);
  const int r = c->r, no = c->norb, nk = c->nk, M = c->om_M;
  const long long ncs = static_cast<long long>(no) * no * nk;
  const double s = c->nspin, beta = c->beta, cg = s / (beta * nk);
  QA_LAUNCH(c, 1, qa::launch_hf_eig(c->d_Hk, c->d_SigHF, no, nk, o.E, o.U, st));
  QA_LAUNCH(c, 1, qa::launch_omega_hf(o.E, o.U, c->d_SigHF, c->d_nk, no, nk, beta, mu, o.part, o.abar,
                                      s / nk * wbar, st));
  QA_LAUNCH(c, 1, qa::launch_herm_scale(c->d_nk, 0, no, nk, -0.5 * s / nk * wbar, o.sig_x, st));
  QA_LAUNCH(c, 1, qa::launch_herm_scale(c->d_SigHF, 1, no, nk, -0.5 * s / nk * wbar, o.nbar_x, st));
  QA_TRY(cudaMemsetAsync(o.sbar_tau, 0, static_cast<size_t>(r) * ncs * 16, st));
  QA_TRY(cudaMemsetAsync(o.gbar_tau, 0, static_cast<size_t>(r) * ncs * 16, st));
  for (int j0 = 0; j0 < 2 * M; j0 += c->om_cf) {
    const int rows = std::min(c->om_cf, 2 * M - j0);
    const double2* E = c->d_omEF + static_cast<size_t>(j0) * r;
    const double2* EH = c->d_omEFH + static_cast<size_t>(j0) * r;
    QA_LAUNCH(c, 1, qa::launch_dlr_apply<double>(E, rows, r, c->d_SigC, o.bufS, ncs, st));
    QA_LAUNCH(c, 1, qa::launch_dlr_apply<double>(E, rows, r, Gin, o.bufG, ncs, st));
    QA_LAUNCH(c, 1, qa::launch_omega_g(c->d_Hk, c->d_SigHF, o.bufS, o.bufG, j0 - M, rows, no, nk, beta, mu,
                                       o.part, o.bufA, -cg * wbar, cg * wbar, c->d_err, st));
    QA_LAUNCH(c, 1, qa::launch_sum_rows(o.bufA, rows, ncs, o.abar, 1, st));
    QA_LAUNCH(c, 1, qa::launch_dlr_apply<double>(EH, r, rows, o.bufS, o.sbar_tau, ncs, st, 1));
    QA_LAUNCH(c, 1, qa::launch_dlr_apply<double>(EH, r, rows, o.bufG, o.gbar_tau, ncs, st, 1));
  }
  return QA_OK;
}

// The ring term's cotangents: Pbar(q, i nu_j) += EB^H Pbar_m, Vbar(q) += sum_m
// (P W P)^H terms; needs P(q, i nu) (d_P) intact.
int omega_bwd_w(qa_ctx* c, double wbar, double2* Pbar_nu, cudaStream_t st) {
  OmScratch o;
  om_layout(c, c->om_cf, c->om_cb, &o);
  const int r = c->r, nk = c->nk, nb = c->nb, M = c->om_M;
  const long long ncb = static_cast<long long>(nb) * nb * nk;
  const double cw = -wbar / (2.0 * c->beta * nk);
  for (int j0 = 0; j0 < 2 * M + 1; j0 += c->om_cb) {
    const int rows = std::min(c->om_cb, 2 * M + 1 - j0);
    QA_LAUNCH(c, 1, qa::launch_dlr_apply<double>(c->d_omEB + static_cast<size_t>(j0) * r, rows, r, c->d_P,
                                                 o.bufP, ncb, st));
    QA_LAUNCH(c, 1, qa::launch_omega_w(o.bufP, static_cast<const double2*>(c->d_Vq), nb, nk, rows, o.part,
                                       o.bufV, cw, c->d_err, st));
    QA_LAUNCH(c, 1, qa::launch_sum_rows(o.bufV, rows, ncb, reinterpret_cast<double2*>(c->d_Vqbar), 1, st));
    QA_LAUNCH(c, 1, qa::launch_dlr_apply<double>(c->d_omEBH + static_cast<size_t>(j0) * r, r, rows, o.bufP,
                                                 Pbar_nu, ncb, st, 1));
  }
  return QA_OK;
}

// Adjoint of one iteration at fixed mu (FP64).  Recomputes the forward
// stages from G_in (P is recomputed, not stored), then pulls the cotangents
// back stage by stage (qa_adjoint.cu).
int gw_backward_impl(qa_ctx* c, const double2* Gin, double mu, const double2* Gbar_out,
                     const double2* Sigbar, const double* nbar, double2* Gbar_in, double* grad_t,
                     double* grad_V, cudaStream_t st, double wbar = 0.0) {
  const qa::FftDev& fft = c->fft64;
  // big tensors in the context's pair basis: nb = npair (full) or rho (reduced)
  const int r = c->r, no2 = c->norb * c->norb, nk = c->nk, np2 = c->npair * c->npair, nb2 = c->nb * c->nb;
  const long long ncs = static_cast<long long>(no2) * nk;
  const long long ncb = static_cast<long long>(nb2) * nk;
  const long long lines_s = static_cast<long long>(no2) * r, lines_b = static_cast<long long>(nb2) * r;
  c->launches = 0;
  if (int rc = reset_err(c, st)) return rc;
  bool timing = c->timing;
  c->timing = false;
  StageTimer tm(c, st);
  c->timing = timing;
  c->keep_lu = true;
  const int frc = forward_sigma<double>(c, Gin, tm, st);
  c->keep_lu = false;
  if (frc) return frc;
  // grand-potential cotangent (wbar != 0): its explicit terms first
  OmScratch om{};
  if (wbar != 0.0) {
    om_layout(c, c->om_cf, c->om_cb, &om);
    if (int rc = omega_bwd_pre(c, Gin, mu, wbar, st)) return rc;
  }
  double2* Giw_bar = static_cast<double2*>(c->d_Giw);
  double2* SigIw_bar = static_cast<double2*>(c->d_Gt);
  double2* Sig_bar = static_cast<double2*>(c->d_SigC);
  double2* Wbig = static_cast<double2*>(c->d_W);
  // outputs -> Gbar(k, i w)
  if (Gbar_out) {
    QA_LAUNCH(c, 1, qa::launch_dlr_apply<double>(c->tH.Twt, r, r, Gbar_out, Giw_bar, ncs, st));
  } else {
    QA_TRY(cudaMemsetAsync(Giw_bar, 0, static_cast<size_t>(ncs) * r * 16, st));
  }
  if (nbar) {
    QA_TRY(cudaMemcpyAsync(c->d_nbar, nbar, no2 * 16, cudaMemcpyHostToDevice, st));
    QA_LAUNCH(c, 1, qa::launch_add_dw_nbar(Giw_bar, static_cast<const double2*>(c->t64.dw), c->d_nbar,
                                           r, no2, nk, st));
  }
  // Dyson for G
  QA_LAUNCH(c, 1, qa::launch_dyson_g_bwd(c->d_Hk, c->d_SigHF, static_cast<const double2*>(c->d_SigIw),
                                         c->d_iw, mu, r, c->norb, nk, Giw_bar, SigIw_bar, c->d_Sbar, st));
  if (wbar != 0.0) QA_LAUNCH(c, 1, qa::launch_axpy(c->d_Sbar, om.abar, 1.0, ncs, st));
  // Sigma^C(k, i w) <- Sigma^C(k, tau) <- Sigma^C(R, tau)
  QA_LAUNCH(c, 1, qa::launch_dlr_apply<double>(c->tH.Ttw, r, r, SigIw_bar, Sig_bar, ncs, st));
  if (Sigbar) QA_LAUNCH(c, 1, qa::launch_axpy(Sig_bar, Sigbar, 1.0, ncs * r, st));
  if (wbar != 0.0) QA_LAUNCH(c, 1, qa::launch_axpy(Sig_bar, om.sbar_tau, 1.0, ncs * r, st));
  QA_LAUNCH(c, 1, qa::launch_fft3d<double>(fft, +1, Sig_bar, Sig_bar, lines_s, st, 1.0));
  // Sigma contraction: Gbar(R) and Wbar(R, tau) (in place over W^C)
  if (c->reduced)
    QA_LAUNCH(c, 1, qa::launch_sigma_bwd_terms(static_cast<const double2*>(c->d_GR), Sig_bar, Wbig, c->d_GRbar,
                                               c->d_tsig, static_cast<const double2*>(c->d_csig), r, nb2,
                                               c->norb, nk, st));
  else
    QA_LAUNCH(c, 1, qa::launch_sigma_bwd(static_cast<const double2*>(c->d_GR), Sig_bar, Wbig, c->d_GRbar,
                                         r, c->norb, nk, st));
  // W^C(R, tau) <- W^C(q, tau) <- W^C(q, i nu)
  QA_LAUNCH(c, 1, qa::launch_fft3d<double>(fft, -1, Wbig, Wbig, lines_b, st, 1.0 / nk));
  QA_LAUNCH(c, 1, qa::launch_dlr_apply<double>(c->tH.Tnt, r, r, Wbig, Wbig, ncb, st));
  // Dyson for W: Pbar (in place) and Vbar(q)
  QA_TRY(cudaMemsetAsync(c->d_Vqbar, 0, static_cast<size_t>(ncb) * 16, st));
  QA_LAUNCH(c, 1, qa::launch_dyson_w_bwd(static_cast<const double2*>(c->d_P),
                                         static_cast<const double2*>(c->d_Vq), Wbig, c->d_Vqbar, r,
                                         c->nb, nk, c->d_err, st,
                                         static_cast<const double2*>(c->d_lu), c->d_piv));
  if (wbar != 0.0)
    if (int rc = omega_bwd_w(c, wbar, Wbig, st)) return rc;
  // P(q, i nu) <- P(q, tau) <- P(R, tau)
  QA_LAUNCH(c, 1, qa::launch_dlr_apply<double>(c->tH.Ttn, r, r, Wbig, Wbig, ncb, st));
  QA_LAUNCH(c, 1, qa::launch_fft3d<double>(fft, +1, Wbig, Wbig, lines_b, st, 1.0));
  // bubble
  if (c->reduced)
    QA_LAUNCH(c, 1, qa::launch_bubble_bwd_terms(static_cast<const double2*>(c->d_GR),
                                                static_cast<const double2*>(c->d_Grefl), c->d_mR, Wbig,
                                                c->d_GRbar, c->d_GLbar, c->d_tbub,
                                                static_cast<const double2*>(c->d_cbub), r, nb2, c->norb, nk, st));
  else
    QA_LAUNCH(c, 1, qa::launch_bubble_bwd(static_cast<const double2*>(c->d_GR),
                                          static_cast<const double2*>(c->d_Grefl), c->d_mR, Wbig,
                                          c->d_GRbar, c->d_GLbar, r, c->norb, nk, c->nspin, st));
  // G(R) <- G(k) and G(-R, beta - tau) <- G(k, beta - tau) <- G(k, tau)
  QA_LAUNCH(c, 1, qa::launch_fft3d<double>(fft, -1, c->d_GRbar, c->d_GRbar, lines_s, st, 1.0 / nk));
  QA_LAUNCH(c, 1, qa::launch_fft3d<double>(fft, -1, c->d_GLbar, c->d_GLbar, lines_s, st, 1.0 / nk));
  double2* gin = Gbar_in ? Gbar_in : reinterpret_cast<double2*>(c->d_Gk);
  QA_LAUNCH(c, 1, qa::launch_dlr_apply<double>(c->tH.Trefl, r, r, c->d_GLbar, gin, ncs, st));
  QA_LAUNCH(c, 1, qa::launch_axpy(gin, c->d_GRbar, 1.0, ncs * r, st));
  if (wbar != 0.0) QA_LAUNCH(c, 1, qa::launch_axpy(gin, om.gbar_tau, 1.0, ncs * r, st));
  // t(R) = -H(R): tbar(R) = -sum_k e^{+ik.R} Hbar(k)
  QA_LAUNCH(c, 1, qa::launch_density_R(c->d_Sbar, c->d_hR, c->nH, no2, nullptr, nk, c->n[0], c->n[1],
                                       c->n[2], c->d_tbar, st));
  QA_LAUNCH(c, 1, qa::launch_scale(c->d_tbar, -static_cast<double>(nk), static_cast<long long>(c->nH) * no2, st));
  // Sigma^HF alone carries the grand potential's double-counting term
  if (wbar != 0.0) QA_LAUNCH(c, 1, qa::launch_axpy(c->d_Sbar, om.sig_x, 1.0, ncs, st));
  // Hartree and Fock: (H, Sigma^HF) bar -> Sigma^H bar, Sigma^F bar(R_v) -> Vbar, nbar
  QA_LAUNCH(c, 1, qa::launch_density_R(c->d_Sbar, c->d_vR, c->nV + 1, no2, nullptr, nk, c->n[0],
                                       c->n[1], c->n[2], c->d_X, st));
  QA_LAUNCH(c, 1, qa::launch_hf_bwd(c->d_vV, c->d_nR, c->d_X, c->nV, c->norb, c->nspin, nk,
                                    c->d_VbarHF, c->d_nbarR, st));
  QA_LAUNCH(c, 1, qa::launch_nbar_k(c->d_nbarR, c->d_vR, c->nV + 1, no2, nk, c->n[0], c->n[1],
                                    c->n[2], c->d_nk, st));
  if (wbar != 0.0) QA_LAUNCH(c, 1, qa::launch_axpy(c->d_nk, om.nbar_x, 1.0, ncs, st));
  QA_LAUNCH(c, 1, qa::launch_dlr_apply<double>(c->tH.dtau, r, 1, c->d_nk, gin, ncs, st, 1));
  // V(R): sum_q e^{+iq.R} Vbar(q) plus the Hartree/Fock part.  On the reduced
  // basis the Dyson adjoint gives the cotangent of S(q) = B^H V(q) B, so
  // Vbar(R) = B Sbar(R) B^H (on the host: nV small matrices).
  if (c->nV > 0) {
    QA_LAUNCH(c, 1, qa::launch_density_R(reinterpret_cast<const double2*>(c->d_Vqbar), c->d_vR, c->nV,
                                         nb2, nullptr, nk, c->n[0], c->n[1], c->n[2], c->d_Vbar, st));
    QA_LAUNCH(c, 1, qa::launch_scale(c->d_Vbar, static_cast<double>(nk), static_cast<long long>(c->nV) * nb2, st));
    if (!c->reduced)
      QA_LAUNCH(c, 1, qa::launch_axpy(c->d_Vbar, c->d_VbarHF, 1.0, static_cast<long long>(c->nV) * np2, st));
  }
  if (grad_t)
    QA_TRY(cudaMemcpyAsync(grad_t, c->d_tbar, static_cast<size_t>(c->nH_user) * no2 * 16,
                           cudaMemcpyDeviceToHost, st));
  std::vector<cd> sbar, vhf;
  if (grad_V && c->nV > 0) {
    if (c->reduced) {
      sbar.resize(static_cast<size_t>(c->nV) * nb2);
      vhf.resize(static_cast<size_t>(c->nV) * np2);
      QA_TRY(cudaMemcpyAsync(sbar.data(), c->d_Vbar, sbar.size() * 16, cudaMemcpyDeviceToHost, st));
      QA_TRY(cudaMemcpyAsync(vhf.data(), c->d_VbarHF, vhf.size() * 16, cudaMemcpyDeviceToHost, st));
    } else {
      QA_TRY(cudaMemcpyAsync(grad_V, c->d_Vbar, static_cast<size_t>(c->nV) * np2 * 16,
                             cudaMemcpyDeviceToHost, st));
    }
  }
  QA_TRY(cudaStreamSynchronize(st));
  if (grad_V && c->nV > 0 && c->reduced) {
    const int np = c->npair, rho = c->rho;
    cd* gv = reinterpret_cast<cd*>(grad_V);
    for (int v = 0; v < c->nV; ++v)
      for (int A = 0; A < np; ++A)
        for (int Bq = 0; Bq < np; ++Bq) {
          cd acc = vhf[(static_cast<size_t>(v) * np + A) * np + Bq];
          for (int i = 0; i < rho; ++i) {
            const cd bai = c->basis[static_cast<size_t>(A) * rho + i];
            if (bai == cd(0, 0)) continue;
            for (int j = 0; j < rho; ++j) {
              const cd bbj = c->basis[static_cast<size_t>(Bq) * rho + j];
              if (bbj == cd(0, 0)) continue;
              acc += bai * sbar[(static_cast<size_t>(v) * rho + i) * rho + j] * std::conj(bbj);
            }
          }
          gv[(static_cast<size_t>(v) * np + A) * np + Bq] = acc;
        }
  }
  return check_err(c, nullptr, st);
}

// ------------------------------------------------- Hartree-Fock loop, QP

// Scratch of the Hartree-Fock loop inside d_Gt: U [N_k][norb^2], E [N_k][norb],
// the previous Sigma^HF [N_k][norb^2].
struct HfScratch {
  double2* U;
  double* E;
  double2* old;
};

bool hf_scratch(qa_ctx* c, HfScratch* h) {
  const size_t nk = c->nk, no = c->norb, no2 = no * no;
  const size_t u = nk * no2 * 16, e = align_up(nk * no * 8), o = nk * no2 * 16;
  if (u + e + o > static_cast<size_t>(c->r) * no2 * nk * 16) return false;
  char* base = static_cast<char*>(c->d_Gt);
  h->U = reinterpret_cast<double2*>(base);
  h->E = reinterpret_cast<double*>(base + u);
  h->old = reinterpret_cast<double2*>(base + u + e);
  return true;
}

int fd_blocks(const qa_ctx* c) {
  const long long n = static_cast<long long>(c->nk) * c->norb;
  return static_cast<int>(std::min<long long>(std::max<long long>((n + 255) / 256, 1), c->nblocks_g));
}

// N(mu) = (s / N_k) sum_{k,i} f(beta (E_ki - mu)) and dN/dmu from the device eigenvalues.
int fd_eval(qa_ctx* c, const double* E, double mu, double* N, double* dN, cudaStream_t st) {
  const long long n = static_cast<long long>(c->nk) * c->norb;
  const int nb = fd_blocks(c);
  QA_LAUNCH(c, 1, qa::launch_fd_sum(E, n, c->beta, mu, c->d_part, nb, st));
  QA_LAUNCH(c, 1, qa::launch_reduce_pairs(c->d_part, nb, 0, c->d_red, st));
  double h[2];
  QA_TRY(cudaStreamSynchronize(st));
  h[0] = c->mb->red[0];
  h[1] = c->mb->red[1];
  *N = c->nspin * h[0] / c->nk;
  *dN = c->nspin * h[1] / c->nk;
  return QA_OK;
}

// Chemical potential of the Fermi-Dirac filling of the eigenvalues E: the
// bracket [E_min - 1 - 40/beta, E_max + 1 + 40/beta] (empty below, full above),
// then bisection with Newton steps taken when they stay inside the bracket
// and shrink faster than bisection; stop at |N - filling| <= 1e-12 max(1,
// filling) or a bracket below 1e-14 max(1, |mu|).
int fd_mu(qa_ctx* c, const double* E, double* mu_out, int* evals, cudaStream_t st) {
  const long long n = static_cast<long long>(c->nk) * c->norb;
  const int nb = fd_blocks(c);
  QA_LAUNCH(c, 1, qa::launch_fd_range(E, n, c->d_part, nb, st));
  QA_LAUNCH(c, 1, qa::launch_reduce_pairs(c->d_part, nb, 1, c->d_red, st));
  double h[2];
  QA_TRY(cudaStreamSynchronize(st));
  h[0] = c->mb->red[0];
  h[1] = c->mb->red[1];
  if (!std::isfinite(h[0]) || !std::isfinite(h[1])) return QA_ERANGE;
  double lo = -h[1] - 1.0 - 40.0 / c->beta, hi = h[0] + 1.0 + 40.0 / c->beta;
  const double target = c->filling, tolN = 1e-12 * std::max(1.0, target);
  double mu = 0.5 * (lo + hi), N = 0, dN = 0, dxold = hi - lo;
  int count = 0;
  for (int it = 0; it < 300; ++it) {
    if (int rc = fd_eval(c, E, mu, &N, &dN, st)) return rc;
    ++count;
    if (!std::isfinite(N)) return QA_ERANGE;
    const double f = N - target;
    if (std::fabs(f) <= tolN) break;
    if (f < 0) lo = mu; else hi = mu;
    if (hi - lo < 1e-14 * std::max(1.0, std::fabs(mu))) break;
    const double cand = mu - f / dN;
    if (dN > 0 && std::isfinite(cand) && cand > lo && cand < hi &&
        std::fabs(2.0 * f) <= std::fabs(dxold * dN)) {
      dxold = std::fabs(f / dN);
      mu = cand;
    } else {
      dxold = 0.5 * (hi - lo);
      mu = 0.5 * (lo + hi);
    }
    if (it == 299) return QA_ENOCONV;
  }
  *mu_out = mu;
  *evals += count;
  return QA_OK;
}

// eigenvalues of H + Sigma^HF (null: H alone), mu of the filling, n(k) into d_nk
int hf_density(qa_ctx* c, const HfScratch& h, const double2* sig, double* mu, int* evals,
               cudaStream_t st) {
  QA_LAUNCH(c, 1, qa::launch_hf_eig(c->d_Hk, sig, c->norb, c->nk, h.E, h.U, st));
  if (int rc = fd_mu(c, h.E, mu, evals, st)) return rc;
  QA_LAUNCH(c, 1, qa::launch_fd_density(h.E, h.U, c->norb, c->nk, c->beta, *mu, c->d_nk, st));
  return QA_OK;
}

// Self-consistent Hartree-Fock (paper Sec. "Hartree-Fock self-consistency",
// Fig. 3(a)): start from the Fermi-Dirac density of H0, then repeat
// Sigma^HF(n) -> mix -> eigenvalues of H0 + Sigma^HF -> mu -> n until the
// largest change of Sigma^HF is <= tol.  G_out: the HF Green's function
// (Dyson with Sigma^HF at the HF mu) on the DLR tau nodes.
int hf_solve_impl(qa_ctx* c, int max_iter, double tol, double mix, void* G_out, double* mu_out,
                  int* iters_out, double* resid_out, double* n_out, cudaStream_t st) {
  HfScratch h;
  if (!hf_scratch(c, &h)) return QA_ENOMEM;
  c->launches = 0;
  if (int rc = reset_err(c, st)) return rc;
  const int no2 = c->norb * c->norb;
  const long long nsig = static_cast<long long>(c->nk) * no2;
  int evals = 0;
  double mu = 0;
  if (int rc = hf_density(c, h, nullptr, &mu, &evals, st)) return rc;
  QA_TRY(cudaMemsetAsync(h.old, 0, nsig * 16, st));
  double resid = INFINITY;
  int it = 0;
  const int nb = fd_blocks(c);
  c->sigc_valid = false;
  for (it = 1; it <= max_iter; ++it) {
    QA_LAUNCH(c, 1, qa::launch_density_R(c->d_nk, c->d_vR, c->nV + 1, no2, nullptr, c->nk, c->n[0],
                                         c->n[1], c->n[2], c->d_nR, st, c->d_phV));
    QA_LAUNCH(c, 2, qa::launch_hf(c->d_vV, c->d_nR, c->d_vR, c->nV, c->norb, c->nspin, nullptr, c->nk,
                                  c->n[0], c->n[1], c->n[2], c->d_sigFR, c->d_SigHF, st, c->d_phV));
    QA_LAUNCH(c, 1, qa::launch_mix(c->d_SigHF, h.old, mix, nsig, c->d_part, nb, st));
    QA_LAUNCH(c, 1, qa::launch_reduce_pairs(c->d_part, nb, 1, c->d_red, st));
    QA_TRY(cudaStreamSynchronize(st));
    resid = c->mb->red[0];                 // read before the mu search reuses the mailbox
    if (int rc = hf_density(c, h, c->d_SigHF, &mu, &evals, st)) return rc;
    if (!std::isfinite(resid)) return QA_ERANGE;
    if (resid <= tol) break;
  }
  c->sighf_valid = true;
  if (it > max_iter) it = max_iter;
  if (G_out || n_out) {
    double bound = 0;
    if (int rc = prepare_g<double>(c, c->d_SigHF, nullptr, mu, &bound, st)) return rc;
    if (G_out) {
      if (int rc = finish_g<double>(c, c->t64, mu, G_out, n_out, st)) return rc;
    } else {
      // local density n(R = 0) of the HF solution: k-average of n(k)
      QA_LAUNCH(c, 1, qa::launch_k_average<double>(c->d_nk, no2, c->nk, c->d_nloc, st));
      QA_TRY(cudaStreamSynchronize(st));
      std::memcpy(n_out, c->mb->nloc, static_cast<size_t>(no2) * 16);
    }
  }
  QA_TRY(cudaStreamSynchronize(st));
  c->mu = mu;
  c->have_mu = true;
  if (mu_out) *mu_out = mu;
  if (iters_out) *iters_out = it;
  if (resid_out) *resid_out = resid;
  if (int herr = check_err(c, nullptr, st)) return herr;
  return resid <= tol ? QA_OK : QA_ENOCONV;
}

// Quasiparticle quantities from the self-energy in the workspace.
template <typename T>
int qp_impl(qa_ctx* c, double2* Z, double2* S0, double2* Hqp, double* eps, cudaStream_t st) {
  if (c->r < 2) return QA_ENOMEM;           // node sums use 2 N_k norb^2 of d_Gt
  if (int rc = reset_err(c, st)) return rc;
  const int r = c->sigc_valid ? c->r : 0;
  QA_LAUNCH(c, r > 0 ? 2 : 1, qa::launch_qp<T>(c->d_Hk, c->d_SigHF, c->sigc_valid ? c->d_SigIw : nullptr, c->d_wq,
                                   c->d_wq + c->r, r, c->norb, c->nk, M_PI / c->beta,
                                   static_cast<double2*>(c->d_Gt), Z, S0, Hqp, eps, c->d_err, st));
  QA_TRY(cudaStreamSynchronize(st));
  return check_err(c, nullptr, st);
}

}  // namespace

namespace qa {
int density_tables(const ::qa_ctx* c, const std::complex<double>** dtau, int* r, int* norb,
                   int* nk, int* nspin) {
  if (!c || c->r < 1) return QA_EINVAL;
  *dtau = c->mats.dtau.data();
  *r = c->r;
  *norb = c->norb;
  *nk = c->nk;
  *nspin = c->nspin;
  return QA_OK;
}
}  // namespace qa

extern "C" {

const char* qa_strerror(int s) {
  switch (s) {
    case QA_OK: return "ok";
    case QA_EINVAL: return "invalid argument";
    case QA_ENOMEM: return "workspace too small";
    case QA_ESINGULAR: return "singular Dyson pivot";
    case QA_ENOCONV: return "chemical potential search did not converge";
    case QA_ERANGE: return "non-finite value or spectrum outside the DLR window";
    case QA_ETIMEOUT: return "device wait timed out";
    case QA_ECUDA: return "CUDA runtime error";
    case QA_ESTATE: return "call out of order";
    case QA_EBOUNDS: return "index-map gather out of range (bounds-checked build)";
    default: return "unknown status";
  }
}

int qa_create(const qa_lattice* lat, const qa_hoppings* hop, const qa_interaction* inter,
              double beta, double Lambda, double eps, double filling, int precision,
              qa_ctx** out) {
  if (!lat || !hop || !inter || !out) return QA_EINVAL;
  *out = nullptr;
  if (precision != QA_FP64 && precision != QA_MIXED && precision != QA_FP32) return QA_EINVAL;
  if (lat->norb < 1 || lat->norb > 5 || lat->nspin < 1) return QA_EINVAL;
  long long nk = 1;
  for (int d = 0; d < 3; ++d) {
    if (lat->n[d] < 1 || lat->n[d] > 4096 || !small_primes_only(lat->n[d])) return QA_EINVAL;
    nk *= lat->n[d];
  }
  if (nk > 12288) return QA_EINVAL;
  if (!(beta > 0) || !(Lambda > 1) || !(eps > 0 && eps < 1)) return QA_EINVAL;
  if (!(filling > 0) || !(filling < static_cast<double>(lat->nspin) * lat->norb)) return QA_EINVAL;
  if (hop->nR < 0 || inter->nR < 0) return QA_EINVAL;
  if ((hop->nR > 0 && (!hop->R || !hop->t)) || (inter->nR > 0 && (!inter->R || !inter->V)))
    return QA_EINVAL;
  qa_ctx* c = new (std::nothrow) qa_ctx();
  if (!c) return QA_ENOMEM;
  c->n[0] = lat->n[0]; c->n[1] = lat->n[1]; c->n[2] = lat->n[2];
  c->nk = static_cast<int>(nk);
  c->norb = lat->norb;
  c->npair = lat->norb * lat->norb;
  c->nspin = lat->nspin;
  c->beta = beta; c->Lambda = Lambda; c->eps = eps; c->filling = filling;
  c->precision = precision;
  const int no = c->norb, no2 = no * no, np2 = c->npair * c->npair;
  // H(R) = -t(R), plus eps on R = 0
  bool have0 = false;
  for (int i = 0; i < hop->nR; ++i) {
    for (int d = 0; d < 3; ++d) c->hopR.push_back(hop->R[3 * i + d]);
    bool zero = hop->R[3 * i] == 0 && hop->R[3 * i + 1] == 0 && hop->R[3 * i + 2] == 0;
    for (int e = 0; e < no2; ++e) {
      cd v(-hop->t[2 * (static_cast<size_t>(i) * no2 + e)], -hop->t[2 * (static_cast<size_t>(i) * no2 + e) + 1]);
      if (zero && e / no == e % no && hop->eps) v += hop->eps[e / no];
      c->hopH.push_back(v);
    }
    have0 |= zero;
  }
  if (!have0) {
    c->hopR.insert(c->hopR.end(), {0, 0, 0});
    for (int e = 0; e < no2; ++e)
      c->hopH.push_back(cd(e / no == e % no && hop->eps ? hop->eps[e / no] : 0.0, 0.0));
  }
  c->nH = static_cast<int>(c->hopR.size() / 3);
  c->nH_user = hop->nR;
  // Hermiticity: H(-R) = H(R)^dagger for every listed R
  double scale = 0;
  for (const cd& v : c->hopH) scale = std::max(scale, std::abs(v));
  for (int i = 0; i < c->nH; ++i) {
    int j = -1;
    for (int k = 0; k < c->nH; ++k)
      if (c->hopR[3 * k] == -c->hopR[3 * i] && c->hopR[3 * k + 1] == -c->hopR[3 * i + 1] &&
          c->hopR[3 * k + 2] == -c->hopR[3 * i + 2]) { j = k; break; }
    if (j < 0) { delete c; return QA_EINVAL; }
    for (int a = 0; a < no; ++a)
      for (int b = 0; b < no; ++b) {
        cd x = c->hopH[static_cast<size_t>(i) * no2 + a * no + b];
        cd y = c->hopH[static_cast<size_t>(j) * no2 + b * no + a];
        if (std::abs(x - std::conj(y)) > 1e-12 * std::max(1.0, scale)) { delete c; return QA_EINVAL; }
      }
  }
  c->nV = inter->nR;
  for (int i = 0; i < c->nV; ++i) {
    for (int d = 0; d < 3; ++d) c->vR.push_back(inter->R[3 * i + d]);
    for (int e = 0; e < np2; ++e)
      c->vV.push_back(cd(inter->V[2 * (static_cast<size_t>(i) * np2 + e)],
                         inter->V[2 * (static_cast<size_t>(i) * np2 + e) + 1]));
  }
  c->vR.insert(c->vR.end(), {0, 0, 0});
  for (const cd& v : c->vV)
    if (!std::isfinite(v.real()) || !std::isfinite(v.imag())) { delete c; return QA_EINVAL; }
  for (const cd& v : c->hopH)
    if (!std::isfinite(v.real()) || !std::isfinite(v.imag())) { delete c; return QA_EINVAL; }
  setup_pairs(c, false);
  // DLR grid and transform matrices
  if (qa::build_dlr(Lambda, eps, &c->grid) != 0) { delete c; return QA_EINVAL; }
  c->r = c->grid.r;
  qa::build_dlr_matrices(c->grid, beta, &c->mats);
  if (precision == QA_MIXED && qa::dlr_oz_supported(c->r)) {
    c->use_oz = true;
    qa::pack_dlr_oz(c->mats.Ttn.data(), c->r, &c->oz_Ttn);
    qa::pack_dlr_oz(c->mats.Tnt.data(), c->r, &c->oz_Tnt);
    qa::pack_dlr_oz(c->mats.Trefl.data(), c->r, &c->oz_Trefl);
    qa::pack_dlr_oz(c->mats.Ttw.data(), c->r, &c->oz_Ttw);
    qa::pack_dlr_oz(c->mats.Twt.data(), c->r, &c->oz_Twt);
  }
  if (precision == QA_FP32 && qa::dlr_tc_supported(c->r, nullptr)) {
    const char* env = std::getenv("QA_DLR_SIMT");
    c->use_tc = !(env && env[0] == '1');
    if (c->use_tc) {
      qa::pack_dlr_tc(c->mats.Ttn.data(), c->r, &c->tc_Ttn);
      qa::pack_dlr_tc(c->mats.Tnt.data(), c->r, &c->tc_Tnt);
      qa::pack_dlr_tc(c->mats.Trefl.data(), c->r, &c->tc_Trefl);
      qa::pack_dlr_tc(c->mats.Ttw.data(), c->r, &c->tc_Ttw);
      qa::pack_dlr_tc(c->mats.Twt.data(), c->r, &c->tc_Twt);
    }
  }
  // FFT plans and the -R map
  for (int d = 0; d < 3; ++d) qa::plan_fft_axis(c->n[d], &c->ax[d], &c->pos[d]);
  c->mR.resize(c->nk);
  for (int i1 = 0; i1 < c->n[0]; ++i1)
    for (int i2 = 0; i2 < c->n[1]; ++i2)
      for (int i3 = 0; i3 < c->n[2]; ++i3)
        c->mR[grid_index(c, i1, i2, i3)] =
            grid_index(c, (c->n[0] - i1) % c->n[0], (c->n[1] - i2) % c->n[1], (c->n[2] - i3) % c->n[2]);
  *out = c;
  return QA_OK;
}

int qa_set_pair_basis(qa_ctx* c, int mode) {
  if (!c || (mode != QA_PAIRS_AUTO && mode != QA_PAIRS_FULL && mode != QA_PAIRS_REDUCED))
    return QA_EINVAL;
  if (c->bound) return QA_ESTATE;
  c->pair_mode = mode;
  return setup_pairs(c, false);
}

int qa_get_pair_basis(const qa_ctx* c, int* rho, int* active, double* B) {
  if (!c) return QA_EINVAL;
  if (rho) *rho = c->rho;
  if (active) *active = c->reduced ? 1 : 0;
  if (B && c->rho > 0) std::memcpy(B, c->basis.data(), c->basis.size() * 16);
  return QA_OK;
}

int qa_workspace_size(const qa_ctx* c, size_t* bytes) {
  if (!c || !bytes) return QA_EINVAL;
  if (c->bound) {                   // the bound layout stays as it is
    *bytes = c->ws_need + kAlign;
    return QA_OK;
  }
  *bytes = layout(const_cast<qa_ctx*>(c), nullptr) + kAlign;
  return QA_OK;
}

int qa_bind(qa_ctx* c, void* workspace, size_t bytes, void* stream) {
  if (!c || !workspace) return QA_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  size_t need = layout(c, nullptr);
  char* base = static_cast<char*>(workspace);
  size_t shift = (kAlign - reinterpret_cast<uintptr_t>(base) % kAlign) % kAlign;
  if (bytes < need + shift) return QA_ENOMEM;
  c->ws = base + shift;
  c->ws_bytes = bytes - shift;
  layout(c, c->ws);
  c->ws_need = need;
  // the scalar results live in a pinned host mailbox written through its device alias
  if (!c->mb) {
    QA_TRY(cudaHostAlloc(reinterpret_cast<void**>(&c->mb), sizeof(QaMailbox), cudaHostAllocMapped));
    QA_TRY(cudaHostGetDevicePointer(reinterpret_cast<void**>(&c->mb_dev), c->mb, 0));
  }
  c->d_red = c->mb_dev->red;
  c->drop_mu_graphs();          // they hold pointers into the previous workspace
  c->d_err = &c->mb_dev->err;
  c->d_bad = &c->mb_dev->bad;
  c->d_nloc = c->mb_dev->nloc;
  const int r = c->r;
  // DLR tables
  const qa::DlrMatrices& m = c->mats;
  std::vector<cd> iw_c;
  QA_TRY(upload_c<double>(c->t64.Trefl, m.Trefl, st));
  QA_TRY(upload_c<double>(c->t64.Ttn, m.Ttn, st));
  QA_TRY(upload_c<double>(c->t64.Tnt, m.Tnt, st));
  QA_TRY(upload_c<double>(c->t64.Ttw, m.Ttw, st));
  QA_TRY(upload_c<double>(c->t64.Twt, m.Twt, st));
  QA_TRY(upload_c<double>(c->t64.dtau, m.dtau, st));
  c->dtau_real = true;
  for (const cd& v : m.dtau) c->dtau_real = c->dtau_real && v.imag() == 0.0;
  QA_TRY(upload_c<double>(c->t64.dw, m.dw, st));
  QA_TRY(upload_c<float>(c->t32.Trefl, m.Trefl, st));
  QA_TRY(upload_c<float>(c->t32.Ttn, m.Ttn, st));
  QA_TRY(upload_c<float>(c->t32.Tnt, m.Tnt, st));
  QA_TRY(upload_c<float>(c->t32.Ttw, m.Ttw, st));
  QA_TRY(upload_c<float>(c->t32.Twt, m.Twt, st));
  QA_TRY(upload_c<float>(c->t32.dtau, m.dtau, st));
  QA_TRY(upload_c<float>(c->t32.dw, m.dw, st));
  QA_TRY(upload_c<qa::dfl>(c->tdf.Trefl, m.Trefl, st));
  QA_TRY(upload_c<qa::dfl>(c->tdf.Ttn, m.Ttn, st));
  QA_TRY(upload_c<qa::dfl>(c->tdf.Tnt, m.Tnt, st));
  QA_TRY(upload_c<qa::dfl>(c->tdf.Ttw, m.Ttw, st));
  QA_TRY(upload_c<qa::dfl>(c->tdf.Twt, m.Twt, st));
  QA_TRY(upload_c<qa::dfl>(c->tdf.dtau, m.dtau, st));
  QA_TRY(upload_c<qa::dfl>(c->tdf.dw, m.dw, st));
  QA_TRY(cudaMemcpyAsync(c->d_iw, m.iw.data(), r * 8, cudaMemcpyHostToDevice, st));
  {
    std::vector<cd> wq(m.wq_p);
    wq.insert(wq.end(), m.wq_m.begin(), m.wq_m.end());
    QA_TRY(upload_c<double>(c->d_wq, wq, st));
    QA_TRY(cudaStreamSynchronize(st));    // wq goes out of scope
  }
  if (c->use_oz) {
    QA_TRY(cudaMemcpyAsync(c->d_oz_Ttn, c->oz_Ttn.data(), c->oz_Ttn.size(), cudaMemcpyHostToDevice, st));
    QA_TRY(cudaMemcpyAsync(c->d_oz_Tnt, c->oz_Tnt.data(), c->oz_Tnt.size(), cudaMemcpyHostToDevice, st));
    QA_TRY(cudaMemcpyAsync(c->d_oz_Trefl, c->oz_Trefl.data(), c->oz_Trefl.size(), cudaMemcpyHostToDevice, st));
    QA_TRY(cudaMemcpyAsync(c->d_oz_Ttw, c->oz_Ttw.data(), c->oz_Ttw.size(), cudaMemcpyHostToDevice, st));
    QA_TRY(cudaMemcpyAsync(c->d_oz_Twt, c->oz_Twt.data(), c->oz_Twt.size(), cudaMemcpyHostToDevice, st));
  }
  if (c->use_tc) {
    QA_TRY(cudaMemcpyAsync(c->d_tc_Ttn, c->tc_Ttn.data(), c->tc_Ttn.size() * 2, cudaMemcpyHostToDevice, st));
    QA_TRY(cudaMemcpyAsync(c->d_tc_Tnt, c->tc_Tnt.data(), c->tc_Tnt.size() * 2, cudaMemcpyHostToDevice, st));
    QA_TRY(cudaMemcpyAsync(c->d_tc_Trefl, c->tc_Trefl.data(), c->tc_Trefl.size() * 2, cudaMemcpyHostToDevice, st));
    QA_TRY(cudaMemcpyAsync(c->d_tc_Ttw, c->tc_Ttw.data(), c->tc_Ttw.size() * 2, cudaMemcpyHostToDevice, st));
    QA_TRY(cudaMemcpyAsync(c->d_tc_Twt, c->tc_Twt.data(), c->tc_Twt.size() * 2, cudaMemcpyHostToDevice, st));
  }
  if (c->precision == QA_FP64) {
    auto ctrans = [r](const std::vector<cd>& T) {
      std::vector<cd> H(T.size());
      for (int i = 0; i < r; ++i)
        for (int j = 0; j < r; ++j) H[static_cast<size_t>(j) * r + i] = std::conj(T[static_cast<size_t>(i) * r + j]);
      return H;
    };
    std::vector<cd> cdt(r);
    for (int j = 0; j < r; ++j) cdt[j] = std::conj(m.dtau[j]);     // an r x 1 matrix
    const std::vector<cd> h1 = ctrans(m.Trefl), h2 = ctrans(m.Ttn), h3 = ctrans(m.Tnt),
                          h4 = ctrans(m.Ttw), h5 = ctrans(m.Twt);
    QA_TRY(upload_c<double>(c->tH.Trefl, h1, st));
    QA_TRY(upload_c<double>(c->tH.Ttn, h2, st));
    QA_TRY(upload_c<double>(c->tH.Tnt, h3, st));
    QA_TRY(upload_c<double>(c->tH.Ttw, h4, st));
    QA_TRY(upload_c<double>(c->tH.Twt, h5, st));
    QA_TRY(upload_c<double>(c->tH.dtau, cdt, st));
    QA_TRY(cudaStreamSynchronize(st));
  }
  // FFT twiddles exp(-2 pi i m / L) per axis, and digit-reversal tables
  std::vector<cd> tw;
  std::vector<int> pos;
  for (int d = 0; d < 3; ++d) {
    c->fft64.n[d] = c->fft32.n[d] = c->fftdf.n[d] = c->n[d];
    c->fft64.nfac[d] = c->fft32.nfac[d] = c->fftdf.nfac[d] = c->ax[d].nfac;
    for (int s = 0; s < qa::kMaxFac; ++s)
      c->fft64.fac[d][s] = c->fft32.fac[d][s] = c->fftdf.fac[d][s] = c->ax[d].fac[s];
    c->fft64.tw_off[d] = c->fft32.tw_off[d] = c->fftdf.tw_off[d] = static_cast<int>(tw.size());
    c->fft64.pos_off[d] = c->fft32.pos_off[d] = c->fftdf.pos_off[d] = static_cast<int>(pos.size());
    const long double two_pi = 6.283185307179586476925286766559005768L;
    for (int k = 0; k < c->n[d]; ++k) {
      long double ang = -two_pi * k / c->n[d];
      tw.push_back(cd(static_cast<double>(std::cos(ang)), static_cast<double>(std::sin(ang))));
    }
    pos.insert(pos.end(), c->pos[d].begin(), c->pos[d].end());
  }
  QA_TRY(upload_c<double>(c->d_tw64, tw, st));
  QA_TRY(upload_c<float>(c->d_tw32, tw, st));
  QA_TRY(upload_c<qa::dfl>(c->d_twdf, tw, st));
  QA_TRY(cudaMemcpyAsync(c->d_pos, pos.data(), pos.size() * 4, cudaMemcpyHostToDevice, st));
  c->fft64.tw = c->d_tw64;
  c->fft32.tw = c->d_tw32;
  c->fftdf.tw = c->d_twdf;
  c->fft64.pos = c->fft32.pos = c->fftdf.pos = c->d_pos;
  QA_TRY(cudaMemcpyAsync(c->d_mR, c->mR.data(), c->nk * 4, cudaMemcpyHostToDevice, st));
  QA_TRY(cudaMemcpyAsync(c->d_hR, c->hopR.data(), c->hopR.size() * 4, cudaMemcpyHostToDevice, st));
  QA_TRY(upload_c<double>(c->d_hH, c->hopH, st));
  QA_TRY(cudaMemcpyAsync(c->d_vR, c->vR.data(), c->vR.size() * 4, cudaMemcpyHostToDevice, st));
  QA_LAUNCH(c, 1, qa::launch_phase_table(c->d_vR, c->nV + 1, c->nk, c->n[0], c->n[1], c->n[2], c->d_phV, st));
  if (c->nV > 0) QA_TRY(upload_c<double>(c->d_vV, c->vV, st));
  // H(k), V(q) (or S(q) on the reduced pair basis)
  const int no2 = c->norb * c->norb;
  QA_LAUNCH(c, 1, qa::launch_ft_table(c->d_hR, c->d_hH, c->nH, no2, nullptr, c->nk, c->n[0], c->n[1],
                             c->n[2], c->d_Hk, st));
  if (int rc = upload_interaction(c, st)) return rc;
  // G0 at mu0 (always FP64)
  if (int rc = reset_err(c, st)) return rc;
  double mu0 = 0, N0 = 0;
  int ev = 0;
  int rc = mu_search<double>(c, nullptr, nullptr, c->t64, 0.0, &mu0, &N0, &ev, st);
  if (rc != QA_OK) return rc;
  rc = finish_g<double>(c, c->t64, mu0, c->d_G0, nullptr, st);
  if (rc != QA_OK) return rc;
  QA_TRY(cudaStreamSynchronize(st));
  rc = check_err(c, nullptr, st);
  if (rc != QA_OK) return rc;
  c->mu0 = mu0;
  c->have_mu = false;
  c->bound = true;
  return QA_OK;
}

int qa_get_grid(const qa_ctx* c, int* r, double* x, double* t_rel, int* nf, int* mb) {
  if (!c) return QA_EINVAL;
  if (r) *r = c->r;
  for (int i = 0; i < c->r; ++i) {
    if (x) x[i] = c->grid.x[i];
    if (t_rel) t_rel[i] = c->grid.t[i];
    if (nf) nf[i] = c->grid.nf[i];
    if (mb) mb[i] = c->grid.mb[i];
  }
  return QA_OK;
}

int qa_get_plan(const qa_ctx* c, int* minus_R, int* fft_pos, int* fft_nfac, int* fft_fac) {
  if (!c) return QA_EINVAL;
  if (minus_R) std::memcpy(minus_R, c->mR.data(), c->mR.size() * 4);
  int off = 0;
  for (int d = 0; d < 3; ++d) {
    if (fft_pos) std::memcpy(fft_pos + off, c->pos[d].data(), c->pos[d].size() * 4);
    off += c->n[d];
    if (fft_nfac) fft_nfac[d] = c->ax[d].nfac;
    if (fft_fac)
      for (int s = 0; s < qa::kMaxFac; ++s) fft_fac[d * qa::kMaxFac + s] = c->ax[d].fac[s];
  }
  return QA_OK;
}

int qa_get_sizes(const qa_ctx* c, int* nk, int* norb, int* r) {
  if (!c) return QA_EINVAL;
  if (nk) *nk = c->nk;
  if (norb) *norb = c->norb;
  if (r) *r = c->r;
  return QA_OK;
}

int qa_set_timing(qa_ctx* c, int enable) {
  if (!c) return QA_EINVAL;
  c->timing = enable != 0;
  return QA_OK;
}

int qa_gw_step(qa_ctx* c, const void* G_in, void* G_out, double* mu_out, double* n_out,
               qa_step_stats* stats, void* stream) {
  if (!c || !G_out) return QA_EINVAL;
  if (!c->bound) return QA_ESTATE;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (c->precision == QA_FP64) return gw_step_impl<double>(c, G_in, G_out, mu_out, n_out, stats, st);
  if (c->precision == QA_MIXED) return gw_step_impl<qa::dfl>(c, G_in, G_out, mu_out, n_out, stats, st);
  return gw_step_impl<float>(c, G_in, G_out, mu_out, n_out, stats, st);
}

int qa_density(qa_ctx* c, const void* G, double* n_out, double* N_total, void* stream) {
  if (!c || !G) return QA_EINVAL;
  if (!c->bound) return QA_ESTATE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int no2 = c->norb * c->norb;
  QA_LAUNCH(c, 1, qa::launch_g_input(static_cast<const double2*>(G), static_cast<const double2*>(c->t64.dtau),
                                     c->r, static_cast<long long>(no2) * c->nk, nullptr, c->d_nk, st,
                                     c->dtau_real));
  QA_LAUNCH(c, 1, qa::launch_k_average<double>(c->d_nk, no2, c->nk, c->d_nloc, st));
  std::vector<double> h(2 * no2);
  QA_TRY(cudaStreamSynchronize(st));
  std::memcpy(h.data(), c->mb->nloc, static_cast<size_t>(no2) * 16);
  double tr = 0;
  for (int a = 0; a < c->norb; ++a) tr += h[2 * (a * c->norb + a)];
  if (n_out) std::memcpy(n_out, h.data(), h.size() * 8);
  if (N_total) *N_total = c->nspin * tr;
  return QA_OK;
}

int qa_get(const qa_ctx* c, int which, void* dst, size_t bytes, void* stream) {
  if (!c || !dst) return QA_EINVAL;
  if (!c->bound) return QA_ESTATE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t es = c->precision == QA_FP32 ? 8 : 16;
  const size_t r = c->r, nk = c->nk, no2 = static_cast<size_t>(c->norb) * c->norb,
               nb2 = static_cast<size_t>(c->nb) * c->nb;
  const void* src = nullptr;
  size_t need = 0;
  switch (which) {
    case QA_P_QNU: src = c->d_Pnu ? c->d_Pnu : c->d_P; need = r * nb2 * nk * es; break;
    case QA_WC_RTAU: src = c->d_W; need = r * nb2 * nk * es; break;
    case QA_SIGC_KTAU: src = c->d_SigC; need = r * no2 * nk * es; break;
    case QA_SIGC_KIW: src = c->d_SigIw; need = r * no2 * nk * es; break;
    case QA_SIGHF_K: src = c->d_SigHF; need = nk * no2 * 16; break;
    case QA_G0: src = c->d_G0; need = r * no2 * nk * 16; break;
    case QA_HK: src = c->d_Hk; need = nk * no2 * 16; break;
    case QA_MU0:
      if (bytes != 8) return QA_EINVAL;
      std::memcpy(dst, &c->mu0, 8);
      return QA_OK;
    default: return QA_EINVAL;
  }
  if (bytes != need) return QA_EINVAL;
  QA_TRY(cudaMemcpyAsync(dst, src, need, cudaMemcpyDefault, st));
  QA_TRY(cudaStreamSynchronize(st));
  return QA_OK;
}

int qa_set_wait_limit(qa_ctx* c, long long polls) {
  if (!c) return QA_EINVAL;
  c->wait_limit = polls < 0 ? -1 : polls;
  return QA_OK;
}

int qa_set_mu(qa_ctx* c, int fixed, double mu) {
  if (!c || !std::isfinite(mu)) return QA_EINVAL;
  c->mu_fixed = fixed != 0;
  c->mu_value = mu;
  return QA_OK;
}

int qa_set_params(qa_ctx* c, const qa_hoppings* hop, const qa_interaction* inter, void* stream) {
  if (!c || !hop || !inter) return QA_EINVAL;
  if (!c->bound) return QA_ESTATE;
  if (hop->nR != c->nH_user || inter->nR != c->nV) return QA_EINVAL;
  const int no = c->norb, no2 = no * no;
  for (int i = 0; i < hop->nR; ++i)
    for (int d = 0; d < 3; ++d)
      if (hop->R[3 * i + d] != c->hopR[3 * i + d]) return QA_EINVAL;
  for (int i = 0; i < inter->nR; ++i)
    for (int d = 0; d < 3; ++d)
      if (inter->R[3 * i + d] != c->vR[3 * i + d]) return QA_EINVAL;
  std::vector<cd> H(c->hopH.size());
  for (int i = 0; i < c->nH; ++i) {
    const bool user = i < hop->nR;
    const bool zero = c->hopR[3 * i] == 0 && c->hopR[3 * i + 1] == 0 && c->hopR[3 * i + 2] == 0;
    for (int e = 0; e < no2; ++e) {
      cd v = user ? cd(-hop->t[2 * (static_cast<size_t>(i) * no2 + e)], -hop->t[2 * (static_cast<size_t>(i) * no2 + e) + 1])
                  : cd(0.0, 0.0);
      if (zero && e / no == e % no && hop->eps) v += hop->eps[e / no];
      H[static_cast<size_t>(i) * no2 + e] = v;
    }
  }
  for (const cd& v : H)
    if (!std::isfinite(v.real()) || !std::isfinite(v.imag())) return QA_EINVAL;
  for (const double* v = inter->V; v < inter->V + 2 * c->vV.size(); ++v)
    if (!std::isfinite(*v)) return QA_EINVAL;
  std::vector<cd> oldV = c->vV;
  for (size_t e = 0; e < c->vV.size(); ++e)
    c->vV[e] = cd(inter->V[2 * e], inter->V[2 * e + 1]);
  // the workspace keeps its pair basis: a new V must keep the basis choice and rank
  if (setup_pairs(c, true) != QA_OK) {
    c->vV = oldV;
    setup_pairs(c, true);
    return QA_EINVAL;
  }
  c->hopH = H;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  QA_TRY(upload_c<double>(c->d_hH, c->hopH, st));
  if (c->nV > 0) QA_TRY(upload_c<double>(c->d_vV, c->vV, st));
  QA_TRY(qa::launch_ft_table(c->d_hR, c->d_hH, c->nH, no2, nullptr, c->nk, c->n[0], c->n[1], c->n[2],
                             c->d_Hk, st));
  return upload_interaction(c, st);
}

int qa_gw_backward(qa_ctx* c, const void* G_in, double mu, const void* Gbar_out, const void* Sigbar,
                   const double* nbar, void* Gbar_in, double* grad_t, double* grad_V,
                   void* stream) {
  if (!c) return QA_EINVAL;
  if (!c->bound) return QA_ESTATE;
  if (c->precision != QA_FP64 || !std::isfinite(mu)) return QA_EINVAL;
  const double2* Gin = static_cast<const double2*>(G_in ? G_in : c->d_G0);
  return gw_backward_impl(c, Gin, mu, static_cast<const double2*>(Gbar_out),
                          static_cast<const double2*>(Sigbar), nbar, static_cast<double2*>(Gbar_in),
                          grad_t, grad_V, static_cast<cudaStream_t>(stream));
}

int qa_free_energy(qa_ctx* c, const void* G_in, double mu, int M, double* omega, double* parts,
                   void* stream) {
  if (!c || M < 1 || M > (1 << 20) || !std::isfinite(mu)) return QA_EINVAL;
  if (!c->bound) return QA_ESTATE;
  if (c->precision != QA_FP64) return QA_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (int rc = ensure_omega(c, M)) return rc;
  const double2* Gin = static_cast<const double2*>(G_in ? G_in : c->d_G0);
  c->launches = 0;
  if (int rc = reset_err(c, st)) return rc;
  const bool timing = c->timing;
  c->timing = false;
  StageTimer tm(c, st);
  c->timing = timing;
  c->keep_lu = true;
  const int frc = forward_sigma<double>(c, Gin, tm, st);
  c->keep_lu = false;
  if (frc) return frc;
  double p[4];
  if (int rc = omega_value(c, Gin, mu, p, st)) return rc;
  if (int herr = check_err(c, nullptr, st)) return herr;
  if (omega) *omega = p[0] + p[1] + p[2] + p[3];
  if (parts)
    for (int i = 0; i < 4; ++i) parts[i] = p[i];
  return QA_OK;
}

int qa_free_energy_backward(qa_ctx* c, const void* G_in, double mu, int M, double omega_bar,
                            void* Gbar_in, double* grad_t, double* grad_V, void* stream) {
  if (!c || M < 1 || M > (1 << 20) || !std::isfinite(mu) || !std::isfinite(omega_bar)) return QA_EINVAL;
  if (!c->bound) return QA_ESTATE;
  if (c->precision != QA_FP64) return QA_EINVAL;
  if (c->reduced) return QA_ESTATE;
  if (int rc = ensure_omega(c, M)) return rc;
  const double2* Gin = static_cast<const double2*>(G_in ? G_in : c->d_G0);
  return gw_backward_impl(c, Gin, mu, nullptr, nullptr, nullptr, static_cast<double2*>(Gbar_in), grad_t,
                          grad_V, static_cast<cudaStream_t>(stream), omega_bar);
}

int qa_hf_solve(qa_ctx* c, int max_iter, double tol, double mix, void* G_out, double* mu_out,
                int* iters_out, double* resid_out, double* n_out, void* stream) {
  if (!c || max_iter < 1 || !(tol >= 0) || !(mix > 0 && mix <= 1)) return QA_EINVAL;
  if (!c->bound) return QA_ESTATE;
  return hf_solve_impl(c, max_iter, tol, mix, G_out, mu_out, iters_out, resid_out, n_out,
                       static_cast<cudaStream_t>(stream));
}

int qa_qp(qa_ctx* c, void* Z, void* Sig0, void* Hqp, double* eps, void* stream) {
  if (!c) return QA_EINVAL;
  if (!c->bound || !c->sighf_valid) return QA_ESTATE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double2* z = static_cast<double2*>(Z);
  double2* s0 = static_cast<double2*>(Sig0);
  double2* hq = static_cast<double2*>(Hqp);
  if (c->precision == QA_FP64) return qp_impl<double>(c, z, s0, hq, eps, st);
  if (c->precision == QA_MIXED) return qp_impl<qa::dfl>(c, z, s0, hq, eps, st);
  return qp_impl<float>(c, z, s0, hq, eps, st);
}

void qa_destroy(qa_ctx* c) { delete c; }

}  // extern "C"
