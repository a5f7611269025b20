// Allocation-free density entry point.
//
// Some callers cannot call cudaMalloc: code that runs where the CUDA
// allocator is off limits (inside a host callback, a signal or error
// handler, a plug-in loaded by a framework that owns every device
// allocation, or a hard-real-time loop where an allocation may block).
// qa_density_static gives them the density of a G without any device
// allocation: its scratch lives in the file-scope array below, which every
// GPU that loads the library holds from module load until process exit.
//
// Rules of the shared scratch:
//   * one array per device, shared by every call on that device; it keeps
//     the last call's contents.  Each call writes every word it later reads
//     (the DLR weights, n(k) and the averaged matrix), so nothing has to
//     start at zero;
//   * calls whose GPU work overlaps (two streams, or two host threads on one
//     device without ordering) race on the array and give wrong results;
//   * the first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (with that device current).
#include <mutex>
#include <vector>

#include "../../include/qa.h"
#include "qa_common.cuh"

namespace qa {
namespace {

constexpr size_t kStaticScratchBytes = 4u << 20;    // 4 MiB per device
__device__ __align__(256) unsigned char g_density_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// Device address of the scratch array on the current device (set-up once per device).
int scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return QA_ECUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_density_scratch) != cudaSuccess || !p) return QA_ECUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return QA_OK;
}

}  // namespace
}  // namespace qa

extern "C" int qa_density_static(const qa_ctx* ctx, const void* G, double* n_out,
                                 double* N_total, void* stream) {
  if (!ctx || !G) return QA_EINVAL;
  const std::complex<double>* dtau = nullptr;
  int r = 0, norb = 0, nk = 0, nspin = 0;
  if (qa::density_tables(ctx, &dtau, &r, &norb, &nk, &nspin) != QA_OK) return QA_EINVAL;
  const int no2 = norb * norb;
  const size_t off_nk = qa::up256(static_cast<size_t>(r) * 16);
  const size_t off_loc = off_nk + qa::up256(static_cast<size_t>(no2) * nk * 16);
  const size_t need = off_loc + qa::up256(static_cast<size_t>(no2) * 16);
  if (need > qa::kStaticScratchBytes) return QA_ENOMEM;   // problem too large for the static scratch
  void* base = nullptr;
  if (int rc = qa::scratch_address(&base)) return rc;
  char* sb = static_cast<char*>(base);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(sb, dtau, static_cast<size_t>(r) * 16, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return QA_ECUDA;
  double2* nkd = reinterpret_cast<double2*>(sb + off_nk);
  double2* loc = reinterpret_cast<double2*>(sb + off_loc);
  if (qa::launch_dlr_apply<double>(sb, 1, r, G, nkd, static_cast<long long>(no2) * nk, st) != cudaSuccess)
    return QA_ECUDA;
  if (qa::launch_k_average<double>(nkd, no2, nk, loc, st) != cudaSuccess) return QA_ECUDA;
  std::vector<double> h(2 * static_cast<size_t>(no2));
  if (cudaMemcpyAsync(h.data(), loc, static_cast<size_t>(no2) * 16, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return QA_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return QA_ECUDA;
  double tr = 0;
  for (int a = 0; a < norb; ++a) tr += h[2 * (a * norb + a)];
  if (n_out)
    for (size_t i = 0; i < h.size(); ++i) n_out[i] = h[i];
  if (N_total) *N_total = nspin * tr;
  return QA_OK;
}
