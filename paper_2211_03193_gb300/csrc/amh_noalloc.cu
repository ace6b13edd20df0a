// amh_noalloc.cu -- amh_grad_noalloc: energy and gradient for a batch of
// torsion vectors without any device allocation.
//
// amh_grad reads the distogram from a table that amh_init prepared in
// memory the library allocated.  This entry point instead prepares the
// table into one file-scope static device array and runs the same gradient
// kernel on it, so a caller that may not allocate device memory can still
// use it.  The array is shared by every call on a device and keeps the last
// call's contents; every entry a call reads is written by that call first.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "amh.h"
#include "amh_internal.h"

using namespace amh;

namespace {

// (value, slope) entries of the prepared table: 2^21 entries = 16 MiB, e.g.
// L <= 332 residues with 37 bins.
static __device__ __align__(256) float2 g_noalloc_table[AMH_NOALLOC_MAX_ENTRIES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float2* g_table_ptr[kMaxDevices] = {nullptr};

amh_status fail(amh_status st, const std::string& m) {
  set_context_free_error(m);  // read back with amh_last_error(NULL)
  return st;
}

bool on_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" amh_status amh_grad_noalloc(int L, int B, const double* table, int table_is_neglog,
                                       const double* edges, const float* theta, int batch,
                                       double* E_out, float* dE_dtheta, void* stream) {
  if (L < 2 || L > 4096) return fail(AMH_EINVAL, "L must be in [2, 4096]");
  if (B < 2 || B > 256) return fail(AMH_EINVAL, "B must be in [2, 256]");
  if (batch < 0) return fail(AMH_EINVAL, "batch must be >= 0");
  if (!edges) return fail(AMH_EINVAL, "edges is NULL");
  const long long rows = (long long)L * (L - 1) / 2;
  const int Bp = (B + 1) & ~1;
  if (rows * Bp > (long long)AMH_NOALLOC_MAX_ENTRIES)
    return fail(AMH_EINVAL, "table of " + std::to_string(rows * Bp) +
                                " entries exceeds the static scratch of " +
                                std::to_string(AMH_NOALLOC_MAX_ENTRIES) + " entries");
  // evenly spaced bin centres (as amh_init)
  std::vector<double> cen(B);
  for (int j = 0; j < B; ++j) {
    if (!(edges[j] < edges[j + 1]) || !std::isfinite(edges[j]))
      return fail(AMH_EINVAL, "edges must be finite and ascending (last may be +inf)");
    if (std::isinf(edges[j + 1])) {
      if (j == 0) return fail(AMH_EINVAL, "open first bin");
      cen[j] = edges[j] + 0.5 * (edges[j] - edges[j - 1]);
    } else {
      cen[j] = 0.5 * (edges[j] + edges[j + 1]);
    }
  }
  const double w = (cen[B - 1] - cen[0]) / (B - 1);
  for (int j = 0; j + 1 < B; ++j)
    if (std::fabs((cen[j + 1] - cen[j]) - w) > 1e-9 * w)
      return fail(AMH_EINVAL, "bin centres are not evenly spaced");
  if (batch == 0) return AMH_OK;
  if (!on_device(table) || !on_device(theta) || !on_device(E_out) || !on_device(dE_dtheta))
    return fail(AMH_EINVAL, "table, theta, E_out and dE_dtheta must be device pointers");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(AMH_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(AMH_EINVAL, "device ordinal too large");
  float2* scratch = nullptr;
  {
    // once per device, with that device current: the device address of the
    // static array (its host-side name is not a device address)
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_table_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_table);
      if (e != cudaSuccess)
        return fail(AMH_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_table_ptr[dev] = (float2*)p;
    }
    scratch = g_table_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  size_t optin = 0;
  {
    static bool smem_set[kMaxDevices] = {false};
    static size_t smem_optin[kMaxDevices] = {0};
    std::lock_guard<std::mutex> lk(g_mu);
    if (!smem_set[dev]) {
      cudaDeviceProp prop;
      e = cudaGetDeviceProperties(&prop, dev);
      if (e == cudaSuccess) e = grad_set_smem<float>(prop.sharedMemPerBlockOptin);
      if (e != cudaSuccess) return fail(AMH_ECUDA, std::string("set-up: ") + cudaGetErrorString(e));
      smem_optin[dev] = prop.sharedMemPerBlockOptin;
      smem_set[dev] = true;
    }
    optin = smem_optin[dev];
  }
  // the gradient kernel keeps one chain's coordinates in shared memory: the
  // same limit amh_grad applies (1 KB left for its static shared memory)
  if (grad_smem_bytes(sizeof(float), L) + 1024 > optin)
    return fail(AMH_EINVAL, "L = " + std::to_string(L) + " is too long for the gradient "
                                "kernel's shared memory");
  e = launch_prep_table<float>(table, rows, B, Bp, table_is_neglog, (float*)scratch, st);
  if (e != cudaSuccess) return fail(AMH_ECUDA, std::string("table kernel: ") + cudaGetErrorString(e));

  Tab<float> tb{};  // tex = 0: the gradient kernel reads entries by plain loads
  tb.E = scratch;
  tb.inv_w = (float)(1.0 / w);
  tb.off = (float)(-cen[0] / w);
  tb.umax = (float)(B - 1);
  tb.k1 = (float)(1.0 / w / (B - 1));
  tb.k2 = (float)(-cen[0] / w / (B - 1));
  tb.Bp = Bp;
  Geom<float> g = ideal_geometry<float>();
  ProteinDev pd;
  memset(&pd, 0, sizeof(pd));
  pd.L = L;
  pd.n = 2 * L;
  e = launch_grad<float>(&pd, 0, L, theta, batch, E_out, dE_dtheta, tb, g, st);
  if (e != cudaSuccess) return fail(AMH_ECUDA, std::string("gradient kernel: ") + cudaGetErrorString(e));
  return AMH_OK;
}
