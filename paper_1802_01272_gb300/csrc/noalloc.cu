// noalloc.cu -- density histogram of caller-owned distributions that
// allocates no memory.
//
// Who needs it: callers that must not call cudaMalloc or any allocating
// routine -- processes whose device memory is handed out by another
// allocator or reserved up front (a serving loop that keeps every lattice
// resident and has budgeted all of HBM), loops that cannot afford the device
// synchronisation an allocation may imply, and callers that keep f in their
// own buffers without a lbm_handle.  lbm_histogram needs a temporary device
// counts buffer on every call; this variant counts into a fixed, file-scope
// device array instead.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "ctulbm.h"
#include "lbm_internal.h"

using namespace ctulbm;

namespace {

// The shared bin counters.  Every device that loads the library holds this
// array (LBM_NOALLOC_MAX_BINS x 8 bytes) until the process exits.
static __device__ __align__(256) unsigned long long g_noalloc_bins[LBM_NOALLOC_MAX_BINS];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_bins_addr[kMaxDevices] = {nullptr};

// The array's name is only a host-side stand-in; the device address is
// looked up once per device, with that device current, and kept for the life
// of the process: it assumes the device's context is not reset
// (cudaDeviceReset) while the library is loaded.
int bins_address(int device, unsigned long long** out) {
  if (device < 0 || device >= kMaxDevices) return LBM_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_bins_addr[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_bins) != cudaSuccess || !p) return LBM_ERR_CUDA;
    g_bins_addr[device] = p;
  }
  *out = static_cast<unsigned long long*>(g_bins_addr[device]);
  return LBM_OK;
}

}  // namespace

extern "C" int lbm_histogram_noalloc(const void* f_device, int32_t Lx, int32_t Ly,
                                     int32_t precision, double rho_ref, int32_t nbins, double lo,
                                     double hi, void* cuda_stream, int64_t* counts) {
  if (!f_device || !counts || Lx < 1 || Ly < 1 || (long long)Lx * Ly > (1LL << 31) - 1)
    return LBM_ERR_INVALID_ARG;
  if (nbins < 1 || nbins > LBM_NOALLOC_MAX_BINS || !(hi > lo)) return LBM_ERR_INVALID_ARG;
  if (precision != LBM_FP64 && precision != LBM_FP32_SHIFTED && precision != LBM_FP16_SHIFTED)
    return LBM_ERR_INVALID_ARG;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return LBM_ERR_CUDA;
  // the bins live on the current device: f must be there too
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, f_device) != cudaSuccess) return LBM_ERR_INVALID_ARG;
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
    return LBM_ERR_INVALID_ARG;
  if (attr.device != device) return LBM_ERR_INVALID_ARG;
  unsigned long long* bins = nullptr;
  const int r = bins_address(device, &bins);
  if (r != LBM_OK) return r;

  AuxArgs a;
  std::memset(&a, 0, sizeof(a));
  a.Lx = Lx;
  a.Ly = Ly;
  a.plane = (long long)Lx * Ly;
  a.storage = precision == LBM_FP64 ? STORE_F64 : (precision == LBM_FP16_SHIFTED ? STORE_F16 : STORE_F32);
  a.rho_ref = precision == LBM_FP64 ? 0.0 : rho_ref;  // rho = rho_ref + sum_k f_k

  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const size_t bytes = sizeof(unsigned long long) * (size_t)nbins;
  if (cudaMemsetAsync(bins, 0, bytes, s) != cudaSuccess) return LBM_ERR_CUDA;
  if (launch_hist(a, f_device, nbins, lo, hi, bins, s) != cudaSuccess) return LBM_ERR_CUDA;
  if (cudaMemcpyAsync(counts, bins, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return LBM_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return LBM_ERR_CUDA;
  return LBM_OK;
}
