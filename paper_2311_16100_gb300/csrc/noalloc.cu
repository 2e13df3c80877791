// Hutchinson's diagonal estimate without any device allocation.
//
// Some callers cannot allocate device memory at the time they need the
// estimate: code running inside a stream capture of a larger application
// (where a cudaMalloc would break or serialise the capture), processes whose
// device memory is owned by a caching allocator that must not be bypassed
// or fragmented, and services that reserve all their memory at start-up and
// forbid allocation afterwards.  cs_hutchinson_diag_noalloc serves them: its
// only scratch, the probe words (one 32-bit word per voxel), lives in a
// fixed file-scope device array sized for grids up to 128^3 (8 MiB), which
// every GPU that loads the library holds until the process exits.  The
// caller passes the rotations, defocus and the output buffer; nothing else
// is allocated, no handle is needed.
#include <cmath>
#include <mutex>

#include "internal.h"

namespace cs {

namespace {

constexpr int kNoAllocMaxM = 128;

// probe-word scratch shared by every call (the last call's words remain)
static __device__ __align__(256) uint32_t g_probe_scratch[kNoAllocMaxM * kNoAllocMaxM * kNoAllocMaxM];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
uint32_t* g_scratch_ptr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};

// Device address of the scratch array and the SM count, fetched once per
// device with that device current.  In host code the array's name is only a
// host-side stand-in, never a device address.  The cached address belongs
// to the device's context as it was at the first call: after a
// cudaDeviceReset of that device the array is reloaded elsewhere, so this
// entry point must not be called on a device that was reset.
cudaError_t setup_device(int dev, uint32_t** scratch, int* num_sms) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_probe_scratch);
    if (e != cudaSuccess) return e;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g_num_sms[dev] = sms;
    g_scratch_ptr[dev] = static_cast<uint32_t*>(p);
  }
  *scratch = g_scratch_ptr[dev];
  *num_sms = g_num_sms[dev];
  return cudaSuccess;
}

}  // namespace

}  // namespace cs

extern "C" int cs_hutchinson_diag_noalloc(const cs_geom* g, const float* rot,
                                          const float* defocus, int B, float lambda,
                                          float scale, int n_probes, uint64_t seed,
                                          uint64_t probe_block, float* diag_out,
                                          void* stream) {
  using namespace cs;
  if (!g || !diag_out) return CS_ERR_ARG;
  if (g->M < 4 || g->M > CS_MAX_M || (g->M & 1)) return CS_ERR_SHAPE;
  if (g->M > kNoAllocMaxM) return CS_ERR_SHAPE;   // beyond the fixed scratch
  if (g->r_max < 1 || g->r_max > g->M / 2 - 1) return CS_ERR_SHAPE;
  if (g->interp != CS_NEAREST && g->interp != CS_TRILINEAR) return CS_ERR_ARG;
  if (B < 0 || n_probes < 1 || n_probes > 32) return CS_ERR_SHAPE;
  if (!std::isfinite(lambda) || !std::isfinite(scale)) return CS_ERR_ARG;
  const long nch = ((long)g->M * g->M + kBlock - 1) / kBlock;
  if ((long)B * nch > 0x7fffffffL) return CS_ERR_SHAPE;
  if (B > 0 && !rot) return CS_ERR_ARG;
  if (B > 0 && g->ctf.enabled && !defocus) return CS_ERR_ARG;
  if (g->ctf.enabled) {
    const cs_ctf& c = g->ctf;
    if (!(std::isfinite(c.kv) && c.kv > 0) || !(std::isfinite(c.pixel_A) && c.pixel_A > 0) ||
        !(std::isfinite(c.cs_mm) && c.cs_mm >= 0) ||
        !(std::isfinite(c.amp) && c.amp >= 0 && c.amp < 1))
      return CS_ERR_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return CS_ERR_CUDA;
  }
  uint32_t* scratch = nullptr;
  int num_sms = 0;
  if (setup_device(dev, &scratch, &num_sms) != cudaSuccess) {
    cudaGetLastError();
    return CS_ERR_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Geo G = make_geo(*g);
  if (g->interp == CS_TRILINEAR &&
      launch_probe_bits(g->M, seed, probe_block, nullptr, scratch, num_sms, s) != cudaSuccess)
    return CS_ERR_CUDA;
  if (launch_hutchinson(G, scratch, rot, defocus, B, lambda, scale, n_probes, diag_out,
                        pixel_grid(num_sms, B, g->M), num_sms, s) != cudaSuccess)
    return CS_ERR_CUDA;
  return CS_OK;
}
