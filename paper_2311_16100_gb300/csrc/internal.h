// Host-side internals of libcryosgd: the handle, its workspace, argument
// preparation and the kernel launchers each translation unit provides.
#pragma once

#include <atomic>
#include <utility>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/cryosgd.h"
#include "device.cuh"
#include "fused_ws.h"

struct cs_handle {
  int device = 0;
  int num_sms = 0;
  std::string err;
  // workspace (grown on demand, released in cs_destroy)
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int algo = 0;            // CS_ALGO_*
  int table_key = -1;      // (M, r_max) of the cached disc pixel table
  // launch shape of the trilinear traversals (cs_set_launch_shape / cs_autotune)
  int block = 256;
  int blocks_per_sm = 8;
  int slabs = 0;           // z-slabs per traversal (0: by footprint, cs_set_slabs)
  // multi-volume workspace
  void* mws = nullptr;
  size_t mws_bytes = 0;
  int mws_generation = 0;
  int mtable_key[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
  // device status word: set by kernels whose bounded waits ran out
  int* status = nullptr;
  // profiler: CS_NPHASES + 1 boundary events per timed step
  bool prof = false;
  int prof_max_steps = 0;
  int prof_steps = 0;
  std::vector<cudaEvent_t> prof_events;
  // double-buffered staging of host batches (cs_precond_sgd_step_host)
  int host_mode = 0;          // CS_HOST_STAGED / CS_HOST_DIRECT
  void* stage = nullptr;
  int stage_M = 0, stage_B = 0;
  unsigned long long stage_calls = 0;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t copy_done[2] = {nullptr, nullptr};
  cudaEvent_t compute_done[2] = {nullptr, nullptr};
  // disc-packed host batches: row starts of the disc of radius disc_r in
  // the packed order (device int[2 disc_r + 2])
  int* disc_rows = nullptr;
  int disc_M = 0, disc_r = -1;
};

namespace cs {

// Kernel launches made by the library (reported by cs_kernel_launches).
extern std::atomic<uint64_t> g_launches;
inline void count_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

// Dynamic shared memory limit of a kernel, raised once per device: the
// attribute belongs to the kernel on the current device, so a process that
// uses several GPUs sets it on each (done: one bit per device below 64;
// devices past that set it at every call).
template <typename K>
cudaError_t ensure_smem_limit(K* kernel, int bytes, std::atomic<uint64_t>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = dev < 64 ? 1ull << dev : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// Launch with programmatic stream serialisation: the kernel's blocks may be
// scheduled while the previous kernel in the stream finishes; the kernel
// must call grid_dep_wait() before its first access to memory.
template <typename... P, typename... A>
cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, cudaStream_t s, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

// Workspace layout for a grid of side M and batches of up to B images:
// offsets are 256-byte aligned.
struct Workspace {
  float2* g;         // gradient, complex [M^3]
  float2* d;         // step direction, complex [M^3]
  float* dhat;       // thresholded preconditioner [M^3]
  float* dest;       // Hutchinson estimate of the batch [M^3]
  uint32_t* bits;    // probe words [M^3]
  double* part;      // block partial sums [kPartSlots]
  // tile engine
  int* tile_count;   // [n_tiles]
  int* tile_list;    // [n_tiles][B]
  int* item_start;   // [n_tiles + 1]
  int* queue;        // [1]
  double* part_items;   // [max items]: loss partials
  double* part_items2;  // [max items]: curvature partials
  FusedWs fw;           // vector-reduction accumulators and disc table
};

constexpr int kPartRegion = 8192;           // doubles per partial-sum region
constexpr int kPartSlots = 4 * kPartRegion; // four regions
constexpr int kBlock = 256;            // threads per block of the pixel kernels

size_t workspace_bytes(int M, int B);
Workspace carve(void* base, int M, int B);

// Geometry for the kernels; FP64 CTF constants folded on the host.
Geo make_geo(const cs_geom& g);

// Number of blocks of the grid-stride pixel kernels.
int pixel_grid(int num_sms, int B, int M);

// ---- launchers (return the cudaError_t of the launch) ----
cudaError_t launch_quat_to_rot(const float* quat, int B, float* rot, cudaStream_t s);
// rotations of batch (*cursor mod n_batches) of a dataset's quaternions
cudaError_t launch_quat_to_rot_cursor(const float* quat, int B, int n_batches,
                                      const double* cursor, float* rot, cudaStream_t s);
cudaError_t launch_slice_project(const Geo& G, const float2* vol, const float* rot,
                                 const float* df, int B, float2* out, int grid,
                                 cudaStream_t s);
cudaError_t launch_backproject(const Geo& G, const float2* img, const float* rot,
                               const float* df, int B, float scale, float2* vol,
                               int grid, cudaStream_t s);
// loss_grad: grad = lambda v (init) then += scatter; data-term partials in
// part_loss[0..grid), |v|^2 partials in part_vv[0..*n_vv); if loss != NULL the
// final loss is written there.
cudaError_t launch_loss_grad(const Geo& G, const float2* vol, const float2* img,
                             const float* rot, const float* df, int B, float lambda,
                             float scale, float2* grad, double* loss, double* part_loss,
                             double* part_vv, int* n_vv, int grid, int num_sms,
                             cudaStream_t s);
// grad = lambda v and |v|^2 partials (part_vv[0..*n_vv)).
cudaError_t launch_init_grad(int n, const float2* vol, float lambda, float2* grad,
                             double* part_vv, int* n_vv, int num_sms, cudaStream_t s);
// loss = scale/2 sum(pl[0..n)) + lambda/2 sum(pv[0..nv)), n = *n_dev if n_dev.
cudaError_t launch_finalize_loss(const double* pl, int n, const int* n_dev, const double* pv,
                                 int nv, float lambda, float scale, double* loss,
                                 cudaStream_t s);
cudaError_t launch_fill(int n, float value, float* out, int num_sms, cudaStream_t s);
cudaError_t launch_scale_copy(int n, const float* z, float lambda, float* out, int num_sms,
                              cudaStream_t s);
cudaError_t launch_hvp(const Geo& G, const float* z, const float* rot, const float* df,
                       int B, float lambda, float scale, float* Hz, int grid,
                       int num_sms, cudaStream_t s);
cudaError_t launch_probe_bits(int M, uint64_t seed, uint64_t block_host,
                              const double* k_dev, uint32_t* bits, int num_sms,
                              cudaStream_t s);
cudaError_t launch_hutchinson(const Geo& G, const uint32_t* bits, const float* rot,
                              const float* df, int B, float lambda, float scale,
                              int n_probes, float* diag, int grid, int num_sms,
                              cudaStream_t s);
cudaError_t launch_exact_diag(const Geo& G, const float* rot, const float* df, int B,
                              float lambda, float scale, float* diag, float* cov,
                              float* c2w, int grid, int num_sms, cudaStream_t s);
cudaError_t launch_alpha(const Geo& G, const float* df, int N, double px_over_pv,
                         double lambda, double scale_alpha, double* alpha,
                         cudaStream_t s);
// SGD step pieces
cudaError_t launch_precond_update(int n, const float* dest, float* D, float* Davg,
                                  float* dhat, const double* scalars, float beta,
                                  int num_sms, cudaStream_t s);
// D = ((k-1)/k) D + (1/k) est (D = est at k = 1, whatever D held).
cudaError_t launch_running_mean(int n, const float* est, float* D, long k, int num_sms,
                                cudaStream_t s);
cudaError_t launch_fixed_dhat(int n, const float* D, float* dhat, const double* scalars,
                              int num_sms, cudaStream_t s);
// d = g / dhat (dhat NULL: d = g); part[0..gb) <- sum |g|^2/dhat,
// part[gb..2gb) <- sum |d|^2; returns gb through *nblk.
cudaError_t launch_direction(int n, const float2* g, const float* dhat, float2* d,
                             double* part, int* nblk, int num_sms, cudaStream_t s);
// part[0..grid) <- sum_i sum_p |C P d|^2
cudaError_t launch_curvature(const Geo& G, const float2* d, const float* rot,
                             const float* df, int B, double* part, int grid,
                             cudaStream_t s);
// n_loss / n_Q are read from *n_dev when n_dev is not NULL (tile items).
cudaError_t launch_eta(double* scalars, const double* part_loss, int n_loss,
                       const double* part_vv, int n_vv, const double* part_G,
                       const double* part_dd, int n_dir, const double* part_Q,
                       int n_Q, const int* n_dev, float lambda, float scale, float c,
                       int max_halvings, cudaStream_t s);
cudaError_t launch_update(int n, float2* v, const float2* d, const double* scalars,
                          int num_sms, cudaStream_t s);
// learned preconditioner network (mlp.cu)
constexpr int kMlpParams = 4481;
cudaError_t launch_mlp_forward(int M, const float* params, const float* cov, const float* c2w,
                               float* out, int exp_out, float offset, bool tc, int* err,
                               int num_sms, cudaStream_t s);
cudaError_t launch_mlp_grad(int M, int r2, float inv_n, const float* params, const float* cov,
                            const float* c2w, const float* target, float* grad, double* sse,
                            bool tc, int* err, int num_sms, cudaStream_t s);
// Failure-handling self-test: a bounded mbarrier wait that runs out.
cudaError_t launch_wait_selftest(long long limit, int* err, cudaStream_t s);
cudaError_t launch_adam(float* p, float* m, float* v, float* g, float gscale, int step,
                        float lr, float b1, float b2, float eps, cudaStream_t s);
// network target: log(max(mean of n_est estimates, floor_rel x mean of the
// positive means)); part: 2 x (grid) doubles of scratch
cudaError_t launch_mlp_target(int M, int n_est, const float* est, float floor_rel,
                              float* target, double* part, int num_sms, cudaStream_t s);

// Spreads disc-packed images (complex64[B][n_px], rows of the disc of radius
// r in order, row starts rows[0 .. 2r+1]) into image layout [B][M][M]; the
// pixels outside the disc are not written.
cudaError_t launch_expand_disc(int M, int r, int B, const int* rows, const float* packed,
                               float* images, cudaStream_t s);

// Rate of 16-byte global reductions (G ops/s) measured on a scratch buffer.
cudaError_t measure_red_rate(void* scratch, size_t bytes, int num_sms, cudaStream_t s,
                             double* gops);
// In-plane shift phase (shifts.cu): images[i] *= T_i (sign +1) or T_i^* (-1).
cudaError_t launch_phase_shift(int M, int B, float2* images, const float* shifts, int sign,
                               int num_sms, cudaStream_t s);
// Per-shell reductions (shells.cu); n_sh <= kMaxShells.
constexpr int kMaxShells = 1024;
cudaError_t launch_fsc(int M, const float2* u, const float2* v, int n_sh, double* sums,
                       double* fsc, int num_sms, cudaStream_t s);
cudaError_t launch_shell_minmax(int M, const float* x, int n_sh, float* lo, float* hi, int* count,
                                int num_sms, cudaStream_t s);
cudaError_t launch_rel_err(const Geo& G, const float2* v, const float2* vref,
                           double* part, double* out, int num_sms, cudaStream_t s);

}  // namespace cs
