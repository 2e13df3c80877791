// C ABI of libcryosgd (declared in include/cryosgd.h): handle, workspace,
// host-side argument validation and the stream-ordered composition of the
// kernels into the calls of the paper's problem statement.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"
#include "tiles.h"
#include "fused.h"

namespace cs {

std::atomic<uint64_t> g_launches{0};

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

size_t workspace_bytes(int M, int B) {
  const size_t n = (size_t)M * M * M;
  const size_t nt = (size_t)tile_count_for(M);
  const size_t items = max_items_for(M, B > 0 ? B : 1);
  return align256(n * sizeof(float2)) * 2 + align256(n * sizeof(float)) * 2 +
         align256(n * sizeof(uint32_t)) + align256(kPartSlots * sizeof(double)) +
         align256(nt * sizeof(int)) + align256(nt * (size_t)(B > 0 ? B : 1) * sizeof(int)) +
         align256((nt + 1) * sizeof(int)) + align256(sizeof(int)) +
         2 * align256(items * sizeof(double)) + align256(fused_ws_bytes(M)) +
         align256(slab_lists_bytes(M, B));
}

Workspace carve(void* base, int M, int B) {
  const size_t n = (size_t)M * M * M;
  const size_t nt = (size_t)tile_count_for(M);
  const size_t items = max_items_for(M, B > 0 ? B : 1);
  char* p = static_cast<char*>(base);
  Workspace w;
  // vector-pass region first: its layout depends on M only
  w.fw = fused_carve(p, M);                p += align256(fused_ws_bytes(M));
  w.g = reinterpret_cast<float2*>(p);      p += align256(n * sizeof(float2));
  w.d = reinterpret_cast<float2*>(p);      p += align256(n * sizeof(float2));
  w.dhat = reinterpret_cast<float*>(p);    p += align256(n * sizeof(float));
  w.dest = reinterpret_cast<float*>(p);    p += align256(n * sizeof(float));
  w.bits = reinterpret_cast<uint32_t*>(p); p += align256(n * sizeof(uint32_t));
  w.part = reinterpret_cast<double*>(p);   p += align256(kPartSlots * sizeof(double));
  w.tile_count = reinterpret_cast<int*>(p); p += align256(nt * sizeof(int));
  w.tile_list = reinterpret_cast<int*>(p);  p += align256(nt * (size_t)(B > 0 ? B : 1) * sizeof(int));
  w.item_start = reinterpret_cast<int*>(p); p += align256((nt + 1) * sizeof(int));
  w.queue = reinterpret_cast<int*>(p);      p += align256(sizeof(int));
  w.part_items = reinterpret_cast<double*>(p); p += align256(items * sizeof(double));
  w.part_items2 = reinterpret_cast<double*>(p); p += align256(items * sizeof(double));
  slab_carve(p, M, B, w.fw);   // per-slab item lists of the slab-split traversals
  return w;
}

Geo make_geo(const cs_geom& g) {
  Geo G{};
  G.M = g.M;
  G.half = g.M / 2;
  G.r2max = g.r_max * g.r_max;
  G.interp = g.interp;
  G.ctf_on = g.ctf.enabled ? 1 : 0;
  if (G.ctf_on) {
    const double V = (double)g.ctf.kv * 1e3;
    const double lam = 12.2643 / std::sqrt(V * (1.0 + 0.978466e-6 * V));
    const double box = (double)g.M * (double)g.ctf.pixel_A;
    const double ka = lam / (box * box);
    const double kb = 0.5 * (double)g.ctf.cs_mm * 1e7 * lam * lam * lam / (box * box * box * box);
    G.ka_hi = (float)ka;
    G.ka_lo = (float)(ka - (double)G.ka_hi);
    G.kb = (float)kb;
    const double A = (double)g.ctf.amp;
    G.wsin = (float)std::sqrt(1.0 - A * A);
    G.wcos = (float)A;
  }
  return G;
}

int pixel_grid(int num_sms, int B, int M) {
  const long nch = ((long)M * M + kBlock - 1) / kBlock;
  const long total = (long)B * nch;
  const long cap = (long)num_sms * 8;   // 8 blocks of 256 threads per SM
  long g = total < cap ? total : cap;
  return (int)(g > 0 ? g : 1);
}

}  // namespace cs

#ifdef CS_DEBUG_BOUNDS
namespace cs {
// readers of every translation unit's range-check flag (debug build)
std::vector<unsigned (*)()>& dbg_readers() {
  static std::vector<unsigned (*)()> v;
  return v;
}
void dbg_register(unsigned (*reader)()) { dbg_readers().push_back(reader); }
}  // namespace cs
#endif

using namespace cs;

namespace {

int fail(cs_handle* h, int code, const char* fmt, ...) {
  if (h) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    h->err = buf;
  }
  return code;
}

int cuda_fail(cs_handle* h, cudaError_t e, const char* what) {
  return fail(h, CS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Makes the handle's device current for the duration of a call.
struct DeviceScope {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) err = cudaSetDevice(dev);
  }
  ~DeviceScope() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool is_finite(double x) { return std::isfinite(x); }

int check_geom(cs_handle* h, const cs_geom* g) {
  if (!g) return fail(h, CS_ERR_ARG, "geometry pointer is NULL");
  if (g->M < 4 || g->M > CS_MAX_M || (g->M & 1))
    return fail(h, CS_ERR_SHAPE, "M=%d must be even and in [4, %d]", g->M, CS_MAX_M);
  if (g->r_max < 1 || g->r_max > g->M / 2 - 1)
    return fail(h, CS_ERR_SHAPE, "r_max=%d must be in [1, M/2-1=%d]", g->r_max, g->M / 2 - 1);
  if (g->interp != CS_NEAREST && g->interp != CS_TRILINEAR)
    return fail(h, CS_ERR_ARG, "interp=%d is not CS_NEAREST or CS_TRILINEAR", g->interp);
  if (g->ctf.enabled) {
    const cs_ctf& c = g->ctf;
    if (!(is_finite(c.kv) && c.kv > 0) || !(is_finite(c.pixel_A) && c.pixel_A > 0) ||
        !(is_finite(c.cs_mm) && c.cs_mm >= 0) || !(is_finite(c.amp) && c.amp >= 0 && c.amp < 1))
      return fail(h, CS_ERR_ARG, "CTF parameters out of range (kv>0, pixel>0, Cs>=0, 0<=A<1)");
  }
  return CS_OK;
}

int check_batch(cs_handle* h, const cs_geom* g, int B, const float* rot,
                const float* defocus) {
  if (B < 0) return fail(h, CS_ERR_SHAPE, "batch size B=%d is negative", B);
  const long nch = ((long)g->M * g->M + kBlock - 1) / kBlock;
  if ((long)B * nch > 0x7fffffffL || (long)B * g->M * g->M * 2 > (long)1 << 62)
    return fail(h, CS_ERR_SHAPE, "batch size B=%d too large for M=%d", B, g->M);
  if (B > 0 && !rot) return fail(h, CS_ERR_ARG, "rot is NULL");
  if (B > 0 && g->ctf.enabled && !defocus)
    return fail(h, CS_ERR_ARG, "defocus is NULL but the CTF is enabled");
  return CS_OK;
}

int ensure_ws(cs_handle* h, int M, int B, Workspace* w) {
  const size_t need = workspace_bytes(M, B);
  if (h->ws_bytes < need) {
    if (const char* f = getenv("CS_FAULT_INJECT_ALLOC"))
      if (f[0] == '1') return fail(h, CS_ERR_ALLOC, "workspace allocation failed (injected)");
    if (h->ws) {
      cudaError_t e = cudaDeviceSynchronize();
      if (e != cudaSuccess) return cuda_fail(h, e, "synchronise before workspace growth");
      cudaFree(h->ws);
      h->ws = nullptr;
      h->ws_bytes = 0;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(h, CS_ERR_ALLOC, "workspace of %zu bytes: %s", need, cudaGetErrorString(e));
    }
    h->ws = p;
    h->ws_bytes = need;
    h->table_key = -1;
  }
  *w = carve(h->ws, M, B);
  return CS_OK;
}

// The traversals of grids split into z-slabs use the tile-ordered disc
// table (whole items outside a slab are skipped); one slab keeps the
// row-ordered table (no idle lanes on the disc's edge tiles).
bool tiled_table(const cs_handle* h, int M) {
  const int S = h->slabs > 0 ? h->slabs : slab_count(M, F_GRAD | F_HUTCH);
  return S > 1;
}

// Disc pixel table of the vector passes for grid M, disc r: rebuilt on the
// stream when the grid, the disc, the layout or the workspace changed.
cudaError_t prepare_vector(cs_handle* h, const Workspace& w, int M, int r, cudaStream_t s) {
  const bool tiled = tiled_table(h, M);
  const int key = ((tiled ? 1 + (h->block == 128) : 0) << 28) | (M << 12) | r;
  if (h->table_key != key) {
    cudaError_t e = tiled ? launch_disc_table_tiled(M, r, h->block, w.fw, s)
                          : launch_disc_table(M, r, w.fw, s);
    if (e != cudaSuccess) return e;
    h->table_key = key;
  }
  return cudaSuccess;
}

bool use_tiles(const cs_handle* h) { return h->algo == CS_ALGO_TILED; }

// Grid of a vector traversal: one block per item up to num_sms x the blocks
// per SM of the handle's launch shape.  The gather-only curvature pass is
// capped at the blocks resident at once (one wave: measured 9% faster at
// 128^3, batch 1024); the passes with reductions run oversubscribed, where
// blocks that finish early are replaced (measured 3% faster than one wave).
int vec_grid(const cs_handle* h, int B, int M, int flags) {
  const long items = (long)B * (((long)M * M + h->block - 1) / h->block);
  int per_sm = h->blocks_per_sm;
  if (flags == F_CURV) {
    // one wave of the kernel that will run (slab-split passes have their own)
    const bool split = tiled_table(h, M) && pass_slabs(M, F_CURV, h->slabs) > 1;
    const int f = split ? (F_CURV | F_SLAB) : F_CURV;
    const int res = fused_resident(f, h->block, false);
    if (res < per_sm) per_sm = res;
  }
  const long cap = (long)h->num_sms * per_sm;
  const long g = items < cap ? items : cap;
  return (int)(g > 0 ? (g < kPartRegion ? g : kPartRegion) : 1);
}
// Vector-reduction passes: the default for trilinear interpolation.
bool use_vector(const cs_handle* h, const cs_geom* g) {
  return (h->algo == CS_ALGO_AUTO || h->algo == CS_ALGO_VECTOR) && g->interp == CS_TRILINEAR;
}

// Bins the batch for the tile engine and fills the common fields of A.
cudaError_t bin_batch(cs_handle* h, const Geo& G, const Workspace& w, const float* rot,
                      const float* df, int B, float scale, TileArgs& A, cudaStream_t s) {
  A = TileArgs{};
  A.df = df;
  A.scale = scale;
  return launch_bin(G, rot, B, A, w.tile_count, w.tile_list, w.item_start, w.queue, s);
}

inline cudaStream_t S(void* s) { return static_cast<cudaStream_t>(s); }

#define CS_TRY(expr)             \
  do {                           \
    int _rc = (expr);            \
    if (_rc != CS_OK) return _rc; \
  } while (0)

#define CS_CUDA(expr, what)                          \
  do {                                               \
    cudaError_t _e = (expr);                         \
    if (_e != cudaSuccess) return cuda_fail(h, _e, what); \
  } while (0)

#define CS_SCOPE(h)                                                   \
  DeviceScope _scope((h)->device);                                    \
  if (_scope.err != cudaSuccess) return cuda_fail((h), _scope.err, "cudaSetDevice")

// NVTX range of the step phase being enqueued by this thread (a tool such
// as Nsight Systems shows it; without one attached the calls do nothing)
thread_local bool t_phase_open = false;

void phase_range(int b) {
  static const char* const kNames[CS_NPHASES] = {"cs step: precond", "cs step: loss_grad",
                                                  "cs step: direction", "cs step: curvature",
                                                  "cs step: update"};
  if (t_phase_open) {       // the previous phase ends (or a step that returned early)
    nvtxRangePop();
    t_phase_open = false;
  }
  if (b < CS_NPHASES) {
    nvtxRangePushA(kNames[b]);
    t_phase_open = true;
  }
}

// Records boundary event `b` (0..CS_NPHASES) of the current step: the NVTX
// phase range, and the timing event when the profiler is on.
void prof_mark(cs_handle* h, int b, cudaStream_t s) {
  phase_range(b);
  if (!h->prof || h->prof_steps >= h->prof_max_steps) return;
  const size_t i = (size_t)h->prof_steps * (CS_NPHASES + 1) + b;
  if (i < h->prof_events.size()) cudaEventRecord(h->prof_events[i], s);
  if (b == CS_NPHASES) ++h->prof_steps;
}

void prof_free(cs_handle* h) {
  for (cudaEvent_t e : h->prof_events) cudaEventDestroy(e);
  h->prof_events.clear();
  h->prof_steps = 0;
  h->prof_max_steps = 0;
}

}  // namespace

extern "C" {

int cs_create(cs_handle** out, int device) {
  if (!out) return CS_ERR_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    return CS_ERR_CUDA;
  }
  if (device < 0 || device >= n) return CS_ERR_ARG;
  cs_handle* h = new (std::nothrow) cs_handle();
  if (!h) return CS_ERR_ALLOC;
  h->device = device;
  {
    DeviceScope scope(device);
    if (scope.err != cudaSuccess ||
        cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device) !=
            cudaSuccess) {
      cudaGetLastError();
      delete h;
      return CS_ERR_CUDA;
    }
  }
  *out = h;
  return CS_OK;
}

int cs_destroy(cs_handle* h) {
  if (!h) return CS_OK;
  {
    DeviceScope scope(h->device);
    if (h->ws) {
      cudaDeviceSynchronize();
      cudaFree(h->ws);
    }
    prof_free(h);
    if (h->mws) cudaFree(h->mws);
    if (h->status) cudaFree(h->status);
    if (h->disc_rows) cudaFree(h->disc_rows);
    if (h->stage || h->copy_stream) {
      cudaDeviceSynchronize();
      if (h->stage) cudaFree(h->stage);
      for (int i = 0; i < 2; ++i) {
        if (h->copy_done[i]) cudaEventDestroy(h->copy_done[i]);
        if (h->compute_done[i]) cudaEventDestroy(h->compute_done[i]);
      }
      if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    }
  }
  delete h;
  return CS_OK;
}

const char* cs_last_error(const cs_handle* h) { return h ? h->err.c_str() : ""; }

const char* cs_status_string(int s) {
  switch (s) {
    case CS_OK: return "CS_OK";
    case CS_ERR_ARG: return "CS_ERR_ARG";
    case CS_ERR_SHAPE: return "CS_ERR_SHAPE";
    case CS_ERR_CUDA: return "CS_ERR_CUDA";
    case CS_ERR_TIMEOUT: return "CS_ERR_TIMEOUT";
    case CS_ERR_INTERNAL: return "CS_ERR_INTERNAL";
    case CS_ERR_ALLOC: return "CS_ERR_ALLOC";
    default: return "CS_UNKNOWN";
  }
}

int cs_reserve(cs_handle* h, int M, int max_batch) {
  if (!h) return CS_ERR_ARG;
  if (M < 4 || M > CS_MAX_M || (M & 1))
    return fail(h, CS_ERR_SHAPE, "M=%d must be even and in [4, %d]", M, CS_MAX_M);
  if (max_batch < 0) return fail(h, CS_ERR_SHAPE, "max_batch=%d is negative", max_batch);
  CS_SCOPE(h);
  Workspace w;
  CS_TRY(ensure_ws(h, M, max_batch, &w));
  CS_CUDA(cudaDeviceSynchronize(), "cs_reserve");
  return CS_OK;
}

size_t cs_workspace_bytes(const cs_handle* h) { return h ? h->ws_bytes : 0; }

int cs_set_algo(cs_handle* h, int algo) {
  if (!h) return CS_ERR_ARG;
  if (algo != CS_ALGO_AUTO && algo != CS_ALGO_PIXEL && algo != CS_ALGO_TILED &&
      algo != CS_ALGO_VECTOR)
    return fail(h, CS_ERR_ARG, "algo=%d is not a CS_ALGO_* value", algo);
  h->algo = algo;
  return CS_OK;
}

int cs_quat_to_rot(cs_handle* h, const float* quat, int B, float* rot, void* stream) {
  if (!h) return CS_ERR_ARG;
  if (B < 0) return fail(h, CS_ERR_SHAPE, "B=%d is negative", B);
  if (B == 0) return CS_OK;
  if (!quat || !rot) return fail(h, CS_ERR_ARG, "quat or rot is NULL");
  CS_SCOPE(h);
  CS_CUDA(launch_quat_to_rot(quat, B, rot, S(stream)), "quat_to_rot launch");
  return CS_OK;
}

int cs_slice_project(cs_handle* h, const cs_geom* g, const float* vol, const float* rot,
                     const float* defocus, int B, float* out, void* stream) {
  if (!h) return CS_ERR_ARG;
  CS_TRY(check_geom(h, g));
  CS_TRY(check_batch(h, g, B, rot, defocus));
  if (B == 0) return CS_OK;
  if (!vol || !out) return fail(h, CS_ERR_ARG, "vol or out is NULL");
  CS_SCOPE(h);
  Geo G = make_geo(*g);
  CS_CUDA(launch_slice_project(G, reinterpret_cast<const float2*>(vol), rot, defocus, B,
                               reinterpret_cast<float2*>(out),
                               pixel_grid(h->num_sms, B, g->M), S(stream)),
          "slice_project launch");
  return CS_OK;
}

int cs_backproject_adjoint(cs_handle* h, const cs_geom* g, const float* images,
                           const float* rot, const float* defocus, int B, float scale,
                           float* vol_accum, void* stream) {
  if (!h) return CS_ERR_ARG;
  CS_TRY(check_geom(h, g));
  CS_TRY(check_batch(h, g, B, rot, defocus));
  if (!is_finite(scale)) return fail(h, CS_ERR_ARG, "scale is not finite");
  if (B == 0) return CS_OK;
  if (!images || !vol_accum) return fail(h, CS_ERR_ARG, "images or vol_accum is NULL");
  CS_SCOPE(h);
  Geo G = make_geo(*g);
  cudaStream_t s = S(stream);
  if (use_vector(h, g)) {
    Workspace w;
    CS_TRY(ensure_ws(h, g->M, B, &w));
    const int grid = vec_grid(h, B, g->M, F_ADJ);
    CS_CUDA(prepare_vector(h, w, g->M, g->r_max, s), "vector pass set-up");
    CS_CUDA(launch_zero_c2(g->M, w.fw, s), "zero accumulators");
    CS_CUDA(launch_fused(F_ADJ, G, w.fw, rot, defocus, B, scale, nullptr, nullptr, nullptr,
                         reinterpret_cast<const float2*>(images), nullptr, 0, 0, nullptr, 1,
                         grid, s, h->block, h->slabs,
                         tiled_table(h, g->M)),
            "adjoint launch");
    CS_CUDA(launch_combine_c2(g->M, reinterpret_cast<const float2*>(vol_accum), 1.0f, w.fw,
                              reinterpret_cast<float2*>(vol_accum), nullptr, nullptr,
                              h->num_sms, s),
            "combine launch");
    return CS_OK;
  }
  if (!use_tiles(h)) {
    CS_CUDA(launch_backproject(G, reinterpret_cast<const float2*>(images), rot, defocus, B,
                               scale, reinterpret_cast<float2*>(vol_accum),
                               pixel_grid(h->num_sms, B, g->M), s),
            "backproject launch");
    return CS_OK;
  }
  Workspace w;
  CS_TRY(ensure_ws(h, g->M, B, &w));
  TileArgs A;
  CS_CUDA(bin_batch(h, G, w, rot, defocus, B, scale, A, s), "binning launch");
  A.img = reinterpret_cast<const float2*>(images);
  A.dst = vol_accum;
  CS_CUDA(launch_tile_op(OP_ADJOINT, A, h->num_sms, s), "adjoint tile launch");
  return CS_OK;
}

int cs_loss_grad(cs_handle* h, const cs_geom* g, const float* vol, const float* images,
                 const float* rot, const float* defocus, int B, float lambda, float scale,
                 float* grad, double* loss, void* stream) {
  if (!h) return CS_ERR_ARG;
  CS_TRY(check_geom(h, g));
  CS_TRY(check_batch(h, g, B, rot, defocus));
  if (!is_finite(lambda) || !is_finite(scale)) return fail(h, CS_ERR_ARG, "lambda/scale not finite");
  if (!vol || !grad || (B > 0 && !images))
    return fail(h, CS_ERR_ARG, "vol, grad or images is NULL");
  CS_SCOPE(h);
  Workspace w;
  CS_TRY(ensure_ws(h, g->M, B, &w));
  Geo G = make_geo(*g);
  cudaStream_t s = S(stream);
  int nvv = 0;
  if (use_vector(h, g) && B > 0) {
    const int grid = vec_grid(h, B, g->M, F_GRAD);
    CS_CUDA(prepare_vector(h, w, g->M, g->r_max, s), "vector pass set-up");
    CS_CUDA(launch_zero_c2(g->M, w.fw, s), "zero accumulators");
    CS_CUDA(launch_pairs(g->M, reinterpret_cast<const float2*>(vol), w.fw.pairs, h->num_sms, s),
            "pairs launch");
    CS_CUDA(launch_fused(F_GRAD, G, w.fw, rot, defocus, B, scale,
                         reinterpret_cast<const float2*>(vol), w.fw.pairs, nullptr,
                         reinterpret_cast<const float2*>(images), w.part, 0, 0, nullptr, 1,
                         grid, s, h->block, h->slabs,
                         tiled_table(h, g->M)),
            "loss_grad launch");
    CS_CUDA(launch_combine_c2(g->M, reinterpret_cast<const float2*>(vol), lambda, w.fw,
                              reinterpret_cast<float2*>(grad), w.part + kPartRegion, &nvv,
                              h->num_sms, s),
            "combine launch");
    if (loss)
      CS_CUDA(launch_finalize_loss(w.part, grid, nullptr, w.part + kPartRegion, nvv, lambda,
                                   scale, loss, s),
              "finalize_loss launch");
    return CS_OK;
  }
  if (!use_tiles(h) || B == 0) {
    CS_CUDA(launch_loss_grad(G, reinterpret_cast<const float2*>(vol),
                             reinterpret_cast<const float2*>(images), rot, defocus, B,
                             lambda, scale, reinterpret_cast<float2*>(grad), loss, w.part,
                             w.part + kPartRegion, &nvv, pixel_grid(h->num_sms, B, g->M),
                             h->num_sms, s),
            "loss_grad launch");
    return CS_OK;
  }
  const int n = g->M * g->M * g->M;
  CS_CUDA(launch_init_grad(n, reinterpret_cast<const float2*>(vol), lambda,
                           reinterpret_cast<float2*>(grad), w.part + kPartRegion, &nvv,
                           h->num_sms, s),
          "init_grad launch");
  TileArgs A;
  CS_CUDA(bin_batch(h, G, w, rot, defocus, B, scale, A, s), "binning launch");
  A.src = vol;
  A.img = reinterpret_cast<const float2*>(images);
  A.dst = grad;
  A.part = w.part_items;
  CS_CUDA(launch_tile_op(OP_LOSS_GRAD, A, h->num_sms, s), "loss_grad tile launch");
  if (loss)
    CS_CUDA(launch_finalize_loss(w.part_items, 0, w.item_start + A.n_tiles,
                                 w.part + kPartRegion, nvv, lambda, scale, loss, s),
            "finalize_loss launch");
  return CS_OK;
}

int cs_hvp(cs_handle* h, const cs_geom* g, const float* z, const float* rot,
           const float* defocus, int B, float lambda, float scale, float* Hz,
           void* stream) {
  if (!h) return CS_ERR_ARG;
  CS_TRY(check_geom(h, g));
  CS_TRY(check_batch(h, g, B, rot, defocus));
  if (!is_finite(lambda) || !is_finite(scale)) return fail(h, CS_ERR_ARG, "lambda/scale not finite");
  if (!z || !Hz) return fail(h, CS_ERR_ARG, "z or Hz is NULL");
  if (z == Hz) return fail(h, CS_ERR_ARG, "z and Hz must not alias");
  CS_SCOPE(h);
  Geo G = make_geo(*g);
  cudaStream_t s = S(stream);
  if (use_vector(h, g) && B > 0) {
    Workspace w;
    CS_TRY(ensure_ws(h, g->M, B, &w));
    const int grid = vec_grid(h, B, g->M, F_HVP);
    CS_CUDA(prepare_vector(h, w, g->M, g->r_max, s), "vector pass set-up");
    CS_CUDA(launch_zero_r4(g->M, w.fw, s), "zero accumulators");
    CS_CUDA(launch_fused(F_HVP, G, w.fw, rot, defocus, B, scale, nullptr, nullptr, z, nullptr,
                         nullptr, 0, 0, nullptr, 1, grid, s, h->block, h->slabs,
                         tiled_table(h, g->M)),
            "hvp launch");
    CS_CUDA(launch_combine_r4(g->M, w.fw, 0.0f, lambda, z, Hz, h->num_sms, s), "combine launch");
    return CS_OK;
  }
  if (!use_tiles(h) || B == 0) {
    CS_CUDA(launch_hvp(G, z, rot, defocus, B, lambda, scale, Hz,
                       pixel_grid(h->num_sms, B, g->M), h->num_sms, s),
            "hvp launch");
    return CS_OK;
  }
  Workspace w;
  CS_TRY(ensure_ws(h, g->M, B, &w));
  CS_CUDA(launch_scale_copy(g->M * g->M * g->M, z, lambda, Hz, h->num_sms, s),
          "scale_copy launch");
  TileArgs A;
  CS_CUDA(bin_batch(h, G, w, rot, defocus, B, scale, A, s), "binning launch");
  A.src = z;
  A.dst = Hz;
  CS_CUDA(launch_tile_op(OP_HVP, A, h->num_sms, s), "hvp tile launch");
  return CS_OK;
}

}  // extern "C"

namespace {

// Enqueues one Hutchinson estimate of a validated batch into `out`
// (workspace already sized for M and B).
int hutch_enqueue(cs_handle* h, const cs_geom* g, const Workspace& w, const float* rot,
                  const float* defocus, int B, float lambda, float scale, int n_probes,
                  uint64_t seed, uint64_t probe_block, float* out, cudaStream_t s) {
  Geo G = make_geo(*g);
  if (use_vector(h, g) && B > 0) {
    const int grid = vec_grid(h, B, g->M, F_HUTCH);
    CS_CUDA(prepare_vector(h, w, g->M, g->r_max, s), "vector pass set-up");
    CS_CUDA(launch_zero_r4(g->M, w.fw, s), "zero accumulators");
    CS_CUDA(launch_fused(F_HUTCH, G, w.fw, rot, defocus, B, scale, nullptr, nullptr, nullptr,
                         nullptr, nullptr, seed, probe_block, nullptr, n_probes, grid, s, h->block,
                         h->slabs, tiled_table(h, g->M)),
            "hutchinson launch");
    CS_CUDA(launch_combine_r4(g->M, w.fw, lambda, 0.0f, nullptr, out, h->num_sms, s),
            "combine launch");
    return CS_OK;
  }
  if (g->interp == CS_TRILINEAR)
    CS_CUDA(launch_probe_bits(g->M, seed, probe_block, nullptr, w.bits, h->num_sms, s),
            "probe_bits launch");
  if (!use_tiles(h) || B == 0) {
    CS_CUDA(launch_hutchinson(G, w.bits, rot, defocus, B, lambda, scale, n_probes, out,
                              pixel_grid(h->num_sms, B, g->M), h->num_sms, s),
            "hutchinson launch");
    return CS_OK;
  }
  CS_CUDA(launch_fill(g->M * g->M * g->M, lambda, out, h->num_sms, s), "fill launch");
  TileArgs A;
  CS_CUDA(bin_batch(h, G, w, rot, defocus, B, scale, A, s), "binning launch");
  A.src = w.bits;
  A.dst = out;
  A.K = n_probes;
  CS_CUDA(launch_tile_op(OP_HUTCH, A, h->num_sms, s), "hutchinson tile launch");
  return CS_OK;
}

}  // namespace

extern "C" {

int cs_hutchinson_diag(cs_handle* h, const cs_geom* g, const float* rot,
                       const float* defocus, int B, float lambda, float scale,
                       int n_probes, uint64_t seed, uint64_t probe_block, float* diag_out,
                       void* stream) {
  if (!h) return CS_ERR_ARG;
  CS_TRY(check_geom(h, g));
  CS_TRY(check_batch(h, g, B, rot, defocus));
  if (!is_finite(lambda) || !is_finite(scale)) return fail(h, CS_ERR_ARG, "lambda/scale not finite");
  if (n_probes < 1 || n_probes > 32)
    return fail(h, CS_ERR_SHAPE, "n_probes=%d must be in [1, 32]", n_probes);
  if (!diag_out) return fail(h, CS_ERR_ARG, "diag_out is NULL");
  CS_SCOPE(h);
  Workspace w;
  CS_TRY(ensure_ws(h, g->M, B, &w));
  return hutch_enqueue(h, g, w, rot, defocus, B, lambda, scale, n_probes, seed, probe_block,
                       diag_out, S(stream));
}

int cs_precompute_preconditioner(cs_handle* h, const cs_geom* g, const float* rot_all,
                                 const float* defocus_all, int N, int B, int n_epochs,
                                 float lambda, int n_probes, uint64_t seed, float* D_out,
                                 void* stream) {
  if (!h) return CS_ERR_ARG;
  CS_TRY(check_geom(h, g));
  if (N < 1 || B < 1 || n_epochs < 1)
    return fail(h, CS_ERR_SHAPE, "N=%d, B=%d and n_epochs=%d must be positive", N, B, n_epochs);
  CS_TRY(check_batch(h, g, B, rot_all, defocus_all));
  if (!is_finite(lambda)) return fail(h, CS_ERR_ARG, "lambda not finite");
  if (n_probes < 1 || n_probes > 32)
    return fail(h, CS_ERR_SHAPE, "n_probes=%d must be in [1, 32]", n_probes);
  if (!D_out) return fail(h, CS_ERR_ARG, "D_out is NULL");
  const long n_batches = ((long)N + B - 1) / B;
  if (n_batches * n_epochs > 0x7fffffffL)
    return fail(h, CS_ERR_SHAPE, "n_epochs=%d too large for %ld batches", n_epochs, n_batches);
  CS_SCOPE(h);
  Workspace w;
  CS_TRY(ensure_ws(h, g->M, B, &w));
  cudaStream_t s = S(stream);
  const int n = g->M * g->M * g->M;
  long k = 0;
  for (int e = 0; e < n_epochs; ++e)
    for (long b = 0; b < n_batches; ++b) {
      ++k;
      const int Bb = (int)std::min<long>(B, N - b * B);
      const float scale = (float)((double)N / Bb);
      CS_TRY(hutch_enqueue(h, g, w, rot_all + 9 * b * B,
                           defocus_all ? defocus_all + b * B : nullptr, Bb, lambda, scale,
                           n_probes, seed, (uint64_t)k, w.dest, s));
      CS_CUDA(launch_running_mean(n, w.dest, D_out, k, h->num_sms, s),
              "running-mean launch");
    }
  return CS_OK;
}

int cs_exact_diag(cs_handle* h, const cs_geom* g, const float* rot, const float* defocus,
                  int B, float lambda, float scale, float* diag_out, float* coverage_out,
                  float* ctf2w_out, void* stream) {
  if (!h) return CS_ERR_ARG;
  CS_TRY(check_geom(h, g));
  CS_TRY(check_batch(h, g, B, rot, defocus));
  if (!is_finite(lambda) || !is_finite(scale)) return fail(h, CS_ERR_ARG, "lambda/scale not finite");
  if (!diag_out && !coverage_out && !ctf2w_out) return CS_OK;
  CS_SCOPE(h);
  Geo G = make_geo(*g);
  CS_CUDA(launch_exact_diag(G, rot, defocus, B, lambda, scale, diag_out, coverage_out,
                            ctf2w_out, pixel_grid(h->num_sms, B, g->M), h->num_sms,
                            S(stream)),
          "exact_diag launch");
  return CS_OK;
}

int cs_threshold_alpha(cs_handle* h, const cs_geom* g, const float* defocus_all, int N,
                       double lambda, double scale_alpha, double* alpha_out,
                       void* stream) {
  if (!h) return CS_ERR_ARG;
  CS_TRY(check_geom(h, g));
  if (N < 0) return fail(h, CS_ERR_SHAPE, "N=%d is negative", N);
  if (!alpha_out) return fail(h, CS_ERR_ARG, "alpha_out is NULL");
  if (N > 0 && g->ctf.enabled && !defocus_all)
    return fail(h, CS_ERR_ARG, "defocus_all is NULL but the CTF is enabled");
  if (!is_finite(lambda) || !is_finite(scale_alpha))
    return fail(h, CS_ERR_ARG, "lambda/scale_alpha not finite");
  // 1-voxel shells round(|k|) = R: R^2 - R + 1 <= |k|^2 <= R^2 + R
  const long R = g->r_max, lo = R * R - R + 1, hi = R * R + R;
  const int M = g->M, half = M / 2;
  long px = 0, pv = 0;
  for (int y = -half; y < half; ++y)
    for (int x = -half; x < half; ++x) {
      const long q2 = (long)x * x + (long)y * y;
      if (q2 >= lo && q2 <= hi) ++px;
      if (q2 > hi) continue;
      for (int z = -half; z < half; ++z) {
        const long q3 = q2 + (long)z * z;
        if (q3 >= lo && q3 <= hi) ++pv;
      }
    }
  if (pv == 0) return fail(h, CS_ERR_INTERNAL, "empty 3-D shell at R=%ld", R);
  CS_SCOPE(h);
  Geo G = make_geo(*g);
  CS_CUDA(launch_alpha(G, defocus_all, N, (double)px / (double)pv, lambda, scale_alpha,
                       alpha_out, S(stream)),
          "alpha launch");
  return CS_OK;
}

// One Algorithm-1 step; img_rows != NULL: images disc-packed with those
// row starts (vector traversal only)
static int precond_step_impl(cs_handle* h, const cs_geom* g, cs_sgd_state* st,
                             const float* images, const float* rot, const float* defocus,
                             int B, float lambda, float scale, void* stream,
                             const int* img_rows) {
  if (!h) return CS_ERR_ARG;
  CS_TRY(check_geom(h, g));
  CS_TRY(check_batch(h, g, B, rot, defocus));
  if (!st) return fail(h, CS_ERR_ARG, "state is NULL");
  if (!is_finite(lambda) || !is_finite(scale)) return fail(h, CS_ERR_ARG, "lambda/scale not finite");
  if (!st->v || !st->scalars || (B > 0 && !images))
    return fail(h, CS_ERR_ARG, "state.v, state.scalars or images is NULL");
  if (st->mode != CS_PLAIN && st->mode != CS_HUTCHINSON && st->mode != CS_FIXED)
    return fail(h, CS_ERR_ARG, "mode=%d is not a cs_sgd_mode", st->mode);
  if (st->mode != CS_PLAIN && !st->D) return fail(h, CS_ERR_ARG, "state.D is NULL");
  if (st->mode == CS_HUTCHINSON) {
    if (!st->D_avg) return fail(h, CS_ERR_ARG, "state.D_avg is NULL");
    if (st->n_probes < 1 || st->n_probes > 32)
      return fail(h, CS_ERR_SHAPE, "n_probes=%d must be in [1, 32]", st->n_probes);
    if (!(st->beta > 0.f && st->beta < 1.f))
      return fail(h, CS_ERR_ARG, "beta=%g must be in (0, 1)", (double)st->beta);
  }
  if (!(st->c > 0.f && st->c < 1.f)) return fail(h, CS_ERR_ARG, "c=%g must be in (0, 1)", (double)st->c);
  if (st->max_halvings < 0) return fail(h, CS_ERR_ARG, "max_halvings is negative");
  CS_SCOPE(h);
  Workspace w;
  CS_TRY(ensure_ws(h, g->M, B, &w));
  const Geo G = make_geo(*g);
  const int n = g->M * g->M * g->M;
  const int grid = pixel_grid(h->num_sms, B, g->M);
  cudaStream_t s = S(stream);
  double* pL = w.part;                   // data-term partials
  double* pV = w.part + kPartRegion;     // |v|^2 partials
  double* pD = w.part + 2 * kPartRegion; // direction partials (G, |d|^2)
  double* pQ = w.part + 3 * kPartRegion; // curvature partials
  const float* dhat = nullptr;
  if (use_vector(h, g) && B > 0) {
    // one traversal computes loss, gradient and (Hutchinson) the estimate
    const bool hutch = st->mode == CS_HUTCHINSON;
    const int vgrid = vec_grid(h, B, g->M, hutch ? (F_GRAD | F_HUTCH) : F_GRAD);
    const int cgrid = vec_grid(h, B, g->M, F_CURV);
    int nvv = 0, nd = 0;
    prof_mark(h, 0, s);
    CS_CUDA(prepare_vector(h, w, g->M, g->r_max, s), "vector pass set-up");
    CS_CUDA(launch_step_prep(g->M, reinterpret_cast<const float2*>(st->v), w.fw, hutch,
                             h->num_sms, s),
            "step set-up launch");
    prof_mark(h, CS_PH_LOSS_GRAD, s);
    CS_CUDA(launch_fused(hutch ? (F_GRAD | F_HUTCH) : F_GRAD, G, w.fw, rot, defocus, B, scale,
                         reinterpret_cast<const float2*>(st->v), w.fw.pairs, nullptr,
                         reinterpret_cast<const float2*>(images), pL, st->seed, 0,
                         st->scalars + CS_S_K, st->n_probes, vgrid, s, h->block, h->slabs,
                         tiled_table(h, g->M), img_rows, g->r_max),
            "fused loss_grad launch");
    prof_mark(h, CS_PH_DIRECTION, s);
    CS_CUDA(launch_step_post(g->M, st->mode, reinterpret_cast<const float2*>(st->v), lambda,
                             st->beta, st->scalars, w.fw, st->D, st->D_avg, pD, pV, &nd,
                             h->num_sms, s),
            "step_post launch");
    CS_CUDA(launch_patches(g->M, w.fw, h->num_sms, s), "patch layout launch");
    nvv = nd;
    prof_mark(h, CS_PH_CURVATURE, s);
    CS_CUDA(launch_fused(F_CURV, G, w.fw, rot, defocus, B, scale, w.d, w.fw.pairs, nullptr,
                         nullptr, pQ, 0, 0, nullptr, 1, cgrid, s, h->block, h->slabs,
                         tiled_table(h, g->M)),
            "curvature launch");
    prof_mark(h, CS_PH_UPDATE, s);
    CS_CUDA(launch_eta(st->scalars, pL, vgrid, pV, nvv, pD, pD + nd, nd, pQ, cgrid, nullptr,
                       lambda, scale, st->c, st->max_halvings, s),
            "eta launch");
    CS_CUDA(launch_update_pairs(g->M, reinterpret_cast<float2*>(st->v), w.fw, st->scalars,
                                h->num_sms, s),
            "update launch");
    prof_mark(h, CS_NPHASES, s);
    return CS_OK;
  }
  if (img_rows && B > 0)
    return fail(h, CS_ERR_INTERNAL, "disc-packed images need the vector traversal");
  const bool tiles = use_tiles(h) && B > 0;
  TileArgs A;
  prof_mark(h, 0, s);
  if (tiles) CS_CUDA(bin_batch(h, G, w, rot, defocus, B, scale, A, s), "binning launch");
  if (st->mode == CS_HUTCHINSON) {
    if (g->interp == CS_TRILINEAR)
      CS_CUDA(launch_probe_bits(g->M, st->seed, 0, st->scalars + CS_S_K, w.bits, h->num_sms, s),
              "probe_bits launch");
    if (tiles) {
      CS_CUDA(launch_fill(n, lambda, w.dest, h->num_sms, s), "fill launch");
      TileArgs T = A;
      T.src = w.bits;
      T.dst = w.dest;
      T.K = st->n_probes;
      CS_CUDA(launch_tile_op(OP_HUTCH, T, h->num_sms, s), "hutchinson tile launch");
    } else {
      CS_CUDA(launch_hutchinson(G, w.bits, rot, defocus, B, lambda, scale, st->n_probes,
                                w.dest, grid, h->num_sms, s),
              "hutchinson launch");
    }
    CS_CUDA(launch_precond_update(n, w.dest, st->D, st->D_avg, w.dhat, st->scalars,
                                  st->beta, h->num_sms, s),
            "precond_update launch");
    dhat = w.dhat;
  } else if (st->mode == CS_FIXED) {
    CS_CUDA(launch_fixed_dhat(n, st->D, w.dhat, st->scalars, h->num_sms, s),
            "fixed_dhat launch");
    dhat = w.dhat;
  }
  int nvv = 0, nd = 0;
  prof_mark(h, CS_PH_LOSS_GRAD, s);
  if (tiles) {
    CS_CUDA(launch_init_grad(n, reinterpret_cast<const float2*>(st->v), lambda, w.g, pV, &nvv,
                             h->num_sms, s),
            "init_grad launch");
    TileArgs T = A;
    T.src = st->v;
    T.img = reinterpret_cast<const float2*>(images);
    T.dst = w.g;
    T.part = w.part_items;
    CS_CUDA(launch_tile_op(OP_LOSS_GRAD, T, h->num_sms, s), "loss_grad tile launch");
  } else {
    CS_CUDA(launch_loss_grad(G, reinterpret_cast<const float2*>(st->v),
                             reinterpret_cast<const float2*>(images), rot, defocus, B, lambda,
                             scale, w.g, nullptr, pL, pV, &nvv, grid, h->num_sms, s),
            "loss_grad launch");
  }
  prof_mark(h, CS_PH_DIRECTION, s);
  CS_CUDA(launch_direction(n, w.g, dhat, w.d, pD, &nd, h->num_sms, s), "direction launch");
  prof_mark(h, CS_PH_CURVATURE, s);
  if (tiles) {
    TileArgs T = A;
    T.src = w.d;
    T.part = w.part_items2;
    CS_CUDA(launch_tile_op(OP_CURVATURE, T, h->num_sms, s), "curvature tile launch");
  } else if (B > 0) {
    CS_CUDA(launch_curvature(G, w.d, rot, defocus, B, pQ, grid, s), "curvature launch");
  }
  prof_mark(h, CS_PH_UPDATE, s);
  if (tiles)
    CS_CUDA(launch_eta(st->scalars, w.part_items, 0, pV, nvv, pD, pD + nd, nd, w.part_items2, 0,
                       w.item_start + A.n_tiles, lambda, scale, st->c, st->max_halvings, s),
            "eta launch");
  else
    CS_CUDA(launch_eta(st->scalars, pL, B > 0 ? grid : 0, pV, nvv, pD, pD + nd, nd, pQ,
                       B > 0 ? grid : 0, nullptr, lambda, scale, st->c, st->max_halvings, s),
            "eta launch");
  CS_CUDA(launch_update(n, reinterpret_cast<float2*>(st->v), w.d, st->scalars, h->num_sms, s),
          "update launch");
  prof_mark(h, CS_NPHASES, s);
  return CS_OK;
}

int cs_precond_sgd_step(cs_handle* h, const cs_geom* g, cs_sgd_state* st,
                        const float* images, const float* rot, const float* defocus, int B,
                        float lambda, float scale, void* stream) {
  return precond_step_impl(h, g, st, images, rot, defocus, B, lambda, scale, stream, nullptr);
}

int cs_profile_enable(cs_handle* h, int enable, int max_steps) {
  if (!h) return CS_ERR_ARG;
  if (enable && max_steps < 1) return fail(h, CS_ERR_ARG, "max_steps=%d must be >= 1", max_steps);
  CS_SCOPE(h);
  if (!enable) {
    h->prof = false;
    return CS_OK;
  }
  CS_CUDA(cudaDeviceSynchronize(), "profile_enable");
  prof_free(h);
  const size_t n = (size_t)max_steps * (CS_NPHASES + 1);
  h->prof_events.reserve(n);
  for (size_t i = 0; i < n; ++i) {
    cudaEvent_t e;
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) {
      prof_free(h);
      return cuda_fail(h, err, "cudaEventCreate");
    }
    h->prof_events.push_back(e);
  }
  h->prof_max_steps = max_steps;
  h->prof_steps = 0;
  h->prof = true;
  return CS_OK;
}

int cs_profile_read(cs_handle* h, double* ms, int* counts) {
  if (!h) return CS_ERR_ARG;
  if (!ms || !counts) return fail(h, CS_ERR_ARG, "ms or counts is NULL");
  CS_SCOPE(h);
  for (int p = 0; p < CS_NPHASES; ++p) {
    ms[p] = 0.0;
    counts[p] = 0;
  }
  for (int st = 0; st < h->prof_steps; ++st) {
    const cudaEvent_t* e = &h->prof_events[(size_t)st * (CS_NPHASES + 1)];
    CS_CUDA(cudaEventSynchronize(e[CS_NPHASES]), "cudaEventSynchronize");
    for (int p = 0; p < CS_NPHASES; ++p) {
      float t = 0.f;
      CS_CUDA(cudaEventElapsedTime(&t, e[p], e[p + 1]), "cudaEventElapsedTime");
      ms[p] += t;
      counts[p] += 1;
    }
  }
  return CS_OK;
}

uint64_t cs_kernel_launches(void) { return g_launches.load(); }

int cs_measure_reduction_rate(cs_handle* h, double* gops) {
  if (!h) return CS_ERR_ARG;
  if (!gops) return fail(h, CS_ERR_ARG, "gops is NULL");
  CS_SCOPE(h);
  const size_t bytes = (size_t)16 << 20;
  void* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, CS_ERR_ALLOC, "calibration buffer: %s", cudaGetErrorString(e));
  }
  e = measure_red_rate(buf, bytes, h->num_sms, nullptr, gops);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_fail(h, e, "reduction-rate calibration");
  return CS_OK;
}

}  // extern "C"

// ----------------------------------------------------------- multi-volume

namespace {

constexpr int kMultiParts = 4 * kPartRegion;   // partial slots per problem

struct ProblemWs {
  FusedWs fw;
  float* rot;       // [B][9]
  double* part;     // kMultiParts doubles: loss | |v|^2 | (G, |d|^2) | Q
};

size_t problem_ws_bytes(int M, int B) {
  return align256(fused_ws_bytes(M)) + align256((size_t)B * 9 * sizeof(float)) +
         align256((size_t)kMultiParts * sizeof(double)) + align256(slab_lists_bytes(M, B));
}

int check_problems(cs_handle* h, const cs_problem* P, int n) {
  if (!P) return fail(h, CS_ERR_ARG, "problems pointer is NULL");
  if (n < 1 || n > CS_MAX_PROBLEMS)
    return fail(h, CS_ERR_SHAPE, "n=%d problems must be in [1, %d]", n, CS_MAX_PROBLEMS);
  for (int p = 0; p < n; ++p) {
    const cs_problem& q = P[p];
    CS_TRY(check_geom(h, &q.geom));
    if (q.geom.interp != CS_TRILINEAR)
      return fail(h, CS_ERR_ARG, "problem %d: the multi-volume step needs trilinear interpolation", p);
    if (q.B < 1 || q.n_batches < 1)
      return fail(h, CS_ERR_SHAPE, "problem %d: B=%d and n_batches=%d must be >= 1", p, q.B, q.n_batches);
    const long nch = ((long)q.geom.M * q.geom.M + 127) / 128;
    if ((long)q.B * nch > 0x7fffffffL || (long)q.B * q.n_batches > 0x7fffffffL)
      return fail(h, CS_ERR_SHAPE, "problem %d: batch too large", p);
    if (!q.images || !q.quat || (q.geom.ctf.enabled && !q.defocus))
      return fail(h, CS_ERR_ARG, "problem %d: images, quat or defocus is NULL", p);
    const cs_sgd_state& st = q.state;
    if (!st.v || !st.scalars) return fail(h, CS_ERR_ARG, "problem %d: state.v or scalars is NULL", p);
    if (st.mode != P[0].state.mode)
      return fail(h, CS_ERR_ARG, "problem %d: all problems must share the SGD mode", p);
    if (st.mode != CS_PLAIN && st.mode != CS_HUTCHINSON && st.mode != CS_FIXED)
      return fail(h, CS_ERR_ARG, "problem %d: mode=%d is not a cs_sgd_mode", p, st.mode);
    if (st.mode != CS_PLAIN && !st.D) return fail(h, CS_ERR_ARG, "problem %d: state.D is NULL", p);
    if (st.mode == CS_HUTCHINSON &&
        (!st.D_avg || st.n_probes < 1 || st.n_probes > 32 || !(st.beta > 0.f && st.beta < 1.f)))
      return fail(h, CS_ERR_ARG, "problem %d: Hutchinson state (D_avg, n_probes, beta) invalid", p);
    if (!(st.c > 0.f && st.c < 1.f) || st.max_halvings < 0)
      return fail(h, CS_ERR_ARG, "problem %d: c or max_halvings invalid", p);
    if (!is_finite(q.lambda) || !is_finite(q.scale))
      return fail(h, CS_ERR_ARG, "problem %d: lambda/scale not finite", p);
  }
  return CS_OK;
}

int ensure_mws(cs_handle* h, const cs_problem* P, int n, ProblemWs* W) {
  size_t need = 0;
  for (int p = 0; p < n; ++p) need += problem_ws_bytes(P[p].geom.M, P[p].B);
  if (h->mws_bytes < need) {
    if (h->mws) {
      cudaError_t e = cudaDeviceSynchronize();
      if (e != cudaSuccess) return cuda_fail(h, e, "synchronise before workspace growth");
      cudaFree(h->mws);
      h->mws = nullptr;
      h->mws_bytes = 0;
    }
    void* ptr = nullptr;
    cudaError_t e = cudaMalloc(&ptr, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(h, CS_ERR_ALLOC, "multi-volume workspace of %zu bytes: %s", need,
                  cudaGetErrorString(e));
    }
    h->mws = ptr;
    h->mws_bytes = need;
    ++h->mws_generation;
    for (int i = 0; i < 8; ++i) h->mtable_key[i] = -1;
  }
  char* c = static_cast<char*>(h->mws);
  for (int p = 0; p < n; ++p) {
    const int M = P[p].geom.M;
    W[p].fw = fused_carve(c, M);                c += align256(fused_ws_bytes(M));
    W[p].rot = reinterpret_cast<float*>(c);     c += align256((size_t)P[p].B * 9 * sizeof(float));
    W[p].part = reinterpret_cast<double*>(c);   c += align256((size_t)kMultiParts * sizeof(double));
    // per-slab item lists (problems whose traversals are split into z-slabs)
    slab_carve(c, M, P[p].B, W[p].fw);
    c += align256(slab_lists_bytes(M, P[p].B));
  }
  return CS_OK;
}

long disc_pixels(int M, int r) {
  long n = 0;
  for (int y = -r; y <= r; ++y) {
    int xr = (int)std::floor(std::sqrt((double)(r * r - y * y)));
    n += 2 * xr + 1;
  }
  (void)M;
  return n;
}

// blocks of the multi-volume traversal, split in proportion to each
// problem's pixel count
void split_blocks(const cs_handle* h, const cs_problem* P, int n, int* start, int* total,
                  int block) {
  (void)block;
  const int G = h->num_sms * h->blocks_per_sm;
  double work[CS_MAX_PROBLEMS], sum = 0;
  for (int p = 0; p < n; ++p) {
    work[p] = (double)P[p].B * (double)disc_pixels(P[p].geom.M, P[p].geom.r_max);
    sum += work[p];
  }
  int acc = 0;
  start[0] = 0;
  for (int p = 0; p < n; ++p) {
    int b = (int)std::lround(G * work[p] / sum);
    if (b < 1) b = 1;
    acc += b;
    start[p + 1] = acc;
  }
  *total = acc;
}

cudaError_t prepare_tables(cs_handle* h, const cs_problem* P, int n, const ProblemWs* W,
                           cudaStream_t s) {
  for (int p = 0; p < n; ++p) {
    const int M = P[p].geom.M, r = P[p].geom.r_max;
    const bool tiled = tiled_table(h, M);
    const int key = ((tiled ? 1 + (h->block == 128) : 0) << 28) | (M << 12) | r;
    if (h->mtable_key[p] != key) {
      cudaError_t e = tiled ? launch_disc_table_tiled(M, r, h->block, W[p].fw, s)
                            : launch_disc_table(M, r, W[p].fw, s);
      if (e != cudaSuccess) return e;
      // a graph captured with the previous table layout must not replay
      if (h->mtable_key[p] != -1) ++h->mws_generation;
      h->mtable_key[p] = key;
    }
  }
  return cudaSuccess;
}

FusedArgs problem_args(const cs_problem& q, const ProblemWs& w, const Geo& G) {
  FusedArgs A{};
  A.G = G;
  A.table = w.fw.table;
  A.n_px_dev = w.fw.n_px;
  A.rot = w.rot;
  A.df = q.defocus;
  A.B = q.B;
  A.scale = q.scale;
  A.vol = reinterpret_cast<const float2*>(q.state.v);
  A.img = reinterpret_cast<const float2*>(q.images);
  A.img_rows = nullptr;
  A.img_r = 0;
  A.E = w.fw.E;
  A.O = w.fw.O;
  A.P = w.fw.P;
  A.K = q.state.n_probes;
  A.vp = w.fw.pairs;
  A.dq = w.fw.dq;
  A.seed = q.state.seed;
  A.k_dev = q.state.scalars + CS_S_K;
  A.cursor = q.state.scalars + CS_S_K;
  A.n_batches = q.n_batches;
  A.part_add = 0;
  return A;
}

// Everything of one multi-volume step, enqueued on s (no allocation, no
// host synchronisation: capturable).  Problems whose grid is split into
// z-slabs (tiled_table) run their traversals as their own slab launches;
// the others share one launch of the multi-volume kernel.
int multi_step_enqueue(cs_handle* h, const cs_problem* P, int n, const ProblemWs* W,
                       cudaStream_t s) {
  const bool hutch = P[0].state.mode == CS_HUTCHINSON;
  const int fl = hutch ? (F_GRAD | F_HUTCH) : F_GRAD;
  bool big[CS_MAX_PROBLEMS];
  int small_idx[CS_MAX_PROBLEMS], n_small = 0;
  cs_problem small[CS_MAX_PROBLEMS];
  for (int p = 0; p < n; ++p) {
    big[p] = tiled_table(h, P[p].geom.M);
    if (!big[p]) {
      small_idx[n_small] = p;
      small[n_small++] = P[p];
    }
  }
  MultiFusedArgs MA{};
  MA.n = n_small;
  int total = 0;
  if (n_small > 0) split_blocks(h, small, n_small, MA.start, &total, h->block);
  FusedArgs BA[CS_MAX_PROBLEMS];
  int nL[CS_MAX_PROBLEMS], nQ[CS_MAX_PROBLEMS];
  for (int p = 0; p < n; ++p) {
    const cs_problem& q = P[p];
    const int M = q.geom.M;
    CS_CUDA(launch_quat_to_rot_cursor(q.quat, q.B, q.n_batches, q.state.scalars + CS_S_K,
                                      W[p].rot, s),
            "quat_to_rot launch");
    CS_CUDA(launch_step_prep(M, reinterpret_cast<const float2*>(q.state.v), W[p].fw, hutch,
                             h->num_sms, s),
            "step set-up launch");
    BA[p] = problem_args(q, W[p], make_geo(q.geom));
    BA[p].part = W[p].part;                     // loss partials
  }
  for (int i = 0; i < n_small; ++i) {
    MA.a[i] = BA[small_idx[i]];
    nL[small_idx[i]] = nQ[small_idx[i]] = MA.start[i + 1] - MA.start[i];
  }
  if (n_small > 0)
    CS_CUDA(launch_fused_multi(fl, MA, total, h->block, s), "multi-volume traversal launch");
  for (int p = 0; p < n; ++p) {
    if (!big[p]) continue;
    nL[p] = vec_grid(h, P[p].B, P[p].geom.M, fl);
    CS_CUDA(launch_fused_args(fl, BA[p], W[p].fw, nL[p], s, h->block, h->slabs, true),
            "slab traversal launch");
  }
  int nd[CS_MAX_PROBLEMS];
  for (int p = 0; p < n; ++p) {
    const cs_problem& q = P[p];
    CS_CUDA(launch_step_post(q.geom.M, q.state.mode, reinterpret_cast<const float2*>(q.state.v),
                             q.lambda, q.state.beta, q.state.scalars, W[p].fw, q.state.D,
                             q.state.D_avg, W[p].part + 2 * kPartRegion, W[p].part + kPartRegion,
                             &nd[p], h->num_sms, s),
            "step_post launch");
    CS_CUDA(launch_patches(q.geom.M, W[p].fw, h->num_sms, s), "patch layout launch");
    BA[p].img = nullptr;
    BA[p].part = W[p].part + 3 * kPartRegion;   // curvature partials
  }
  for (int i = 0; i < n_small; ++i) MA.a[i] = BA[small_idx[i]];
  if (n_small > 0)
    CS_CUDA(launch_fused_multi(F_CURV, MA, total, h->block, s), "multi-volume curvature launch");
  for (int p = 0; p < n; ++p) {
    if (!big[p]) continue;
    nQ[p] = vec_grid(h, P[p].B, P[p].geom.M, F_CURV);
    CS_CUDA(launch_fused_args(F_CURV, BA[p], W[p].fw, nQ[p], s, h->block, h->slabs, true),
            "slab curvature launch");
  }
  for (int p = 0; p < n; ++p) {
    const cs_problem& q = P[p];
    double* pD = W[p].part + 2 * kPartRegion;
    CS_CUDA(launch_eta(q.state.scalars, W[p].part, nL[p], W[p].part + kPartRegion, nd[p], pD,
                       pD + nd[p], nd[p], W[p].part + 3 * kPartRegion, nQ[p], nullptr, q.lambda,
                       q.scale, q.state.c, q.state.max_halvings, s),
            "eta launch");
    CS_CUDA(launch_update_pairs(q.geom.M, reinterpret_cast<float2*>(q.state.v), W[p].fw,
                                q.state.scalars, h->num_sms, s),
            "update launch");
  }
  return CS_OK;
}

}  // namespace

struct cs_graph {
  cs_handle* h = nullptr;
  int device = 0;
  int generation = 0;
  uint64_t n_kernels = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

extern "C" {

int cs_multi_step(cs_handle* h, const cs_problem* probs, int n, void* stream) {
  if (!h) return CS_ERR_ARG;
  CS_TRY(check_problems(h, probs, n));
  CS_SCOPE(h);
  ProblemWs W[CS_MAX_PROBLEMS];
  CS_TRY(ensure_mws(h, probs, n, W));
  cudaStream_t s = S(stream);
  CS_CUDA(prepare_tables(h, probs, n, W, s), "pixel table launch");
  return multi_step_enqueue(h, probs, n, W, s);
}

int cs_multi_step_graph(cs_handle* h, const cs_problem* probs, int n, cs_graph** out) {
  if (!h || !out) return CS_ERR_ARG;
  *out = nullptr;
  CS_TRY(check_problems(h, probs, n));
  CS_SCOPE(h);
  ProblemWs W[CS_MAX_PROBLEMS];
  CS_TRY(ensure_mws(h, probs, n, W));
  cudaStream_t cs_stream = nullptr;
  CS_CUDA(cudaStreamCreateWithFlags(&cs_stream, cudaStreamNonBlocking), "cudaStreamCreate");
  cudaError_t e = prepare_tables(h, probs, n, W, cs_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs_stream);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs_stream);
    return cuda_fail(h, e, "pixel tables before capture");
  }
  cs_graph* g = new (std::nothrow) cs_graph();
  if (!g) {
    cudaStreamDestroy(cs_stream);
    return fail(h, CS_ERR_ALLOC, "graph object");
  }
  const uint64_t l0 = g_launches.load();
  e = cudaStreamBeginCapture(cs_stream, cudaStreamCaptureModeThreadLocal);
  int rc = CS_OK;
  if (e == cudaSuccess) rc = multi_step_enqueue(h, probs, n, W, cs_stream);
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(cs_stream, &graph) : e;
  const uint64_t captured = g_launches.load() - l0;
  g_launches.fetch_sub(captured);   // captured, not executed
  cudaStreamDestroy(cs_stream);
  if (rc != CS_OK || e != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    delete g;
    if (rc != CS_OK) return rc;
    return cuda_fail(h, e != cudaSuccess ? e : e2, "stream capture");
  }
  e = cudaGraphInstantiate(&g->exec, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    delete g;
    return cuda_fail(h, e, "cudaGraphInstantiate");
  }
  g->graph = graph;
  g->h = h;
  g->device = h->device;
  g->generation = h->mws_generation;
  g->n_kernels = captured;
  *out = g;
  return CS_OK;
}

int cs_graph_launch(cs_graph* g, void* stream) {
  if (!g || !g->exec) return CS_ERR_ARG;
  cs_handle* h = g->h;
  if (g->generation != h->mws_generation)
    return fail(h, CS_ERR_ARG, "the handle's multi-volume workspace changed since the capture");
  CS_SCOPE(h);
  CS_CUDA(cudaGraphLaunch(g->exec, S(stream)), "cudaGraphLaunch");
  count_launches((int)g->n_kernels);
  return CS_OK;
}

int cs_graph_destroy(cs_graph* g) {
  if (!g) return CS_OK;
  {
    DeviceScope scope(g->device);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
  }
  delete g;
  return CS_OK;
}

int cs_set_slabs(cs_handle* h, int slabs) {
  if (!h) return CS_ERR_ARG;
  if (slabs < 0 || slabs > 16) return fail(h, CS_ERR_ARG, "slabs=%d must be in [0, 16]", slabs);
  h->slabs = slabs;
  return CS_OK;
}

int cs_set_host_mode(cs_handle* h, int mode) {
  if (!h) return CS_ERR_ARG;
  if (mode != CS_HOST_STAGED && mode != CS_HOST_DIRECT)
    return fail(h, CS_ERR_ARG, "host mode %d is not CS_HOST_STAGED or CS_HOST_DIRECT", mode);
  h->host_mode = mode;
  return CS_OK;
}

int cs_set_launch_shape(cs_handle* h, int block, int bps) {
  if (!h) return CS_ERR_ARG;
  if (block != 128 && block != 256)
    return fail(h, CS_ERR_ARG, "block_threads=%d must be 128 or 256", block);
  if (bps < 1 || bps > (block == 256 ? 32 : 64))
    return fail(h, CS_ERR_ARG, "blocks_per_sm=%d out of range", bps);
  h->block = block;
  h->blocks_per_sm = bps;
  return CS_OK;
}

int cs_autotune(cs_handle* h, const cs_problem* probs, int n, int* block_out, int* bps_out) {
  if (!h) return CS_ERR_ARG;
  CS_TRY(check_problems(h, probs, n));
  CS_SCOPE(h);
  ProblemWs W[CS_MAX_PROBLEMS];
  CS_TRY(ensure_mws(h, probs, n, W));
  cudaStream_t s = nullptr;
  CS_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "cudaStreamCreate");
  const bool hutch = probs[0].state.mode == CS_HUTCHINSON;
  cudaError_t e = prepare_tables(h, probs, n, W, s);
  // the shape of the shared multi-volume launch is tuned on the problems it
  // carries (those not split into z-slabs)
  cs_problem small[CS_MAX_PROBLEMS];
  int n_small = 0;
  MultiFusedArgs MA{};
  for (int p = 0; p < n && e == cudaSuccess; ++p) {
    const cs_problem& q = probs[p];
    if (tiled_table(h, q.geom.M)) continue;
    e = launch_quat_to_rot_cursor(q.quat, q.B, q.n_batches, q.state.scalars + CS_S_K, W[p].rot, s);
    if (e == cudaSuccess) e = launch_pairs(q.geom.M, reinterpret_cast<const float2*>(q.state.v),
                                           W[p].fw.pairs, h->num_sms, s);
    MA.a[n_small] = problem_args(q, W[p], make_geo(q.geom));
    MA.a[n_small].part = W[p].part;
    small[n_small++] = q;
  }
  MA.n = n_small;
  cudaEvent_t a = nullptr, b = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  const int old_block = h->block, old_bps = h->blocks_per_sm;
  struct Shape { int block, bps; };
  const Shape cands[] = {{256, 4},  {256, 6},  {256, 8},  {256, 12}, {256, 16},
                         {128, 8},  {128, 12}, {128, 16}, {128, 24}, {128, 32}};
  float best = 1e30f;
  Shape pick = {old_block, old_bps};
  for (const Shape& c : cands) {
    if (e != cudaSuccess || n_small == 0) break;
    h->block = c.block;
    h->blocks_per_sm = c.bps;
    int total = 0;
    split_blocks(h, small, n_small, MA.start, &total, c.block);
    if (total > kPartRegion) continue;
    float tmin = 1e30f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
      cudaEventRecord(a, s);
      e = launch_fused_multi(hutch ? (F_GRAD | F_HUTCH) : F_GRAD, MA, total, c.block, s);
      cudaEventRecord(b, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(b);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
      if (e == cudaSuccess && ms < tmin) tmin = ms;
    }
    if (e == cudaSuccess && tmin < best) {
      best = tmin;
      pick = c;
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaStreamDestroy(s);
  if (e != cudaSuccess) {
    h->block = old_block;
    h->blocks_per_sm = old_bps;
    return cuda_fail(h, e, "autotune");
  }
  h->block = pick.block;
  h->blocks_per_sm = pick.bps;
  if (block_out) *block_out = pick.block;
  if (bps_out) *bps_out = pick.bps;
  return CS_OK;
}

int cs_phase_shift(cs_handle* h, int M, float* images, const float* shifts, int B, int sign,
                   void* stream) {
  if (!h) return CS_ERR_ARG;
  if (M < 4 || M > CS_MAX_M || (M & 1))
    return fail(h, CS_ERR_SHAPE, "M=%d must be even and in [4, %d]", M, CS_MAX_M);
  if (B < 0) return fail(h, CS_ERR_SHAPE, "batch size B=%d is negative", B);
  if (sign != 1 && sign != -1) return fail(h, CS_ERR_ARG, "sign=%d must be +1 or -1", sign);
  if (B == 0) return CS_OK;
  if (!images || !shifts) return fail(h, CS_ERR_ARG, "images or shifts is NULL");
  CS_SCOPE(h);
  CS_CUDA(launch_phase_shift(M, B, reinterpret_cast<float2*>(images), shifts, sign, h->num_sms,
                             S(stream)),
          "phase shift launch");
  return CS_OK;
}

int cs_fsc(cs_handle* h, int M, const float* u, const float* v, int n_shells, double* sums,
           double* fsc, void* stream) {
  if (!h) return CS_ERR_ARG;
  if (M < 4 || M > CS_MAX_M || (M & 1))
    return fail(h, CS_ERR_SHAPE, "M=%d must be even and in [4, %d]", M, CS_MAX_M);
  if (n_shells < 1 || n_shells > kMaxShells)
    return fail(h, CS_ERR_SHAPE, "n_shells=%d must be in [1, %d]", n_shells, kMaxShells);
  if (!u || !v || !sums) return fail(h, CS_ERR_ARG, "u, v or sums is NULL");
  CS_SCOPE(h);
  CS_CUDA(launch_fsc(M, reinterpret_cast<const float2*>(u), reinterpret_cast<const float2*>(v),
                     n_shells, sums, fsc, h->num_sms, S(stream)),
          "fsc launch");
  return CS_OK;
}

int cs_shell_minmax(cs_handle* h, int M, const float* x, int n_shells, float* min_out,
                    float* max_out, int* count_out, void* stream) {
  if (!h) return CS_ERR_ARG;
  if (M < 4 || M > CS_MAX_M || (M & 1))
    return fail(h, CS_ERR_SHAPE, "M=%d must be even and in [4, %d]", M, CS_MAX_M);
  if (n_shells < 1 || n_shells > kMaxShells)
    return fail(h, CS_ERR_SHAPE, "n_shells=%d must be in [1, %d]", n_shells, kMaxShells);
  if (!x || !min_out || !max_out || !count_out)
    return fail(h, CS_ERR_ARG, "x, min_out, max_out or count_out is NULL");
  CS_SCOPE(h);
  CS_CUDA(launch_shell_minmax(M, x, n_shells, min_out, max_out, count_out, h->num_sms,
                              S(stream)),
          "shell min/max launch");
  return CS_OK;
}

int cs_rel_err(cs_handle* h, const cs_geom* g, const float* v, const float* v_ref,
               double* out, void* stream) {
  if (!h) return CS_ERR_ARG;
  CS_TRY(check_geom(h, g));
  if (!v || !v_ref || !out) return fail(h, CS_ERR_ARG, "v, v_ref or out is NULL");
  CS_SCOPE(h);
  Workspace w;
  CS_TRY(ensure_ws(h, g->M, 1, &w));
  Geo G = make_geo(*g);
  CS_CUDA(launch_rel_err(G, reinterpret_cast<const float2*>(v),
                         reinterpret_cast<const float2*>(v_ref), w.part, out, h->num_sms,
                         S(stream)),
          "rel_err launch");
  return CS_OK;
}

}  // extern "C"

// ------------------------------------------------ learned preconditioner

namespace {

int ensure_status(cs_handle* h) {
  if (h->status) return CS_OK;
  int* p = nullptr;
  cudaError_t e = cudaMalloc(&p, sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, CS_ERR_ALLOC, "status word: %s", cudaGetErrorString(e));
  }
  e = cudaMemset(p, 0, sizeof(int));
  if (e != cudaSuccess) {
    cudaFree(p);
    return cuda_fail(h, e, "status word");
  }
  h->status = p;
  return CS_OK;
}

long ball_count(int M, int r) {
  const int half = M / 2;
  long n = 0;
  for (int z = -half; z < half; ++z)
    for (int y = -half; y < half; ++y) {
      const long q = (long)z * z + (long)y * y;
      if (q > (long)r * r) continue;
      const int xr = (int)std::floor(std::sqrt((double)((long)r * r - q)));
      const int lo = -xr < -half ? -half : -xr, hi = xr > half - 1 ? half - 1 : xr;
      n += hi - lo + 1;
    }
  return n;
}

}  // namespace

extern "C" {

int cs_mlp_forward(cs_handle* h, int M, const float* params, const float* cov, const float* c2w,
                   float* out, int exp_out, float offset, int tc, void* stream) {
  if (!h) return CS_ERR_ARG;
  if (M < 4 || M > CS_MAX_M || (M & 1)) return fail(h, CS_ERR_SHAPE, "M=%d invalid", M);
  if (!params || !cov || !c2w || !out) return fail(h, CS_ERR_ARG, "NULL pointer argument");
  if (!is_finite(offset)) return fail(h, CS_ERR_ARG, "offset is not finite");
  CS_SCOPE(h);
  CS_TRY(ensure_status(h));
  CS_CUDA(launch_mlp_forward(M, params, cov, c2w, out, exp_out, offset, tc != 0, h->status,
                             h->num_sms, S(stream)),
          "mlp_forward launch");
  return CS_OK;
}

int cs_mlp_target(cs_handle* h, int M, int n_est, const float* est, float floor_rel,
                  float* target, void* stream) {
  if (!h) return CS_ERR_ARG;
  if (M < 4 || M > CS_MAX_M || (M & 1)) return fail(h, CS_ERR_SHAPE, "M=%d invalid", M);
  if (n_est < 1 || n_est > 4096) return fail(h, CS_ERR_SHAPE, "n_est=%d invalid", n_est);
  if (!est || !target) return fail(h, CS_ERR_ARG, "NULL pointer argument");
  if (!(floor_rel > 0.f && floor_rel <= 1.f))
    return fail(h, CS_ERR_ARG, "floor_rel must be in (0, 1]");
  CS_SCOPE(h);
  Workspace w;
  CS_TRY(ensure_ws(h, M, 1, &w));
  CS_CUDA(launch_mlp_target(M, n_est, est, floor_rel, target, w.part, h->num_sms, S(stream)),
          "mlp_target launch");
  return CS_OK;
}

int cs_mlp_grad(cs_handle* h, int M, int r_ball, const float* params, const float* cov,
                const float* c2w, const float* target, float* grad, double* sse, int tc,
                void* stream) {
  if (!h) return CS_ERR_ARG;
  if (M < 4 || M > CS_MAX_M || (M & 1)) return fail(h, CS_ERR_SHAPE, "M=%d invalid", M);
  if (r_ball < 1 || r_ball > M / 2) return fail(h, CS_ERR_SHAPE, "r_ball=%d invalid", r_ball);
  if (!params || !cov || !c2w || !target || !grad || !sse)
    return fail(h, CS_ERR_ARG, "NULL pointer argument");
  CS_SCOPE(h);
  CS_TRY(ensure_status(h));
  const long nb = ball_count(M, r_ball);
  CS_CUDA(launch_mlp_grad(M, r_ball * r_ball, 1.0f / (float)nb, params, cov, c2w, target, grad,
                          sse, tc != 0, h->status, h->num_sms, S(stream)),
          "mlp_grad launch");
  return CS_OK;
}

int cs_mlp_adam_step(cs_handle* h, float* params, float* m, float* v, float* grad,
                     float grad_scale, int step, float lr, float b1, float b2, float eps,
                     void* stream) {
  if (!h) return CS_ERR_ARG;
  if (!params || !m || !v || !grad) return fail(h, CS_ERR_ARG, "NULL pointer argument");
  if (step < 1 || !(lr > 0) || !(b1 >= 0 && b1 < 1) || !(b2 >= 0 && b2 < 1) || !(eps > 0))
    return fail(h, CS_ERR_ARG, "Adam hyper-parameters out of range");
  if (!(is_finite(grad_scale) && grad_scale > 0))
    return fail(h, CS_ERR_ARG, "grad_scale must be finite and positive");
  CS_SCOPE(h);
  CS_CUDA(launch_adam(params, m, v, grad, grad_scale, step, lr, b1, b2, eps, S(stream)),
          "adam launch");
  return CS_OK;
}

int cs_selftest_wait_timeout(cs_handle* h, long long spins, void* stream) {
  if (!h) return CS_ERR_ARG;
  if (spins < 1 || spins > (1ll << 24))
    return fail(h, CS_ERR_ARG, "spins=%lld must be in [1, 2^24]", spins);
  CS_SCOPE(h);
  CS_TRY(ensure_status(h));
  CS_CUDA(launch_wait_selftest(spins, h->status, S(stream)), "wait self-test launch");
  return CS_OK;
}

int cs_check_device_status(cs_handle* h) {
  if (!h) return CS_ERR_ARG;
#ifdef CS_DEBUG_BOUNDS
  {
    CS_SCOPE(h);
    CS_CUDA(cudaDeviceSynchronize(), "synchronise");
    unsigned bad = 0;
    for (unsigned (*rd)() : dbg_readers()) bad |= rd();
    if (bad) return fail(h, CS_ERR_INTERNAL, "a device-side index range check failed");
  }
#endif
  if (!h->status) return CS_OK;
  CS_SCOPE(h);
  CS_CUDA(cudaDeviceSynchronize(), "synchronise");
  int flag = 0;
  CS_CUDA(cudaMemcpy(&flag, h->status, sizeof(int), cudaMemcpyDeviceToHost), "status read");
  if (flag) {
    CS_CUDA(cudaMemset(h->status, 0, sizeof(int)), "status reset");
    return fail(h, CS_ERR_TIMEOUT, "a bounded device-side wait ran out (tensor-core kernel)");
  }
  return CS_OK;
}

int cs_build_flags(void) {
#ifdef CS_DEBUG_BOUNDS
  return CS_BUILD_DEBUG_BOUNDS;
#else
  return 0;
#endif
}

}  // extern "C"

// ------------------------------------------- steps fed from host memory
//
// Double-buffered staging: two device slots hold a batch (images, poses,
// defocus, rotations).  Step n copies its batch into slot n mod 2 on the
// handle's copy stream, after the step that last used that slot has
// finished, and computes on the caller's stream once its copy is done; so
// the copy of batch n+1 runs while step n computes.

namespace {

struct StageSlot {
  float* images;
  float* quat;
  float* defocus;
  float* rot;
  float* packed;    // disc-packed images of a cs_precond_sgd_step_host_disc batch
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// disc pixels of radius r: rows ky = -r .. r of 2 floor(sqrt(r^2 - ky^2)) + 1
long disc_count(int r) {
  long n = 0;
  for (int ky = -r; ky <= r; ++ky) {
    int xr = 0;
    while ((long)(xr + 1) * (xr + 1) <= (long)r * r - (long)ky * ky) ++xr;
    n += 2 * xr + 1;
  }
  return n;
}

size_t slot_bytes(int M, int B) {
  return align256((size_t)B * M * M * 8) + align256((size_t)B * 16) + align256((size_t)B * 4) +
         align256((size_t)B * 36) + align256((size_t)B * disc_count(M / 2 - 1) * 8);
}

StageSlot stage_slot(const cs_handle* h, int slot) {
  unsigned char* p = static_cast<unsigned char*>(h->stage) + slot * slot_bytes(h->stage_M, h->stage_B);
  StageSlot s;
  s.images = reinterpret_cast<float*>(p);
  p += align256((size_t)h->stage_B * h->stage_M * h->stage_M * 8);
  s.quat = reinterpret_cast<float*>(p);
  p += align256((size_t)h->stage_B * 16);
  s.defocus = reinterpret_cast<float*>(p);
  p += align256((size_t)h->stage_B * 4);
  s.rot = reinterpret_cast<float*>(p);
  p += align256((size_t)h->stage_B * 36);
  s.packed = reinterpret_cast<float*>(p);
  return s;
}

// Device address of page-locked host memory that the runtime has mapped
// into the device's address space, or NULL (pageable or device memory, or
// a host allocation without a device mapping).
const float* mapped_device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  // unified addressing: the device address of mapped host memory is the
  // host address; anything else takes the staged path
  if (a.type != cudaMemoryTypeHost || a.devicePointer != p) return nullptr;
  return static_cast<const float*>(a.devicePointer);
}

int ensure_stage(cs_handle* h, int M, int B) {
  if (!h->copy_stream) {
    CS_CUDA(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking), "copy stream");
    for (int i = 0; i < 2; ++i) {
      CS_CUDA(cudaEventCreateWithFlags(&h->copy_done[i], cudaEventDisableTiming), "event");
      CS_CUDA(cudaEventCreateWithFlags(&h->compute_done[i], cudaEventDisableTiming), "event");
    }
  }
  if (h->stage && h->stage_M == M && h->stage_B >= B) return CS_OK;
  const int Bn = (h->stage && h->stage_M == M && h->stage_B > B) ? h->stage_B : B;
  const size_t need = 2 * slot_bytes(M, Bn);
  if (h->stage) {
    // slots may still be read by in-flight steps or written by copies
    CS_CUDA(cudaDeviceSynchronize(), "synchronise before staging growth");
    cudaFree(h->stage);
    h->stage = nullptr;
  }
  void* p = nullptr;
  if (cudaMalloc(&p, need) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, CS_ERR_ALLOC, "staging allocation of %zu bytes failed", need);
  }
  // pixels a disc-packed batch does not write are zero (never read)
  CS_CUDA(cudaMemset(p, 0, need), "staging reset");
  h->stage = p;
  h->stage_M = M;
  h->stage_B = Bn;
  return CS_OK;
}

// Row starts of the disc of radius r in packed order, on the device.
int ensure_disc_rows(cs_handle* h, int M, int r) {
  if (h->disc_rows && h->disc_M == M && h->disc_r == r) return CS_OK;
  std::vector<int> rows(2 * r + 2, 0);
  for (int k = 0; k <= 2 * r; ++k) {
    const int ky = k - r;
    int xr = 0;
    while ((long)(xr + 1) * (xr + 1) <= (long)r * r - (long)ky * ky) ++xr;
    rows[k + 1] = rows[k] + 2 * xr + 1;
  }
  if (h->disc_rows) {
    CS_CUDA(cudaDeviceSynchronize(), "synchronise before disc table change");
    cudaFree(h->disc_rows);
    h->disc_rows = nullptr;
  }
  int* d = nullptr;
  if (cudaMalloc(&d, rows.size() * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, CS_ERR_ALLOC, "disc row table allocation failed");
  }
  h->disc_rows = d;
  CS_CUDA(cudaMemcpy(d, rows.data(), rows.size() * sizeof(int), cudaMemcpyHostToDevice),
          "disc row table");
  h->disc_M = M;
  h->disc_r = r;
  return CS_OK;
}

}  // namespace

extern "C" {

int cs_precond_sgd_step_host(cs_handle* h, const cs_geom* g, cs_sgd_state* st,
                             const float* images_host, const float* quat_host,
                             const float* defocus_host, int B, float lambda, float scale,
                             double* loss_host, void* stream) {
  if (!h) return CS_ERR_ARG;
  CS_TRY(check_geom(h, g));
  if (!st) return fail(h, CS_ERR_ARG, "state is NULL");
  if (B < 1) return fail(h, CS_ERR_SHAPE, "batch size B=%d must be positive", B);
  if (!images_host || !quat_host) return fail(h, CS_ERR_ARG, "images_host or quat_host is NULL");
  if (g->ctf.enabled && !defocus_host)
    return fail(h, CS_ERR_ARG, "defocus_host is NULL but the CTF is enabled");
  CS_SCOPE(h);
  CS_TRY(ensure_stage(h, g->M, B));
  const int slot = (int)(h->stage_calls & 1u);
  const StageSlot d = stage_slot(h, slot);
  cudaStream_t cs = S(stream), cp = h->copy_stream;
  const float* dimg =
      h->host_mode == CS_HOST_DIRECT ? mapped_device_pointer(images_host) : nullptr;
  if (dimg) {
    // direct: the traversal reads the images from host memory; the poses
    // and defoci (a few KB) are copied on the compute stream
    CS_CUDA(cudaMemcpyAsync(d.quat, quat_host, (size_t)B * 16, cudaMemcpyHostToDevice, cs),
            "pose copy");
    if (defocus_host)
      CS_CUDA(cudaMemcpyAsync(d.defocus, defocus_host, (size_t)B * 4, cudaMemcpyHostToDevice, cs),
              "defocus copy");
    CS_TRY(cs_quat_to_rot(h, d.quat, B, d.rot, stream));
    CS_TRY(cs_precond_sgd_step(h, g, st, dimg, d.rot, defocus_host ? d.defocus : nullptr, B,
                               lambda, scale, stream));
    if (loss_host)
      CS_CUDA(cudaMemcpyAsync(loss_host, st->scalars + CS_S_LOSS, sizeof(double),
                              cudaMemcpyDeviceToHost, cs),
              "loss read-back");
    // the staged slots are not touched, but keep the slot events ordered
    // after this step so that a later staged call waits for it
    CS_CUDA(cudaEventRecord(h->compute_done[slot], cs), "compute event");
    ++h->stage_calls;
    return CS_OK;
  }
  const size_t nimg = (size_t)B * g->M * g->M * 8;
  CS_CUDA(cudaStreamWaitEvent(cp, h->compute_done[slot], 0), "copy stream wait");
  CS_CUDA(cudaMemcpyAsync(d.images, images_host, nimg, cudaMemcpyHostToDevice, cp), "image copy");
  CS_CUDA(cudaMemcpyAsync(d.quat, quat_host, (size_t)B * 16, cudaMemcpyHostToDevice, cp),
          "pose copy");
  if (defocus_host)
    CS_CUDA(cudaMemcpyAsync(d.defocus, defocus_host, (size_t)B * 4, cudaMemcpyHostToDevice, cp),
            "defocus copy");
  CS_CUDA(cudaEventRecord(h->copy_done[slot], cp), "copy event");
  CS_CUDA(cudaStreamWaitEvent(cs, h->copy_done[slot], 0), "compute stream wait");
  CS_TRY(cs_quat_to_rot(h, d.quat, B, d.rot, stream));
  CS_TRY(cs_precond_sgd_step(h, g, st, d.images, d.rot, defocus_host ? d.defocus : nullptr, B,
                             lambda, scale, stream));
  if (loss_host)
    CS_CUDA(cudaMemcpyAsync(loss_host, st->scalars + CS_S_LOSS, sizeof(double),
                            cudaMemcpyDeviceToHost, cs),
            "loss read-back");
  CS_CUDA(cudaEventRecord(h->compute_done[slot], cs), "compute event");
  ++h->stage_calls;
  return CS_OK;
}

int cs_disc_pixels(int M, int r_max) {
  if (M < 4 || M > CS_MAX_M || (M & 1) || r_max < 1 || r_max > M / 2 - 1) return -1;
  return (int)disc_count(r_max);
}

int cs_precond_sgd_step_host_disc(cs_handle* h, const cs_geom* g, cs_sgd_state* st,
                                  const float* images_disc_host, const float* quat_host,
                                  const float* defocus_host, int B, float lambda, float scale,
                                  double* loss_host, void* stream) {
  if (!h) return CS_ERR_ARG;
  CS_TRY(check_geom(h, g));
  if (!st) return fail(h, CS_ERR_ARG, "state is NULL");
  if (B < 1) return fail(h, CS_ERR_SHAPE, "batch size B=%d must be positive", B);
  if (!images_disc_host || !quat_host)
    return fail(h, CS_ERR_ARG, "images_disc_host or quat_host is NULL");
  if (g->ctf.enabled && !defocus_host)
    return fail(h, CS_ERR_ARG, "defocus_host is NULL but the CTF is enabled");
  CS_SCOPE(h);
  CS_TRY(ensure_stage(h, g->M, B));
  CS_TRY(ensure_disc_rows(h, g->M, g->r_max));
  const int slot = (int)(h->stage_calls & 1u);
  const StageSlot d = stage_slot(h, slot);
  cudaStream_t cs = S(stream), cp = h->copy_stream;
  const size_t npk = (size_t)B * disc_count(g->r_max) * 8;
  // the vector traversal reads the packed pixels where they land; the other
  // scatter algorithms get them spread into image layout first
  const bool packed = use_vector(h, g);
  CS_CUDA(cudaStreamWaitEvent(cp, h->compute_done[slot], 0), "copy stream wait");
  CS_CUDA(cudaMemcpyAsync(d.packed, images_disc_host, npk, cudaMemcpyHostToDevice, cp),
          "image copy");
  if (!packed)
    CS_CUDA(launch_expand_disc(g->M, g->r_max, B, h->disc_rows, d.packed, d.images, cp),
            "disc expansion launch");
  CS_CUDA(cudaMemcpyAsync(d.quat, quat_host, (size_t)B * 16, cudaMemcpyHostToDevice, cp),
          "pose copy");
  if (defocus_host)
    CS_CUDA(cudaMemcpyAsync(d.defocus, defocus_host, (size_t)B * 4, cudaMemcpyHostToDevice, cp),
            "defocus copy");
  CS_CUDA(cudaEventRecord(h->copy_done[slot], cp), "copy event");
  CS_CUDA(cudaStreamWaitEvent(cs, h->copy_done[slot], 0), "compute stream wait");
  CS_TRY(cs_quat_to_rot(h, d.quat, B, d.rot, stream));
  CS_TRY(precond_step_impl(h, g, st, packed ? d.packed : d.images, d.rot,
                           defocus_host ? d.defocus : nullptr, B, lambda, scale, stream,
                           packed ? h->disc_rows : nullptr));
  if (loss_host)
    CS_CUDA(cudaMemcpyAsync(loss_host, st->scalars + CS_S_LOSS, sizeof(double),
                            cudaMemcpyDeviceToHost, cs),
            "loss read-back");
  CS_CUDA(cudaEventRecord(h->compute_done[slot], cs), "compute event");
  ++h->stage_calls;
  return CS_OK;
}

}  // extern "C"
