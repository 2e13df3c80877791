// Vector-reduction pixel passes (see fused.cu).
#pragma once

#include "internal.h"

namespace cs {

enum FusedFlags { F_ADJ = 1, F_GRAD = 2, F_HUTCH = 4, F_HVP = 8, F_CURV = 16,
                  // kernel variant with the z-slab / tile-ordered table logic
                  // (compiled out of the one-slab launches)
                  F_SLAB = 32,
                  // one-slab launch over the tile-ordered table (skips its holes)
                  F_HOLES = 64,
                  // F_GRAD on disc-packed images (FusedArgs::img_rows)
                  F_PACKED = 128 };

constexpr int kMaxProblems = 8;   // volumes per multi-volume launch



struct FusedArgs {
  Geo G;
  const int* table;
  const int* n_px_dev;
  const float* rot;
  const float* df;
  int B;
  float scale;
  const float2* vol;    // F_GRAD: volume; F_CURV: direction d
  const float* zr;      // F_HVP: real vector z
  const float2* img;    // F_ADJ, F_GRAD
  // F_GRAD: images disc-packed (rows[k] = first pixel of disc row k, k = ky +
  // img_r, rows[2 img_r + 1] = pixels per image) instead of [B][M][M]; NULL:
  // image layout
  const int* img_rows;
  int img_r;
  float2* E;
  float2* O;
  double* part;         // F_GRAD: data-term partials; F_CURV: curvature partials
  float* P;             // F_HUTCH, F_HVP
  int K;
  const float4* vp;     // pair layout of vol (F_GRAD)
  const float4* dq;     // F_CURV: 2 x 2 patch layout of the direction d
  uint64_t seed;        // F_HUTCH: probe stream
  uint64_t block_host;  // F_HUTCH: probe block, or
  const double* k_dev;  //   (iterations done + 1) read from the SGD state
  // batch selection on the device (multi-volume step): when cursor is set,
  // img and df point at all n_batches batches and batch (k mod n_batches)
  // is used, k = iterations done (*cursor)
  const double* cursor;
  int n_batches;
  // part_add: add the block partial to part[] instead of storing it (slab
  // launches after the first)
  int part_add;
  // tile-ordered table: chunk ch covers the 16 x tile_h pixels with origin
  // tile_org[ch] (packed like table entries); NULL for the row-ordered table
  const int* tile_org;
  int tile_h;
  // F_SLAB: this launch's items are slab_items[slab_se[0] .. slab_se[1])
  // (item = image * chunks + chunk)
  const int* slab_items;
  const int* slab_se;
};

struct MultiFusedArgs {
  int n;                              // problems
  int start[kMaxProblems + 1];        // first block of each problem
  FusedArgs a[kMaxProblems];
};

size_t fused_ws_bytes(int M);
// tile-ordered table sizes: entries and tile origins
size_t table_entries(int M);
size_t tile_slots(int M);
// per-slab item lists for batches of up to B images: bytes, and the carving
// of a region of that size into w's slab fields
size_t slab_lists_bytes(int M, int B);
void slab_carve(void* region, int M, int B, FusedWs& w);
constexpr int kMaxSlabs = 16;
FusedWs fused_carve(void* base, int M);

cudaError_t launch_disc_table(int M, int r, const FusedWs& w, cudaStream_t s);
// Tile-ordered table for traversals split into z-slabs: one chunk of `block`
// entries per 16 x (block/16) pixel tile that meets the disc, entries of
// pixels outside the disc are -1; w.tile_org[ch] is chunk ch's origin.
cudaError_t launch_disc_table_tiled(int M, int r, int block, const FusedWs& w, cudaStream_t s);
// One trilinear traversal with the given flags (partials: one per block).
// vol: natural layout, vp: its pair layout (F_GRAD; F_CURV reads the patch
// layout of the direction, w.dq, written by launch_patches); probe words
// (F_HUTCH) come from (seed, block), block = *k_dev + 1 when k_dev != NULL.
// block = threads per block (128 or 256); slabs = z-slabs (one launch each;
// 0: slab_count).
// tiled: the table in w is tile-ordered (launch_disc_table_tiled with the
// same block size).
cudaError_t launch_fused(int flags, const Geo& G, const FusedWs& w, const float* rot,
                         const float* df, int B, float scale, const float2* vol,
                         const float4* vp, const float* zr, const float2* img, double* part,
                         uint64_t seed, uint64_t block_host, const double* k_dev, int K,
                         int grid, cudaStream_t s, int block = 256,
                         int slabs = 0,
                         bool tiled = false, const int* img_rows = nullptr, int img_r = 0);
// One launch over several problems (flags F_GRAD, F_GRAD|F_HUTCH or F_CURV).
// Number of z-slabs a traversal of an M^3 grid is split into: one launch
// per slab keeps the slab's accumulators and gathered volume in L2.
int slab_count(int M, int flags);
// Slabs a split traversal actually uses: the override `slabs` (> 0) or
// slab_count, at most M/16 and kMaxSlabs.
int pass_slabs(int M, int flags, int slabs);
// launch_fused with the kernel arguments already filled in (the slab fields
// are set here): used by the multi-volume step for its large volumes, whose
// arguments select the batch on the device (cursor).
cudaError_t launch_fused_args(int flags, FusedArgs A, const FusedWs& w, int grid, cudaStream_t s,
                              int block, int slabs, bool tiled);
// Blocks of a traversal kernel (flags, block size; multi: the multi-volume
// kernel; F_CURV | F_SLAB: the slab-split curvature kernel) that fit on one
// SM at once.  A traversal grid larger than
// num_sms x this would run in more than one wave, the last one part-empty.
int fused_resident(int flags, int block, bool multi);
cudaError_t launch_fused_multi(int flags, const MultiFusedArgs& MA, int grid, int block,
                               cudaStream_t s);

// Element-wise work of one step between the fused traversal and the
// curvature pass (see fused.cu), writing d into w.dn; partG holds the
// |g|^2/D-hat partials then the |d|^2 partials (*nb each), partV the |v|^2
// partials.
cudaError_t launch_step_post(int M, int mode, const float2* v, float lambda, float beta,
                             const double* scalars, const FusedWs& w, float* D, float* Davg,
                             double* partG, double* partV, int* nb, int num_sms,
                             cudaStream_t s);
// 2 x 2 patch layout w.dq of the direction w.dn (read by the curvature pass:
// two 32-byte loads per pixel instead of four 16-byte ones from a pair
// layout; 0.137 -> 0.107 ms at 128^3, batch 1024).
cudaError_t launch_patches(int M, const FusedWs& w, int num_sms, cudaStream_t s);
// v -= eta d with d = w.dn.
cudaError_t launch_update_pairs(int M, float2* v, const FusedWs& w, const double* scalars,
                                int num_sms, cudaStream_t s);
// vp[j] = (v[j], v[j+1]), 0 past each row's end.
cudaError_t launch_pairs(int M, const float2* v, float4* vp, int num_sms, cudaStream_t s);
// zero E, O (and P when zero_p) and write the pair layout of v, in one pass
cudaError_t launch_step_prep(int M, const float2* v, const FusedWs& w, bool zero_p, int num_sms,
                             cudaStream_t s);
cudaError_t launch_zero_c2(int M, const FusedWs& w, cudaStream_t s);
cudaError_t launch_zero_r4(int M, const FusedWs& w, cudaStream_t s);
// g = lambda v + E + shift(O) (v may be NULL); |v|^2 partials if part_vv.
cudaError_t launch_combine_c2(int M, const float2* v, float lambda, const FusedWs& w,
                              float2* g, double* part_vv, int* n_vv, int num_sms,
                              cudaStream_t s);
// out = base + coef * add + (patch buffers); add may be NULL.
cudaError_t launch_combine_r4(int M, const FusedWs& w, float base, float coef,
                              const float* add, float* out, int num_sms, cudaStream_t s);

}  // namespace cs
