// Tile engine interface (see tiles.cu).
#pragma once

#include "internal.h"

namespace cs {

constexpr int kT = 16;            // tile edge (voxels)
constexpr int kImgPerItem = 64;   // images per work item

enum TileOp { OP_ADJOINT = 0, OP_LOSS_GRAD = 1, OP_HVP = 2, OP_HUTCH = 3, OP_CURVATURE = 4 };

struct TileArgs {
  Geo G;
  const float* rot = nullptr;      // [B][9]
  const float* df = nullptr;       // [B] (CTF on)
  int B = 0;
  float scale = 1.f;
  int K = 1;                       // probes (OP_HUTCH)
  const void* src = nullptr;       // gathered operand: volume, real vector or probe words
  const float2* img = nullptr;     // images (OP_ADJOINT, OP_LOSS_GRAD)
  void* dst = nullptr;             // accumulation target in global memory
  double* part = nullptr;          // per-item partial sums (OP_LOSS_GRAD, OP_CURVATURE)
  // binning
  int tpa = 0, n_tiles = 0, list_stride = 1;
  const int* tile_count = nullptr;
  const int* tile_list = nullptr;
  const int* item_start = nullptr; // [n_tiles + 1]; item_start[n_tiles] = number of items
  int* queue = nullptr;            // work counter
};

int tiles_per_axis(int M);
inline int tile_count_for(int M) { int t = tiles_per_axis(M); return t * t * t; }
inline size_t max_items_for(int M, int B) {
  return (size_t)tile_count_for(M) * (size_t)((B + kImgPerItem - 1) / kImgPerItem);
}

// Bins the batch's images by tile and builds the item table; fills the
// binning fields of A.
cudaError_t launch_bin(const Geo& G, const float* rot, int B, TileArgs& A, int* count,
                       int* list, int* item_start, int* queue, cudaStream_t s);
// Runs one tile operation over the binned batch (resets the work counter).
cudaError_t launch_tile_op(int op, const TileArgs& A, int num_sms, cudaStream_t s);

}  // namespace cs
