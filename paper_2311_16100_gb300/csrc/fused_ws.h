// Workspace of the vector-reduction passes (see fused.cu).
#pragma once

#include <cuda_runtime.h>

namespace cs {

struct FusedWs {
  float2* E;      // complex accumulator, natural layout [M^3]
  float2* O;      // complex accumulator shifted by one voxel along x [M^3]
  float* P;       // four real 2x2-patch accumulators [4][M^3]
  float4* pairs;  // pair layout (v[j], v[j+1]) of the gathered volume [M^3]
  int* table;     // disc pixel table (row order, or tile order: see fused.cu)
  int* tile_org;  // tile order: origin of each table chunk
  int* n_px;      // number of table entries
  // per-slab item lists of a slab-split traversal (single-problem workspace
  // only; NULL otherwise): span of each (image, tile) item, per-image counts,
  // slab starts [S+1], the lists
  int* slab_span;
  int* slab_cnt;
  int* slab_se;
  int* slab_items;
  int slab_cap_B;
};

}  // namespace cs
