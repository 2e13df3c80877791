// Workspace of the vector-reduction passes (see fused.cu).
#pragma once

#include <cuda_runtime.h>

namespace cs {

struct FusedWs {
  float2* E;      // complex accumulator, natural layout [M^3]
  float2* O;      // complex accumulator shifted by one voxel along x [M^3]
  float* P;       // four real 2x2-patch accumulators [4][M^3]
  float4* pairs;  // pair layout (v[j], v[j+1]) of the gathered volume [M^3]
  float2* dn;     // search direction d of a step, natural layout [M^3]
  float4* dq;     // d as 2 x 2 (x, y) patches, 32 bytes per voxel [2 M^3]:
                  // (d[j], d[j+1], d[j+M], d[j+M+1]), 0 past the grid's edge
  int* table;     // disc pixel table (row order, or tile order: see fused.cu)
  int* tile_org;  // tile order: origin of each table chunk
  int* n_px;      // number of table entries
  // per-slab item lists of a slab-split traversal (NULL in workspaces
  // without a slab region): span and region of each (image, tile) item,
  // per-(slab, region, image) counts (then offsets), per-(slab, region)
  // totals and list starts, slab starts [S+1], the lists
  int* slab_span;
  int* slab_cnt;
  int* slab_tot;
  int* slab_base;
  int* slab_se;
  int* slab_items;
  int slab_cap_B;
};

}  // namespace cs
