// Pixel-parallel adjoint passes with vector reductions into parity-split
// accumulators.
//
// Global floating-point reductions are executed in L2 at a fixed rate of
// operations, whatever their width (measured on GB300: ~211 G reductions/s
// for f32, v2.f32 and v4.f32 alike, with or without lanes sharing an
// address).  The adjoint of trilinear interpolation (Definition 2.1) adds to
// the 8 corners of each pixel's cell; the passes here pack those additions
// into 16-byte reductions:
//   * complex accumulators: corners (x0, x0+1) of a cell row are 16
//     contiguous bytes, aligned when x0 is even.  Two buffers are kept, E
//     (natural layout) and O (shifted by one voxel along x), so that every
//     pair is one aligned v4 reduction into E (x0 even) or O (x0 odd):
//     4 reductions per pixel instead of 8;
//   * real accumulators: four buffers P[px][py] hold the grid as 2x2 (x, y)
//     patches whose origin has parity (px, py); each z-plane of a cell is one
//     patch in exactly one buffer: 2 reductions per pixel instead of 8.
// A combine pass folds the buffers into the natural layout.  Pixels are
// enumerated from a table of the disc's pixels (no idle lanes outside the
// disc); images are read once with an evict-first policy so that the
// accumulators and the volume stay in L2.
//
// The fused pass of the SGD step computes, for one mini-batch and one
// traversal of its pixels, the loss, the gradient (Eq. optim cp) and
// Hutchinson's estimate (Eq. hutch) from bit-packed probes.
#include <climits>
#include <cmath>

#include "internal.h"
#include "fused.h"

namespace cs {

namespace {

// pixel table: entry p = (kx + half) | (ky + half) << 16 for the disc's
// pixels in row-major order
__global__ void k_disc_table(int M, int r, int* __restrict__ table, int* __restrict__ n_out) {
  // one block; rows handled in order with a running offset
  __shared__ int row_off[CS_MAX_M + 1];
  const int half = M / 2;
  for (int ky = -r + (int)threadIdx.x; ky <= r; ky += blockDim.x) {
    int xr = (int)sqrtf((float)(r * r - ky * ky));
    while (xr * xr > r * r - ky * ky) --xr;
    while ((xr + 1) * (xr + 1) <= r * r - ky * ky) ++xr;
    row_off[ky + r + 1] = 2 * xr + 1;
  }
  if (threadIdx.x == 0) row_off[0] = 0;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int i = 1; i <= 2 * r + 1; ++i) row_off[i] += row_off[i - 1];
  __syncthreads();
  for (int ky = -r + (int)threadIdx.x; ky <= r; ky += blockDim.x) {
    const int o = row_off[ky + r], n = row_off[ky + r + 1] - o, xr = (n - 1) / 2;
    for (int i = 0; i < n; ++i)
      table[o + i] = ((i - xr) + half) | ((ky + half) << 16);
  }
  if (threadIdx.x == 0) *n_out = row_off[2 * r + 1];
}

// Tile-ordered table: tiles of 16 x th pixels (th = block / 16) in row-major
// tile order over [-half, half)^2; each tile meeting the disc gets one chunk
// of `block` entries, slot i = pixel (x0 + i % 16, y0 + i / 16), -1 outside
// the disc.  One block; the tile count is at most (512/16) x (512/8).
__global__ void k_disc_table_tiled(int M, int r, int block, int* __restrict__ table,
                                   int* __restrict__ org, int* __restrict__ n_out) {
  __shared__ int off[2049];
  const int half = M / 2, th = block / 16;
  const int ntx = (M + 15) / 16, nty = (M + th - 1) / th, nt = ntx * nty;
  const int r2 = r * r;
  for (int t = threadIdx.x; t < nt; t += blockDim.x) {
    const int x0 = (t % ntx) * 16 - half, y0 = (t / ntx) * th - half;
    // nearest point of the tile to the origin decides whether it meets the disc
    const int nx = x0 > 0 ? x0 : (x0 + 15 < 0 ? x0 + 15 : 0);
    const int ny = y0 > 0 ? y0 : (y0 + th - 1 < 0 ? y0 + th - 1 : 0);
    off[t + 1] = nx * nx + ny * ny <= r2 ? 1 : 0;
  }
  if (threadIdx.x == 0) off[0] = 0;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int t = 1; t <= nt; ++t) off[t] += off[t - 1];
  __syncthreads();
  for (int t = threadIdx.x; t < nt; t += blockDim.x) {
    if (off[t + 1] == off[t]) continue;
    const int c = off[t];
    const int x0 = (t % ntx) * 16 - half, y0 = (t / ntx) * th - half;
    org[c] = (x0 + half) | ((y0 + half) << 16);
    for (int i = 0; i < block; ++i) {
      const int kx = x0 + i % 16, ky = y0 + i / 16;
      table[(size_t)c * block + i] =
          kx * kx + ky * ky <= r2 ? (kx + half) | ((ky + half) << 16) : -1;
    }
  }
  if (threadIdx.x == 0) *n_out = off[nt] * block;
}

struct Cell {
  int x0, y0, z0;
  float tx, ty, tz;
};

__device__ __forceinline__ Cell cell_of(const Geo& G, const Rot& R, int kx, int ky) {
  const float fx = (float)kx, fy = (float)ky;
  // the fraction is taken from the centred coordinate: adding M/2 first
  // would round it to the coarser spacing of floats near M/2 .. M
  const float sx = fmaf(R.r1x, fy, R.r0x * fx);
  const float sy = fmaf(R.r1y, fy, R.r0y * fx);
  const float sz = fmaf(R.r1z, fy, R.r0z * fx);
  const float flx = floorf(sx), fly = floorf(sy), flz = floorf(sz);
  Cell c;
  c.x0 = (int)flx + G.half; c.y0 = (int)fly + G.half; c.z0 = (int)flz + G.half;
  c.tx = sx - flx; c.ty = sy - fly; c.tz = sz - flz;
  return c;
}

__device__ __forceinline__ float corner_w(const Cell& c, int k);
__device__ __forceinline__ bool corner_in(const Geo& G, const Cell& c, int k);

// per-corner gather from the pair layout (element j's first half is v[j]);
// used for cells whose base corner is outside the grid
__device__ __forceinline__ float2 gather_cell_pairs_slow(const Geo& G, const Cell& c,
                                                         const float4* __restrict__ vp) {
  float re = 0.f, im = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (!corner_in(G, c, k)) continue;
    const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
    const size_t j = ((size_t)(c.z0 + dz) * G.M + (c.y0 + dy)) * G.M + (c.x0 + dx);
    if (!CS_IN(j, (size_t)G.M * G.M * G.M)) continue;
    const float4 a = __ldg(vp + j);
    const float w = corner_w(c, k);
    re = fmaf(w, a.x, re);
    im = fmaf(w, a.y, im);
  }
  return make_float2(re, im);
}

__device__ __forceinline__ float corner_w(const Cell& c, int k) {
  const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
  return (dx ? c.tx : 1.f - c.tx) * (dy ? c.ty : 1.f - c.ty) * (dz ? c.tz : 1.f - c.tz);
}

__device__ __forceinline__ bool corner_in(const Geo& G, const Cell& c, int k) {
  const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
  return (unsigned)(c.x0 + dx) < (unsigned)G.M && (unsigned)(c.y0 + dy) < (unsigned)G.M &&
         (unsigned)(c.z0 + dz) < (unsigned)G.M;
}

// A cell whose base corner lies inside the grid (always the case for
// rotations and r_max <= M/2 - 1); other cells take the per-corner path.
__device__ __forceinline__ bool base_in(const Geo& G, const Cell& c) {
  return (unsigned)c.x0 < (unsigned)G.M && (unsigned)c.y0 < (unsigned)G.M &&
         (unsigned)c.z0 < (unsigned)G.M;
}

// Corner weights of a cell whose base corner is inside the grid, k = dx +
// 2 dy + 4 dz; corners past the grid's upper edge get weight 0.
// The products are taken two at a time (packed pairs, the same roundings).
__device__ __forceinline__ void cell_weights(const Geo& G, const Cell& c, float w8[8]) {
  const float wx1 = c.x0 + 1 < G.M ? c.tx : 0.f, wy1 = c.y0 + 1 < G.M ? c.ty : 0.f;
  const float wz1 = c.z0 + 1 < G.M ? c.tz : 0.f;
  const float wx0 = 1.f - c.tx, wy0 = 1.f - c.ty, wz0 = 1.f - c.tz;
  const float2 wy = make_float2(wy0, wy1), wx = make_float2(wx0, wx1);
  const float2 z0 = mul2(dup2(wz0), wy), z1 = mul2(dup2(wz1), wy);
  const float wzy[4] = {z0.x, z0.y, z1.x, z1.y};
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const float2 q = mul2(dup2(wzy[r]), wx);
    w8[2 * r] = q.x;
    w8[2 * r + 1] = q.y;
  }
}

// gather from the pair layout with precomputed corner weights (base_in cells)
__device__ __forceinline__ float2 gather_pairs_w(const Geo& G, const Cell& c,
                                                 const float4* __restrict__ vp,
                                                 const float w8[8]) {
  const int M = G.M;
  float2 acc = make_float2(0.f, 0.f);        // (re, im), packed pairs
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int y = c.y0 + (r & 1), z = c.z0 + (r >> 1);
    if (z >= M || y >= M) continue;
    const size_t j = ((size_t)z * M + y) * M + c.x0;
    if (!CS_IN(j, (size_t)M * M * M)) continue;
    const float4 a = __ldg(vp + j);
    acc = fma2(dup2(w8[2 * r]), make_float2(a.x, a.y),
               fma2(dup2(w8[2 * r + 1]), make_float2(a.z, a.w), acc));
  }
  return acc;
}

// 32-byte load of one 2 x 2 (x, y) patch of complex values:
// (re, im) of (x, y), (x+1, y), (x, y+1), (x+1, y+1)
__device__ __forceinline__ void ld_patch(const float4* __restrict__ p, float (&a)[8]) {
  asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=f"(a[0]), "=f"(a[1]), "=f"(a[2]), "=f"(a[3]), "=f"(a[4]), "=f"(a[5]), "=f"(a[6]),
        "=f"(a[7])
      : "l"(p));
}

// Place of voxel (x, y, z)'s patch in the patch buffer: the grid in 2 x 2 x 2
// blocks of voxels, block-major, z-, y-, x-major within a block, so that a
// z-plane of a block (4 patches) is one 128-byte line and cells a step apart
// share lines more often than in row order
__device__ __forceinline__ size_t patch_slot(int M, int x, int y, int z) {
  const int Mh = M >> 1;
  return ((((size_t)(z >> 1) * Mh + (y >> 1)) * Mh + (x >> 1)) << 3) +
         (((z & 1) << 2) | ((y & 1) << 1) | (x & 1));
}

// gather from the 2 x 2 patch layout with precomputed corner weights
// (base_in cells): one 32-byte load per z-plane of the cell; weight
// w8[4 dz + 2 dy + dx] goes with patch element dx + 2 dy
__device__ __forceinline__ float2 gather_patch_w(const Geo& G, const Cell& c,
                                                 const float4* __restrict__ dq,
                                                 const float w8[8]) {
  const int M = G.M;
  float2 acc = make_float2(0.f, 0.f);        // (re, im), packed pairs
#pragma unroll
  for (int dz = 0; dz < 2; ++dz) {
    const int z = c.z0 + dz;
    if (z >= M) continue;
    const size_t j = patch_slot(M, c.x0, c.y0, z);
    if (!CS_IN(j, (size_t)M * M * M)) continue;
    float a[8];
    ld_patch(dq + 2 * j, a);
    const float* w = w8 + 4 * dz;
    acc = fma2(dup2(w[0]), make_float2(a[0], a[1]),
               fma2(dup2(w[1]), make_float2(a[2], a[3]),
                    fma2(dup2(w[2]), make_float2(a[4], a[5]),
                         fma2(dup2(w[3]), make_float2(a[6], a[7]), acc))));
  }
  return acc;
}

// per-corner gather from the patch layout (element 0 of patch j is d[j]);
// cells whose base corner is outside the grid
__device__ __forceinline__ float2 gather_cell_patch_slow(const Geo& G, const Cell& c,
                                                         const float4* __restrict__ dq) {
  float re = 0.f, im = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (!corner_in(G, c, k)) continue;
    const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
    const size_t j = patch_slot(G.M, c.x0 + dx, c.y0 + dy, c.z0 + dz);
    if (!CS_IN(j, (size_t)G.M * G.M * G.M)) continue;
    const float4 a = __ldg(dq + 2 * j);
    const float w = corner_w(c, k);
    re = fmaf(w, a.x, re);
    im = fmaf(w, a.y, im);
  }
  return make_float2(re, im);
}

// L2 policy that keeps lines (the accumulators) in L2 ahead of others, and
// a 16-byte reduction under it
__device__ __forceinline__ uint64_t l2_keep_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void red_add_keep(float4* p, float4 v, uint64_t pol) {
  asm volatile("red.global.add.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;"
               :: "l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "l"(pol) : "memory");
}

// scatter of val * w8 into E / O (base_in cells), one v4 reduction per row
__device__ __forceinline__ void scatter_c2_w(const Geo& G, const Cell& c, float2 val,
                                             float2* __restrict__ E, float2* __restrict__ O,
                                             const float w8[8], uint64_t pol) {
  const int M = G.M;
  const bool odd = c.x0 & 1;
  float2* base = odd ? O : E;
  const int xb = odd ? c.x0 - 1 : c.x0;      // even slot of the pair
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int y = c.y0 + (r & 1), z = c.z0 + (r >> 1);
    if (z >= M || y >= M) continue;
    const float a0 = w8[2 * r], a1 = w8[2 * r + 1];
    const size_t j = ((size_t)z * M + y) * M + xb;
    if (!CS_IN(j + 1, (size_t)M * M * M)) continue;     // the pair (j, j + 1)
    float4* p = reinterpret_cast<float4*>(base + j);
    const float2 q0 = mul2(dup2(a0), val), q1 = mul2(dup2(a1), val);
    red_add_keep(p, make_float4(q0.x, q0.y, q1.x, q1.y), pol);
  }
}

// adds val * w(corner) to the 8 corners of a cell: one v4 reduction per
// (y, z) corner row, into E (x0 even) or O (x0 odd, shifted by one voxel)
__device__ __forceinline__ void scatter_cell_c2(const Geo& G, const Cell& c, float2 val,
                                                float2* __restrict__ E, float2* __restrict__ O) {
  const int M = G.M;
  if (!base_in(G, c)) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (!corner_in(G, c, k)) continue;
      const float w = corner_w(c, k);
      const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
      const size_t j = ((size_t)(c.z0 + dz) * M + (c.y0 + dy)) * M + (c.x0 + dx);
      if (!CS_IN(j, (size_t)M * M * M)) continue;
      atomicAdd(E + j, make_float2(w * val.x, w * val.y));
    }
    return;
  }
  const bool odd = c.x0 & 1;
  float2* base = odd ? O : E;
  const int xb = odd ? c.x0 - 1 : c.x0;      // even slot of the pair
  const float w0x = 1.f - c.tx, w1x = c.tx;
#pragma unroll
  for (int dz = 0; dz < 2; ++dz) {
    const int z = c.z0 + dz;
    const float wz = dz ? c.tz : 1.f - c.tz;
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      const int y = c.y0 + dy;
      if (z >= M || y >= M) continue;
      const float wzy = wz * (dy ? c.ty : 1.f - c.ty);
      const float a0 = wzy * w0x, a1 = wzy * w1x;
      const size_t j = ((size_t)z * M + y) * M + xb;
      if (!CS_IN(j + 1, (size_t)M * M * M)) continue;   // the pair (j, j + 1)
      float4* p = reinterpret_cast<float4*>(base + j);
      atomicAdd(p, make_float4(a0 * val.x, a0 * val.y, a1 * val.x, a1 * val.y));
    }
  }
}

// adds per-corner real values to the 2x2 (x, y) patch buffers, one v4
// reduction per z-plane.  vals[k] for corner k = dx + 2 dy + 4 dz.
__device__ __forceinline__ void scatter_cell_r4(const Geo& G, const Cell& c, const float* vals,
                                                float* __restrict__ P, uint64_t pol) {
  const int M = G.M, Mh = G.M / 2;
  const size_t nb = (size_t)M * M * M;
  if (!base_in(G, c)) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (!corner_in(G, c, k)) continue;
      const int x = c.x0 + (k & 1), y = c.y0 + ((k >> 1) & 1), z = c.z0 + (k >> 2);
      float* buf = P + (size_t)((y & 1) * 2 + (x & 1)) * nb;
      const size_t j = 4 * (((size_t)z * Mh + (y >> 1)) * Mh + (x >> 1));
      if (!CS_IN(j, nb)) continue;
      atomicAdd(buf + j, vals[k]);
    }
    return;
  }
  const int px = c.x0 & 1, py = c.y0 & 1;
  float* buf = P + (size_t)(py * 2 + px) * nb;
  const int X = (c.x0 - px) >> 1, Y = (c.y0 - py) >> 1;
#pragma unroll
  for (int dz = 0; dz < 2; ++dz) {
    const int z = c.z0 + dz;
    if (z >= M) continue;
    const size_t j = 4 * (((size_t)z * Mh + Y) * Mh + X);
    if (!CS_IN(j + 3, nb)) continue;                    // the patch j .. j + 3
    float4* p = reinterpret_cast<float4*>(buf + j);
    red_add_keep(p, make_float4(vals[4 * dz + 0], vals[4 * dz + 1], vals[4 * dz + 2],
                                vals[4 * dz + 3]), pol);
  }
}


// real trilinear gather (corners outside the grid read 0)
__device__ __forceinline__ float gather_cell_r(const Geo& G, const Cell& c,
                                               const float* __restrict__ z) {
  float a = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (!corner_in(G, c, k)) continue;
    const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
    const size_t j = ((size_t)(c.z0 + dz) * G.M + (c.y0 + dy)) * G.M + (c.x0 + dx);
    if (!CS_IN(j, (size_t)G.M * G.M * G.M)) continue;
    a = fmaf(corner_w(c, k), __ldg(z + j), a);
  }
  return a;
}





// One traversal of the batch's disc pixels (trilinear).  Work item =
// (image, 256 consecutive disc pixels); a fixed grid walks the items, so
// the per-block partial sums are deterministic.
//   F_ADJ   : E/O += scale C y                    (adjoint of the forward model)
//   F_GRAD  : r = C P v - x; loss += |r|^2; E/O += scale C r     (Eq. optim cp)
//   F_HUTCH : P4 += scale C^2 w_j sum_l w_l Z_jl  (Eq. hutch, bit-packed probes)
//   F_HVP   : P4 += scale C^2 w_j (P z)           (Eq. hessian)
//   F_CURV  : part += C^2 |P d|^2                 (curvature of the Armijo step)
// ---- per-slab item lists (deterministic)
//
// Item (b, t) = image b, table chunk t (a 16 x tile_h pixel tile).  Each
// item belongs to exactly one slab launch, that of the z coordinate of its
// tile's centre (R[0][2] kx + R[1][2] ky + M/2 at the middle of the tile's
// range), and that launch processes all of its pixels, so every pixel is
// processed once.  A tile spans at most ~23 voxels in z, so a launch also
// touches accumulators up to about half a tile beyond its slab: every lane
// stays busy, at the price of a slightly larger L2 footprint per launch.
//
// Within a slab the items are grouped by the region of the slab their tile
// centre falls in (kSlabQ x kSlabQ columns of the grid in x, y), region by
// region, each region's items image by image.  The blocks of a launch then
// work on the items of one or two regions at a time, and the accumulators
// and volume they touch (a few MB) stay in L2 until the region is done,
// instead of every image's band across the whole slab being touched at once.

constexpr int kSlabQ = 4;                      // regions per axis (x, y)
constexpr int kSlabKeys = kSlabQ * kSlabQ;     // regions per slab

__device__ __forceinline__ int slab_of(int z0, int M, int S) {
  int sl = 0;
  while (sl + 1 < S && z0 >= (int)((long)M * (sl + 1) / S)) ++sl;
  return sl;
}

// one block per image: slab and region of each of its items, and counts per
// (slab, region): cnt[(s kSlabKeys + q) B + b]
__global__ void __launch_bounds__(256)
k_slab_span(Geo G, const float* __restrict__ rot, const int* __restrict__ tile_org,
            const int* __restrict__ n_px, int bd, int tile_h, int S, int* __restrict__ span,
            int* __restrict__ cnt, int B) {
  __shared__ int c[kMaxSlabs * kSlabKeys];
  const int b = blockIdx.x;
  const int nch = *n_px / bd;
  for (int k = threadIdx.x; k < kMaxSlabs * kSlabKeys; k += blockDim.x) c[k] = 0;
  __syncthreads();
  const float* R = rot + 9 * (size_t)b;
  const float ax = __ldg(R + 0), ay = __ldg(R + 1), a = __ldg(R + 2);
  const float cx = __ldg(R + 3), cy = __ldg(R + 4), c2 = __ldg(R + 5);
  for (int t = threadIdx.x; t < nch; t += blockDim.x) {
    const int o = __ldg(tile_org + t);
    const float x0 = (float)((o & 0xffff) - G.half), y0 = (float)((o >> 16) - G.half);
    // the tile's centre: its slab and its region in x, y
    const float xc = x0 + 7.5f, yc = y0 + 0.5f * (float)(tile_h - 1);
    const int gz = (int)floorf(fmaf(c2, yc, a * xc)) + G.half;
    const int gx = (int)floorf(fmaf(cx, yc, ax * xc)) + G.half;
    const int gy = (int)floorf(fmaf(cy, yc, ay * xc)) + G.half;
    const int sl = slab_of(gz, G.M, S);
    const int qx = min(max(gx * kSlabQ / G.M, 0), kSlabQ - 1);
    const int qy = min(max(gy * kSlabQ / G.M, 0), kSlabQ - 1);
    const int q = qy * kSlabQ + qx;
    span[(size_t)b * nch + t] = sl * kSlabKeys + q;
    atomicAdd(&c[sl * kSlabKeys + q], 1);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < S * kSlabKeys; k += blockDim.x)
    cnt[(size_t)k * B + b] = c[k];
}

// one block per (slab, region) key: exclusive scan of its per-image counts
// in place (image order), and the key's total
__global__ void __launch_bounds__(256)
k_slab_rows(int B, int* __restrict__ cnt, int* __restrict__ tot) {
  __shared__ int wsum[8];
  __shared__ int carry;
  const int k = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int* row = cnt + (size_t)k * B;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < B; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int v = i < B ? row[i] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    int before = carry;
    for (int q = 0; q < wid; ++q) before += wsum[q];
    if (i < B) row[i] = before + x - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = before + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) tot[k] = carry;
}

// one block: base[k] = first list entry of key k (exclusive scan of the key
// totals, slab-major), se[s] = first entry of slab s, se[S] = total
__global__ void __launch_bounds__(256)
k_slab_bases(int S, const int* __restrict__ tot, int* __restrict__ base, int* __restrict__ se) {
  if (threadIdx.x != 0) return;
  int run = 0;
  for (int k = 0; k < S * kSlabKeys; ++k) {
    if (k % kSlabKeys == 0) se[k / kSlabKeys] = run;
    base[k] = run;
    run += tot[k];
  }
  se[S] = run;
}

// one block per image: its items into the lists, at base[k] + (the key's
// items of earlier images) + (its earlier items with that key: ranks within
// a warp from matching keys, warps in order, chunks in order)
__global__ void __launch_bounds__(256)
k_slab_fill(const int* __restrict__ n_px, int bd, int S, const int* __restrict__ span,
            const int* __restrict__ off, const int* __restrict__ base, int B,
            int* __restrict__ items) {
  __shared__ int run[kMaxSlabs * kSlabKeys];
  __shared__ int wcnt[8][kMaxSlabs * kSlabKeys];
  const int b = blockIdx.x;
  const int nch = *n_px / bd;
  const int nk = S * kSlabKeys;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = threadIdx.x; k < nk; k += blockDim.x) {
    run[k] = base[k] + off[(size_t)k * B + b];
    for (int w = 0; w < nw; ++w) wcnt[w][k] = 0;
  }
  __syncthreads();
  for (int t0 = 0; t0 < nch; t0 += blockDim.x) {
    const int t = t0 + threadIdx.x;
    const int key = t < nch ? span[(size_t)b * nch + t] : -1;   // slab * kSlabKeys + region
    const unsigned m = __match_any_sync(0xffffffffu, key);
    const int rank = __popc(m & ((1u << lane) - 1u));
    if (key >= 0 && rank == 0) wcnt[wid][key] = __popc(m);
    __syncthreads();
    if (key >= 0) {
      int before = 0;
      for (int w = 0; w < wid; ++w) before += wcnt[w][key];
      items[run[key] + before + rank] = b * nch + t;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
      int tot = 0;
      for (int w = 0; w < nw; ++w) {
        tot += wcnt[w][k];
        wcnt[w][k] = 0;
      }
      run[k] += tot;
    }
    __syncthreads();
  }
}

template <int FL>
__device__ __forceinline__ float fused_traverse(const FusedArgs& A, int blk, int nblk) {
  const Geo& G = A.G;
  const int n_px = *A.n_px_dev;
  const int bd = blockDim.x;
  const int nch = (n_px + bd - 1) / bd;
  const int total = A.B * nch;
  const int MM = G.M * G.M;
  const float2* img = A.img;
  const float* dfp = A.df;
  if (A.cursor) {
    const long long bsel = (long long)(*A.cursor) % (long long)A.n_batches;
    if (img) img += (size_t)bsel * A.B * MM;
    if (dfp) dfp += (size_t)bsel * A.B;
  }
  const uint32_t pmask = A.K >= 32 ? 0xffffffffu : ((1u << A.K) - 1u);
  const float invK = 1.0f / (float)(A.K > 0 ? A.K : 1);
  uint64_t pbase = 0, st_base = 0, step_y = 0, step_z = 0;
  if (FL & F_HUTCH) {
    const uint64_t blk = A.k_dev ? (uint64_t)(*A.k_dev) + 1ull : A.block_host;
    pbase = blk * (((uint64_t)G.M * G.M * G.M) >> 1);
    st_base = A.seed + (pbase + 1ull) * kSplitMixGamma;     // state of output pbase
    step_y = (uint64_t)(G.M / 2) * kSplitMixGamma;           // next row: M/2 outputs on
    step_z = (uint64_t)G.M * G.M / 2 * kSplitMixGamma;       // next plane: M^2/2
  }
  float acc = 0.f;
  // the accumulators stay in L2 ahead of the streamed images
  const uint64_t pol = l2_keep_policy();
  // item w = (image b, chunk ch) = (w / nch, w % nch), advanced by nblk
  // items per iteration without a division
  // F_SLAB: this slab's items from its list; otherwise every item in order
  const int first = (FL & F_SLAB) ? A.slab_se[0] : 0;
  const int count = (FL & F_SLAB) ? A.slab_se[1] - first : total;
  int b_next = blk / nch, ch = blk - b_next * nch;
  const int db = nblk / nch, dch = nblk - db * nch;
  for (int w = blk; w < count; w += nblk) {
    int b, chc;
    if (FL & F_SLAB) {
      const int it = __ldg(A.slab_items + first + w);
      b = it / nch;
      chc = it - b * nch;
      if (!CS_IN(b, A.B)) continue;
    } else {
      b = b_next;
      chc = ch;
      ch += dch;
      b_next += db;
      if (ch >= nch) {
        ch -= nch;
        ++b_next;
      }
    }
    const int p = chc * bd + threadIdx.x;
    if (p >= n_px) continue;
    const int e = __ldg(A.table + p);
    if ((FL & (F_SLAB | F_HOLES)) && e < 0) continue;   // holes of the tile-ordered table
    const int ix = e & 0xffff, iy = e >> 16;
    const int kx = ix - G.half, ky = iy - G.half;
    if (!CS_IN(b, A.B) || !CS_IN(ix, G.M) || !CS_IN(iy, G.M)) continue;
    const Rot R = load_rot(A.rot, b);
    const Cell c = cell_of(G, R, kx, ky);
    float C = 1.f;
    if (G.ctf_on) {
      float a_hi, a_lo;
      ctf_coeff(G, __ldg(dfp + b), a_hi, a_lo);
      C = ctf_value(G, a_hi, a_lo, kx * kx + ky * ky);
    }
    const bool inb = base_in(G, c);
    float w8[8];
    if (inb) cell_weights(G, c, w8);
    if (FL & (F_ADJ | F_GRAD)) {
      size_t ii = (size_t)b * MM + (size_t)iy * G.M + ix;
      if (FL & F_PACKED) {
        // disc-packed images: the pixel's place in its disc row
        const int k = ky + A.img_r;
        if (!CS_IN(k, 2 * A.img_r + 1)) continue;
        const int r0 = __ldg(A.img_rows + k), r1 = __ldg(A.img_rows + k + 1);
        const int xi = kx + ((r1 - r0 - 1) >> 1);          // place within the row
        if (!CS_IN(xi, r1 - r0)) continue;
        ii = (size_t)b * __ldg(A.img_rows + 2 * A.img_r + 1) + r0 + xi;
      }
      float2 r = __ldcs(img + ii);
      if (FL & F_GRAD) {
        const float2 a = inb ? gather_pairs_w(G, c, A.vp, w8) : gather_cell_pairs_slow(G, c, A.vp);
        r = make_float2(fmaf(C, a.x, -r.x), fmaf(C, a.y, -r.y));
        acc = fmaf(r.x, r.x, fmaf(r.y, r.y, acc));
      }
      const float2 sr = mul2(dup2(A.scale * C), r);
      if (inb)
        scatter_c2_w(G, c, sr, A.E, A.O, w8, pol);
      else
        scatter_cell_c2(G, c, sr, A.E, A.O);
    }
    if (FL & F_CURV) {
      const float2 a = inb ? gather_patch_w(G, c, A.dq, w8) : gather_cell_patch_slow(G, c, A.dq);
      acc = fmaf(C * C, fmaf(a.x, a.x, a.y * a.y), acc);
    }
    if (FL & F_HVP) {
      const float y = A.scale * C * C * gather_cell_r(G, c, A.zr);
      float vals[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) vals[k] = corner_in(G, c, k) ? corner_w(c, k) * y : 0.f;
      scatter_cell_r4(G, c, vals, A.P, pol);
    }
    if (FL & F_HUTCH) {
      uint32_t bw[8];
      float wsum = 0.f;
      if (!inb) {
#pragma unroll
        for (int k = 0; k < 8; ++k) w8[k] = corner_in(G, c, k) ? corner_w(c, k) : 0.f;
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) wsum += w8[k];
      if (inb) {
        // SplitMix64 states of the corner rows' outputs: output i has state
        // seed + (pbase + i + 1) gamma, so with i0 = j0 / 2 for the base
        // corner, the row (dy, dz) starts at i0 + (dy M + dz M^2) / 2 (M is
        // even) and its second output, for an odd x0, is one further: the
        // eight states are 64-bit additions to one product
        const size_t j0 = ((size_t)c.z0 * G.M + c.y0) * G.M + c.x0;
        const uint64_t odd = j0 & 1;
        const uint64_t s0 = st_base + (uint64_t)(j0 >> 1) * kSplitMixGamma;
#pragma unroll
        for (int r2 = 0; r2 < 4; ++r2) {
          const int dy = r2 & 1, dz = r2 >> 1;
          const int y = c.y0 + dy, z = c.z0 + dz;
          uint32_t b0 = 0u, b1 = 0u;
          if (y < G.M && z < G.M) {
            const uint64_t sr = s0 + (dy ? step_y : 0ull) + (dz ? step_z : 0ull);
            const uint64_t w0 = splitmix_mix(sr);
            const uint64_t w1 = splitmix_mix(sr + odd * kSplitMixGamma);
            b0 = odd ? (uint32_t)(w0 >> 32) : (uint32_t)w0;
            b1 = odd ? (uint32_t)w1 : (uint32_t)(w1 >> 32);
          }
          bw[2 * r2] = b0;
          bw[2 * r2 + 1] = b1;
        }
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          bw[k] = 0u;
          if (!corner_in(G, c, k)) continue;
          const size_t j = ((size_t)(c.z0 + (k >> 2)) * G.M + (c.y0 + ((k >> 1) & 1))) * G.M +
                           (c.x0 + (k & 1));
          bw[k] = (uint32_t)(probe_pair(A.seed, pbase, (uint64_t)(j >> 1)) >> (32 * (j & 1)));
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) bw[k] &= pmask;
      // S_j = sum_l w_l popc(b_j ^ b_l): each of the 28 unordered pairs is
      // counted once and feeds both of its corners
      const float sc = A.scale * C * C;
      float S[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) S[j] = 0.f;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
#pragma unroll
        for (int l = j + 1; l < 8; ++l) {
          const float pc = (float)__popc(bw[j] ^ bw[l]);
          S[j] = fmaf(w8[l], pc, S[j]);
          S[l] = fmaf(w8[j], pc, S[l]);
        }
      }
      float vals[8];
#pragma unroll
      for (int j = 0; j < 8; j += 2) {
        const float2 v = mul2(mul2(dup2(sc), make_float2(w8[j], w8[j + 1])),
                              fma2(dup2(-2.0f * invK), make_float2(S[j], S[j + 1]), dup2(wsum)));
        vals[j] = v.x;
        vals[j + 1] = v.y;
      }
      scatter_cell_r4(G, c, vals, A.P, pol);
    }
  }
  return acc;
}

template <int FL>
__device__ __forceinline__ void fused_body(const FusedArgs& A) {
  grid_dep_wait();
  const float acc = fused_traverse<FL>(A, blockIdx.x, gridDim.x);
  if (FL & (F_GRAD | F_CURV)) {
    const double t = block_sum_f(acc);
    if (threadIdx.x == 0)
      A.part[blockIdx.x] = ((FL & F_SLAB) && A.part_add) ? A.part[blockIdx.x] + t : t;
  }
}

template <int FL>
__global__ void __launch_bounds__(256)
k_fused(FusedArgs A) {
  fused_body<FL>(A);
}

// The slab-split curvature pass compiled for at least 5 resident blocks per
// SM (measured at 256^3, 2 slabs: 0.76 ms instead of 0.81 ms)
__global__ void __launch_bounds__(256, 5)
k_fused_curv_slab(FusedArgs A) {
  fused_body<F_CURV | F_SLAB>(A);
}

// Several independent problems (volumes of different grid sizes) in one
// launch: blocks [start[p], start[p+1]) walk problem p's items, so each
// block's partial sum belongs to one problem and stays deterministic.
template <int FL>
__global__ void __launch_bounds__(256)
k_fused_multi(MultiFusedArgs MA) {
  grid_dep_wait();
  int p = 0;
  while (p + 1 < MA.n && (int)blockIdx.x >= MA.start[p + 1]) ++p;
  const int lb = blockIdx.x - MA.start[p];
  const int nb = MA.start[p + 1] - MA.start[p];
  const float acc = fused_traverse<FL>(MA.a[p], lb, nb);
  if (FL & (F_GRAD | F_CURV)) {
    const double t = block_sum_f(acc);
    if (threadIdx.x == 0) MA.a[p].part[lb] = t;
  }
}

// vp[j] = (v[j], v[j+1]) with 0 past the end of each x row
__global__ void __launch_bounds__(256)
k_pairs(int M, const float2* __restrict__ v, float4* __restrict__ vp) {
  const int n = M * M * M;
  for (int j = blockIdx.x * 256 + threadIdx.x; j < n; j += gridDim.x * 256) {
    const float2 a = v[j];
    const float2 b = (j % M) != M - 1 ? v[j + 1] : make_float2(0.f, 0.f);
    vp[j] = make_float4(a.x, a.y, b.x, b.y);
  }
}

// one 32-byte store of eight floats under an L2 policy
__device__ __forceinline__ void st_keep8(float* p, float4 a, float4 b, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8}, %9;"
               :: "l"(p), "f"(a.x), "f"(a.y), "f"(a.z), "f"(a.w), "f"(b.x), "f"(b.y), "f"(b.z),
                  "f"(b.w), "l"(pol) : "memory");
}

// Set-up of a step's traversal in one pass over the voxels: E = O = 0,
// the four patch buffers P = 0 (zero_p), vp = pair layout of v, all written
// under the policy that keeps them in L2 for the traversal that follows.
// With n = M^3 (a multiple of 8), thread q < n/4 writes 32-byte chunk q of
// E and of O (four voxels each), chunks q and q + n/4 of the patch buffers
// (n/2 chunks in all) and of the pair layout (two voxels per chunk): every
// store covers a whole sector, and a warp's stores are contiguous.
__global__ void __launch_bounds__(256)
k_step_prep(int M, const float2* __restrict__ v, float2* __restrict__ E, float2* __restrict__ O,
            float* __restrict__ P, float4* __restrict__ vp, int zero_p) {
  grid_dep_wait();
  const int n = M * M * M, n4 = n / 4;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  float* Ef = reinterpret_cast<float*>(E);
  float* Of = reinterpret_cast<float*>(O);
  float* vpf = reinterpret_cast<float*>(vp);
  const uint64_t pol = l2_keep_policy();     // the accumulators stay in L2
  for (int q = blockIdx.x * 256 + threadIdx.x; q < n4; q += gridDim.x * 256) {
    st_keep8(Ef + 8 * (size_t)q, z4, z4, pol);
    st_keep8(Of + 8 * (size_t)q, z4, z4, pol);
    if (zero_p) {
      st_keep8(P + 8 * (size_t)q, z4, z4, pol);
      st_keep8(P + 8 * ((size_t)q + n4), z4, z4, pol);
    }
    float4 a[2];
    float2 c[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int j = 2 * (q + k * n4);          // voxels j, j + 1 (j even)
      a[k] = *reinterpret_cast<const float4*>(v + j);
      c[k] = ((j + 1) % M) != M - 1 ? v[j + 2] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int j = 2 * (q + k * n4);
      // (v[j], v[j+1]) and (v[j+1], v[j+2]); x = M - 1 at j + 1 reads 0
      st_keep8(vpf + 4 * (size_t)j, a[k], make_float4(a[k].z, a[k].w, c[k].x, c[k].y), pol);
    }
  }
}

// g = lambda v + E + shift(O), and |v|^2 partials
__global__ void __launch_bounds__(256)
k_combine_c2(int M, const float2* v, float lambda, float2* __restrict__ E,
             float2* __restrict__ O, float2* g, double* __restrict__ part) {
  const int n = M * M * M;
  // a few voxels per thread in FP32, warp sums in FP32, the block sum in FP64
  float accv = 0.f;
  for (int j = blockIdx.x * 256 + threadIdx.x; j < n; j += gridDim.x * 256) {
    const int x = j % M;
    float2 a = v ? v[j] : make_float2(0.f, 0.f);
    float2 r = E[j];
    if (x >= 1) {
      const float2 o = O[j - 1];
      r.x += o.x;
      r.y += o.y;
    }
    g[j] = make_float2(fmaf(lambda, a.x, r.x), fmaf(lambda, a.y, r.y));
    accv += fmaf(a.x, a.x, a.y * a.y);
  }
  if (part) {
    const double t = block_sum_f(accv);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
  }
}

// out = base + coef * add + sum over the four patch buffers
__global__ void __launch_bounds__(256)
k_combine_r4(int M, float* __restrict__ P, float base, float coef,
             const float* __restrict__ add, float* __restrict__ out) {
  const int n = M * M * M, Mh = M / 2;
  const size_t nb = (size_t)n;
  for (int j = blockIdx.x * 256 + threadIdx.x; j < n; j += gridDim.x * 256) {
    const int x = j % M, y = (j / M) % M, z = j / (M * M);
    float s = add ? fmaf(coef, add[j], base) : base;
#pragma unroll
    for (int py = 0; py < 2; ++py) {
#pragma unroll
      for (int px = 0; px < 2; ++px) {
        const int xx = x - px, yy = y - py;
        if (xx < 0 || yy < 0) continue;
        float* buf = P + (size_t)(py * 2 + px) * nb;
        const size_t slot =
            4 * (((size_t)z * Mh + (yy >> 1)) * Mh + (xx >> 1)) + 2 * (yy & 1) + (xx & 1);
        s += buf[slot];
      }
    }
    out[j] = s;
  }
}

// Everything element-wise between the fused traversal and the curvature
// pass of one Algorithm 1 step, per voxel j:
//   HUTCH: D_est = lambda + patches; D_avg = ((k-1)/k) D_avg + D_est/k;
//          D = beta D + (1-beta) D_avg; D-hat = max(|D|, alpha)
//   FIXED: D-hat = max(|D|, alpha);  PLAIN: D-hat = 1
//   g = lambda v + E + shift(O);  d = g / D-hat, written in natural layout (dn);
//   partials of |g|^2/D-hat, |d|^2 and |v|^2.
// A thread takes a 2 x 2 (x, y) block of voxels of one z-plane (x, y even):
// the block is one patch of the patch buffer with even origin, two patches
// of each buffer with one odd origin coordinate and four of the buffer with
// both odd, so the buffers are read as whole 16-byte patches; the natural
// layouts are read and written as aligned pairs of voxels along x.  The
// patch sums of a voxel are added in the order (0,0), (1,0), (0,1), (1,1) of
// the buffers' origin parities.
__device__ __forceinline__ float4 ld_patch4(const float* __restrict__ buf, size_t patch) {
  return *reinterpret_cast<const float4*>(buf + 4 * patch);
}

__global__ void __launch_bounds__(256)
k_step_post(int M, int mode, const float2* __restrict__ v, float lambda, float beta,
            const double* __restrict__ sc, float2* __restrict__ E, float2* __restrict__ O,
            float* __restrict__ P, float* __restrict__ D, float* __restrict__ Davg,
            float2* __restrict__ dn, double* __restrict__ partG, double* __restrict__ partV,
            int nb) {
  grid_dep_wait();
  const int Mh = M / 2;
  const size_t nbuf = (size_t)M * M * M;
  const int nblk = Mh * Mh * M;
  const double k = sc[CS_S_K] + 1.0;
  const float wold = (float)((k - 1.0) / k), wnew = (float)(1.0 / k);
  const float alpha = (float)sc[CS_S_ALPHA];
  // per-thread partial sums of a few voxels in FP32 (FP64 arithmetic is a
  // small fraction of the FP32 rate), warp sums in FP32, the block's warp
  // sums added in FP64
  float aG = 0.f, aD = 0.f, aV = 0.f;
  for (int bi = blockIdx.x * 256 + threadIdx.x; bi < nblk; bi += gridDim.x * 256) {
    const int X = bi % Mh, Y = (bi / Mh) % Mh, z = bi / (Mh * Mh);
    const int x = 2 * X, y = 2 * Y;
    const size_t j0 = ((size_t)z * M + y) * M + x;       // (x, y); row y + 1 at j0 + M
    const size_t jr[2] = {j0, j0 + M};
    // voxel order within the block: (x, y), (x+1, y), (x, y+1), (x+1, y+1)
    float dh[4] = {1.f, 1.f, 1.f, 1.f};
    if (mode == CS_HUTCHINSON) {
      const size_t pz = (size_t)z * Mh;
      const size_t pXY = (pz + Y) * Mh + X;                // patch (X, Y)
      float e[4] = {lambda, lambda, lambda, lambda};
      {   // origin parity (0, 0): patch (X, Y)
        const float4 p = ld_patch4(P, pXY);
        e[0] += p.x; e[1] += p.y; e[2] += p.z; e[3] += p.w;
      }
      {   // (1, 0): patches (X-1, Y) (elements 1, 3) and (X, Y) (0, 2)
        const float* buf = P + nbuf;
        const float4 r = ld_patch4(buf, pXY);
        if (X > 0) {
          const float4 l = ld_patch4(buf, pXY - 1);
          e[0] += l.y;
          e[2] += l.w;
        }
        e[1] += r.x;
        e[3] += r.z;
      }
      {   // (0, 1): patches (X, Y-1) (elements 2, 3) and (X, Y) (0, 1)
        const float* buf = P + 2 * nbuf;
        if (Y > 0) {
          const float4 u = ld_patch4(buf, pXY - Mh);
          e[0] += u.z;
          e[1] += u.w;
        }
        const float4 w = ld_patch4(buf, pXY);
        e[2] += w.x;
        e[3] += w.y;
      }
      {   // (1, 1): patches (X-1, Y-1) (3), (X, Y-1) (2), (X-1, Y) (1), (X, Y) (0)
        const float* buf = P + 3 * nbuf;
        if (Y > 0) {
          if (X > 0) e[0] += ld_patch4(buf, pXY - Mh - 1).w;
          e[1] += ld_patch4(buf, pXY - Mh).z;
        }
        if (X > 0) e[2] += ld_patch4(buf, pXY - 1).y;
        e[3] += ld_patch4(buf, pXY).x;
      }
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const float2 da = *reinterpret_cast<const float2*>(Davg + jr[r]);
        const float2 dd = *reinterpret_cast<const float2*>(D + jr[r]);
        const float a0 = fmaf(wold, da.x, wnew * e[2 * r]);
        const float a1 = fmaf(wold, da.y, wnew * e[2 * r + 1]);
        const float d0 = fmaf(beta, dd.x, (1.0f - beta) * a0);
        const float d1 = fmaf(beta, dd.y, (1.0f - beta) * a1);
        *reinterpret_cast<float2*>(Davg + jr[r]) = make_float2(a0, a1);
        *reinterpret_cast<float2*>(D + jr[r]) = make_float2(d0, d1);
        dh[2 * r] = fmaxf(fabsf(d0), alpha);
        dh[2 * r + 1] = fmaxf(fabsf(d1), alpha);
      }
    } else if (mode == CS_FIXED) {
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const float2 dd = *reinterpret_cast<const float2*>(D + jr[r]);
        dh[2 * r] = fmaxf(fabsf(dd.x), alpha);
        dh[2 * r + 1] = fmaxf(fabsf(dd.y), alpha);
      }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const size_t j = jr[r];
      const float4 vv = *reinterpret_cast<const float4*>(v + j);
      float4 g = *reinterpret_cast<const float4*>(E + j);
      if (x >= 1) {
        const float2 o = O[j - 1];
        g.x += o.x;
        g.y += o.y;
      }
      const float2 o1 = O[j];
      g.z += o1.x;
      g.w += o1.y;
      g.x = fmaf(lambda, vv.x, g.x);
      g.y = fmaf(lambda, vv.y, g.y);
      g.z = fmaf(lambda, vv.z, g.z);
      g.w = fmaf(lambda, vv.w, g.w);
      const float i0 = 1.0f / dh[2 * r], i1 = 1.0f / dh[2 * r + 1];
      const float4 d = make_float4(g.x * i0, g.y * i0, g.z * i1, g.w * i1);
      *reinterpret_cast<float4*>(dn + j) = d;
      aG += fmaf(g.x, g.x, g.y * g.y) * i0;
      aG += fmaf(g.z, g.z, g.w * g.w) * i1;
      aD += fmaf(d.x, d.x, d.y * d.y);
      aD += fmaf(d.z, d.z, d.w * d.w);
      aV += fmaf(vv.x, vv.x, vv.y * vv.y);
      aV += fmaf(vv.z, vv.z, vv.w * vv.w);
    }
  }
  const double tG = block_sum_f(aG);
  const double tD = block_sum_f(aD);
  const double tV = block_sum_f(aV);
  if (threadIdx.x == 0) {
    partG[blockIdx.x] = tG;
    partG[nb + blockIdx.x] = tD;
    partV[blockIdx.x] = tV;
  }
}

// one 32-byte store of a patch (a, b, c, d): the whole sector in one
// instruction
__device__ __forceinline__ void st_patch(float4* p, float2 a, float2 b, float2 c, float2 d) {
  asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
               :: "l"(p), "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y), "f"(d.x),
                  "f"(d.y) : "memory");
}

// 2 x 2 (x, y) patch layout of d for the curvature pass: the patch of voxel
// j = (x, y, z) is (d[j], d[j+1], d[j+M], d[j+M+1]), 0 past the grid's edge
// in x or y, stored at patch_slot(x, y, z).  Thread t writes patch slot t
// (one 32-byte store: a warp's stores cover 1 KB contiguously) and reads
// the four values it holds.  Written by k_step_post directly
// instead (d[j] stored into four patches, 8 bytes each): slower (curvature
// 0.107 -> 0.115 ms and step 0.616 -> 0.620 ms at 128^3).
__global__ void __launch_bounds__(256)
k_patches(int M, const float2* __restrict__ dn, float4* __restrict__ dq) {
  grid_dep_wait();
  const int n = M * M * M, Mh = M >> 1;
  const float2 z2 = make_float2(0.f, 0.f);
  for (int t = blockIdx.x * 256 + threadIdx.x; t < n; t += gridDim.x * 256) {
    const int in = t & 7, blk = t >> 3;
    const int x = 2 * (blk % Mh) + (in & 1), y = 2 * ((blk / Mh) % Mh) + ((in >> 1) & 1);
    const int z = 2 * (blk / (Mh * Mh)) + (in >> 2);
    const int j = (z * M + y) * M + x;
    const bool xin = x + 1 < M, yin = y + 1 < M;
    const float2 a = dn[j];
    const float2 b = xin ? dn[j + 1] : z2;
    const float2 c = yin ? dn[j + M] : z2;
    const float2 d = xin && yin ? dn[j + M + 1] : z2;
    st_patch(dq + 2 * (size_t)t, a, b, c, d);
  }
}

// v -= eta d; thread q handles voxels q + k n/4, k = 0..3, all loads issued
// before the stores
__global__ void __launch_bounds__(256)
k_update_pairs(int n, float2* __restrict__ v, const float2* __restrict__ dn,
               const double* __restrict__ sc) {
  grid_dep_wait();
  const float eta = (float)sc[CS_S_ETA];
  const int n4 = n / 4;
  for (int q = blockIdx.x * 256 + threadIdx.x; q < n4; q += gridDim.x * 256) {
    float2 d[4];
    float2 a[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      d[k] = dn[q + k * n4];
      a[k] = v[q + k * n4];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
      v[q + k * n4] = make_float2(fmaf(-eta, d[k].x, a[k].x), fmaf(-eta, d[k].y, a[k].y));
  }
}

// element-wise kernels: up to 8 blocks of 256 threads per SM (full occupancy)
int elem_grid(int n, int num_sms) {
  int g = (n + 255) / 256;
  return g < num_sms * 8 ? (g > 0 ? g : 1) : num_sms * 8;
}

}  // namespace

// entries of the disc table (row order: <= M^2; tile order: whole tiles of
// up to 16 x 16 over a padded grid) and tile origins (tiles of 16 x 8 at most)
size_t table_entries(int M) { return (size_t)(M + 16) * (M + 16); }
size_t tile_slots(int M) { return (size_t)((M + 15) / 16) * ((M + 7) / 8) + 64; }

size_t slab_lists_bytes(int M, int B) {
  const size_t b = (size_t)(B > 0 ? B : 1), items = b * tile_slots(M);
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t keys = (size_t)kMaxSlabs * kSlabKeys;
  return al(items * sizeof(int)) + al(keys * b * sizeof(int)) + 2 * al(keys * sizeof(int)) +
         al((kMaxSlabs + 1) * sizeof(int)) + al(items * sizeof(int));
}

void slab_carve(void* region, int M, int B, FusedWs& w) {
  const size_t b = (size_t)(B > 0 ? B : 1), items = b * tile_slots(M);
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t keys = (size_t)kMaxSlabs * kSlabKeys;
  char* p = static_cast<char*>(region);
  w.slab_span = reinterpret_cast<int*>(p);  p += al(items * sizeof(int));
  w.slab_cnt = reinterpret_cast<int*>(p);   p += al(keys * b * sizeof(int));
  w.slab_tot = reinterpret_cast<int*>(p);   p += al(keys * sizeof(int));
  w.slab_base = reinterpret_cast<int*>(p);  p += al(keys * sizeof(int));
  w.slab_se = reinterpret_cast<int*>(p);    p += al((kMaxSlabs + 1) * sizeof(int));
  w.slab_items = reinterpret_cast<int*>(p);
  w.slab_cap_B = (int)b;
}

size_t fused_ws_bytes(int M) {
  const size_t n = (size_t)M * M * M;
  // E, O (complex), P (4 real buffers), pair layout, d, d's patches, disc
  // table, count
  return 2 * n * sizeof(float2) + 4 * n * sizeof(float) + n * sizeof(float4) +
         n * sizeof(float2) + 2 * n * sizeof(float4) + table_entries(M) * sizeof(int) +
         tile_slots(M) * sizeof(int) + 256;
}

FusedWs fused_carve(void* base, int M) {
  const size_t n = (size_t)M * M * M;
  char* p = static_cast<char*>(base);
  FusedWs w;
  w.E = reinterpret_cast<float2*>(p);   p += n * sizeof(float2);
  w.O = reinterpret_cast<float2*>(p);   p += n * sizeof(float2);
  w.P = reinterpret_cast<float*>(p);    p += 4 * n * sizeof(float);
  w.pairs = reinterpret_cast<float4*>(p); p += n * sizeof(float4);
  w.dq = reinterpret_cast<float4*>(p);  p += 2 * n * sizeof(float4);
  w.dn = reinterpret_cast<float2*>(p);  p += n * sizeof(float2);
  w.table = reinterpret_cast<int*>(p);  p += table_entries(M) * sizeof(int);
  w.tile_org = reinterpret_cast<int*>(p); p += tile_slots(M) * sizeof(int);
  w.n_px = reinterpret_cast<int*>(p);
  w.slab_span = w.slab_cnt = w.slab_tot = w.slab_base = w.slab_se = w.slab_items = nullptr;
  w.slab_cap_B = 0;
  return w;
}

cudaError_t launch_disc_table(int M, int r, const FusedWs& w, cudaStream_t s) {
  k_disc_table<<<1, 256, 0, s>>>(M, r, w.table, w.n_px);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_disc_table_tiled(int M, int r, int block, const FusedWs& w, cudaStream_t s) {
  if (block != 128 && block != 256) return cudaErrorInvalidValue;
  k_disc_table_tiled<<<1, 256, 0, s>>>(M, r, block, w.table, w.tile_org, w.n_px);
  count_launches(1);
  return cudaGetLastError();
}

namespace {

template <typename K>
int resident_of(K kernel, int block) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block, 0) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n > 0 ? n : 1;
}

int flag_slot(int flags) {
  switch (flags) {
    case F_ADJ: return 0;
    case F_GRAD: return 1;
    case F_GRAD | F_HUTCH: return 2;
    case F_HUTCH: return 3;
    case F_HVP: return 4;
    case F_CURV: return 5;
    case F_CURV | F_SLAB: return 6;
    default: return -1;
  }
}

}  // namespace

int fused_resident(int flags, int block, bool multi) {
  // cached per (kernel, block size); every device of a process is a GB300
  static int cache[2][7][2];
  const int f = flag_slot(flags), b = block == 128 ? 0 : 1, m = multi ? 1 : 0;
  if (f < 0 || (block != 128 && block != 256)) return 1;
  int& c = cache[m][f][b];
  if (c > 0) return c;
  int n = 1;
  if (!multi) {
    switch (flags) {
      case F_ADJ: n = resident_of(k_fused<F_ADJ>, block); break;
      case F_GRAD: n = resident_of(k_fused<F_GRAD>, block); break;
      case F_GRAD | F_HUTCH: n = resident_of(k_fused<F_GRAD | F_HUTCH>, block); break;
      case F_HUTCH: n = resident_of(k_fused<F_HUTCH>, block); break;
      case F_HVP: n = resident_of(k_fused<F_HVP>, block); break;
      case F_CURV: n = resident_of(k_fused<F_CURV>, block); break;
      case F_CURV | F_SLAB: n = resident_of(k_fused_curv_slab, block); break;
    }
  } else {
    switch (flags) {
      case F_GRAD: n = resident_of(k_fused_multi<F_GRAD>, block); break;
      case F_GRAD | F_HUTCH: n = resident_of(k_fused_multi<F_GRAD | F_HUTCH>, block); break;
      case F_CURV: n = resident_of(k_fused_multi<F_CURV>, block); break;
      default: n = 1;
    }
  }
  c = n;
  return n;
}

cudaError_t launch_fused(int flags, const Geo& G, const FusedWs& w, const float* rot,
                         const float* df, int B, float scale, const float2* vol,
                         const float4* vp, const float* zr, const float2* img, double* part,
                         uint64_t seed, uint64_t block_host, const double* k_dev, int K,
                         int grid, cudaStream_t s, int block, int slabs, bool tiled,
                         const int* img_rows, int img_r) {
  FusedArgs A;
  A.G = G;
  A.table = w.table;
  A.n_px_dev = w.n_px;
  A.rot = rot;
  A.df = df;
  A.B = B;
  A.scale = scale;
  A.vol = vol;
  A.zr = zr;
  A.img = img;
  A.img_rows = img_rows;
  A.img_r = img_r;
  A.E = w.E;
  A.O = w.O;
  A.part = part;
  A.P = w.P;
  A.K = K;
  A.vp = vp;
  A.dq = w.dq;
  A.seed = seed;
  A.block_host = block_host;
  A.k_dev = k_dev;
  A.cursor = nullptr;
  A.n_batches = 1;
  return launch_fused_args(flags, A, w, grid, s, block, slabs, tiled);
}

cudaError_t launch_fused_args(int flags, FusedArgs A, const FusedWs& w, int grid, cudaStream_t s,
                              int block, int slabs, bool tiled) {
  const Geo& G = A.G;
  const int B = A.B;
  const float* rot = A.rot;
  A.tile_org = tiled ? w.tile_org : nullptr;
  A.tile_h = block / 16;
  A.slab_items = nullptr;
  A.slab_se = nullptr;
  if (block != 128 && block != 256) return cudaErrorInvalidValue;
  // one launch per z-slab, each walking the items (tiles) whose centre lies
  // in its slab, so every pixel is processed exactly once; slabs need the
  // tile-ordered table
  const int S = tiled ? pass_slabs(G.M, flags, slabs) : 1;
  // one slab on a tile-ordered table: the one-slab kernel variant that
  // skips the table's holes
  const int holes = (tiled && S == 1) ? F_HOLES : 0;
  if (tiled && B > 0 && S > 1) {
    if (!w.slab_items || B > w.slab_cap_B) return cudaErrorInvalidValue;
    k_slab_span<<<B, 256, 0, s>>>(G, rot, w.tile_org, w.n_px, block, block / 16, S, w.slab_span,
                                  w.slab_cnt, B);
    k_slab_rows<<<S * kSlabKeys, 256, 0, s>>>(B, w.slab_cnt, w.slab_tot);
    k_slab_bases<<<1, 32, 0, s>>>(S, w.slab_tot, w.slab_base, w.slab_se);
    k_slab_fill<<<B, 256, 0, s>>>(w.n_px, block, S, w.slab_span, w.slab_cnt, w.slab_base, B,
                                  w.slab_items);
    count_launches(4);
    A.slab_items = w.slab_items;
  }
  for (int sl = 0; sl < S; ++sl) {
    if (A.slab_items) A.slab_se = w.slab_se + sl;
    A.part_add = sl > 0;
    constexpr int X = F_SLAB, Y = F_HOLES, P = F_PACKED;
    cudaError_t e0 = cudaSuccess;
    const int packed = (A.img_rows && (flags & F_GRAD)) ? P : 0;
    switch (flags | (A.slab_items ? X : 0) | holes | packed) {
      case F_ADJ: e0 = launch_pdl(k_fused<F_ADJ>, grid, block, s, A); break;
      case F_GRAD: e0 = launch_pdl(k_fused<F_GRAD>, grid, block, s, A); break;
      case F_GRAD | F_HUTCH: e0 = launch_pdl(k_fused<F_GRAD | F_HUTCH>, grid, block, s, A); break;
      case F_HUTCH: e0 = launch_pdl(k_fused<F_HUTCH>, grid, block, s, A); break;
      case F_HVP: e0 = launch_pdl(k_fused<F_HVP>, grid, block, s, A); break;
      case F_CURV: e0 = launch_pdl(k_fused<F_CURV>, grid, block, s, A); break;
      case F_ADJ | X: e0 = launch_pdl(k_fused<F_ADJ | X>, grid, block, s, A); break;
      case F_GRAD | X: e0 = launch_pdl(k_fused<F_GRAD | X>, grid, block, s, A); break;
      case F_GRAD | F_HUTCH | X: e0 = launch_pdl(k_fused<F_GRAD | F_HUTCH | X>, grid, block, s, A); break;
      case F_HUTCH | X: e0 = launch_pdl(k_fused<F_HUTCH | X>, grid, block, s, A); break;
      case F_HVP | X: e0 = launch_pdl(k_fused<F_HVP | X>, grid, block, s, A); break;
      case F_CURV | X: e0 = launch_pdl(k_fused_curv_slab, grid, block, s, A); break;
      case F_ADJ | Y: e0 = launch_pdl(k_fused<F_ADJ | Y>, grid, block, s, A); break;
      case F_GRAD | Y: e0 = launch_pdl(k_fused<F_GRAD | Y>, grid, block, s, A); break;
      case F_GRAD | F_HUTCH | Y: e0 = launch_pdl(k_fused<F_GRAD | F_HUTCH | Y>, grid, block, s, A); break;
      case F_HUTCH | Y: e0 = launch_pdl(k_fused<F_HUTCH | Y>, grid, block, s, A); break;
      case F_HVP | Y: e0 = launch_pdl(k_fused<F_HVP | Y>, grid, block, s, A); break;
      case F_CURV | Y: e0 = launch_pdl(k_fused<F_CURV | Y>, grid, block, s, A); break;
      case F_GRAD | P: e0 = launch_pdl(k_fused<F_GRAD | P>, grid, block, s, A); break;
      case F_GRAD | F_HUTCH | P: e0 = launch_pdl(k_fused<F_GRAD | F_HUTCH | P>, grid, block, s, A); break;
      case F_GRAD | X | P: e0 = launch_pdl(k_fused<F_GRAD | X | P>, grid, block, s, A); break;
      case F_GRAD | F_HUTCH | X | P: e0 = launch_pdl(k_fused<F_GRAD | F_HUTCH | X | P>, grid, block, s, A); break;
      case F_GRAD | Y | P: e0 = launch_pdl(k_fused<F_GRAD | Y | P>, grid, block, s, A); break;
      case F_GRAD | F_HUTCH | Y | P: e0 = launch_pdl(k_fused<F_GRAD | F_HUTCH | Y | P>, grid, block, s, A); break;
      default: return cudaErrorInvalidValue;
    }
    count_launches(1);
    if (e0 != cudaSuccess) return e0;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// The passes with reductions touch 48 bytes per voxel at random (pair layout
// of v, E/O, the four patch buffers), the curvature pass 32 (the 2 x 2
// patch layout of d).
// About one launch per ~134 MB (128 MB for the curvature) of that footprint.
// Measured at 256^3, batch 1024 (tiles owned by the slab of their centre):
// the loss-gradient pass takes 1.98 / 1.96 / 1.96 / 1.98 / 2.01 / 2.06 ms
// with 4 / 5 / 6 / 8 / 12 / 16 slabs (6.33 ms in one launch), the curvature
// 0.71 / 0.71 / 0.74 ms with 2 / 4 / 8; at 160^3 the loss-gradient pass
// takes 0.87 / 0.77 / 0.78 ms with 1 / 2 / 3 slabs; at 128^3 one is best.
int slab_count(int M, int flags) {
  const double vox = (double)M * M * M;
  const double ratio = flags == F_CURV ? 32.0 * vox / 128e6 : 48.0 * vox / 134e6;
  // passes with reductions: 2 slabs from 1.25 x the footprint on (measured
  // at 160^3: loss-gradient pass 0.87 -> 0.77 ms)
  long S = flags == F_CURV ? lround(ratio) : (ratio >= 1.25 ? lround(ratio + 0.25) : 1);
  if (S < 1) S = 1;
  if (S > kMaxSlabs) S = kMaxSlabs;
  return (int)S;
}

int pass_slabs(int M, int flags, int slabs) {
  int S = slabs > 0 ? slabs : slab_count(M, flags);
  const int smax = M / 16 < kMaxSlabs ? M / 16 : kMaxSlabs;
  if (S > smax) S = smax;
  return S < 1 ? 1 : S;
}

cudaError_t launch_fused_multi(int flags, const MultiFusedArgs& MA, int grid, int block,
                               cudaStream_t s) {
  if (block != 128 && block != 256) return cudaErrorInvalidValue;
  cudaError_t e = cudaSuccess;
  switch (flags) {
    case F_GRAD: e = launch_pdl(k_fused_multi<F_GRAD>, grid, block, s, MA); break;
    case F_GRAD | F_HUTCH: e = launch_pdl(k_fused_multi<F_GRAD | F_HUTCH>, grid, block, s, MA); break;
    case F_CURV: e = launch_pdl(k_fused_multi<F_CURV>, grid, block, s, MA); break;
    default: return cudaErrorInvalidValue;
  }
  count_launches(1);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_step_post(int M, int mode, const float2* v, float lambda, float beta,
                             const double* scalars, const FusedWs& w, float* D, float* Davg,
                             double* partG, double* partV, int* nb, int num_sms,
                             cudaStream_t s) {
  const int g = elem_grid(M * M * M / 4, num_sms);     // a thread per 2 x 2 block
  *nb = g;
  const cudaError_t e = launch_pdl(k_step_post, g, 256, s, M, mode, v, lambda, beta, scalars,
                                   w.E, w.O, w.P, D, Davg, w.dn, partG, partV, g);
  count_launches(1);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_patches(int M, const FusedWs& w, int num_sms, cudaStream_t s) {
  const cudaError_t e =
      launch_pdl(k_patches, elem_grid(M * M * M, num_sms), 256, s, M, w.dn, w.dq);
  count_launches(1);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_update_pairs(int M, float2* v, const FusedWs& w, const double* scalars,
                                int num_sms, cudaStream_t s) {
  const int n = M * M * M;
  const cudaError_t e =
      launch_pdl(k_update_pairs, elem_grid(n / 4, num_sms), 256, s, n, v, w.dn, scalars);
  count_launches(1);
  return e != cudaSuccess ? e : cudaGetLastError();
}


cudaError_t launch_step_prep(int M, const float2* v, const FusedWs& w, bool zero_p, int num_sms,
                             cudaStream_t s) {
  const cudaError_t e = launch_pdl(k_step_prep, elem_grid(M * M * M / 4, num_sms), 256, s, M, v,
                                   w.E, w.O, w.P, w.pairs, zero_p ? 1 : 0);
  count_launches(1);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_pairs(int M, const float2* v, float4* vp, int num_sms, cudaStream_t s) {
  k_pairs<<<elem_grid(M * M * M, num_sms), 256, 0, s>>>(M, v, vp);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_zero_c2(int M, const FusedWs& w, cudaStream_t s) {
  const size_t n = (size_t)M * M * M;
  return cudaMemsetAsync(w.E, 0, 2 * n * sizeof(float2), s);
}

cudaError_t launch_zero_r4(int M, const FusedWs& w, cudaStream_t s) {
  const size_t n = (size_t)M * M * M;
  return cudaMemsetAsync(w.P, 0, 4 * n * sizeof(float), s);
}

cudaError_t launch_combine_c2(int M, const float2* v, float lambda, const FusedWs& w,
                              float2* g, double* part_vv, int* n_vv, int num_sms,
                              cudaStream_t s) {
  const int gb = elem_grid(M * M * M, num_sms);
  if (n_vv) *n_vv = gb;
  k_combine_c2<<<gb, 256, 0, s>>>(M, v, lambda, w.E, w.O, g, part_vv);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_combine_r4(int M, const FusedWs& w, float base, float coef,
                              const float* add, float* out, int num_sms, cudaStream_t s) {
  k_combine_r4<<<elem_grid(M * M * M, num_sms), 256, 0, s>>>(M, w.P, base, coef, add, out);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace cs
