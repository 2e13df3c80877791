// Tile engine: the scatter-heavy passes of the hot path with their adjoint
// accumulation in shared memory instead of global atomics.
//
// The volume grid is cut into kT^3 tiles.  A binning pass lists, per tile
// and in image order, the images whose central slice (Fourier slice theorem,
// Section 2.1) can reach the tile.  A work item is (tile, up to kImgPerItem
// consecutive listed images); persistent CTAs take items from a global
// counter.  For each item the CTA stages the tile plus a one-voxel halo of
// the gathered operand (volume, probe words or real vector) in shared
// memory, zeroes a shared accumulator for the tile, and each warp walks the
// pixels of one image whose interpolation cell touches the tile: the rows of
// the image that cross the tile are found from the tile's box, each row's
// pixel interval from the three slab constraints, and every candidate pixel
// is then tested exactly with the same single-precision sample point as
// every other kernel of the library.  A pixel whose cell straddles tiles is
// processed by each of them, and each adds only the corners it owns, so every
// (pixel, corner) contribution is added exactly once.  Per-pixel scalar sums
// (loss, curvature) are counted only in the tile holding the pixel's base
// corner.  At the end of the item the accumulator is added to global memory
// once per touched voxel.
//
// Operations: OP_ADJOINT (P^* C y), OP_LOSS_GRAD (Eq. optim cp gradient +
// loss), OP_HVP (Eq. hessian), OP_HUTCH (Eq. hutch, bit-packed probes),
// OP_CURVATURE (|C P d|^2 of the Armijo step).
#include "tiles.h"

namespace cs {

namespace {

constexpr int kH = kT + 2;              // halo edge
constexpr int kTileThreads = 512;
constexpr int kWarps = kTileThreads / 32;

template <int OP> struct OpTraits;
template <> struct OpTraits<OP_ADJOINT> {
  using Halo = float; using Acc = float2;
  static constexpr bool kGather = false, kScatter = true, kSum = false;
};
template <> struct OpTraits<OP_LOSS_GRAD> {
  using Halo = float2; using Acc = float2;
  static constexpr bool kGather = true, kScatter = true, kSum = true;
};
template <> struct OpTraits<OP_HVP> {
  using Halo = float; using Acc = float;
  static constexpr bool kGather = true, kScatter = true, kSum = false;
};
template <> struct OpTraits<OP_HUTCH> {
  using Halo = uint32_t; using Acc = float;
  static constexpr bool kGather = true, kScatter = true, kSum = false;
};
template <> struct OpTraits<OP_CURVATURE> {
  using Halo = float2; using Acc = float;
  static constexpr bool kGather = true, kScatter = false, kSum = true;
};

template <int OP>
constexpr size_t smem_bytes() {
  using T = OpTraits<OP>;
  return (T::kGather ? sizeof(typename T::Halo) * kH * kH * kH : 0) +
         (T::kScatter ? sizeof(typename T::Acc) * kT * kT * kT : 0);
}

__device__ __forceinline__ bool in_box(int v, int lo, int hi) { return v >= lo && v <= hi; }

__device__ __forceinline__ int isqrt_floor(int n) {
  int r = (int)sqrtf((float)n);
  while (r * r > n) --r;
  while ((r + 1) * (r + 1) <= n) ++r;
  return r;
}

// Conservative test: can the disc slice of rotation R reach the box
// [lo, hi]^3 (index space)?  Plane through the centre c with normal row 2
// of R, and distance from c to the box at most r + 1.
__device__ __forceinline__ bool slice_meets_box(const float* R, float3 lo, float3 hi,
                                                float c, float rr) {
  const float nx = R[6], ny = R[7], nz = R[8];
  const float bx = 0.5f * (lo.x + hi.x) - c, by = 0.5f * (lo.y + hi.y) - c,
              bz = 0.5f * (lo.z + hi.z) - c;
  const float hx = 0.5f * (hi.x - lo.x), hy = 0.5f * (hi.y - lo.y), hz = 0.5f * (hi.z - lo.z);
  const float d = fabsf(nx * bx + ny * by + nz * bz);
  const float reach = fabsf(nx) * hx + fabsf(ny) * hy + fabsf(nz) * hz + 0.05f;
  if (d > reach) return false;
  const float ex = fmaxf(0.f, fmaxf(lo.x - c, c - hi.x));
  const float ey = fmaxf(0.f, fmaxf(lo.y - c, c - hi.y));
  const float ez = fmaxf(0.f, fmaxf(lo.z - c, c - hi.z));
  return ex * ex + ey * ey + ez * ez <= (rr + 1.0f) * (rr + 1.0f);
}

// One warp per tile: list the images whose slice can reach the tile, in
// image order (ballot + popcount keeps the order deterministic).
__global__ void __launch_bounds__(256)
k_bin(Geo G, const float* __restrict__ rot, int B, int tpa, int n_tiles,
      int* __restrict__ count, int* __restrict__ list, int stride) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n_tiles) return;
  const int tx = warp % tpa, ty = (warp / tpa) % tpa, tz = warp / (tpa * tpa);
  const float pad = G.interp ? 1.0f : 0.5f;
  // index-space box of sample points whose cell (or nearest voxel) is in the tile
  const float3 lo = make_float3(tx * kT - pad, ty * kT - pad, tz * kT - pad);
  const float3 hi = make_float3(tx * kT + kT - 1 + (G.interp ? 1.0f : 0.5f),
                                ty * kT + kT - 1 + (G.interp ? 1.0f : 0.5f),
                                tz * kT + kT - 1 + (G.interp ? 1.0f : 0.5f));
  const float rr = sqrtf((float)G.r2max);
  int n = 0;
  for (int base = 0; base < B; base += 32) {
    const int b = base + lane;
    bool hit = false;
    if (b < B) {
      float R[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) R[i] = __ldg(rot + 9 * (size_t)b + i);
      hit = slice_meets_box(R, lo, hi, (float)G.half, rr);
    }
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    if (hit) list[(size_t)warp * stride + n + __popc(m & ((1u << lane) - 1u))] = b;
    n += __popc(m);
  }
  if (lane == 0) count[warp] = n;
}

// Exclusive prefix of per-tile item counts; item_start[n_tiles] = total.
__global__ void __launch_bounds__(1024)
k_items(const int* __restrict__ count, int n_tiles, int per_item, int* __restrict__ item_start,
        int* __restrict__ queue) {
  __shared__ int sums[1024];
  const int t = threadIdx.x;
  const int chunk = (n_tiles + blockDim.x - 1) / blockDim.x;
  const int a = t * chunk, e = min(n_tiles, a + chunk);
  int s = 0;
  for (int i = a; i < e; ++i) s += (count[i] + per_item - 1) / per_item;
  sums[t] = s;
  __syncthreads();
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {
    int v = t >= off ? sums[t - off] : 0;
    __syncthreads();
    sums[t] += v;
    __syncthreads();
  }
  int run = sums[t] - s;
  for (int i = a; i < e; ++i) {
    item_start[i] = run;
    run += (count[i] + per_item - 1) / per_item;
  }
  if (t == blockDim.x - 1) {
    item_start[n_tiles] = sums[t];
    *queue = 0;
  }
}

template <typename T>
__device__ __forceinline__ T load_or_zero(const T* p, bool ok) {
  return ok ? __ldg(p) : T{};
}
template <>
__device__ __forceinline__ float2 load_or_zero<float2>(const float2* p, bool ok) {
  return ok ? __ldg(p) : make_float2(0.f, 0.f);
}

__device__ __forceinline__ void acc_add(float* a, float v) { atomicAdd(a, v); }
__device__ __forceinline__ void acc_add(float2* a, float2 v) {
  atomicAdd(&a->x, v.x);
  atomicAdd(&a->y, v.y);
}
__device__ __forceinline__ bool nonzero(float v) { return v != 0.0f; }
__device__ __forceinline__ bool nonzero(float2 v) { return v.x != 0.0f || v.y != 0.0f; }
__device__ __forceinline__ void global_add(float* p, float v) { atomicAdd(p, v); }
__device__ __forceinline__ void global_add(float2* p, float2 v) { atomicAdd(p, v); }

// Corner c = (dx, dy, dz) of a pixel's interpolation cell, relative to the
// halo origin (tile origin - 1): weight, halo index, accumulator index and
// whether the tile owns the corner (inside the tile and the grid).
template <int I>
struct Corners {
  static constexpr int N = I ? 8 : 1;
  int hx, hy, hz, gx0, gy0, gz0, M;
  float tx, ty, tz;
  __device__ __forceinline__ Corners(int hx_, int hy_, int hz_, float tx_, float ty_, float tz_,
                                     int ax, int ay, int az, int M_)
      : hx(hx_), hy(hy_), hz(hz_), gx0(ax - 1 + hx_), gy0(ay - 1 + hy_), gz0(az - 1 + hz_),
        M(M_), tx(tx_), ty(ty_), tz(tz_) {}
  __device__ __forceinline__ float w(int c) const {
    if (!I) return 1.0f;
    const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
    return (dx ? tx : 1.f - tx) * (dy ? ty : 1.f - ty) * (dz ? tz : 1.f - tz);
  }
  __device__ __forceinline__ int halo(int c) const {
    const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
    return ((hz + dz) * kH + (hy + dy)) * kH + (hx + dx);
  }
  __device__ __forceinline__ int acc(int c) const {
    const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
    return ((hz + dz - 1) * kT + (hy + dy - 1)) * kT + (hx + dx - 1);
  }
  __device__ __forceinline__ bool mine(int c) const {
    const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
    const int X = hx + dx, Y = hy + dy, Z = hz + dz;
    return X >= 1 && X <= kT && Y >= 1 && Y <= kT && Z >= 1 && Z <= kT && gx0 + dx < M &&
           gy0 + dy < M && gz0 + dz < M;
  }
};

template <int OP, int I>
__global__ void __launch_bounds__(kTileThreads, 2)
k_tile(TileArgs A) {
  using Tr = OpTraits<OP>;
  using HaloT = typename Tr::Halo;
  using AccT = typename Tr::Acc;
  constexpr bool kGather = Tr::kGather && !(OP == OP_HUTCH && I == 0);
  extern __shared__ __align__(16) unsigned char smem[];
  HaloT* halo = reinterpret_cast<HaloT*>(smem);
  AccT* acc = reinterpret_cast<AccT*>(smem + (Tr::kGather ? sizeof(HaloT) * kH * kH * kH : 0));
  __shared__ int s_item;

  const Geo& G = A.G;
  const int M = G.M, half = G.half;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n_items = A.item_start[A.n_tiles];
  const uint32_t pmask = A.K >= 32 ? 0xffffffffu : ((1u << A.K) - 1u);
  const float invK = 1.0f / (float)(A.K > 0 ? A.K : 1);
  const int r2 = G.r2max;
  const int r = isqrt_floor(r2);

  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(A.queue, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= n_items) break;
    // tile of the item: last t with item_start[t] <= item
    int lo_t = 0, hi_t = A.n_tiles - 1;
    while (lo_t < hi_t) {
      const int mid = (lo_t + hi_t + 1) >> 1;
      if (__ldg(A.item_start + mid) <= item) lo_t = mid; else hi_t = mid - 1;
    }
    const int t = lo_t;
    const int seg = item - __ldg(A.item_start + t);
    const int cnt = __ldg(A.tile_count + t);
    const int i_beg = seg * kImgPerItem, i_end = min(cnt, i_beg + kImgPerItem);
    const int tpa = A.tpa;
    const int ax = (t % tpa) * kT, ay = ((t / tpa) % tpa) * kT, az = (t / (tpa * tpa)) * kT;

    if (kGather) {
      const HaloT* src = reinterpret_cast<const HaloT*>(A.src);
      for (int i = threadIdx.x; i < kH * kH * kH; i += kTileThreads) {
        const int hx = i % kH, hy = (i / kH) % kH, hz = i / (kH * kH);
        const int gx = ax - 1 + hx, gy = ay - 1 + hy, gz = az - 1 + hz;
        const bool ok = (unsigned)gx < (unsigned)M && (unsigned)gy < (unsigned)M &&
                        (unsigned)gz < (unsigned)M;
        halo[i] = load_or_zero(src + ((size_t)(ok ? gz : 0) * M + (ok ? gy : 0)) * M + (ok ? gx : 0), ok);
      }
    }
    if (Tr::kScatter) {
      for (int i = threadIdx.x; i < kT * kT * kT; i += kTileThreads) acc[i] = AccT{};
    }
    __syncthreads();

    float part = 0.f;
    for (int ii = i_beg + warp; ii < i_end; ii += kWarps) {
      const int b = __ldg(A.tile_list + (size_t)t * A.list_stride + ii);
      const float* Rp = A.rot + 9 * (size_t)b;
      const float ux = __ldg(Rp + 0), uy = __ldg(Rp + 1), uz = __ldg(Rp + 2);
      const float wx = __ldg(Rp + 3), wy = __ldg(Rp + 4), wz = __ldg(Rp + 5);
      float a_hi = 0.f, a_lo = 0.f;
      if (G.ctf_on) ctf_coeff(G, __ldg(A.df + b), a_hi, a_lo);
      // box of admissible sample points (index space), as in k_bin
      const float pad_lo = I ? 1.0f : 0.5f, pad_hi = I ? 1.0f : 0.5f;
      const float lox = ax - pad_lo, loy = ay - pad_lo, loz = az - pad_lo;
      const float hix = ax + kT - 1 + pad_hi, hiy = ay + kT - 1 + pad_hi, hiz = az + kT - 1 + pad_hi;
      const float hf = (float)half;
      // rows: ky = (s - c) . w over the box
      const float kymin = fminf(wx * (lox - hf), wx * (hix - hf)) +
                          fminf(wy * (loy - hf), wy * (hiy - hf)) +
                          fminf(wz * (loz - hf), wz * (hiz - hf));
      const float kymax = fmaxf(wx * (lox - hf), wx * (hix - hf)) +
                          fmaxf(wy * (loy - hf), wy * (hiy - hf)) +
                          fmaxf(wz * (loz - hf), wz * (hiz - hf));
      const int ky0 = max(-r, (int)floorf(kymin) - 1);
      const int ky1 = min(r, (int)ceilf(kymax) + 1);
      for (int rb = ky0; rb <= ky1; rb += 32) {
        const int ky = rb + lane;
        int n_row = 0, x_lo = 0;
        if (ky <= ky1) {
          const int xr = isqrt_floor(r2 - ky * ky);
          float L = (float)-xr, H = (float)xr;
          const float fy = (float)ky;
          const float base[3] = {fmaf(wx, fy, hf), fmaf(wy, fy, hf), fmaf(wz, fy, hf)};
          const float uu[3] = {ux, uy, uz};
          const float lo3[3] = {lox, loy, loz}, hi3[3] = {hix, hiy, hiz};
          bool empty = false;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            if (fabsf(uu[a]) > 1e-6f) {
              const float inv = 1.0f / uu[a];
              const float t0 = (lo3[a] - base[a]) * inv, t1 = (hi3[a] - base[a]) * inv;
              L = fmaxf(L, fminf(t0, t1));
              H = fminf(H, fmaxf(t0, t1));
            } else if (base[a] < lo3[a] - 1.0f || base[a] > hi3[a] + 1.0f) {
              empty = true;
            }
          }
          if (!empty && L <= H + 2.0f) {
            x_lo = max(-xr, (int)floorf(L) - 1);
            const int x_hi = min(xr, (int)ceilf(H) + 1);
            n_row = max(0, x_hi - x_lo + 1);
          }
        }
        // inclusive scan of row lengths across the warp
        int incl = n_row;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        // lane l takes the contiguous candidate run [l*per, (l+1)*per): lanes of
        // one instruction then sit ~per pixels apart, so their cells (and the
        // shared-memory words they accumulate into) rarely coincide
        const int per = (total + 31) >> 5;
        for (int j = 0; j < per; ++j) {
          const int f = lane * per + j;
          int pos = 0;
#pragma unroll
          for (int s = 16; s >= 1; s >>= 1) {
            const int v = __shfl_sync(0xffffffffu, incl, pos + s - 1);
            if (v <= f) pos += s;
          }
          const int prev = __shfl_sync(0xffffffffu, incl, pos > 0 ? pos - 1 : 0);
          const int xl = __shfl_sync(0xffffffffu, x_lo, pos);
          if (f >= total) continue;
          const int kx = xl + f - (pos > 0 ? prev : 0);
          const int kyp = rb + pos;
          const float fx = (float)kx, fy = (float)kyp;
          const int q = kx * kx + kyp * kyp;
          // ---- exact membership and stencil (same arithmetic as make_stencil)
          int hxx, hyy, hzz;
          float tx = 0.f, ty = 0.f, tz = 0.f;
          if (I == 0) {
            const int nx = nearest_axis(ux, wx, fx, fy, half);
            const int ny = nearest_axis(uy, wy, fx, fy, half);
            const int nz = nearest_axis(uz, wz, fx, fy, half);
            if (!(in_box(nx, ax, ax + kT - 1) && in_box(ny, ay, ay + kT - 1) &&
                  in_box(nz, az, az + kT - 1)))
              continue;
            hxx = nx - ax + 1; hyy = ny - ay + 1; hzz = nz - az + 1;
          } else {
            const float sx = fmaf(wx, fy, ux * fx);
            const float sy = fmaf(wy, fy, uy * fx);
            const float sz = fmaf(wz, fy, uz * fx);
            const float flx = floorf(sx), fly = floorf(sy), flz = floorf(sz);
            const int x0 = (int)flx + half, y0 = (int)fly + half, z0 = (int)flz + half;
            if (!(in_box(x0, ax - 1, ax + kT - 1) && in_box(y0, ay - 1, ay + kT - 1) &&
                  in_box(z0, az - 1, az + kT - 1)))
              continue;
            hxx = x0 - ax + 1; hyy = y0 - ay + 1; hzz = z0 - az + 1;
            tx = sx - flx; ty = sy - fly; tz = sz - flz;
          }
          // base corner inside the tile: this tile counts the pixel's scalar terms
          const bool owner = hxx >= 1 && hyy >= 1 && hzz >= 1;
          const float C = ctf_value(G, a_hi, a_lo, q);
          const Corners<I> K8(hxx, hyy, hzz, tx, ty, tz, ax, ay, az, M);
          if (OP == OP_ADJOINT || OP == OP_LOSS_GRAD) {
            const float2 x = __ldg(A.img + (size_t)b * M * M + (size_t)(kyp + half) * M + (kx + half));
            float2 res = x;
            if (OP == OP_LOSS_GRAD) {
              float re = 0.f, im = 0.f;
#pragma unroll
              for (int c = 0; c < Corners<I>::N; ++c) {
                const float2 v = reinterpret_cast<const float2*>(halo)[K8.halo(c)];
                re = fmaf(K8.w(c), v.x, re);
                im = fmaf(K8.w(c), v.y, im);
              }
              res = make_float2(fmaf(C, re, -x.x), fmaf(C, im, -x.y));
              if (owner) part = fmaf(res.x, res.x, fmaf(res.y, res.y, part));
            }
            const float sc = A.scale * C;
            const float2 v = make_float2(sc * res.x, sc * res.y);
            float2* ac = reinterpret_cast<float2*>(acc);
#pragma unroll
            for (int c = 0; c < Corners<I>::N; ++c)
              if (K8.mine(c)) acc_add(ac + K8.acc(c), make_float2(K8.w(c) * v.x, K8.w(c) * v.y));
          } else if (OP == OP_HVP) {
            float a = 0.f;
#pragma unroll
            for (int c = 0; c < Corners<I>::N; ++c)
              a = fmaf(K8.w(c), reinterpret_cast<const float*>(halo)[K8.halo(c)], a);
            const float y = A.scale * C * C * a;
            float* ac = reinterpret_cast<float*>(acc);
#pragma unroll
            for (int c = 0; c < Corners<I>::N; ++c)
              if (K8.mine(c)) acc_add(ac + K8.acc(c), K8.w(c) * y);
          } else if (OP == OP_HUTCH) {
            const float sc = A.scale * C * C;
            float* ac = reinterpret_cast<float*>(acc);
            if (I == 0) {
              if (K8.mine(0)) acc_add(ac + K8.acc(0), sc);
            } else {
              uint32_t bw[8];
              float wsum = 0.f;
#pragma unroll
              for (int c = 0; c < 8; ++c) {
                bw[c] = reinterpret_cast<const uint32_t*>(halo)[K8.halo(c)];
                wsum += K8.w(c);
              }
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                if (!K8.mine(j)) continue;
                float pc = 0.f;
#pragma unroll
                for (int l = 0; l < 8; ++l)
                  if (l != j) pc = fmaf(K8.w(l), (float)__popc((bw[j] ^ bw[l]) & pmask), pc);
                acc_add(ac + K8.acc(j), sc * K8.w(j) * fmaf(-2.0f * invK, pc, wsum));
              }
            }
          } else if (OP == OP_CURVATURE) {
            if (owner) {
              float re = 0.f, im = 0.f;
#pragma unroll
              for (int c = 0; c < Corners<I>::N; ++c) {
                const float2 v = reinterpret_cast<const float2*>(halo)[K8.halo(c)];
                re = fmaf(K8.w(c), v.x, re);
                im = fmaf(K8.w(c), v.y, im);
              }
              part = fmaf(C * C, fmaf(re, re, im * im), part);
            }
          }
        }
      }
    }
    __syncthreads();
    if (Tr::kScatter) {
      AccT* dst = reinterpret_cast<AccT*>(A.dst);
      for (int i = threadIdx.x; i < kT * kT * kT; i += kTileThreads) {
        const int lx = i % kT, ly = (i / kT) % kT, lz = i / (kT * kT);
        const int gx = ax + lx, gy = ay + ly, gz = az + lz;
        const AccT v = acc[i];
        const size_t j = ((size_t)gz * M + gy) * M + gx;
        if (gx < M && gy < M && gz < M && nonzero(v) && CS_IN(j, (size_t)M * M * M))
          global_add(dst + j, v);
      }
    }
    if (Tr::kSum) {
      const double s = block_sum_f(part);
      if (threadIdx.x == 0) A.part[item] = s;
    }
    __syncthreads();
  }
}

template <int OP, int I>
cudaError_t launch_engine(const TileArgs& A, int num_sms, cudaStream_t s) {
  constexpr size_t sm = smem_bytes<OP>();
  // the shared-memory limit per device; the residency once (every device
  // of a process is the same GB300)
  static std::atomic<uint64_t> configured{0};
  static std::atomic<int> blocks_per_sm{0};
  cudaError_t e = ensure_smem_limit(k_tile<OP, I>, (int)sm, configured);
  if (e != cudaSuccess) return e;
  int bps = blocks_per_sm.load(std::memory_order_acquire);
  if (bps < 1) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_tile<OP, I>, kTileThreads, sm);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
    blocks_per_sm.store(bps, std::memory_order_release);
  }
  k_tile<OP, I><<<num_sms * bps, kTileThreads, sm, s>>>(A);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

int tiles_per_axis(int M) { return (M + kT - 1) / kT; }

cudaError_t launch_bin(const Geo& G, const float* rot, int B, TileArgs& A, int* count,
                       int* list, int* item_start, int* queue, cudaStream_t s) {
  const int tpa = tiles_per_axis(G.M);
  const int n_tiles = tpa * tpa * tpa;
  A.G = G;
  A.rot = rot;
  A.B = B;
  A.tpa = tpa;
  A.n_tiles = n_tiles;
  A.tile_count = count;
  A.tile_list = list;
  A.list_stride = B > 0 ? B : 1;
  A.item_start = item_start;
  A.queue = queue;
  k_bin<<<(n_tiles * 32 + 255) / 256, 256, 0, s>>>(G, rot, B, tpa, n_tiles, count, list,
                                                  A.list_stride);
  count_launches(1);
  k_items<<<1, 1024, 0, s>>>(count, n_tiles, kImgPerItem, item_start, queue);
  count_launches(1);
  return cudaGetLastError();
}


cudaError_t launch_tile_op(int op, const TileArgs& A, int num_sms, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(A.queue, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const bool tri = A.G.interp != 0;
  switch (op) {
    case OP_ADJOINT: return tri ? launch_engine<OP_ADJOINT, 1>(A, num_sms, s)
                                : launch_engine<OP_ADJOINT, 0>(A, num_sms, s);
    case OP_LOSS_GRAD: return tri ? launch_engine<OP_LOSS_GRAD, 1>(A, num_sms, s)
                                  : launch_engine<OP_LOSS_GRAD, 0>(A, num_sms, s);
    case OP_HVP: return tri ? launch_engine<OP_HVP, 1>(A, num_sms, s)
                            : launch_engine<OP_HVP, 0>(A, num_sms, s);
    case OP_HUTCH: return tri ? launch_engine<OP_HUTCH, 1>(A, num_sms, s)
                              : launch_engine<OP_HUTCH, 0>(A, num_sms, s);
    case OP_CURVATURE: return tri ? launch_engine<OP_CURVATURE, 1>(A, num_sms, s)
                                  : launch_engine<OP_CURVATURE, 0>(A, num_sms, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cs
