// Device-side building blocks shared by the kernels of libcryosgd:
// grid geometry, the interpolation stencils of Definition 2.1, the CTF and
// the SplitMix64 probe generator.  sm_103a only.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "debug_bounds.cuh"

namespace cs {

// Packed FP32 pairs (sm_100 family): one instruction performs two IEEE
// round-to-nearest operations, each lane bit-identical to the scalar one.
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// Kernel-side copy of the geometry.  The CTF phase (in units of pi) is
//   chi/pi = a_i q - b q^2,  a_i = ka * defocus_i,
// ka = lam / (M pix)^2 and b = Cs lam^3 / (2 (M pix)^4), prepared on the
// host in FP64; ka is carried as an unevaluated float pair (hi + lo) so that
// the large term a_i q can be reduced modulo 2 without losing accuracy.
struct Geo {
  int M;
  int half;       // M / 2
  int r2max;      // r_max^2
  int interp;     // 0 nearest, 1 trilinear
  int ctf_on;
  float ka_hi, ka_lo;
  float kb;
  float wsin;     // sqrt(1 - A^2)
  float wcos;     // A
};

// Per-image CTF coefficient a_i = ka * df as a float pair (error-free
// product of ka_hi and df via fmaf, plus the ka_lo term).
__device__ __forceinline__ void ctf_coeff(const Geo& G, float df, float& a_hi,
                                          float& a_lo) {
  float p = G.ka_hi * df;
  float e = fmaf(G.ka_hi, df, -p);
  a_hi = p;
  a_lo = fmaf(G.ka_lo, df, e);
}

// C_i at pixel radius^2 q.  The product a_hi*q is split exactly into its
// rounded value p and error e (fmaf), p is reduced modulo 2 exactly
// (p - 2 rint(p/2) is exact by Sterbenz' lemma), and the small remaining
// terms are added to the reduced phase before sincospif.
__device__ __forceinline__ float ctf_value(const Geo& G, float a_hi, float a_lo,
                                           int q) {
  if (!G.ctf_on) return 1.0f;
  float fq = (float)q;
  float p = a_hi * fq;
  float e = fmaf(a_hi, fq, -p);
  float r = p - 2.0f * rintf(0.5f * p);
  r += fmaf(a_lo, fq, e);
  r = fmaf(-G.kb, fq * fq, r);
  float s, c;
  sincospif(r, &s, &c);
  return -(G.wsin * s + G.wcos * c);
}

// Rotation of one image, row-major R[0..8].
struct Rot {
  float r0x, r0y, r0z, r1x, r1y, r1z;   // rows 0 and 1 of R
};

__device__ __forceinline__ Rot load_rot(const float* __restrict__ rot, int b) {
  const float* p = rot + 9 * (size_t)b;
  Rot R;
  R.r0x = __ldg(p + 0); R.r0y = __ldg(p + 1); R.r0z = __ldg(p + 2);
  R.r1x = __ldg(p + 3); R.r1y = __ldg(p + 4); R.r1z = __ldg(p + 5);
  return R;
}

// Interpolation stencil of one pixel: up to 8 voxel indices and weights.
// Corners outside the grid get weight 0 and a clamped (valid) index, so a
// gather or scatter through the stencil never leaves the volume.
struct Stencil {
  int n;          // 1 (nearest) or 8 (trilinear)
  int idx[8];
  float w[8];
};

// Nearest rule: coordinate a = R[0][a]*kx + R[1][a]*ky as two rounded
// products and a rounded sum (no contraction), rounded half to even.
__device__ __forceinline__ int nearest_axis(float r0, float r1, float kx, float ky,
                                            int half) {
  float c = __fadd_rn(__fmul_rn(r0, kx), __fmul_rn(r1, ky));
  return (int)rintf(c) + half;
}

template <int INTERP>
__device__ __forceinline__ void make_stencil(const Geo& G, const Rot& R, int kx,
                                             int ky, Stencil& S) {
  const float fx = (float)kx, fy = (float)ky;
  const int M = G.M;
  if (INTERP == 0) {
    int ix = nearest_axis(R.r0x, R.r1x, fx, fy, G.half);
    int iy = nearest_axis(R.r0y, R.r1y, fx, fy, G.half);
    int iz = nearest_axis(R.r0z, R.r1z, fx, fy, G.half);
    bool ok = (unsigned)ix < (unsigned)M && (unsigned)iy < (unsigned)M &&
              (unsigned)iz < (unsigned)M;
    S.n = 1;
    S.idx[0] = ok ? (iz * M + iy) * M + ix : 0;
    S.w[0] = ok ? 1.0f : 0.0f;
    return;
  }
  // trilinear: cell of s = R^T r, weights (1-t, t) per axis
  // fraction of the centred coordinate (adding M/2 first would round it to
  // the coarser float spacing near M/2 .. M)
  float sx = fmaf(R.r1x, fy, R.r0x * fx);
  float sy = fmaf(R.r1y, fy, R.r0y * fx);
  float sz = fmaf(R.r1z, fy, R.r0z * fx);
  float flx = floorf(sx), fly = floorf(sy), flz = floorf(sz);
  int x0 = (int)flx + G.half, y0 = (int)fly + G.half, z0 = (int)flz + G.half;
  float tx = sx - flx, ty = sy - fly, tz = sz - flz;
  S.n = 8;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
    int ix = x0 + dx, iy = y0 + dy, iz = z0 + dz;
    bool ok = (unsigned)ix < (unsigned)M && (unsigned)iy < (unsigned)M &&
              (unsigned)iz < (unsigned)M;
    int cx = min(max(ix, 0), M - 1), cy = min(max(iy, 0), M - 1),
        cz = min(max(iz, 0), M - 1);
    float w = (dx ? tx : 1.0f - tx) * (dy ? ty : 1.0f - ty) * (dz ? tz : 1.0f - tz);
    S.idx[c] = (cz * M + cy) * M + cx;
    S.w[c] = ok ? w : 0.0f;
  }
}

// SplitMix64 (Steele, Lea & Flood 2014): output number c of the stream
// seeded with `seed` is mix(seed + (c + 1) * golden_gamma).
constexpr uint64_t kSplitMixGamma = 0x9E3779B97F4A7C15ull;

// The output function of SplitMix64 applied to the state z.
__device__ __forceinline__ uint64_t splitmix_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t c) {
  return splitmix_mix(seed + (c + 1ull) * kSplitMixGamma);
}

// Probe words: voxels (2i, 2i+1) take the low / high 32 bits of SplitMix64
// output number block * (n_vox / 2) + i (n_vox = M^3 is even).
__device__ __forceinline__ uint64_t probe_pair(uint64_t seed, uint64_t pair_base, uint64_t i) {
  return splitmix64(seed, pair_base + i);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while the kernel before it in the stream is still
// running; it waits here, before touching anything, until that kernel has
// completed and its writes are visible (a no-op for an ordinary launch).
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Block-wide sum in a fixed order (deterministic); every thread must call.
// Result valid in thread 0.  Needs blockDim.x a multiple of 32, <= 1024.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    t = lane < nw ? red[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;
}

// Sum of p[0 .. n) by one warp in a fixed order: lane l adds p[l], p[l + 32],
// ... in four FP64 chains, then the warp adds its lanes.  FP64 arithmetic runs
// at a small fraction of the FP32 rate on this part: a warp per array, instead
// of a block-wide FP64 tree, keeps the count of FP64 warp instructions low.
// Every lane must call; the result is valid in every lane.
__device__ __forceinline__ double warp_sum_array(const double* p, int n) {
  const int lane = threadIdx.x & 31;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int i = lane;
  for (; i + 96 < n; i += 128) {
    s0 += p[i];
    s1 += p[i + 32];
    s2 += p[i + 64];
    s3 += p[i + 96];
  }
  for (; i < n; i += 32) s0 += p[i];
  return warp_sum((s0 + s1) + (s2 + s3));
}

// Block-wide sum of FP32 per-thread values: each warp adds its lanes in
// FP32 (a fixed butterfly), and thread 0 adds the warp sums in FP64 in warp
// order.  FP64 arithmetic runs at a small fraction of the FP32 rate on this
// part, so only that last level uses it.  Deterministic; every thread must
// call; result valid in thread 0.  blockDim.x a multiple of 32, <= 1024.
__device__ __forceinline__ double block_sum_f(float v) {
  __shared__ double redf[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) redf[wid] = (double)v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    for (int q = 0; q < nw; ++q) t += redf[q];
  }
  return t;
}

}  // namespace cs
