// Per-pixel operator kernels of libcryosgd: forward slice (Definition 2.1,
// Eq. fwd model), adjoint scatter, fused loss + gradient (Eq. optim cp),
// Hessian-vector product (Eq. hessian), Hutchinson's estimator (Eq. hutch),
// exact diagonal and the line-search curvature.
//
// Work decomposition: a work item is (image b, chunk of kBlock consecutive
// pixels of that image); a fixed grid of blocks walks the items with a grid
// stride, so the number of blocks (and hence the number of partial sums of
// the reductions) does not depend on the batch size.  The volume (16 MiB at
// M = 128) stays L2-resident; images are streamed once with coalesced 8-byte
// accesses; adjoint contributions are FP32 reductions into global memory.
#include "internal.h"

namespace cs {

namespace {

struct PixelItem {
  int b, p, kx, ky, q;
  bool inside;
};

__device__ __forceinline__ PixelItem pixel_item(const Geo& G, int w, int nch) {
  PixelItem it;
  it.b = w / nch;
  const int ch = w - it.b * nch;
  it.p = ch * kBlock + threadIdx.x;
  const int MM = G.M * G.M;
  if (it.p >= MM) {
    it.inside = false;
    it.kx = it.ky = it.q = 0;
    return it;
  }
  const int iy = it.p / G.M, ix = it.p - iy * G.M;
  it.kx = ix - G.half;
  it.ky = iy - G.half;
  it.q = it.kx * it.kx + it.ky * it.ky;
  it.inside = it.q <= G.r2max;
  return it;
}

__device__ __forceinline__ float image_ctf(const Geo& G, const float* __restrict__ df,
                                           int b, int q) {
  if (!G.ctf_on) return 1.0f;
  float a_hi, a_lo;
  ctf_coeff(G, __ldg(df + b), a_hi, a_lo);
  return ctf_value(G, a_hi, a_lo, q);
}

template <int I>
__device__ __forceinline__ float2 gather(const Stencil& S, const float2* __restrict__ v,
                                         int n = 0x7fffffff) {
  float re = 0.f, im = 0.f;
#pragma unroll
  for (int c = 0; c < (I ? 8 : 1); ++c) {
    if (!CS_IN(S.idx[c], n)) continue;
    float2 x = __ldg(v + S.idx[c]);
    re = fmaf(S.w[c], x.x, re);
    im = fmaf(S.w[c], x.y, im);
  }
  return make_float2(re, im);
}

template <int I>
__device__ __forceinline__ float gather_real(const Stencil& S, const float* __restrict__ v,
                                             int n = 0x7fffffff) {
  float a = 0.f;
#pragma unroll
  for (int c = 0; c < (I ? 8 : 1); ++c)
    if (CS_IN(S.idx[c], n)) a = fmaf(S.w[c], __ldg(v + S.idx[c]), a);
  return a;
}

template <int I>
__device__ __forceinline__ void scatter(const Stencil& S, float2 val, float2* v,
                                        int n = 0x7fffffff) {
#pragma unroll
  for (int c = 0; c < (I ? 8 : 1); ++c) {
    if (S.w[c] != 0.0f && CS_IN(S.idx[c], n))
      atomicAdd(v + S.idx[c], make_float2(S.w[c] * val.x, S.w[c] * val.y));
  }
}

template <int I>
__device__ __forceinline__ void scatter_real(const Stencil& S, float val, float* v,
                                             int n = 0x7fffffff) {
#pragma unroll
  for (int c = 0; c < (I ? 8 : 1); ++c)
    if (S.w[c] != 0.0f && CS_IN(S.idx[c], n)) atomicAdd(v + S.idx[c], S.w[c] * val);
}

// ------------------------------------------------------------- kernels
template <int I>
__global__ void __launch_bounds__(kBlock)
k_slice_project(Geo G, const float2* __restrict__ vol, const float* __restrict__ rot,
                const float* __restrict__ df, int B, float2* __restrict__ out) {
  const int MM = G.M * G.M, nch = (MM + kBlock - 1) / kBlock, total = B * nch;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    PixelItem it = pixel_item(G, w, nch);
    if (it.p >= MM) continue;
    float2 y = make_float2(0.f, 0.f);
    if (it.inside) {
      Rot R = load_rot(rot, it.b);
      Stencil S;
      make_stencil<I>(G, R, it.kx, it.ky, S);
      float2 a = gather<I>(S, vol, G.M * G.M * G.M);
      float C = image_ctf(G, df, it.b, it.q);
      y = make_float2(C * a.x, C * a.y);
    }
    out[(size_t)it.b * MM + it.p] = y;
  }
}

template <int I>
__global__ void __launch_bounds__(kBlock)
k_backproject(Geo G, const float2* __restrict__ img, const float* __restrict__ rot,
              const float* __restrict__ df, int B, float scale, float2* vol) {
  const int MM = G.M * G.M, nch = (MM + kBlock - 1) / kBlock, total = B * nch;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    PixelItem it = pixel_item(G, w, nch);
    if (!it.inside) continue;
    float2 y = __ldg(img + (size_t)it.b * MM + it.p);
    Rot R = load_rot(rot, it.b);
    Stencil S;
    make_stencil<I>(G, R, it.kx, it.ky, S);
    float sc = scale * image_ctf(G, df, it.b, it.q);
    scatter<I>(S, make_float2(sc * y.x, sc * y.y), vol, G.M * G.M * G.M);
  }
}

// grad = lambda * v, and partial sums of |v|^2
__global__ void __launch_bounds__(kBlock)
k_init_grad(int n, const float2* __restrict__ v, float lambda, float2* __restrict__ g,
            double* __restrict__ part) {
  // a few voxels per thread in FP32, warp sums in FP32, the block sum in FP64
  float acc = 0.f;
  for (int j = blockIdx.x * kBlock + threadIdx.x; j < n; j += gridDim.x * kBlock) {
    float2 x = v[j];
    g[j] = make_float2(lambda * x.x, lambda * x.y);
    acc += fmaf(x.x, x.x, x.y * x.y);
  }
  double t = block_sum_f(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

template <int I>
__global__ void __launch_bounds__(kBlock)
k_loss_grad(Geo G, const float2* __restrict__ vol, const float2* __restrict__ img,
            const float* __restrict__ rot, const float* __restrict__ df, int B,
            float scale, float2* grad, double* __restrict__ part) {
  const int MM = G.M * G.M, nch = (MM + kBlock - 1) / kBlock, total = B * nch;
  float acc = 0.f;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    PixelItem it = pixel_item(G, w, nch);
    if (!it.inside) continue;
    Rot R = load_rot(rot, it.b);
    Stencil S;
    make_stencil<I>(G, R, it.kx, it.ky, S);
    float2 a = gather<I>(S, vol, G.M * G.M * G.M);
    float2 x = __ldg(img + (size_t)it.b * MM + it.p);
    float C = image_ctf(G, df, it.b, it.q);
    float rr = fmaf(C, a.x, -x.x), ri = fmaf(C, a.y, -x.y);
    acc = fmaf(rr, rr, fmaf(ri, ri, acc));
    float sc = scale * C;
    scatter<I>(S, make_float2(sc * rr, sc * ri), grad, G.M * G.M * G.M);
  }
  double t = block_sum_f(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// loss = scale/2 * sum(pl) + lambda/2 * sum(pv), fixed summation order (one
// warp per array)
__global__ void __launch_bounds__(64)
k_finalize_loss(const double* __restrict__ pl, int nl, const int* __restrict__ nl_dev,
                const double* __restrict__ pv, int nv, float lambda, float scale,
                double* loss) {
  __shared__ double st[2];
  if (nl_dev) nl = *nl_dev;
  const int a = threadIdx.x >> 5;
  const double v = a == 0 ? warp_sum_array(pl, nl) : warp_sum_array(pv, nv);
  if ((threadIdx.x & 31) == 0) st[a] = v;
  __syncthreads();
  if (threadIdx.x == 0) *loss = 0.5 * (double)scale * st[0] + 0.5 * (double)lambda * st[1];
}

__global__ void __launch_bounds__(kBlock)
k_scale_copy(int n, const float* __restrict__ z, float lambda, float* __restrict__ out) {
  for (int j = blockIdx.x * kBlock + threadIdx.x; j < n; j += gridDim.x * kBlock)
    out[j] = lambda * z[j];
}

__global__ void __launch_bounds__(kBlock)
k_fill(int n, float value, float* __restrict__ out) {
  for (int j = blockIdx.x * kBlock + threadIdx.x; j < n; j += gridDim.x * kBlock)
    out[j] = value;
}

template <int I>
__global__ void __launch_bounds__(kBlock)
k_hvp(Geo G, const float* __restrict__ z, const float* __restrict__ rot,
      const float* __restrict__ df, int B, float scale, float* Hz) {
  const int MM = G.M * G.M, nch = (MM + kBlock - 1) / kBlock, total = B * nch;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    PixelItem it = pixel_item(G, w, nch);
    if (!it.inside) continue;
    Rot R = load_rot(rot, it.b);
    Stencil S;
    make_stencil<I>(G, R, it.kx, it.ky, S);
    float a = gather_real<I>(S, z, G.M * G.M * G.M);
    float C = image_ctf(G, df, it.b, it.q);
    scatter_real<I>(S, scale * C * C * a, Hz, G.M * G.M * G.M);
  }
}

__global__ void __launch_bounds__(kBlock)
k_probe_bits(int n, uint64_t seed, uint64_t block_host, const double* __restrict__ k_dev,
             uint32_t* __restrict__ bits) {
  // probe block: block_host, or (iterations done + 1) read from the SGD state
  const uint64_t blk = k_dev ? (uint64_t)(*k_dev) + 1ull : block_host;
  const int np = n >> 1;
  const uint64_t base = blk * (uint64_t)np;
  for (int i = blockIdx.x * kBlock + threadIdx.x; i < np; i += gridDim.x * kBlock) {
    const uint64_t w = probe_pair(seed, base, (uint64_t)i);
    reinterpret_cast<uint2*>(bits)[i] = make_uint2((uint32_t)w, (uint32_t)(w >> 32));
  }
}

// D_j += scale C^2 w_j sum_l w_l Z_jl with Z_jl = (K - 2 popc((b_j ^ b_l) & mask)) / K,
// the probe average of z_kj z_kl: (1/K) sum_k z_kj (H z_k)_j expanded over the
// stencil of each pixel, exact for any K <= 32.
template <int I>
__global__ void __launch_bounds__(kBlock)
k_hutchinson(Geo G, const uint32_t* __restrict__ bits, const float* __restrict__ rot,
             const float* __restrict__ df, int B, float scale, int K, float* diag) {
  const int MM = G.M * G.M, nch = (MM + kBlock - 1) / kBlock, total = B * nch;
  const uint32_t mask = K >= 32 ? 0xffffffffu : ((1u << K) - 1u);
  const float invK = 1.0f / (float)K;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    PixelItem it = pixel_item(G, w, nch);
    if (!it.inside) continue;
    Rot R = load_rot(rot, it.b);
    Stencil S;
    make_stencil<I>(G, R, it.kx, it.ky, S);
    float C = image_ctf(G, df, it.b, it.q);
    const float sc = scale * C * C;
    [[maybe_unused]] const int nv = G.M * G.M * G.M;   // range checks (debug build)
    if (I == 0) {
      if (S.w[0] != 0.0f && CS_IN(S.idx[0], nv)) atomicAdd(diag + S.idx[0], sc);
      continue;
    }
    uint32_t bw[8];
    float wsum = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      bw[c] = CS_IN(S.idx[c], nv) ? __ldg(bits + S.idx[c]) : 0u;
      wsum += S.w[c];
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      // sum_l w_l (K - 2 popc) / K = wsum - (2/K) sum_l w_l popc(b_j ^ b_l)
      float pc = 0.f;
#pragma unroll
      for (int l = 0; l < 8; ++l)
        if (l != j) pc = fmaf(S.w[l], (float)__popc((bw[j] ^ bw[l]) & mask), pc);
      float sj = fmaf(-2.0f * invK, pc, wsum);
      if (S.w[j] != 0.0f && CS_IN(S.idx[j], nv)) atomicAdd(diag + S.idx[j], sc * S.w[j] * sj);
    }
  }
}

template <int I>
__global__ void __launch_bounds__(kBlock)
k_exact_diag(Geo G, const float* __restrict__ rot, const float* __restrict__ df, int B,
             float scale, float* diag, float* cov, float* c2w) {
  const int MM = G.M * G.M, nch = (MM + kBlock - 1) / kBlock, total = B * nch;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    PixelItem it = pixel_item(G, w, nch);
    if (!it.inside) continue;
    Rot R = load_rot(rot, it.b);
    Stencil S;
    make_stencil<I>(G, R, it.kx, it.ky, S);
    float C = image_ctf(G, df, it.b, it.q);
    const float c2 = C * C;
#pragma unroll
    for (int c = 0; c < (I ? 8 : 1); ++c) {
      const float wc = S.w[c];
      if (wc == 0.0f || !CS_IN(S.idx[c], G.M * G.M * G.M)) continue;
      if (diag) atomicAdd(diag + S.idx[c], scale * c2 * wc * wc);
      if (cov) atomicAdd(cov + S.idx[c], scale * wc);
      if (c2w) atomicAdd(c2w + S.idx[c], scale * c2 * wc);
    }
  }
}

template <int I>
__global__ void __launch_bounds__(kBlock)
k_curvature(Geo G, const float2* __restrict__ d, const float* __restrict__ rot,
            const float* __restrict__ df, int B, double* __restrict__ part) {
  const int MM = G.M * G.M, nch = (MM + kBlock - 1) / kBlock, total = B * nch;
  float acc = 0.f;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    PixelItem it = pixel_item(G, w, nch);
    if (!it.inside) continue;
    Rot R = load_rot(rot, it.b);
    Stencil S;
    make_stencil<I>(G, R, it.kx, it.ky, S);
    float2 a = gather<I>(S, d, G.M * G.M * G.M);
    float C = image_ctf(G, df, it.b, it.q);
    acc = fmaf(C * C, fmaf(a.x, a.x, a.y * a.y), acc);
  }
  double t = block_sum_f(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

int elem_grid(int n, int num_sms) {
  int g = (n + kBlock - 1) / kBlock;
  return g < num_sms * 8 ? (g > 0 ? g : 1) : num_sms * 8;
}

}  // namespace

#define CS_DISPATCH(G, KER, ...)                                        \
  do {                                                                  \
    if ((G).interp == 0) KER<0><<<grid, kBlock, 0, s>>>(__VA_ARGS__);   \
    else KER<1><<<grid, kBlock, 0, s>>>(__VA_ARGS__);                   \
  } while (0)

cudaError_t launch_slice_project(const Geo& G, const float2* vol, const float* rot,
                                 const float* df, int B, float2* out, int grid,
                                 cudaStream_t s) {
  CS_DISPATCH(G, k_slice_project, G, vol, rot, df, B, out);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_backproject(const Geo& G, const float2* img, const float* rot,
                               const float* df, int B, float scale, float2* vol,
                               int grid, cudaStream_t s) {
  CS_DISPATCH(G, k_backproject, G, img, rot, df, B, scale, vol);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_loss_grad(const Geo& G, const float2* vol, const float2* img,
                             const float* rot, const float* df, int B, float lambda,
                             float scale, float2* grad, double* loss, double* part_loss,
                             double* part_vv, int* n_vv, int grid, int num_sms,
                             cudaStream_t s) {
  const int n = G.M * G.M * G.M;
  const int gi = elem_grid(n, num_sms);
  *n_vv = gi;
  k_init_grad<<<gi, kBlock, 0, s>>>(n, vol, lambda, grad, part_vv);
  count_launches(1);
  if (B > 0) { CS_DISPATCH(G, k_loss_grad, G, vol, img, rot, df, B, scale, grad, part_loss); count_launches(1); }
  if (loss) {
    k_finalize_loss<<<1, 64, 0, s>>>(part_loss, B > 0 ? grid : 0, nullptr, part_vv, gi,
                                       lambda, scale, loss);
    count_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_hvp(const Geo& G, const float* z, const float* rot, const float* df,
                       int B, float lambda, float scale, float* Hz, int grid,
                       int num_sms, cudaStream_t s) {
  const int n = G.M * G.M * G.M;
  k_scale_copy<<<elem_grid(n, num_sms), kBlock, 0, s>>>(n, z, lambda, Hz);
  count_launches(1);
  CS_DISPATCH(G, k_hvp, G, z, rot, df, B, scale, Hz);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_probe_bits(int M, uint64_t seed, uint64_t block_host,
                              const double* k_dev, uint32_t* bits, int num_sms,
                              cudaStream_t s) {
  const int n = M * M * M;
  k_probe_bits<<<elem_grid(n, num_sms), kBlock, 0, s>>>(n, seed, block_host, k_dev, bits);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_hutchinson(const Geo& G, const uint32_t* bits, const float* rot,
                              const float* df, int B, float lambda, float scale,
                              int n_probes, float* diag, int grid, int num_sms,
                              cudaStream_t s) {
  const int n = G.M * G.M * G.M;
  k_fill<<<elem_grid(n, num_sms), kBlock, 0, s>>>(n, lambda, diag);
  count_launches(1);
  CS_DISPATCH(G, k_hutchinson, G, bits, rot, df, B, scale, n_probes, diag);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_exact_diag(const Geo& G, const float* rot, const float* df, int B,
                              float lambda, float scale, float* diag, float* cov,
                              float* c2w, int grid, int num_sms, cudaStream_t s) {
  const int n = G.M * G.M * G.M;
  const int ge = elem_grid(n, num_sms);
  if (diag) { k_fill<<<ge, kBlock, 0, s>>>(n, lambda, diag); count_launches(1); }
  if (cov) { k_fill<<<ge, kBlock, 0, s>>>(n, 0.0f, cov); count_launches(1); }
  if (c2w) { k_fill<<<ge, kBlock, 0, s>>>(n, 0.0f, c2w); count_launches(1); }
  CS_DISPATCH(G, k_exact_diag, G, rot, df, B, scale, diag, cov, c2w);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_curvature(const Geo& G, const float2* d, const float* rot,
                             const float* df, int B, double* part, int grid,
                             cudaStream_t s) {
  CS_DISPATCH(G, k_curvature, G, d, rot, df, B, part);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_init_grad(int n, const float2* vol, float lambda, float2* grad,
                             double* part_vv, int* n_vv, int num_sms, cudaStream_t s) {
  const int gi = elem_grid(n, num_sms);
  *n_vv = gi;
  k_init_grad<<<gi, kBlock, 0, s>>>(n, vol, lambda, grad, part_vv);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_finalize_loss(const double* pl, int n, const int* n_dev, const double* pv,
                                 int nv, float lambda, float scale, double* loss,
                                 cudaStream_t s) {
  k_finalize_loss<<<1, 64, 0, s>>>(pl, n, n_dev, pv, nv, lambda, scale, loss);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_fill(int n, float value, float* out, int num_sms, cudaStream_t s) {
  k_fill<<<elem_grid(n, num_sms), kBlock, 0, s>>>(n, value, out);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_scale_copy(int n, const float* z, float lambda, float* out, int num_sms,
                              cudaStream_t s) {
  k_scale_copy<<<elem_grid(n, num_sms), kBlock, 0, s>>>(n, z, lambda, out);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace cs
