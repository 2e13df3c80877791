// Element-wise and scalar kernels of Algorithm 1 (Section 3.4): pose
// conversion, the preconditioner update (Eqs. hutch update, exp avg update,
// thresh), the step direction, the closed-form stochastic Armijo step
// (Eq. stochastic armijo), the threshold alpha (Eq. thresh value) and the
// relative volume error.
#include "internal.h"

namespace cs {

namespace {

int elem_grid(int n, int num_sms) {
  int g = (n + kBlock - 1) / kBlock;
  return g < num_sms * 8 ? (g > 0 ? g : 1) : num_sms * 8;
}

__global__ void k_quat_to_rot(const float* __restrict__ q, int B, float* __restrict__ R) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float w = q[4 * b], x = q[4 * b + 1], y = q[4 * b + 2], z = q[4 * b + 3];
  float inv = rsqrtf(w * w + x * x + y * y + z * z);
  w *= inv; x *= inv; y *= inv; z *= inv;
  float* r = R + 9 * b;
  r[0] = 1.f - 2.f * (y * y + z * z);
  r[1] = 2.f * (x * y - w * z);
  r[2] = 2.f * (x * z + w * y);
  r[3] = 2.f * (x * y + w * z);
  r[4] = 1.f - 2.f * (x * x + z * z);
  r[5] = 2.f * (y * z - w * x);
  r[6] = 2.f * (x * z - w * y);
  r[7] = 2.f * (y * z + w * x);
  r[8] = 1.f - 2.f * (x * x + y * y);
}

// Rotations of batch (k mod n_batches) of a dataset's quaternions, k read
// from the SGD state (iterations done).
__global__ void k_quat_to_rot_cursor(const float* __restrict__ q, int B, int n_batches,
                                     const double* __restrict__ cursor, float* __restrict__ R) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const long long bsel = (long long)(*cursor) % (long long)n_batches;
  const float* qq = q + 4 * ((size_t)bsel * B + b);
  float w = qq[0], x = qq[1], y = qq[2], z = qq[3];
  float inv = rsqrtf(w * w + x * x + y * y + z * z);
  w *= inv; x *= inv; y *= inv; z *= inv;
  float* r = R + 9 * b;
  r[0] = 1.f - 2.f * (y * y + z * z);
  r[1] = 2.f * (x * y - w * z);
  r[2] = 2.f * (x * z + w * y);
  r[3] = 2.f * (x * y + w * z);
  r[4] = 1.f - 2.f * (x * x + z * z);
  r[5] = 2.f * (y * z - w * x);
  r[6] = 2.f * (x * z - w * y);
  r[7] = 2.f * (y * z + w * x);
  r[8] = 1.f - 2.f * (x * x + y * y);
}

// Running mean of the Hutchinson estimates, EMA and threshold, for step
// k = (iterations done) + 1.
__global__ void __launch_bounds__(kBlock)
k_precond_update(int n, const float* __restrict__ dest, float* __restrict__ D,
                 float* __restrict__ Davg, float* __restrict__ dhat,
                 const double* __restrict__ sc, float beta) {
  const double k = sc[CS_S_K] + 1.0;
  const float wold = (float)((k - 1.0) / k), wnew = (float)(1.0 / k);
  const float alpha = (float)sc[CS_S_ALPHA];
  for (int j = blockIdx.x * kBlock + threadIdx.x; j < n; j += gridDim.x * kBlock) {
    float a = fmaf(wold, Davg[j], wnew * dest[j]);
    float d = fmaf(beta, D[j], (1.0f - beta) * a);
    Davg[j] = a;
    D[j] = d;
    dhat[j] = fmaxf(fabsf(d), alpha);
  }
}

__global__ void __launch_bounds__(kBlock)
k_fixed_dhat(int n, const float* __restrict__ D, float* __restrict__ dhat,
             const double* __restrict__ sc) {
  const float alpha = (float)sc[CS_S_ALPHA];
  for (int j = blockIdx.x * kBlock + threadIdx.x; j < n; j += gridDim.x * kBlock)
    dhat[j] = fmaxf(fabsf(D[j]), alpha);
}

// Running mean of the k-th estimate (Eq. diag est rule); at k = 1 the
// estimate is copied so that D's previous contents never leak in.
__global__ void __launch_bounds__(kBlock)
k_running_mean(int n, const float* __restrict__ est, float* __restrict__ D, float a, float b,
               int first) {
  for (int j = blockIdx.x * kBlock + threadIdx.x; j < n; j += gridDim.x * kBlock)
    D[j] = first ? est[j] : a * D[j] + b * est[j];
}

__global__ void __launch_bounds__(kBlock)
k_direction(int n, const float2* __restrict__ g, const float* __restrict__ dhat,
            float2* __restrict__ d, double* __restrict__ part) {
  // a few voxels per thread in FP32, warp sums in FP32, block sums in FP64
  float aG = 0.f, aD = 0.f;
  for (int j = blockIdx.x * kBlock + threadIdx.x; j < n; j += gridDim.x * kBlock) {
    float2 x = g[j];
    float inv = dhat ? 1.0f / dhat[j] : 1.0f;
    float2 y = make_float2(x.x * inv, x.y * inv);
    d[j] = y;
    aG += fmaf(x.x, x.x, x.y * x.y) * inv;
    aD += fmaf(y.x, y.x, y.y * y.y);
  }
  double tG = block_sum_f(aG);
  double tD = block_sum_f(aD);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = tG;
    part[gridDim.x + blockIdx.x] = tD;
  }
}

// Closed-form stochastic Armijo: f_I(v - eta d) = f_I(v) - eta G + eta^2 Q/2
// (f_I quadratic), so the halving loop of Algorithm 1 stops at the first
// eta = eta_prev 2^-m with eta <= 2 (1 - c) G / Q.
// The five partial arrays (data term, |v|^2, G, |d|^2, curvature) are
// summed one per warp (warp_sum_array).
__global__ void __launch_bounds__(160)
k_eta(double* sc, const double* pl, int nl, const double* pv, int nv, const double* pG,
      const double* pD, int nd, const double* pQ, int nq, const int* n_dev, float lambda,
      float scale, float c, int max_halvings) {
  __shared__ double sum5[5];
  grid_dep_wait();
  if (n_dev) {
    nl = *n_dev;
    nq = *n_dev;
  }
  const int lane = threadIdx.x & 31, a = threadIdx.x >> 5;
  const double* p = a == 0 ? pl : a == 1 ? pv : a == 2 ? pG : a == 3 ? pD : pQ;
  const int n = a == 0 ? nl : a == 1 ? nv : a == 4 ? nq : nd;
  const double t = warp_sum_array(p, n);
  if (lane == 0) sum5[a] = t;
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double L = sum5[0], V = sum5[1], G = sum5[2], DD = sum5[3], Qd = sum5[4];
  double Q = (double)scale * Qd + (double)lambda * DD;
  double eta = sc[CS_S_ETA];
  int h = 0;
  double status = 1.0;
  if (G > 0.0 && Q > 0.0) {
    const double bound = 2.0 * (1.0 - (double)c) * G / Q;
    while (eta > bound && h < max_halvings) {
      eta *= 0.5;
      ++h;
    }
    status = 0.0;
  }
  sc[CS_S_LOSS] = 0.5 * (double)scale * L + 0.5 * (double)lambda * V;
  sc[CS_S_G] = G;
  sc[CS_S_Q] = Q;
  sc[CS_S_HALVINGS] = (double)h;
  sc[CS_S_ETA] = eta;
  sc[CS_S_STATUS] = status;
  sc[CS_S_K] = sc[CS_S_K] + 1.0;
}

__global__ void __launch_bounds__(kBlock)
k_update(int n, float2* __restrict__ v, const float2* __restrict__ d,
         const double* __restrict__ sc) {
  const float eta = (float)sc[CS_S_ETA];
  for (int j = blockIdx.x * kBlock + threadIdx.x; j < n; j += gridDim.x * kBlock) {
    float2 a = v[j], b = d[j];
    v[j] = make_float2(fmaf(-eta, b.x, a.x), fmaf(-eta, b.y, a.y));
  }
}

// sum_i C_i(R)^2 over the dataset, then alpha.
__global__ void __launch_bounds__(1024)
k_alpha(Geo G, const float* __restrict__ df, int N, int q, double px_over_pv,
        double lambda, double scale_alpha, double* alpha) {
  double a = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    float C = 1.0f;
    if (G.ctf_on) {
      float a_hi, a_lo;
      ctf_coeff(G, df[i], a_hi, a_lo);
      C = ctf_value(G, a_hi, a_lo, q);
    }
    a += (double)C * (double)C;
  }
  a = block_sum(a);
  if (threadIdx.x == 0) *alpha = px_over_pv * scale_alpha * a + lambda;
}

__global__ void __launch_bounds__(kBlock)
k_rel_err_part(Geo G, const float2* __restrict__ v, const float2* __restrict__ r,
               double* __restrict__ part) {
  const int n = G.M * G.M * G.M;
  // a few voxels per thread in FP32, warp sums in FP32, block sums in FP64
  float e = 0.f, t = 0.f;
  for (int j = blockIdx.x * kBlock + threadIdx.x; j < n; j += gridDim.x * kBlock) {
    int x = j % G.M, y = (j / G.M) % G.M, z = j / (G.M * G.M);
    int kx = x - G.half, ky = y - G.half, kz = z - G.half;
    if (kx * kx + ky * ky + kz * kz > G.r2max) continue;
    float2 a = v[j], b = r[j];
    float dx = a.x - b.x, dy = a.y - b.y;
    e += fmaf(dx, dx, dy * dy);
    t += fmaf(b.x, b.x, b.y * b.y);
  }
  double se = block_sum_f(e);
  double st = block_sum_f(t);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = se;
    part[gridDim.x + blockIdx.x] = st;
  }
}

// two warps: the error and reference partials
__global__ void __launch_bounds__(64)
k_rel_err_final(const double* part, int nb, double* out) {
  __shared__ double st[2];
  const int a = threadIdx.x >> 5;
  const double v = warp_sum_array(part + a * nb, nb);
  if ((threadIdx.x & 31) == 0) st[a] = v;
  __syncthreads();
  if (threadIdx.x == 0) *out = st[1] > 0.0 ? sqrt(st[0] / st[1]) : 0.0;
}

}  // namespace

cudaError_t launch_quat_to_rot(const float* quat, int B, float* rot, cudaStream_t s) {
  k_quat_to_rot<<<(B + 127) / 128, 128, 0, s>>>(quat, B, rot);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_quat_to_rot_cursor(const float* quat, int B, int n_batches,
                                      const double* cursor, float* rot, cudaStream_t s) {
  k_quat_to_rot_cursor<<<(B + 127) / 128, 128, 0, s>>>(quat, B, n_batches, cursor, rot);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_precond_update(int n, const float* dest, float* D, float* Davg,
                                  float* dhat, const double* scalars, float beta,
                                  int num_sms, cudaStream_t s) {
  k_precond_update<<<elem_grid(n, num_sms), kBlock, 0, s>>>(n, dest, D, Davg, dhat,
                                                            scalars, beta);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_running_mean(int n, const float* est, float* D, long k, int num_sms,
                                cudaStream_t s) {
  const double kd = (double)k;
  k_running_mean<<<elem_grid(n, num_sms), kBlock, 0, s>>>(n, est, D, (float)((kd - 1.0) / kd),
                                                          (float)(1.0 / kd), k == 1);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_fixed_dhat(int n, const float* D, float* dhat, const double* scalars,
                              int num_sms, cudaStream_t s) {
  k_fixed_dhat<<<elem_grid(n, num_sms), kBlock, 0, s>>>(n, D, dhat, scalars);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_direction(int n, const float2* g, const float* dhat, float2* d,
                             double* part, int* nblk, int num_sms, cudaStream_t s) {
  const int gb = elem_grid(n, num_sms);
  *nblk = gb;
  k_direction<<<gb, kBlock, 0, s>>>(n, g, dhat, d, part);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_eta(double* scalars, const double* part_loss, int n_loss,
                       const double* part_vv, int n_vv, const double* part_G,
                       const double* part_dd, int n_dir, const double* part_Q, int n_Q,
                       const int* n_dev, float lambda, float scale, float c,
                       int max_halvings, cudaStream_t s) {
  const cudaError_t e = launch_pdl(k_eta, 1, 160, s, scalars, part_loss, n_loss, part_vv, n_vv,
                                   part_G, part_dd, n_dir, part_Q, n_Q, n_dev, lambda, scale, c,
                                   max_halvings);
  count_launches(1);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_update(int n, float2* v, const float2* d, const double* scalars,
                          int num_sms, cudaStream_t s) {
  k_update<<<elem_grid(n, num_sms), kBlock, 0, s>>>(n, v, d, scalars);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_alpha(const Geo& G, const float* df, int N, double px_over_pv,
                         double lambda, double scale_alpha, double* alpha,
                         cudaStream_t s) {
  const int R = (int)llround(sqrt((double)G.r2max));
  k_alpha<<<1, 1024, 0, s>>>(G, df, N, R * R, px_over_pv, lambda, scale_alpha, alpha);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_rel_err(const Geo& G, const float2* v, const float2* vref,
                           double* part, double* out, int num_sms, cudaStream_t s) {
  const int n = G.M * G.M * G.M;
  const int gb = elem_grid(n, num_sms);
  k_rel_err_part<<<gb, kBlock, 0, s>>>(G, v, vref, part);
  count_launches(1);
  k_rel_err_final<<<1, 64, 0, s>>>(part, gb, out);
  count_launches(1);
  return cudaGetLastError();
}

namespace {

// One block per (disc row, image): row k (ky = k - r) holds the pixels
// kx = -xr .. xr, xr = (rows[k+1] - rows[k] - 1) / 2, packed at rows[k]
__global__ void __launch_bounds__(128)
k_expand_disc(int M, int r, const int* __restrict__ rows, const float2* __restrict__ packed,
              int n_px, float2* __restrict__ images) {
  const int k = blockIdx.x, b = blockIdx.y;
  const int start = __ldg(rows + k), len = __ldg(rows + k + 1) - start;
  const int xr = (len - 1) / 2, half = M / 2;
  const float2* src = packed + (size_t)b * n_px + start;
  float2* dst = images + (size_t)b * M * M + (size_t)(half + k - r) * M + (half - xr);
  for (int t = threadIdx.x; t < len; t += blockDim.x) dst[t] = __ldcs(src + t);
}

}  // namespace

cudaError_t launch_expand_disc(int M, int r, int B, const int* rows, const float* packed,
                               float* images, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  int n_px = 0;
  for (int ky = -r; ky <= r; ++ky) {
    int xr = 0;
    while ((xr + 1) * (xr + 1) <= r * r - ky * ky) ++xr;
    n_px += 2 * xr + 1;
  }
  k_expand_disc<<<dim3(2 * r + 1, B), 128, 0, s>>>(M, r, rows,
                                                   reinterpret_cast<const float2*>(packed), n_px,
                                                   reinterpret_cast<float2*>(images));
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace cs
