// Per-shell reductions over a Fourier volume: the Fourier shell correlation
// of two volumes (Eq. fsc, Section 4) and the per-shell count, minimum and
// maximum of a real field (the conditioning analysis of Section 3.1, where
// the diagonal of H is read shell by shell).
//
// Shell of voxel k (k = index - M/2 on each axis): r = round(|k|), i.e. the
// integer r with r^2 - r + 1 <= |k|^2 <= r^2 + r (r = 0 for k = 0); |k|^2 is
// an integer so no rounding tie can occur.  Voxels with r >= n_shells are
// ignored.  Each block accumulates in shared memory and flushes one global
// atomic per shell and quantity.
#include "internal.h"

namespace cs {

namespace {

constexpr int kShellThreads = 512;

__device__ __forceinline__ int shell_of(int q) {
  int r = (int)sqrt((double)q);          // exact floor for q < 2^52
  if (r * r > q) --r;
  if ((r + 1) * (r + 1) <= q) ++r;
  return q > r * r + r ? r + 1 : r;
}

__device__ __forceinline__ unsigned ordered(float x) {
  const unsigned u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float unordered(unsigned u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// sums[r] = (Re sum u conj(v), sum |u|^2, sum |v|^2) over shell r.
__global__ void __launch_bounds__(kShellThreads)
k_fsc_accum(int M, const float2* __restrict__ u, const float2* __restrict__ v, int n_sh,
            double* __restrict__ sums) {
  extern __shared__ double sh[];
  for (int i = threadIdx.x; i < 3 * n_sh; i += blockDim.x) sh[i] = 0.0;
  __syncthreads();
  const int half = M / 2;
  const long n = (long)M * M * M;
  for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n;
       j += (long)gridDim.x * blockDim.x) {
    const int x = (int)(j % M), y = (int)((j / M) % M), z = (int)(j / ((long)M * M));
    const int kx = x - half, ky = y - half, kz = z - half;
    const int r = shell_of(kx * kx + ky * ky + kz * kz);
    if (r >= n_sh) continue;
    const float2 a = u[j], b = v[j];
    atomicAdd(&sh[3 * r], (double)a.x * b.x + (double)a.y * b.y);
    atomicAdd(&sh[3 * r + 1], (double)a.x * a.x + (double)a.y * a.y);
    atomicAdd(&sh[3 * r + 2], (double)b.x * b.x + (double)b.y * b.y);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 3 * n_sh; i += blockDim.x)
    if (sh[i] != 0.0) atomicAdd(&sums[i], sh[i]);
}

__global__ void k_fsc_final(int n_sh, const double* __restrict__ sums, double* __restrict__ fsc) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_sh) return;
  const double d = sums[3 * r + 1] * sums[3 * r + 2];
  fsc[r] = d > 0.0 ? sums[3 * r] / sqrt(d) : 0.0;
}

// count[r], and min/max of x over shell r as order-preserving words.
__global__ void __launch_bounds__(kShellThreads)
k_shell_minmax(int M, const float* __restrict__ x, int n_sh, unsigned* __restrict__ lo,
               unsigned* __restrict__ hi, int* __restrict__ count) {
  extern __shared__ unsigned shu[];
  unsigned* slo = shu;
  unsigned* shi = shu + n_sh;
  int* scnt = reinterpret_cast<int*>(shu + 2 * n_sh);
  for (int i = threadIdx.x; i < n_sh; i += blockDim.x) {
    slo[i] = 0xffffffffu;
    shi[i] = 0u;
    scnt[i] = 0;
  }
  __syncthreads();
  const int half = M / 2;
  const long n = (long)M * M * M;
  for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n;
       j += (long)gridDim.x * blockDim.x) {
    const int ix = (int)(j % M), iy = (int)((j / M) % M), iz = (int)(j / ((long)M * M));
    const int kx = ix - half, ky = iy - half, kz = iz - half;
    const int r = shell_of(kx * kx + ky * ky + kz * kz);
    if (r >= n_sh) continue;
    const unsigned o = ordered(x[j]);
    atomicMin(&slo[r], o);
    atomicMax(&shi[r], o);
    atomicAdd(&scnt[r], 1);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n_sh; i += blockDim.x) {
    if (scnt[i] == 0) continue;
    atomicMin(&lo[i], slo[i]);
    atomicMax(&hi[i], shi[i]);
    atomicAdd(&count[i], scnt[i]);
  }
}

__global__ void k_shell_minmax_final(int n_sh, unsigned* __restrict__ lo, unsigned* __restrict__ hi,
                                     const int* __restrict__ count) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_sh) return;
  float* flo = reinterpret_cast<float*>(lo);
  float* fhi = reinterpret_cast<float*>(hi);
  if (count[r] == 0) {
    flo[r] = __int_as_float(0x7f800000);     // +inf
    fhi[r] = __int_as_float(0xff800000);     // -inf
  } else {
    flo[r] = unordered(lo[r]);
    fhi[r] = unordered(hi[r]);
  }
}

__global__ void k_fill_u32(int n, unsigned* __restrict__ p, unsigned val) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = val;
}

int shell_grid(int num_sms, long n) {
  const long want = (n + kShellThreads - 1) / kShellThreads;
  const long cap = 2L * num_sms;
  return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

cudaError_t launch_fsc(int M, const float2* u, const float2* v, int n_sh, double* sums,
                       double* fsc, int num_sms, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(sums, 0, sizeof(double) * 3 * n_sh, s);
  if (e != cudaSuccess) return e;
  const long n = (long)M * M * M;
  const size_t smem = sizeof(double) * 3 * n_sh;
  k_fsc_accum<<<shell_grid(num_sms, n), kShellThreads, smem, s>>>(M, u, v, n_sh, sums);
  count_launches(1);
  if (fsc) {
    k_fsc_final<<<(n_sh + 127) / 128, 128, 0, s>>>(n_sh, sums, fsc);
    count_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_shell_minmax(int M, const float* x, int n_sh, float* lo, float* hi, int* count,
                                int num_sms, cudaStream_t s) {
  unsigned* ulo = reinterpret_cast<unsigned*>(lo);
  unsigned* uhi = reinterpret_cast<unsigned*>(hi);
  const int g = (n_sh + 127) / 128;
  k_fill_u32<<<g, 128, 0, s>>>(n_sh, ulo, 0xffffffffu);
  k_fill_u32<<<g, 128, 0, s>>>(n_sh, uhi, 0u);
  count_launches(2);
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * n_sh, s);
  if (e != cudaSuccess) return e;
  const long n = (long)M * M * M;
  const size_t smem = sizeof(unsigned) * 3 * n_sh;
  k_shell_minmax<<<shell_grid(num_sms, n), kShellThreads, smem, s>>>(M, x, n_sh, ulo, uhi, count);
  k_shell_minmax_final<<<g, 128, 0, s>>>(n_sh, ulo, uhi, count);
  count_launches(2);
  return cudaGetLastError();
}

}  // namespace cs
