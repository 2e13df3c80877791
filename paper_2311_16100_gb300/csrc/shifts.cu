// In-plane shift operator T_i of Definition 2.1: a diagonal phase factor on
// the image grid, T_jj = exp(-2 pi i (kx tx + ky ty) / M) for a shift
// (tx, ty) in pixels (the Fourier shift theorem for a real-space shift by
// +t).  T is unitary and commutes with the diagonal CTF, so
//   |x - C T S v| = |T^* x - C S v|:
// the library's operators use the unshifted slice S and a dataset with
// known shifts is phase-corrected once (sign -1); the forward model applies
// T after the slice (sign +1).
//
// Phase reduction: 2 (kx tx + ky ty) / M is reduced modulo 2 exactly by
// splitting t = n / 1024 + t_lo (n integer, |t_lo| <= 1/2048): the integer
// part kx n + ky n' is reduced modulo 1024 M in 64-bit integers, and only the
// small t_lo term is rounded.
#include "internal.h"

namespace cs {

namespace {

__global__ void __launch_bounds__(256)
k_phase_shift(int M, int B, float2* __restrict__ img, const float* __restrict__ shifts,
              float sgn) {
  const long n_px = (long)M * M;
  const long total = n_px * B;
  const long L = 1024L * M;
  const float inv2L = 2.0f / (float)L;
  const float inv2M = 2.0f / (float)M;
  const int half = M / 2;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const long i = e / n_px;
    const int p = (int)(e - i * n_px);
    const int kx = p % M - half, ky = p / M - half;
    const float tx = shifts[2 * i], ty = shifts[2 * i + 1];
    const long long nx = __float2ll_rn(tx * 1024.0f), ny = __float2ll_rn(ty * 1024.0f);
    const float lx = tx - (float)nx * (1.0f / 1024.0f), ly = ty - (float)ny * (1.0f / 1024.0f);
    long long m = ((long long)kx * nx + (long long)ky * ny) % L;
    if (m < 0) m += L;
    const float ph = fmaf((float)m, inv2L, inv2M * fmaf((float)kx, lx, (float)ky * ly));
    float s, c;
    sincospif(ph, &s, &c);
    const float2 x = img[e];
    const float si = -sgn * s;                       // T = cos - i sin (sign +1)
    img[e] = make_float2(x.x * c - x.y * si, x.x * si + x.y * c);
  }
}

}  // namespace

cudaError_t launch_phase_shift(int M, int B, float2* images, const float* shifts, int sign,
                               int num_sms, cudaStream_t s) {
  const long total = (long)M * M * B;
  long g = (total + 255) / 256;
  if (g > (long)num_sms * 16) g = (long)num_sms * 16;
  if (g < 1) g = 1;
  k_phase_shift<<<(int)g, 256, 0, s>>>(M, B, images, shifts, sign > 0 ? 1.0f : -1.0f);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace cs
