// Learned diagonal preconditioner: a 3 -> 64 -> 64 -> 1 GELU network that
// maps per-voxel features (|k| / (M/2), log1p(pose coverage),
// log1p(sum C^2 w)) to log D, trained by mean squared error against
// Hutchinson estimates of the diagonal (Eq. hutch).  Not in the paper.
//
// Two implementations of forward and gradient:
//  * tensor cores (sm_103a): one CTA of 128 threads per tile of 128 voxels
//    (thread t owns voxel row t = TMEM lane t).  The 64 x 64 layer
//    H1 W2^T and the input gradient dA2 W2 are tcgen05.mma kind::f16
//    (BF16 operands in shared memory, FP32 accumulators in tensor memory,
//    M = 128, N = 64, K = 64).  In the gradient kernel each voxel's row
//    [bf(dA2) | bf(H1)] (128 features) is one row of a shared buffer; the
//    weight gradient dA2^T H1 comes from the same buffer read as
//    MN-major operands (M = 128 features, N = the 64 H1 features, K = 128
//    voxels: rows 0..63 of the product), accumulated in tensor memory over
//    all tiles of the CTA.  The 3 -> 64 and 64 -> 1 layers and the bias /
//    small-layer gradients run on the FP32 pipes.  Operands use the
//    no-swizzle canonical layouts: 8-row x 16-byte core matrices; K-major:
//    LBO = next core matrix along K, SBO = next 8-row group; MN-major:
//    LBO = next 8 rows along K, SBO = next core matrix along M (or N).
//  * FP32 reference (any GPU): the same arithmetic (same BF16 rounding
//    points) with plain FMAs, used to cross-check the tensor-core kernels.
#include <cuda_bf16.h>

#include "internal.h"

namespace cs {

namespace {

constexpr int kHid = 64;
constexpr int kRows = 128;                      // voxels per tile
constexpr int oW1 = 0, ob1 = 192, oW2 = 256, ob2 = 4352, ow3 = 4416, ob3 = 4480;
constexpr int kNP = 4481;                        // parameters
constexpr int kSmall = 192 + 64 + 64 + 64 + 1;  // dW1, db1, db2, dw3, db3
constexpr long long kWaitLimit = 1ll << 26;     // bounded mbarrier waits

// GELU with the tanh approximation; tanh from the hardware instruction
// tanh.approx.f32 (maximum relative error about 2^-11: below the BF16
// rounding the hidden layer takes, and a few 1e-4 of the output).
__device__ __forceinline__ float tanh_hw(float u) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(u));
  return t;
}
// s = 0.5 (1 + tanh(u)),  u = sqrt(2/pi) (x + 0.044715 x^3)
__device__ __forceinline__ float gelu_sig(float x) {
  const float c = 0.7978845608028654f;           // sqrt(2/pi)
  return fmaf(0.5f, tanh_hw(c * fmaf(0.044715f * x * x, x, x)), 0.5f);
}
// GELU(x) = x s = 0.5 x + 0.5 x tanh(u), with u = x (c + c 0.044715 x^2):
// six operations (the same u up to rounding)
__device__ __forceinline__ float gelu_f(float x) {
  const float c = 0.7978845608028654f, c3 = 0.7978845608028654f * 0.044715f;
  const float t = tanh_hw(x * fmaf(c3, x * x, c));
  const float hx = 0.5f * x;
  return fmaf(hx, t, hx);
}
// d/dx GELU = s + x s (1 - s) 2c (1 + 3 * 0.044715 x^2), s = 0.5 (1 + tanh(u))
__device__ __forceinline__ float gelu_grad_s(float x, float s) {
  const float c = 0.7978845608028654f;
  return fmaf(x * s * (1.f - s), 2.f * c * fmaf(3.f * 0.044715f, x * x, 1.f), s);
}
__device__ __forceinline__ float gelu_grad_f(float x) { return gelu_grad_s(x, gelu_sig(x)); }
__device__ __forceinline__ float bf16r(float x) {
  return __bfloat162float(__float2bfloat16_rn(x));
}
__device__ __forceinline__ unsigned short bf16bits(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// ---- the activations of two units at once, with the packed FP32 pairs of
// device.cuh (fma2 and kin): the scalar work around the MMAs (the
// activations and their derivatives) is what bounds the tensor-core
// kernels, and pairing halves its instruction count.
constexpr float kGc = 0.7978845608028654f;       // sqrt(2/pi)
constexpr float kGc3 = 0.7978845608028654f * 0.044715f;
__device__ __forceinline__ float2 tanh2(float2 u) { return make_float2(tanh_hw(u.x), tanh_hw(u.y)); }
// 2 GELU(x) = x + x tanh(u) of both lanes: five operations.  Exactly twice
// gelu_f (a power of two scales every rounding alike); the forward kernel
// takes the factor 1/2 into the next layer's weights instead.
__device__ __forceinline__ float2 gelu2_x2(float2 x) {
  const float2 t = tanh2(mul2(x, fma2(dup2(kGc3), mul2(x, x), dup2(kGc))));
  return fma2(x, t, x);
}
// gelu_f of both lanes
__device__ __forceinline__ float2 gelu_x2(float2 x) {
  const float2 t = tanh2(mul2(x, fma2(dup2(kGc3), mul2(x, x), dup2(kGc))));
  const float2 hx = mul2(dup2(0.5f), x);
  return fma2(hx, t, hx);
}
// gelu_sig of both lanes
__device__ __forceinline__ float2 gelu_sig_x2(float2 x) {
  const float2 q = mul2(mul2(dup2(0.044715f), x), x);
  const float2 t = tanh2(mul2(dup2(kGc), fma2(q, x, x)));
  return fma2(dup2(0.5f), t, dup2(0.5f));
}
// gelu_grad_s of both lanes, given xs = x s (1 - s is s (-1) + 1: exact
// product, one rounding, as the scalar subtraction)
__device__ __forceinline__ float2 gelu_grad_x2(float2 x, float2 s, float2 xs) {
  const float2 p = mul2(xs, fma2(s, dup2(-1.f), dup2(1.f)));
  const float2 g = mul2(dup2(2.f * kGc), fma2(dup2(3.f * 0.044715f), mul2(x, x), dup2(1.f)));
  return fma2(p, g, s);
}
// two BF16 (round to nearest even), the first in the low half
__device__ __forceinline__ uint32_t bf16x2_bits(float2 v) {
  const __nv_bfloat162 b = __floats2bfloat162_rn(v.x, v.y);
  return *reinterpret_cast<const uint32_t*>(&b);
}

// Grid of the features: M, M/2 and their reciprocals.
struct FeatGrid {
  int M, half;
  float inv_M, inv_half;
};
__device__ __forceinline__ FeatGrid feat_grid(int M) {
  return FeatGrid{M, M / 2, 1.f / (float)M, 1.f / (float)(M / 2)};
}
// q = a / d, *rem = a mod d for 0 <= a < 2^27, 1 <= d <= 512: the float
// quotient a * (1/d) is within 20/d of a/d (float(a) within 4, 1/d and the
// product within 2^-24 relative each), so below 1 for d >= 20 and far below
// it for smaller d (then a < 2^24 and float(a) is exact); one correction
// step makes it exact.
__device__ __forceinline__ int div_grid(int a, int d, float inv_d, int* rem) {
  int q = (int)((float)a * inv_d);
  int r = a - q * d;
  if (r < 0) {
    --q;
    r += d;
  } else if (r >= d) {
    ++q;
    r -= d;
  }
  *rem = r;
  return q;
}
// features of voxel j (cov_j, c2w_j: its inputs); in_ball: |k|^2 <= r2.
// log1p(c) for c >= 0 as the hardware logarithm of 1 + c (absolute error a
// few 1e-7: far below the BF16 rounding of the first hidden layer)
__device__ __forceinline__ void features(int j, const FeatGrid& G, float cov_j, float c2w_j,
                                         float x[3], int r2, bool& in_ball) {
  int ix, iy;
  const int jm = div_grid(j, G.M, G.inv_M, &ix);
  const int iz = div_grid(jm, G.M, G.inv_M, &iy);
  const int kx = ix - G.half, ky = iy - G.half, kz = iz - G.half;
  const int q = kx * kx + ky * ky + kz * kz;
  x[0] = sqrtf((float)q) * G.inv_half;
  x[1] = __logf(1.f + fmaxf(cov_j, 0.f));
  x[2] = __logf(1.f + fmaxf(c2w_j, 0.f));
  in_ball = q <= r2;
}

// ------------------------------------------------------------------ PTX
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// K-major, no-swizzle descriptor: start, LBO (K step), SBO (8-row step)
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;                       // descriptor version of sm_100 family
  return d;                                     // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: BF16 A and B, FP32 D, K-major A and B
// (mn_major: both MN-major instead)
__host__ __device__ constexpr uint32_t umma_idesc(int m, int n, bool mn_major = false) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (mn_major ? (3u << 15) : 0u) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(bar) : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void bar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar) : "memory");
}

// waits for phase `parity` of the barrier; false if the wait ran out
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity,
                                         long long limit = kWaitLimit) {
  for (long long it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 8 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive FP32 columns, issued without waiting: the registers are
// valid after tmem_wait16 on the same array, which names them as operands so
// that no use of them is scheduled before the wait
__device__ __forceinline__ void tmem_issue16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait16(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :: "memory");
}

// byte offset of element (row, k) in a K-major canonical tile with K extent
// kext (LBO = 128 bytes, SBO = kext/8 * 128 bytes)
__device__ __forceinline__ uint32_t core_off(int row, int k, int kext) {
  return (uint32_t)((row >> 3) * (kext / 8) * 128 + (k >> 3) * 128 + (row & 7) * 16 +
                    (k & 7) * 2);
}


// Warp reduce-scatter: on return, lane l holds in v[0 .. N/32) the warp-wide
// sums of elements l*N/32 .. (l+1)*N/32 - 1 (five butterfly rounds, each
// lane sending the half it does not keep).  N is a multiple of 32.
template <int N>
__device__ __forceinline__ void warp_reduce_scatter(float (&v)[N], int lane) {
#pragma unroll
  for (int s = 16, L = N; s > 0; s >>= 1, L >>= 1) {
    const bool up = (lane & s) != 0;
#pragma unroll
    for (int i = 0; i < L / 2; ++i) {
      const float lo = v[i], hi = v[i + L / 2];
      const float got = __shfl_xor_sync(0xffffffffu, up ? lo : hi, s);
      v[i] = (up ? hi : lo) + got;
    }
  }
}

// ------------------------------------------------------ shared layouts
struct FwdSmem {
  unsigned short W2[kHid * kHid];       // B operand: rows o (N), K = i; bf(W2 / 2)
  unsigned short H1[kRows * kHid];      // A operand: rows = voxels, K = i; bf(2 H1)
  float4 L1[kHid];                      // layer 1 by unit pairs: see pair_l1
  float4 b2[kHid / 4];                  // b2, four units per load
  float4 w3[kHid / 4];                  // w3 / 2, four units per load
  float b3;
  unsigned long long bar;
  uint32_t tmem;
};

constexpr int kFeat = 2 * kHid;        // a voxel's row of the gradient kernel: dA2 | H1
constexpr int kSmallTc = 2 * kHid + 1;  // db2, dw3, db3 (tensor-core gradient kernel)
struct GradSmem {
  // [voxel][feature], K-major with K extent 128: features 0..63 = bf(dA2)
  // (A of the backward MMA), 64..127 = bf(H1) (A of the forward MMA); read
  // as MN-major operands by the weight-gradient MMA
  unsigned short XV[kRows * kFeat];
  unsigned short W2[kHid * kHid];       // forward B: rows o, K = i
  unsigned short W2T[kHid * kHid];      // backward B: rows i, K = o
  float4 L1[kHid];                      // layer 1 by unit pairs: see pair_l1
  float4 L2[kHid / 2];                  // (b2[o], b2[o+1], w3[o], w3[o+1]), o even
  float4 X[kRows];                      // (x0, x1, x2, 1) of the tile's voxels
  float b3;
  float small[kSmallTc];                // db2, dw3, db3 of this CTA
  unsigned long long bar;
  uint32_t tmem;
};

// Dynamic shared memory of the gradient kernel (four CTAs fit on an SM).
constexpr size_t kGradSmemBytes = sizeof(GradSmem);

__device__ __forceinline__ void load_params(const float* __restrict__ p, float* W1, float* b1,
                                            float* b2, float* w3, float* b3) {
  for (int i = threadIdx.x; i < 192; i += blockDim.x) W1[i] = p[oW1 + i];
  for (int i = threadIdx.x; i < 64; i += blockDim.x) {
    b1[i] = p[ob1 + i];
    b2[i] = p[ob2 + i];
    w3[i] = p[ow3 + i];
  }
  if (threadIdx.x == 0) *b3 = p[ob3];
}

// Layer 1 in unit pairs: entries 2p and 2p+1 of L1 hold units 2p, 2p+1 as
// (W1[2p][0], W1[2p+1][0], W1[2p][1], W1[2p+1][1]) and
// (W1[2p][2], W1[2p+1][2], b1[2p], b1[2p+1]).
__device__ __forceinline__ void pair_l1(const float* __restrict__ params, float4* L1) {
  for (int p = threadIdx.x; p < kHid / 2; p += blockDim.x) {
    const float* w = params + oW1 + 6 * p;
    L1[2 * p] = make_float4(w[0], w[3], w[1], w[4]);
    L1[2 * p + 1] = make_float4(w[2], w[5], params[ob1 + 2 * p], params[ob1 + 2 * p + 1]);
  }
}
// pre-activations of units 2p, 2p+1: ((W1 x_0 + b1) + W1 x_1) + W1 x_2, the
// order of the scalar kernels
__device__ __forceinline__ float2 layer1_x2(const float4* L1, int p, float2 X0, float2 X1,
                                           float2 X2) {
  const float4 qa = L1[2 * p], qb = L1[2 * p + 1];
  float2 a = fma2(make_float2(qa.x, qa.y), X0, make_float2(qb.z, qb.w));
  a = fma2(make_float2(qa.z, qa.w), X1, a);
  return fma2(make_float2(qb.x, qb.y), X2, a);
}

// ------------------------------------------------------ tensor-core kernels
// logd[j] = MLP(features(j)) + offset (exp_out: exp(logd) + offset instead)
__global__ void __launch_bounds__(kRows, 8)
k_mlp_forward_tc(int M, const float* __restrict__ params, const float* __restrict__ cov,
                 const float* __restrict__ c2w, float* __restrict__ out, int exp_out,
                 float offset, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  FwdSmem& S = *reinterpret_cast<FwdSmem*>(smem_raw);
  const int t = threadIdx.x, warp = t >> 5;
  const int n = M * M * M;
  const FeatGrid G = feat_grid(M);
  const int n_tiles = (n + kRows - 1) / kRows;
  // Both activations are evaluated as 2 GELU (gelu2_x2, one multiplication
  // fewer each); the factor 1/2 goes into W2 (halving commutes with the BF16
  // rounding) and into w3, so every product and sum equals the plain
  // network's.
  pair_l1(params, S.L1);
  for (int i = threadIdx.x; i < kHid / 4; i += blockDim.x) {
    S.b2[i] = make_float4(params[ob2 + 4 * i], params[ob2 + 4 * i + 1], params[ob2 + 4 * i + 2],
                          params[ob2 + 4 * i + 3]);
    S.w3[i] = make_float4(0.5f * params[ow3 + 4 * i], 0.5f * params[ow3 + 4 * i + 1],
                          0.5f * params[ow3 + 4 * i + 2], 0.5f * params[ow3 + 4 * i + 3]);
  }
  if (t == 0) S.b3 = params[ob3];
  for (int e = t; e < kHid * kHid; e += kRows) {
    const int o = e / kHid, i = e % kHid;
    *reinterpret_cast<unsigned short*>(reinterpret_cast<unsigned char*>(S.W2) +
                                       core_off(o, i, kHid)) = bf16bits(0.5f * params[oW2 + e]);
  }
  if (t == 0) bar_init(smem_u32(&S.bar));
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;"
                 :: "r"(smem_u32(&S.tmem)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = S.tmem;
  const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
  const uint32_t bar = smem_u32(&S.bar);
  const uint32_t idesc = umma_idesc(128, 64);
  uint32_t phase = 0;
  bool ok = true;
  // inputs of the next tile, loaded one tile ahead
  float cov_n = 0.f, c2w_n = 0.f;
  if (blockIdx.x * kRows + t < n) {
    cov_n = __ldg(cov + blockIdx.x * kRows + t);
    c2w_n = __ldg(c2w + blockIdx.x * kRows + t);
  }
  for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
    const int j = tile * kRows + t;
    const float cov_j = cov_n, c2w_j = c2w_n;
    const int jn = j + (int)gridDim.x * kRows;
    if (jn < n) {
      cov_n = __ldg(cov + jn);
      c2w_n = __ldg(c2w + jn);
    }
    float x[3] = {0.f, 0.f, 0.f};
    bool inb = false;
    if (j < n) features(j, G, cov_j, c2w_j, x, 0x7fffffff, inb);
    unsigned char* H1b = reinterpret_cast<unsigned char*>(S.H1);
    const float2 X0 = dup2(x[0]), X1 = dup2(x[1]), X2 = dup2(x[2]);
#pragma unroll 2
    for (int i0 = 0; i0 < kHid; i0 += 8) {
      uint32_t w[4];
#pragma unroll
      for (int p = 0; p < 4; ++p)
        w[p] = bf16x2_bits(gelu2_x2(layer1_x2(S.L1, i0 / 2 + p, X0, X1, X2)));
      *reinterpret_cast<uint4*>(H1b + core_off(t, i0, kHid)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (t == 0) {
      fence_after();
      const uint32_t aB = smem_u32(S.H1), bB = smem_u32(S.W2);
#pragma unroll
      for (int kc = 0; kc < kHid / 16; ++kc)
        mma_bf16(tmem, umma_desc(aB + 256 * kc, 128, 1024), umma_desc(bB + 256 * kc, 128, 1024),
                 idesc, kc > 0);
      mma_commit(bar);
    }
    ok = __syncthreads_and(bar_wait(bar, phase)) != 0;
    phase ^= 1u;
    fence_after();
    if (!ok) break;
    // output: units 4m, 4m+1 and 4m+2, 4m+3 summed in four chains, then
    // added; the next 16 columns are loaded while these are evaluated
    float2 ya = make_float2(S.b3, 0.f), yb = make_float2(0.f, 0.f);
    uint32_t a2[2][16];
    tmem_issue16(lane_addr, a2[0]);
    tmem_wait16(a2[0]);
#pragma unroll
    for (int c = 0; c < kHid; c += 16) {
      uint32_t (&cur)[16] = a2[(c / 16) & 1];
      if (c + 16 < kHid) tmem_issue16(lane_addr + c + 16, a2[(c / 16 + 1) & 1]);
#pragma unroll
      for (int u = 0; u < 16; u += 4) {
        const float4 bb = S.b2[(c + u) / 4], ww = S.w3[(c + u) / 4];
        ya = fma2(make_float2(ww.x, ww.y),
                  gelu2_x2(add2(make_float2(__uint_as_float(cur[u]), __uint_as_float(cur[u + 1])),
                                make_float2(bb.x, bb.y))),
                  ya);
        yb = fma2(make_float2(ww.z, ww.w),
                  gelu2_x2(add2(make_float2(__uint_as_float(cur[u + 2]),
                                            __uint_as_float(cur[u + 3])),
                                make_float2(bb.z, bb.w))),
                  yb);
      }
      if (c + 16 < kHid) tmem_wait16(a2[(c / 16 + 1) & 1]);
    }
    const float y = (ya.x + ya.y) + (yb.x + yb.y);
    if (j < n) out[j] = (exp_out ? expf(y) : y) + offset;
    fence_before();
    __syncthreads();
  }
  if (!ok && t == 0) atomicExch(err, 1);
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" :: "r"(tmem));
  }
}

// Gradient of L = (1/n_ball) sum_{|k| <= r} (y_j - target_j)^2 (accumulated
// into grad with atomics), and the sum of squared residuals into *sse.
// 128 TMEM columns per CTA (the layer-2 accumulator, reused for the
// backward product, and the weight gradient) and at most 128 registers per
// thread: four CTAs per SM.  Units are evaluated in pairs with packed FP32
// instructions.  dW1 and db1 are sums over voxels of dA1 x: each tile's dA1
// (FP32, the tile's rows of the shared buffer once the MMAs have read them)
// is summed column-wise, thread t accumulating unit t/2 over every other
// voxel across all the CTA's tiles, so no per-tile reduction is needed.
// Byte offset of dA1[v][i] in that buffer: rows of 64 floats, 16-byte chunks
// permuted by a bit reversal of v mod 8, so that the row-wise stores and
// the column-wise loads are both free of bank conflicts.
__device__ __forceinline__ uint32_t da1_off(int v, int i) {
  const int r = v & 7;
  const int sw = ((r & 1) << 2) | (r & 2) | (r >> 2);
  return (uint32_t)(v * 256 + (((i >> 2) ^ sw) << 4) + ((i & 3) << 2));
}

__global__ void __launch_bounds__(kRows, 4)
k_mlp_grad_tc(int M, int r2, float inv_n, const float* __restrict__ params,
              const float* __restrict__ cov, const float* __restrict__ c2w,
              const float* __restrict__ target, float* __restrict__ grad, double* __restrict__ sse,
              int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  GradSmem& S = *reinterpret_cast<GradSmem*>(smem_raw);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int n = M * M * M;
  const FeatGrid G = feat_grid(M);
  const int n_tiles = (n + kRows - 1) / kRows;
  pair_l1(params, S.L1);
  for (int p = threadIdx.x; p < kHid / 2; p += blockDim.x)
    S.L2[p] = make_float4(params[ob2 + 2 * p], params[ob2 + 2 * p + 1], params[ow3 + 2 * p],
                          params[ow3 + 2 * p + 1]);
  if (t == 0) S.b3 = params[ob3];
  for (int e = t; e < kHid * kHid; e += kRows) {
    const int o = e / kHid, i = e % kHid;
    const unsigned short w = bf16bits(params[oW2 + e]);
    *reinterpret_cast<unsigned short*>(reinterpret_cast<unsigned char*>(S.W2) +
                                       core_off(o, i, kHid)) = w;
    *reinterpret_cast<unsigned short*>(reinterpret_cast<unsigned char*>(S.W2T) +
                                       core_off(i, o, kHid)) = w;
  }
  for (int i = t; i < kSmallTc; i += kRows) S.small[i] = 0.f;
  if (t == 0) bar_init(smem_u32(&S.bar));
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;"
                 :: "r"(smem_u32(&S.tmem)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = S.tmem;
  const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
  // columns 0..63: layer-2 pre-activation, then the backward product dA2 W2;
  // columns 64..127: the weight gradient (rows 0..63 of its product)
  const uint32_t d1 = tmem, d3 = tmem + 64;
  const uint32_t bar = smem_u32(&S.bar);
  const uint32_t idesc64 = umma_idesc(128, 64), idesc_w = umma_idesc(128, 64, true);
  uint32_t phase = 0;
  bool ok = true;
  int tiles_done = 0;
  double my_sse = 0.0;
  unsigned char* XVb = reinterpret_cast<unsigned char*>(S.XV);
  // dW1 column sums of this thread: unit iu, voxels of parity hv
  const int iu = t >> 1, hv = t & 1;
  float2 g01 = make_float2(0.f, 0.f), g23 = make_float2(0.f, 0.f);
  uint32_t coff[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) coff[q] = da1_off(2 * q + hv, iu) - (uint32_t)((2 * q + hv) * 256);
  // inputs of the next tile, loaded one tile ahead
  float cov_n = 0.f, c2w_n = 0.f, tgt_n = 0.f;
  if (blockIdx.x * kRows + t < n) {
    cov_n = __ldg(cov + blockIdx.x * kRows + t);
    c2w_n = __ldg(c2w + blockIdx.x * kRows + t);
    tgt_n = __ldg(target + blockIdx.x * kRows + t);
  }
  for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
    const int j = tile * kRows + t;
    const float cov_j = cov_n, c2w_j = c2w_n, tgt_j = tgt_n;
    const int jn = j + (int)gridDim.x * kRows;
    if (jn < n) {
      cov_n = __ldg(cov + jn);
      c2w_n = __ldg(c2w + jn);
      tgt_n = __ldg(target + jn);
    }
    float x[3] = {0.f, 0.f, 0.f};
    bool inb = false;
    if (j < n) features(j, G, cov_j, c2w_j, x, r2, inb);
    S.X[t] = make_float4(x[0], x[1], x[2], 1.f);
    const float2 X0 = dup2(x[0]), X1 = dup2(x[1]), X2 = dup2(x[2]);
    // ---- forward, layer 1 -> features 64..127 of this voxel's row
#pragma unroll 2
    for (int i0 = 0; i0 < kHid; i0 += 8) {
      uint32_t w[4];
#pragma unroll
      for (int p = 0; p < 4; ++p)
        w[p] = bf16x2_bits(gelu_x2(layer1_x2(S.L1, i0 / 2 + p, X0, X1, X2)));
      *reinterpret_cast<uint4*>(XVb + core_off(t, kHid + i0, kFeat)) =
          make_uint4(w[0], w[1], w[2], w[3]);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (t == 0) {
      fence_after();
      const uint32_t aB = smem_u32(S.XV) + core_off(0, kHid, kFeat), bB = smem_u32(S.W2);
#pragma unroll
      for (int kc = 0; kc < kHid / 16; ++kc)
        mma_bf16(d1, umma_desc(aB + 256 * kc, 128, 2048), umma_desc(bB + 256 * kc, 128, 1024),
                 idesc64, kc > 0);
      mma_commit(bar);
    }
    ok = __syncthreads_and(bar_wait(bar, phase)) != 0;
    phase ^= 1u;
    fence_after();
    if (!ok) break;
    // ---- forward, layers 2-3, loss, backward through layer 3 (the
    // pre-activation is read from tensor memory twice instead of being held
    // in 64 registers)
    float2 ya = make_float2(S.b3, 0.f), yb = make_float2(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < kHid; c += 16) {
      float a2[16];
      tmem_ld16(d1 + lane_off + c, a2);
#pragma unroll
      for (int u = 0; u < 16; u += 4) {
        const float4 q = S.L2[(c + u) / 2], q1 = S.L2[(c + u) / 2 + 1];
        ya = fma2(make_float2(q.z, q.w),
                  gelu_x2(add2(make_float2(a2[u], a2[u + 1]), make_float2(q.x, q.y))), ya);
        yb = fma2(make_float2(q1.z, q1.w),
                  gelu_x2(add2(make_float2(a2[u + 2], a2[u + 3]), make_float2(q1.x, q1.y))), yb);
      }
    }
    const float y = (ya.x + ya.y) + (yb.x + yb.y);
    const float r = inb ? y - tgt_j : 0.f;
    my_sse += (double)r * r;
    const float dy = 2.f * r * inv_n;
    const float2 DY = dup2(dy);
    float acc_db3 = dy;
    // dA2 -> features 0..63 of this voxel's row; dw3, db2
#pragma unroll
    for (int c = 0; c < kHid; c += 16) {
      float v[32], a2[16];
      uint32_t dab[4];
      tmem_ld16(d1 + lane_off + c, a2);
#pragma unroll
      for (int u = 0; u < 16; u += 2) {
        const float4 q = S.L2[(c + u) / 2];
        const float2 a = add2(make_float2(a2[u], a2[u + 1]), make_float2(q.x, q.y));
        const float2 sg = gelu_sig_x2(a);       // one tanh for GELU and GELU'
        const float2 h2 = mul2(a, sg);
        const float2 da = mul2(mul2(DY, make_float2(q.z, q.w)), gelu_grad_x2(a, sg, h2));
        dab[(u & 7) >> 1] = bf16x2_bits(da);
        if ((u & 7) == 6)
          *reinterpret_cast<uint4*>(XVb + core_off(t, c + u - 6, kFeat)) =
              make_uint4(dab[0], dab[1], dab[2], dab[3]);
        const float2 dw = mul2(DY, h2);
        v[u] = dw.x;             // dw3[o]
        v[u + 1] = dw.y;
        v[16 + u] = da.x;        // db2[o]
        v[17 + u] = da.y;
      }
      warp_reduce_scatter(v, lane);
      // lane l holds element l: dw3[c + l] (l < 16) or db2[c + l - 16]
      atomicAdd(&S.small[lane < 16 ? kHid + c + lane : c + lane - 16], v[0]);
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) acc_db3 += __shfl_xor_sync(0xffffffffu, acc_db3, s);
    if (lane == 0) atomicAdd(&S.small[2 * kHid], acc_db3);
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (t == 0) {
      fence_after();
      const uint32_t xB = smem_u32(S.XV), bB = smem_u32(S.W2T);
      // dH1 = bf(dA2) W2 into columns 0..63 (layer 2's pre-activation has
      // been read by every thread)
#pragma unroll
      for (int kc = 0; kc < kHid / 16; ++kc)
        mma_bf16(d1, umma_desc(xB + 256 * kc, 128, 2048), umma_desc(bB + 256 * kc, 128, 1024),
                 idesc64, kc > 0);
      // weight gradient: rows = the 128 features of the tile's rows, columns =
      // the H1 features 64..127, K = voxels; MN-major without swizzling: 8
      // features per 16-byte core row, next 8 voxels (LBO) 2048 bytes on,
      // next 8 features (SBO) 128 bytes on
#pragma unroll
      for (int kc = 0; kc < kRows / 16; ++kc)
        mma_bf16(d3, umma_desc(xB + 4096 * kc, 2048, 128),
                 umma_desc(xB + core_off(0, kHid, kFeat) + 4096 * kc, 2048, 128), idesc_w,
                 (tiles_done > 0 || kc > 0) ? 1u : 0u);
      mma_commit(bar);
    }
    ok = __syncthreads_and(bar_wait(bar, phase)) != 0;
    phase ^= 1u;
    fence_after();
    if (!ok) break;
    ++tiles_done;
    // ---- backward through layer 1: dA1 = dH1 * gelu'(A1) into this
    // voxel's row of the buffer (both MMAs have read it)
#pragma unroll
    for (int c = 0; c < kHid; c += 8) {
      float dh[8];
      tmem_ld8(d1 + lane_off + c, dh);
      float4 da1[2];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const float2 a = layer1_x2(S.L1, c / 2 + p, X0, X1, X2);
        const float2 sg = gelu_sig_x2(a);
        const float2 d = mul2(make_float2(dh[2 * p], dh[2 * p + 1]),
                              gelu_grad_x2(a, sg, mul2(a, sg)));
        if (p & 1) { da1[p >> 1].z = d.x; da1[p >> 1].w = d.y; }
        else { da1[p >> 1].x = d.x; da1[p >> 1].y = d.y; }
      }
      *reinterpret_cast<float4*>(XVb + da1_off(t, c)) = da1[0];
      *reinterpret_cast<float4*>(XVb + da1_off(t, c + 4)) = da1[1];
    }
    __syncthreads();
    // dW1[iu][0..2], db1[iu] += sum over this parity's voxels of dA1 (x, 1)
    {
      const unsigned char* col = XVb + hv * 256;
      const float4* xs = S.X + hv;
#pragma unroll 4
      for (int k = 0; k < kRows / 2; ++k) {
        const float d = *reinterpret_cast<const float*>(col + k * 512 + coff[k & 3]);
        const float4 xv = xs[2 * k];
        g01 = fma2(dup2(d), make_float2(xv.x, xv.y), g01);
        g23 = fma2(dup2(d), make_float2(xv.z, xv.w), g23);
      }
    }
    fence_before();
    __syncthreads();
  }
  if (!ok && t == 0) atomicExch(err, 1);
  fence_before();
  __syncthreads();
  fence_after();
  // dW2[o][i] = row o (lanes 0..63: warps 0 and 1), column i of the weight
  // gradient's accumulator
  if (ok && tiles_done > 0 && t < 64) {
#pragma unroll
    for (int c = 0; c < kHid; c += 16) {
      float gv[16];
      tmem_ld16(d3 + lane_off + c, gv);
#pragma unroll
      for (int u = 0; u < 16; ++u) atomicAdd(grad + oW2 + t * kHid + c + u, gv[u]);
    }
  }
  // dW1, db1: the two voxel parities of unit iu, added by the even thread
  g01.x += __shfl_xor_sync(0xffffffffu, g01.x, 1);
  g01.y += __shfl_xor_sync(0xffffffffu, g01.y, 1);
  g23.x += __shfl_xor_sync(0xffffffffu, g23.x, 1);
  g23.y += __shfl_xor_sync(0xffffffffu, g23.y, 1);
  if (ok && tiles_done > 0 && hv == 0) {
    atomicAdd(grad + oW1 + 3 * iu, g01.x);
    atomicAdd(grad + oW1 + 3 * iu + 1, g01.y);
    atomicAdd(grad + oW1 + 3 * iu + 2, g23.x);
    atomicAdd(grad + ob1 + iu, g23.y);
  }
  __syncthreads();
  for (int i = t; i < kSmallTc; i += kRows) {
    const float v = S.small[i];
    const int dst = i < kHid ? ob2 + i : (i < 2 * kHid ? ow3 + (i - kHid) : ob3);
    atomicAdd(grad + dst, v);
  }
  double s = block_sum(my_sse);
  if (t == 0) atomicAdd(sse, s);
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" :: "r"(tmem));
  }
}

// ------------------------------------------------------ FP32 reference kernels
__global__ void __launch_bounds__(128)
k_mlp_forward_ref(int M, const float* __restrict__ params, const float* __restrict__ cov,
                  const float* __restrict__ c2w, float* __restrict__ out, int exp_out,
                  float offset) {
  __shared__ float W1[192], b1[64], W2[kHid * kHid], b2[64], w3[64], b3;
  load_params(params, W1, b1, b2, w3, &b3);
  for (int e = threadIdx.x; e < kHid * kHid; e += blockDim.x) W2[e] = bf16r(params[oW2 + e]);
  __syncthreads();
  const int n = M * M * M;
  const FeatGrid G = feat_grid(M);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    float x[3];
    bool inb;
    features(j, G, __ldg(cov + j), __ldg(c2w + j), x, 0x7fffffff, inb);
    float h1[kHid];
#pragma unroll
    for (int i = 0; i < kHid; ++i)
      h1[i] = bf16r(gelu_f(fmaf(W1[3 * i + 2], x[2], fmaf(W1[3 * i + 1], x[1],
                                                          fmaf(W1[3 * i], x[0], b1[i])))));
    float y = b3;
    for (int o = 0; o < kHid; ++o) {
      float a = 0.f;
#pragma unroll
      for (int i = 0; i < kHid; ++i) a = fmaf(W2[o * kHid + i], h1[i], a);
      y = fmaf(w3[o], gelu_f(a + b2[o]), y);
    }
    out[j] = (exp_out ? expf(y) : y) + offset;
  }
}

__global__ void __launch_bounds__(128)
k_mlp_grad_ref(int M, int r2, float inv_n, const float* __restrict__ params,
               const float* __restrict__ cov, const float* __restrict__ c2w,
               const float* __restrict__ target, float* __restrict__ grad,
               double* __restrict__ sse) {
  __shared__ float W1[192], b1[64], b2[64], w3[64], b3;
  __shared__ float small[kSmall];
  extern __shared__ float dyn[];
  float* W2 = dyn;                                            // [64][64]
  float (*H1s)[kHid + 1] = reinterpret_cast<float (*)[kHid + 1]>(dyn + kHid * kHid);
  float (*DAs)[kHid + 1] = reinterpret_cast<float (*)[kHid + 1]>(dyn + kHid * kHid +
                                                                 kRows * (kHid + 1));
  load_params(params, W1, b1, b2, w3, &b3);
  for (int e = threadIdx.x; e < kHid * kHid; e += blockDim.x) W2[e] = bf16r(params[oW2 + e]);
  for (int i = threadIdx.x; i < kSmall; i += blockDim.x) small[i] = 0.f;
  const int t = threadIdx.x;
  // this thread's 32 outputs of dW2: entries t*32 .. t*32+31
  float gW2[32];
#pragma unroll
  for (int u = 0; u < 32; ++u) gW2[u] = 0.f;
  double my_sse = 0.0;
  __syncthreads();
  const int n = M * M * M;
  const FeatGrid G = feat_grid(M);
  const int n_tiles = (n + kRows - 1) / kRows;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int j = tile * kRows + t;
    float x[3] = {0.f, 0.f, 0.f};
    bool inb = false;
    if (j < n) features(j, G, __ldg(cov + j), __ldg(c2w + j), x, r2, inb);
    float h1[kHid];
#pragma unroll
    for (int i = 0; i < kHid; ++i) {
      h1[i] = bf16r(gelu_f(fmaf(W1[3 * i + 2], x[2], fmaf(W1[3 * i + 1], x[1],
                                                          fmaf(W1[3 * i], x[0], b1[i])))));
      H1s[t][i] = h1[i];
    }
    float a2[kHid];
    float y = b3;
    for (int o = 0; o < kHid; ++o) {
      float a = 0.f;
#pragma unroll
      for (int i = 0; i < kHid; ++i) a = fmaf(W2[o * kHid + i], h1[i], a);
      a2[o] = a + b2[o];
      y = fmaf(w3[o], gelu_f(a2[o]), y);
    }
    const float r = inb ? y - target[j] : 0.f;
    my_sse += (double)r * r;
    const float dy = 2.f * r * inv_n;
    atomicAdd(&small[kSmall - 1], dy);
    for (int o = 0; o < kHid; ++o) {
      const float da = dy * w3[o] * gelu_grad_f(a2[o]);
      DAs[t][o] = bf16r(da);
      atomicAdd(&small[320 + o], dy * gelu_f(a2[o]));
      atomicAdd(&small[256 + o], da);
    }
    // dH1 = bf(dA2) W2, then dA1
    for (int i = 0; i < kHid; ++i) {
      float dh = 0.f;
      for (int o = 0; o < kHid; ++o) dh = fmaf(DAs[t][o], W2[o * kHid + i], dh);
      const float a = fmaf(W1[3 * i + 2], x[2], fmaf(W1[3 * i + 1], x[1],
                                                     fmaf(W1[3 * i], x[0], b1[i])));
      const float da1 = dh * gelu_grad_f(a);
      atomicAdd(&small[3 * i], da1 * x[0]);
      atomicAdd(&small[3 * i + 1], da1 * x[1]);
      atomicAdd(&small[3 * i + 2], da1 * x[2]);
      atomicAdd(&small[192 + i], da1);
    }
    __syncthreads();
    // dW2[o][i] += sum_v bf(dA2)[v][o] bf(H1)[v][i], outputs t*32..t*32+31
#pragma unroll 4
    for (int u = 0; u < 32; ++u) {
      const int e = t * 32 + u, o = e / kHid, i = e % kHid;
      float s = 0.f;
      for (int v = 0; v < kRows; ++v) s = fmaf(DAs[v][o], H1s[v][i], s);
      gW2[u] += s;
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 32; ++u) atomicAdd(grad + oW2 + t * 32 + u, gW2[u]);
  __syncthreads();
  for (int i = t; i < kSmall; i += blockDim.x) {
    int dst;
    if (i < 192) dst = oW1 + i;
    else if (i < 256) dst = ob1 + (i - 192);
    else if (i < 320) dst = ob2 + (i - 256);
    else if (i < 384) dst = ow3 + (i - 320);
    else dst = ob3;
    atomicAdd(grad + dst, small[i]);
  }
  double s = block_sum(my_sse);
  if (t == 0) atomicAdd(sse, s);
}

// Adam (Kingma & Ba 2015) on the FP32 master parameters, gradient gs * g;
// g is zeroed.
__global__ void k_adam(int np, float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       float* __restrict__ g, float gs, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
    const float gi = gs * g[i];
    const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
    const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    g[i] = 0.f;
  }
}

// Network target, pass 1: m_j = mean of the n_est estimates of voxel j into
// out; per block, the sum and the count of the positive m_j (part[b],
// part[gridDim.x + b]).
__global__ void __launch_bounds__(256)
k_target_mean(int n, int n_est, const float* __restrict__ est, float* __restrict__ out,
              double* __restrict__ part) {
  const float inv = 1.f / (float)n_est;
  float s = 0.f, c = 0.f;
  for (int j = blockIdx.x * 256 + threadIdx.x; j < n; j += gridDim.x * 256) {
    float a = 0.f;
    for (int e = 0; e < n_est; ++e) a += __ldg(est + (size_t)e * n + j);
    a *= inv;
    out[j] = a;
    if (a > 0.f) {
      s += a;
      c += 1.f;
    }
  }
  const double ts = block_sum_f(s);
  const double tc = block_sum_f(c);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = ts;
    part[gridDim.x + blockIdx.x] = tc;
  }
}

// pass 2: every block sums pass 1's nb partials (warp 0), then
// out_j = log(max(m_j, floor_rel * mean of the positive m))
__global__ void __launch_bounds__(256)
k_target_log(int n, int nb, const double* __restrict__ part, float floor_rel,
             float* __restrict__ out) {
  __shared__ float fl;
  if (threadIdx.x < 32) {
    double s = 0.0, c = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) {
      s += part[b];
      c += part[nb + b];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_xor_sync(0xffffffffu, s, o);
      c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if (threadIdx.x == 0) fl = c > 0.0 ? (float)(floor_rel * (s / c)) : floor_rel;
  }
  __syncthreads();
  const float f = fl;
  for (int j = blockIdx.x * 256 + threadIdx.x; j < n; j += gridDim.x * 256)
    out[j] = logf(fmaxf(out[j], f));
}

}  // namespace

size_t mlp_fwd_smem() { return sizeof(FwdSmem); }
size_t mlp_grad_smem() { return kGradSmemBytes; }

namespace {

// One block whose mbarrier wait can never complete (one arrival expected,
// none made): the wait gives up after `limit` polls and records the expiry
// in the status word, as the tensor-core kernels do.
__global__ void k_wait_selftest(long long limit, int* __restrict__ err) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) bar_init(smem_u32(&bar));
  __syncthreads();
  const bool ok = bar_wait(smem_u32(&bar), 0u, limit);
  if (!ok && threadIdx.x == 0) atomicExch(err, 1);
}

}  // namespace

cudaError_t launch_wait_selftest(long long limit, int* err, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(limit, err);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_mlp_forward(int M, const float* params, const float* cov, const float* c2w,
                               float* out, int exp_out, float offset, bool tc, int* err,
                               int num_sms, cudaStream_t s) {
  const int n = M * M * M;
  if (!tc) {
    const int g = (n + 127) / 128;
    k_mlp_forward_ref<<<g < num_sms * 16 ? g : num_sms * 16, 128, 0, s>>>(M, params, cov, c2w,
                                                                         out, exp_out, offset);
    count_launches(1);
    return cudaGetLastError();
  }
  static std::atomic<uint64_t> configured{0};
  {
    const cudaError_t e = ensure_smem_limit(k_mlp_forward_tc, (int)sizeof(FwdSmem), configured);
    if (e != cudaSuccess) return e;
  }
  // eight CTAs per SM: 8 x 64 TMEM columns, the whole tensor memory
  const int tiles = (n + kRows - 1) / kRows;
  const int g = tiles < num_sms * 8 ? tiles : num_sms * 8;
  k_mlp_forward_tc<<<g, kRows, sizeof(FwdSmem), s>>>(M, params, cov, c2w, out, exp_out, offset,
                                                     err);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_mlp_grad(int M, int r2, float inv_n, const float* params, const float* cov,
                            const float* c2w, const float* target, float* grad, double* sse,
                            bool tc, int* err, int num_sms, cudaStream_t s) {
  const int n = M * M * M;
  const int tiles = (n + kRows - 1) / kRows;
  if (!tc) {
    const size_t dyn = sizeof(float) * (kHid * kHid + 2 * kRows * (kHid + 1));
    static std::atomic<uint64_t> configured_ref{0};
    {
      const cudaError_t e = ensure_smem_limit(k_mlp_grad_ref, (int)dyn, configured_ref);
      if (e != cudaSuccess) return e;
    }
    const int g = tiles < num_sms * 2 ? tiles : num_sms * 2;
    k_mlp_grad_ref<<<g, kRows, dyn, s>>>(M, r2, inv_n, params, cov, c2w, target, grad, sse);
    count_launches(1);
    return cudaGetLastError();
  }
  static std::atomic<uint64_t> configured{0};
  {
    const cudaError_t e = ensure_smem_limit(k_mlp_grad_tc, (int)kGradSmemBytes, configured);
    if (e != cudaSuccess) return e;
  }
  // four CTAs per SM: 4 x 128 TMEM columns, the whole tensor memory
  const int g = tiles < num_sms * 4 ? tiles : num_sms * 4;
  k_mlp_grad_tc<<<g, kRows, kGradSmemBytes, s>>>(M, r2, inv_n, params, cov, c2w, target, grad,
                                                 sse, err);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* p, float* m, float* v, float* g, float gscale, int step,
                        float lr, float b1, float b2, float eps, cudaStream_t s) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adam<<<(kNP + 255) / 256, 256, 0, s>>>(kNP, p, m, v, g, gscale, lr, b1, b2, eps, c1, c2);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_mlp_target(int M, int n_est, const float* est, float floor_rel,
                              float* target, double* part, int num_sms, cudaStream_t s) {
  const int n = M * M * M;
  int g = (n + 255) / 256;
  if (g > num_sms * 4) g = num_sms * 4;
  k_target_mean<<<g, 256, 0, s>>>(n, n_est, est, target, part);
  k_target_log<<<g, 256, 0, s>>>(n, g, part, floor_rel, target);
  count_launches(2);
  return cudaGetLastError();
}

}  // namespace cs
