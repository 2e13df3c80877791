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
// 2 GELU(x) = x + x tanh(u): five operations.  Exactly twice gelu_f (a power
// of two scales every rounding alike); the forward kernel takes the factor
// 1/2 into the next layer's weights instead.
__device__ __forceinline__ float gelu2_f(float x) {
  const float c = 0.7978845608028654f, c3 = 0.7978845608028654f * 0.044715f;
  const float t = tanh_hw(x * fmaf(c3, x * x, c));
  return fmaf(x, t, x);
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

// features of voxel j; in_ball: |k|^2 <= r2
__device__ __forceinline__ void features(int j, int M, const float* __restrict__ cov,
                                         const float* __restrict__ c2w, float x[3], int r2,
                                         bool& in_ball) {
  const int half = M / 2;
  const int ix = j % M, iy = (j / M) % M, iz = j / (M * M);
  const int kx = ix - half, ky = iy - half, kz = iz - half;
  const int q = kx * kx + ky * ky + kz * kz;
  x[0] = sqrtf((float)q) / (float)half;
  x[1] = log1pf(fmaxf(__ldg(cov + j), 0.f));
  x[2] = log1pf(fmaxf(__ldg(c2w + j), 0.f));
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

// byte offset of element (row, k) in a K-major canonical tile with K extent
// kext (LBO = 128 bytes, SBO = kext/8 * 128 bytes)
__device__ __forceinline__ uint32_t core_off(int row, int k, int kext) {
  return (uint32_t)((row >> 3) * (kext / 8) * 128 + (k >> 3) * 128 + (row & 7) * 16 +
                    (k & 7) * 2);
}


// eight consecutive K elements of one row of a K-major canonical tile are
// 16 contiguous bytes: stored with one 128-bit shared-memory store
__device__ __forceinline__ void st_bf16x8(unsigned char* base, uint32_t off, const float* v) {
  uint4 q;
  q.x = (uint32_t)bf16bits(v[0]) | ((uint32_t)bf16bits(v[1]) << 16);
  q.y = (uint32_t)bf16bits(v[2]) | ((uint32_t)bf16bits(v[3]) << 16);
  q.z = (uint32_t)bf16bits(v[4]) | ((uint32_t)bf16bits(v[5]) << 16);
  q.w = (uint32_t)bf16bits(v[6]) | ((uint32_t)bf16bits(v[7]) << 16);
  *reinterpret_cast<uint4*>(base + off) = q;
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
  float4 L1[kHid];                      // (W1[i][0..2], b1[i]): one load per unit
  float4 b2[kHid / 4];                  // b2, four units per load
  float4 w3[kHid / 4];                  // w3 / 2, four units per load
  float b3;
  unsigned long long bar;
  uint32_t tmem;
};

constexpr int kFeat = 2 * kHid;        // a voxel's row of the gradient kernel: dA2 | H1
struct GradSmem {
  // [voxel][feature], K-major with K extent 128: features 0..63 = bf(dA2)
  // (A of the backward MMA), 64..127 = bf(H1) (A of the forward MMA); read
  // as MN-major operands by the weight-gradient MMA
  unsigned short XV[kRows * kFeat];
  unsigned short W2[kHid * kHid];       // forward B: rows o, K = i
  unsigned short W2T[kHid * kHid];      // backward B: rows i, K = o
  float4 L1[kHid];                      // (W1[i][0..2], b1[i])
  float2 L2[kHid];                      // (b2[o], w3[o])
  float b3;
  float small[kSmall];                  // dW1, db1, db2, dw3, db3 of this CTA
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

// ------------------------------------------------------ tensor-core kernels
// logd[j] = MLP(features(j)) + offset (exp_out: exp(logd) + offset instead)
__global__ void __launch_bounds__(kRows)
k_mlp_forward_tc(int M, const float* __restrict__ params, const float* __restrict__ cov,
                 const float* __restrict__ c2w, float* __restrict__ out, int exp_out,
                 float offset, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  FwdSmem& S = *reinterpret_cast<FwdSmem*>(smem_raw);
  const int t = threadIdx.x, warp = t >> 5;
  const int n = M * M * M;
  const int n_tiles = (n + kRows - 1) / kRows;
  // Both activations are evaluated as 2 GELU (gelu2_f, one multiplication
  // fewer each); the factor 1/2 goes into W2 (halving commutes with the BF16
  // rounding) and into w3, so every product and sum equals the plain
  // network's.
  for (int i = threadIdx.x; i < kHid; i += blockDim.x)
    S.L1[i] = make_float4(params[oW1 + 3 * i], params[oW1 + 3 * i + 1], params[oW1 + 3 * i + 2],
                          params[ob1 + i]);
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
  for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
    const int j = tile * kRows + t;
    float x[3] = {0.f, 0.f, 0.f};
    bool inb = false;
    if (j < n) features(j, M, cov, c2w, x, 0x7fffffff, inb);
    unsigned char* H1b = reinterpret_cast<unsigned char*>(S.H1);
#pragma unroll 2
    for (int i0 = 0; i0 < kHid; i0 += 8) {
      float h[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = i0 + u;
        const float4 q = S.L1[i];
        h[u] = gelu2_f(fmaf(q.z, x[2], fmaf(q.y, x[1], fmaf(q.x, x[0], q.w))));
      }
      st_bf16x8(H1b, core_off(t, i0, kHid), h);
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
    float y = S.b3;
#pragma unroll
    for (int c = 0; c < kHid; c += 16) {
      float a2[16];
      tmem_ld16(lane_addr + c, a2);
#pragma unroll
      for (int u = 0; u < 16; u += 4) {
        const float4 bb = S.b2[(c + u) / 4], ww = S.w3[(c + u) / 4];
        y = fmaf(ww.x, gelu2_f(a2[u] + bb.x), y);
        y = fmaf(ww.y, gelu2_f(a2[u + 1] + bb.y), y);
        y = fmaf(ww.z, gelu2_f(a2[u + 2] + bb.z), y);
        y = fmaf(ww.w, gelu2_f(a2[u + 3] + bb.w), y);
      }
    }
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
// thread: four CTAs per SM (gradient 0.72 -> 0.63 ms at 128^3 against the
// earlier build with a separate transposed Gram operand, 256 columns and
// two CTAs per SM).
__global__ void __launch_bounds__(kRows, 4)
k_mlp_grad_tc(int M, int r2, float inv_n, const float* __restrict__ params,
              const float* __restrict__ cov, const float* __restrict__ c2w,
              const float* __restrict__ target, float* __restrict__ grad, double* __restrict__ sse,
              int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  GradSmem& S = *reinterpret_cast<GradSmem*>(smem_raw);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int n = M * M * M;
  const int n_tiles = (n + kRows - 1) / kRows;
  for (int i = threadIdx.x; i < kHid; i += blockDim.x) {
    S.L1[i] = make_float4(params[oW1 + 3 * i], params[oW1 + 3 * i + 1], params[oW1 + 3 * i + 2],
                          params[ob1 + i]);
    S.L2[i] = make_float2(params[ob2 + i], params[ow3 + i]);
  }
  if (t == 0) S.b3 = params[ob3];
  for (int e = t; e < kHid * kHid; e += kRows) {
    const int o = e / kHid, i = e % kHid;
    const unsigned short w = bf16bits(params[oW2 + e]);
    *reinterpret_cast<unsigned short*>(reinterpret_cast<unsigned char*>(S.W2) +
                                       core_off(o, i, kHid)) = w;
    *reinterpret_cast<unsigned short*>(reinterpret_cast<unsigned char*>(S.W2T) +
                                       core_off(i, o, kHid)) = w;
  }
  for (int i = t; i < kSmall; i += kRows) S.small[i] = 0.f;
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
  for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
    const int j = tile * kRows + t;
    float x[3] = {0.f, 0.f, 0.f};
    bool inb = false;
    if (j < n) features(j, M, cov, c2w, x, r2, inb);
    // ---- forward, layer 1 -> features 64..127 of this voxel's row
#pragma unroll 2
    for (int i0 = 0; i0 < kHid; i0 += 8) {
      float h[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float4 q = S.L1[i0 + u];
        h[u] = gelu_f(fmaf(q.z, x[2], fmaf(q.y, x[1], fmaf(q.x, x[0], q.w))));
      }
      st_bf16x8(XVb, core_off(t, kHid + i0, kFeat), h);
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
    // in 64 registers: 86 registers, no spills, gradient 0.631 -> 0.620 ms)
    float y = S.b3;
#pragma unroll
    for (int c = 0; c < kHid; c += 16) {
      float a2[16];
      tmem_ld16(d1 + lane_off + c, a2);
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const float2 q = S.L2[c + u];
        y = fmaf(q.y, gelu_f(a2[u] + q.x), y);
      }
    }
    const float r = inb ? y - __ldg(target + j) : 0.f;
    my_sse += (double)r * r;
    const float dy = 2.f * r * inv_n;
    float acc_db3 = dy;
    // dA2 -> features 0..63 of this voxel's row; dw3, db2
#pragma unroll
    for (int c = 0; c < kHid; c += 16) {
      float v[32], dab[8], a2[16];
      tmem_ld16(d1 + lane_off + c, a2);
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int o = c + u;
        const float a = a2[u] + S.L2[o].x;
        const float sg = gelu_sig(a);             // one tanh for GELU and GELU'
        const float h2 = a * sg;
        const float da = dy * S.L2[o].y * gelu_grad_s(a, sg);
        dab[u & 7] = da;
        if ((u & 7) == 7) st_bf16x8(XVb, core_off(t, o - 7, kFeat), dab);
        v[u] = dy * h2;          // dw3[o]
        v[16 + u] = da;          // db2[o]
      }
      warp_reduce_scatter(v, lane);
      // lane l holds element l: dw3[c + l] (l < 16) or db2[c + l - 16]
      atomicAdd(&S.small[lane < 16 ? 192 + 64 + 64 + c + lane : 192 + 64 + c + lane - 16], v[0]);
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) acc_db3 += __shfl_xor_sync(0xffffffffu, acc_db3, s);
    if (lane == 0) atomicAdd(&S.small[kSmall - 1], acc_db3);
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
    // ---- backward through layer 1: dA1 = dH1 * gelu'(A1); dW1, db1
#pragma unroll
    for (int c = 0; c < kHid; c += 8) {
      float dh[8];
      tmem_ld8(d1 + lane_off + c, dh);
      // v[4u + f] = dA1 x_f (f < 3) and dA1 (f = 3) of unit c + u
      float v[32];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float4 q = S.L1[c + u];
        const float a = fmaf(q.z, x[2], fmaf(q.y, x[1], fmaf(q.x, x[0], q.w)));
        const float da1 = dh[u] * gelu_grad_f(a);
        v[4 * u] = da1 * x[0];
        v[4 * u + 1] = da1 * x[1];
        v[4 * u + 2] = da1 * x[2];
        v[4 * u + 3] = da1;
      }
      warp_reduce_scatter(v, lane);
      // lane l holds element l: unit c + l/4, quantity l%4 (x0, x1, x2, bias)
      {
        const int i = c + (lane >> 2), f = lane & 3;
        atomicAdd(f < 3 ? &S.small[3 * i + f] : &S.small[192 + i], v[0]);
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
  __syncthreads();
  for (int i = t; i < kSmall; i += kRows) {
    const float v = S.small[i];
    int dst;
    if (i < 192) dst = oW1 + i;
    else if (i < 256) dst = ob1 + (i - 192);
    else if (i < 320) dst = ob2 + (i - 256);
    else if (i < 384) dst = ow3 + (i - 320);
    else dst = ob3;
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
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    float x[3];
    bool inb;
    features(j, M, cov, c2w, x, 0x7fffffff, inb);
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
  const int n_tiles = (n + kRows - 1) / kRows;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int j = tile * kRows + t;
    float x[3] = {0.f, 0.f, 0.f};
    bool inb = false;
    if (j < n) features(j, M, cov, c2w, x, r2, inb);
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
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_forward_tc,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(FwdSmem));
    if (e != cudaSuccess) return e;
    configured = true;
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
    static bool configured_ref = false;
    if (!configured_ref) {
      cudaError_t e = cudaFuncSetAttribute(k_mlp_grad_ref,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
      if (e != cudaSuccess) return e;
      configured_ref = true;
    }
    const int g = tiles < num_sms * 2 ? tiles : num_sms * 2;
    k_mlp_grad_ref<<<g, kRows, dyn, s>>>(M, r2, inv_n, params, cov, c2w, target, grad, sse);
    count_launches(1);
    return cudaGetLastError();
  }
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kGradSmemBytes);
    if (e != cudaSuccess) return e;
    configured = true;
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
