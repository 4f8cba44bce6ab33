// K7: the learned drag closure's network on the 5th-generation tensor cores.
//
// MLP 6 -> 128 -> 128 -> 128 -> 128 -> 3 with ReLU, BF16 operands and FP32
// accumulation.  Every layer product (forward: H_l = act(H_{l-1} W_l^T + b);
// backward: dH_{l-1} = (dH_l W_l) * relu'(H_{l-1})) is a 128-sample tile
// times a weight matrix, issued as tcgen05.mma (kind::f16, M = 128, N = 16 or
// 128, K = 16 per instruction) by one thread of the CTA, with both operands
// in shared memory in the canonical K-major layout without swizzle (8x8
// core matrices of 128 contiguous bytes; LBO = stride between core matrices
// along K, SBO = stride between 8-row groups) and the accumulator in tensor
// memory.  Completion is signalled through tcgen05.commit on an mbarrier;
// the epilogue reads the accumulator with tcgen05.ld (32 lanes x 16 columns
// per instruction), adds the bias, applies ReLU and writes the next operand.
// Weight gradients dW_l = dH_l^T H_{l-1} are a reduction over the minibatch
// done on the FP32 cores; Adam keeps FP32 master weights and refreshes the
// BF16 tiles (W in [out][in] and W^T in [in][out] core-matrix order).
//
// Every wait on an mbarrier is bounded: after the poll limit the kernel sets
// an error flag, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "lbm_internal.cuh"

namespace mlp {

constexpr int H = 128;      // hidden width
constexpr int IN = 6;       // features
constexpr int OUT = 3;      // outputs
constexpr int KIN = 16;     // padded input width
constexpr int NOUT = 16;    // padded output width
constexpr int TILE = 128;   // samples per CTA tile
constexpr long long kPollLimit = 1ll << 26;
enum : int { MERR_TIMEOUT = 1 };

// layer shapes (out, in) and padded (N, K) of the forward products
__host__ __device__ constexpr int lay_out(int l) { return l == 4 ? OUT : H; }
__host__ __device__ constexpr int lay_in(int l) { return l == 0 ? IN : H; }
__host__ __device__ constexpr int lay_N(int l) { return l == 4 ? NOUT : H; }
__host__ __device__ constexpr int lay_K(int l) { return l == 0 ? KIN : H; }

// --------------------------------------------------------------------------
// canonical K-major layout without swizzle: element (r, k) of an R x K tile
// --------------------------------------------------------------------------
__host__ __device__ __forceinline__ int cm_index(int r, int k, int K) {
  return (((r >> 3) * (K >> 3) + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor (tcgen05): start, LBO, SBO in 16-byte
// units, descriptor version 1 at bit 46, no swizzle
__device__ __forceinline__ uint64_t smem_desc(const void* base, int K) {
  const uint64_t addr = smem_u32(base);
  const uint64_t lbo = 128;                    // next core matrix along K
  const uint64_t sbo = (uint64_t)(K >> 3) * 128;  // next 8-row group
  return ((addr >> 4) & 0x3FFF) | (((lbo >> 4) & 0x3FFF) << 16) | (((sbo >> 4) & 0x3FFF) << 32) |
         (1ull << 46);
}

// instruction descriptor, kind::f16: D F32, A and B BF16, both K-major
__device__ __forceinline__ uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// bounded wait for the phase with the given parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long long i = 0; i < kPollLimit; i++) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T, one instruction (K = 16)
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       int accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 lanes (rows) x 16 columns of FP32 accumulator into registers
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&r)[16]) {
  uint32_t u[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
        "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; i++) r[i] = __uint_as_float(u[i]);
}

// tensor memory of the CTA: 256 columns (accumulators of up to N = 128 twice)
constexpr uint32_t kTmemCols = 256;

__device__ __forceinline__ void tmem_alloc(uint32_t* slot) {
  // one full warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(kTmemCols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_free(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTmemCols));
}

// D (128 x N) = A (128 x K) * B (N x K)^T, issued by thread 0, waited by all;
// returns false on timeout.  Caller has fenced the operand writes.
__device__ __forceinline__ bool tc_gemm(const __nv_bfloat16* A, const __nv_bfloat16* B, int N, int K,
                                        uint32_t tmem_d, uint64_t* bar, uint32_t& phase) {
  if (threadIdx.x == 0) {
    tc_fence_after();
    const uint32_t idesc = instr_desc(128, N);
    for (int kk = 0; kk < K; kk += 16) {
      // the K-chunk starts at core-matrix column kk/8: byte offset (kk/8)*128
      const uint64_t ad = smem_desc(A + (kk >> 3) * 64, K);
      const uint64_t bd = smem_desc(B + (kk >> 3) * 64, K);
      tc_mma(tmem_d, ad, bd, idesc, kk > 0 ? 1 : 0);
    }
    tc_commit(bar);
  }
  const bool ok = mbar_wait(bar, phase);
  phase ^= 1u;
  tc_fence_after();
  return __syncthreads_and(ok) != 0;  // one verdict for the whole CTA
}

// --------------------------------------------------------------------------
// parameter block (device), see lbm_imb_mlp_* in the header
// --------------------------------------------------------------------------
struct Params {
  float* w[5];             // FP32 master weights [out][in]
  float* b[5];             // FP32 biases
  float* mw[5];            // Adam first moments
  float* vw[5];            // Adam second moments
  float* mb[5];
  float* vb[5];
  float* gw[5];            // weight gradients
  float* gb[5];
  __nv_bfloat16* wt[5];    // BF16 W in [N][K] core-matrix order (forward B operand)
  __nv_bfloat16* wtt[5];   // BF16 W^T in [N=in][K=out] core-matrix order (backward B operand)
  float* norm;             // x_mean[6], x_std[6], y_mean[3], y_std[3]
  // activations of the current minibatch (BF16, row-major [sample][feature])
  __nv_bfloat16* act[5];   // act[0] = normalised input (KIN wide), act[l] = H_l (H wide)
  __nv_bfloat16* dact[5];  // dact[l] = dL/dpre-activation of layer l (N wide)
  float* y;                // network output, normalised [B][NOUT]
  float* loss;             // [1]
  int* err;                // [1]
};

__device__ __forceinline__ void stage_weights(__nv_bfloat16* dst, const __nv_bfloat16* src, int elems) {
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* d = reinterpret_cast<uint4*>(dst);
  for (int i = threadIdx.x; i < elems / 8; i += blockDim.x) d[i] = s[i];
}

// shared memory of the forward/backward kernels
struct SmemFwd {
  __nv_bfloat16 w1[H * KIN];
  __nv_bfloat16 w[3][H * H];
  __nv_bfloat16 w5[NOUT * H];
  __nv_bfloat16 a[TILE * H];     // current activation tile (K-major)
  __nv_bfloat16 x[TILE * KIN];   // input tile
  uint64_t bar;
  uint32_t tmem;
};

// forward pass over tiles of 128 samples; train = 1 keeps the activations
__global__ void __launch_bounds__(128) mlp_forward_kernel(Params P, const float* x, int B, int train,
                                                          float* y_out) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  SmemFwd& S = *reinterpret_cast<SmemFwd*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5;
  stage_weights(S.w1, P.wt[0], H * KIN);
  for (int l = 0; l < 3; l++) stage_weights(S.w[l], P.wt[l + 1], H * H);
  stage_weights(S.w5, P.wt[4], NOUT * H);
  if (tid == 0) mbar_init(&S.bar, 1);
  if (warp == 0) tmem_alloc(&S.tmem);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem;
  uint32_t phase = 0;
  bool ok = true;
  const float* nm = P.norm;
  const int ntiles = (B + TILE - 1) / TILE;
  for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
    const int row = t * TILE + tid;  // this thread's sample (row of the tile)
    const bool valid = row < B;
    // normalised input -> BF16 operand
#pragma unroll
    for (int k = 0; k < KIN; k++) {
      float v = 0.f;
      if (k < IN && valid) v = (x[(size_t)row * IN + k] - nm[k]) / nm[IN + k];
      const __nv_bfloat16 bv = __float2bfloat16_rn(v);
      S.x[cm_index(tid, k, KIN)] = bv;
      if (train && valid) P.act[0][(size_t)row * KIN + k] = bv;
    }
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    for (int l = 0; l < 5 && ok; l++) {
      const __nv_bfloat16* A = l == 0 ? S.x : S.a;
      const __nv_bfloat16* Bm = l == 0 ? S.w1 : (l == 4 ? S.w5 : S.w[l - 1]);
      ok = tc_gemm(A, Bm, lay_N(l), lay_K(l), tmem, &S.bar, phase);
      if (!ok) break;
      // epilogue: this warp's 32 rows
      const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
      const float* bias = P.b[l];
      for (int c0 = 0; c0 < lay_N(l); c0 += 16) {
        float r[16];
        tc_ld16(lane_base + c0, r);
        if (l < 4) {
#pragma unroll
          for (int i = 0; i < 16; i++) {
            const float hv = fmaxf(r[i] + bias[c0 + i], 0.f);
            const __nv_bfloat16 bv = __float2bfloat16_rn(hv);
            S.a[cm_index(tid, c0 + i, H)] = bv;
            if (train && valid) P.act[l + 1][(size_t)row * H + c0 + i] = bv;
          }
        } else if (valid) {
#pragma unroll
          for (int i = 0; i < OUT; i++) {
            const float yv = r[i] + bias[i];
            if (train) P.y[(size_t)row * NOUT + i] = yv;
            if (y_out) y_out[(size_t)row * OUT + i] = yv * nm[2 * IN + OUT + i] + nm[2 * IN + i];
          }
        }
      }
      proxy_fence();
      tc_fence_before();
      __syncthreads();
    }
  }
  if (!ok && tid == 0) atomicOr(P.err, MERR_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_free(tmem);
}

// backward (data) pass: dY from the loss, then dH_{l-1} = (dH_l W_l) * relu'(H_{l-1})
struct SmemBwd {
  __nv_bfloat16 w5t[H * NOUT];   // W5^T: N = 128 (in), K = 16 (out, padded)
  __nv_bfloat16 wt[3][H * H];    // W4^T, W3^T, W2^T
  __nv_bfloat16 d[TILE * H];     // current gradient tile (K-major)
  uint64_t bar;
  uint32_t tmem;
};

__global__ void __launch_bounds__(128) mlp_backward_kernel(Params P, const float* tgt, int B) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  SmemBwd& S = *reinterpret_cast<SmemBwd*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5;
  stage_weights(S.w5t, P.wtt[4], H * NOUT);
  for (int l = 0; l < 3; l++) stage_weights(S.wt[l], P.wtt[3 - l], H * H);  // W4^T, W3^T, W2^T
  if (tid == 0) mbar_init(&S.bar, 1);
  if (warp == 0) tmem_alloc(&S.tmem);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem;
  uint32_t phase = 0;
  bool ok = true;
  const float* nm = P.norm;
  const float scale = 2.f / (float)(B * OUT);
  const int ntiles = (B + TILE - 1) / TILE;
  float lsum = 0.f;
  for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
    const int row = t * TILE + tid;
    const bool valid = row < B;
    // dL/dy of the normalised output (mean squared error)
#pragma unroll
    for (int k = 0; k < NOUT; k++) {
      float g = 0.f;
      if (k < OUT && valid) {
        const float th = (tgt[(size_t)row * OUT + k] - nm[2 * IN + k]) / nm[2 * IN + OUT + k];
        const float e = P.y[(size_t)row * NOUT + k] - th;
        lsum += e * e;
        g = scale * e;
      }
      const __nv_bfloat16 bg = __float2bfloat16_rn(g);
      S.d[cm_index(tid, k, NOUT)] = bg;
      if (valid) P.dact[4][(size_t)row * NOUT + k] = bg;
    }
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    // layers 4..1: product with W_l, then the ReLU mask of H_l's pre-activation
    for (int l = 4; l >= 1 && ok; l--) {
      // B operand of step l is W_l^T (staged: w5t = W_4^T, wt[3 - l] = W_l^T)
      const __nv_bfloat16* Bt = l == 4 ? S.w5t : S.wt[3 - l];
      ok = tc_gemm(S.d, Bt, H, l == 4 ? NOUT : H, tmem, &S.bar, phase);
      if (!ok) break;
      const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
      for (int c0 = 0; c0 < H; c0 += 16) {
        float r[16];
        tc_ld16(lane_base + c0, r);
#pragma unroll
        for (int i = 0; i < 16; i++) {
          float g = 0.f;
          if (valid) {
            const float hv = __bfloat162float(P.act[l][(size_t)row * H + c0 + i]);
            g = hv > 0.f ? r[i] : 0.f;
          }
          const __nv_bfloat16 bg = __float2bfloat16_rn(g);
          S.d[cm_index(tid, c0 + i, H)] = bg;
          if (valid) P.dact[l - 1][(size_t)row * H + c0 + i] = bg;
        }
      }
      proxy_fence();
      tc_fence_before();
      __syncthreads();
    }
  }
  // loss (mean squared error of this minibatch)
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, o);
  if ((tid & 31) == 0 && lsum != 0.f) atomicAdd(P.loss, lsum / (float)(B * OUT));
  if (!ok && tid == 0) atomicOr(P.err, MERR_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_free(tmem);
}

// dW_l[o][i] = sum_m dact[l][m][o] * act[l][m][i],  db_l[o] = sum_m dact[l][m][o]
// (FP32 cores; one 32x32 output block per CTA, minibatch in chunks of 64)
__global__ void __launch_bounds__(256) mlp_wgrad_kernel(Params P, int B, int l) {
  const int OUTl = lay_out(l), INl = lay_in(l);
  const int Nst = lay_N(l), Kst = lay_K(l);  // row strides of dact[l] and act[l]
  const int o0 = blockIdx.y * 32, i0 = blockIdx.x * 32;
  __shared__ float sd[64][33], sa[64][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  float bacc = 0.f;
  for (int m0 = 0; m0 < B; m0 += 64) {
    for (int e = threadIdx.x; e < 64 * 32; e += 256) {
      const int mm = e >> 5, c = e & 31, m = m0 + mm;
      sd[mm][c] = (m < B && o0 + c < OUTl) ? __bfloat162float(P.dact[l][(size_t)m * Nst + o0 + c]) : 0.f;
      sa[mm][c] = (m < B && i0 + c < INl) ? __bfloat162float(P.act[l][(size_t)m * Kst + i0 + c]) : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int mm = 0; mm < 64; mm++) {
      const float av = sa[mm][tx];
#pragma unroll
      for (int j = 0; j < 4; j++) acc[j] += sd[mm][ty + 8 * j] * av;
      if (blockIdx.x == 0 && ty == 0) bacc += sd[mm][tx];
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; j++) {
    const int o = o0 + ty + 8 * j, i = i0 + tx;
    if (o < OUTl && i < INl) P.gw[l][o * INl + i] = acc[j];
  }
  if (blockIdx.x == 0 && ty == 0 && o0 + tx < OUTl) P.gb[l][o0 + tx] = bacc;
}

// Adam on the FP32 masters, then the BF16 operand tiles
__global__ void mlp_adam_kernel(Params P, int l, float lr, float c1, float c2) {
  const int OUTl = lay_out(l), INl = lay_in(l);
  const int nw = OUTl * INl;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  if (i < nw) {
    const float g = P.gw[l][i];
    const float m = b1 * P.mw[l][i] + (1.f - b1) * g;
    const float v = b2 * P.vw[l][i] + (1.f - b2) * g * g;
    P.mw[l][i] = m;
    P.vw[l][i] = v;
    P.w[l][i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
  }
  if (i < OUTl) {
    const float g = P.gb[l][i];
    const float m = b1 * P.mb[l][i] + (1.f - b1) * g;
    const float v = b2 * P.vb[l][i] + (1.f - b2) * g * g;
    P.mb[l][i] = m;
    P.vb[l][i] = v;
    P.b[l][i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
  }
}

// FP32 masters -> BF16 operand tiles (zero padded)
__global__ void mlp_pack_kernel(Params P, int l) {
  const int OUTl = lay_out(l), INl = lay_in(l), N = lay_N(l), K = lay_K(l);
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * K) return;
  const int n = e / K, k = e % K;  // forward operand: [n = out][k = in]
  const float wv = (n < OUTl && k < INl) ? P.w[l][n * INl + k] : 0.f;
  P.wt[l][cm_index(n, k, K)] = __float2bfloat16_rn(wv);
  // backward operand W^T: [n' = in][k' = out], K' = N (padded out width)
  P.wtt[l][cm_index(k, n, N)] = __float2bfloat16_rn(wv);
}

__global__ void mlp_zero_kernel(float* p, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = 0.f;
}

// GEMM probe: D (128 x N) = A (128 x K) * B (N x K)^T through the same
// tcgen05 path (test hook for the operand layout)
__global__ void __launch_bounds__(128) mlp_probe_kernel(const __nv_bfloat16* a, const __nv_bfloat16* b, int N,
                                                        int K, float* d, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __nv_bfloat16* A = reinterpret_cast<__nv_bfloat16*>(smem_raw);
  __nv_bfloat16* Bs = A + 128 * 128;
  uint64_t* bar = reinterpret_cast<uint64_t*>(Bs + 128 * 128);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int e = tid; e < 128 * K; e += 128) A[cm_index(e / K, e % K, K)] = a[e];
  for (int e = tid; e < N * K; e += 128) Bs[cm_index(e / K, e % K, K)] = b[e];
  if (tid == 0) mbar_init(bar, 1);
  if (warp == 0) tmem_alloc(tslot);
  proxy_fence();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  uint32_t phase = 0;
  const bool ok = tc_gemm(A, Bs, N, K, tmem, bar, phase);
  if (ok) {
    for (int c0 = 0; c0 < N; c0 += 16) {
      float r[16];
      tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c0, r);
#pragma unroll
      for (int i = 0; i < 16; i++) d[tid * N + c0 + i] = r[i];
    }
  } else if (tid == 0) {
    atomicOr(err, MERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_free(tmem);
}

}  // namespace mlp

// ============================================================================
// C ABI
// ============================================================================
using namespace mlp;

struct lbm_imb_mlp {
  Params P;
  cudaStream_t stream;
  int64_t max_batch;
  int64_t adam_t;
  int grid;
  float* loss_host_tmp;
};

namespace {
size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

struct MlpLayout {
  size_t off[64];
  size_t total;
};

// sizes of every array of the parameter block, in a fixed order
void mlp_sizes(int64_t B, size_t* sz, int* n) {
  int k = 0;
  for (int l = 0; l < 5; l++) {
    const size_t nw = (size_t)lay_out(l) * lay_in(l), nb = lay_out(l);
    sz[k++] = nw * 4;  // w
    sz[k++] = nb * 4;  // b
    sz[k++] = nw * 4;  // mw
    sz[k++] = nw * 4;  // vw
    sz[k++] = nb * 4;  // mb
    sz[k++] = nb * 4;  // vb
    sz[k++] = nw * 4;  // gw
    sz[k++] = nb * 4;  // gb
    sz[k++] = (size_t)lay_N(l) * lay_K(l) * 2;  // wt
    sz[k++] = (size_t)lay_N(l) * lay_K(l) * 2;  // wtt
  }
  sz[k++] = 32 * 4;                              // norm
  for (int l = 0; l < 5; l++) sz[k++] = (size_t)B * (l == 0 ? KIN : H) * 2;  // act
  for (int l = 0; l < 5; l++) sz[k++] = (size_t)B * (l == 4 ? NOUT : H) * 2;  // dact
  sz[k++] = (size_t)B * NOUT * 4;                // y
  sz[k++] = 16;                                  // loss
  sz[k++] = 16;                                  // err
  *n = k;
}

int mlp_layout(int64_t B, MlpLayout* L) {
  if (B < 1 || B > (1ll << 24)) return LBM_IMB_EINVAL;
  size_t sz[64];
  int n = 0;
  mlp_sizes(B, sz, &n);
  size_t o = 0;
  for (int i = 0; i < n; i++) {
    L->off[i] = o;
    o = up256(o + sz[i]);
  }
  L->total = o;
  return LBM_IMB_OK;
}

void mlp_bind(lbm_imb_mlp* h, unsigned char* base, const MlpLayout& L) {
  int k = 0;
  Params& P = h->P;
  for (int l = 0; l < 5; l++) {
    P.w[l] = (float*)(base + L.off[k++]);
    P.b[l] = (float*)(base + L.off[k++]);
    P.mw[l] = (float*)(base + L.off[k++]);
    P.vw[l] = (float*)(base + L.off[k++]);
    P.mb[l] = (float*)(base + L.off[k++]);
    P.vb[l] = (float*)(base + L.off[k++]);
    P.gw[l] = (float*)(base + L.off[k++]);
    P.gb[l] = (float*)(base + L.off[k++]);
    P.wt[l] = (__nv_bfloat16*)(base + L.off[k++]);
    P.wtt[l] = (__nv_bfloat16*)(base + L.off[k++]);
  }
  P.norm = (float*)(base + L.off[k++]);
  for (int l = 0; l < 5; l++) P.act[l] = (__nv_bfloat16*)(base + L.off[k++]);
  for (int l = 0; l < 5; l++) P.dact[l] = (__nv_bfloat16*)(base + L.off[k++]);
  P.y = (float*)(base + L.off[k++]);
  P.loss = (float*)(base + L.off[k++]);
  P.err = (int*)(base + L.off[k++]);
}

int n_params() {
  int n = 0;
  for (int l = 0; l < 5; l++) n += lay_out(l) * lay_in(l) + lay_out(l);
  return n;
}

cudaError_t pack_all(lbm_imb_mlp* h) {
  for (int l = 0; l < 5; l++) {
    const int ne = lay_N(l) * lay_K(l);
    mlp_pack_kernel<<<(ne + 255) / 256, 256, 0, h->stream>>>(h->P, l);
  }
  return cudaGetLastError();
}

int smem_fwd() { return (int)sizeof(SmemFwd) + 1024; }
int smem_bwd() { return (int)sizeof(SmemBwd) + 1024; }

int read_mlp_err(lbm_imb_mlp* h) {
  int bits = 0;
  if (cudaMemcpyAsync(&bits, h->P.err, 4, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return LBM_IMB_ECUDA;
  if (bits) {
    cudaMemsetAsync(h->P.err, 0, 4, h->stream);
    cudaStreamSynchronize(h->stream);
    return LBM_IMB_ETIMEOUT;
  }
  return LBM_IMB_OK;
}

cudaError_t launch_forward(lbm_imb_mlp* h, const float* x, int B, int train, float* y) {
  const int tiles = (B + TILE - 1) / TILE;
  const int grid = tiles < h->grid ? tiles : h->grid;
  mlp_forward_kernel<<<grid, 128, smem_fwd(), h->stream>>>(h->P, x, B, train, y);
  return cudaGetLastError();
}

cudaError_t launch_backward(lbm_imb_mlp* h, const float* t, int B) {
  const int tiles = (B + TILE - 1) / TILE;
  const int grid = tiles < h->grid ? tiles : h->grid;
  mlp_backward_kernel<<<grid, 128, smem_bwd(), h->stream>>>(h->P, t, B);
  return cudaGetLastError();
}

cudaError_t launch_wgrad(lbm_imb_mlp* h, int B) {
  for (int l = 0; l < 5; l++) {
    dim3 g((lay_in(l) + 31) / 32, (lay_out(l) + 31) / 32);
    mlp_wgrad_kernel<<<g, 256, 0, h->stream>>>(h->P, B, l);
  }
  return cudaGetLastError();
}
}  // namespace

extern "C" {

size_t lbm_imb_mlp_required_bytes(int64_t max_batch) {
  MlpLayout L;
  if (mlp_layout(max_batch, &L) != LBM_IMB_OK) return 0;
  return L.total;
}

int lbm_imb_mlp_init(void* dev_buf, size_t bytes, int64_t max_batch, uint64_t seed, void* stream,
                     lbm_imb_mlp_t** out) {
  if (!dev_buf || !out || ((uintptr_t)dev_buf) % 256) return LBM_IMB_EINVAL;
  MlpLayout L;
  int st = mlp_layout(max_batch, &L);
  if (st) return st;
  if (bytes < L.total) return LBM_IMB_ENOMEM;
  lbm_imb_mlp* h = new lbm_imb_mlp();
  h->stream = static_cast<cudaStream_t>(stream);
  h->max_batch = max_batch;
  mlp_bind(h, static_cast<unsigned char*>(dev_buf), L);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  h->grid = sms > 0 ? sms : 1;
  cudaError_t e = cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_fwd());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bwd());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 128 * 128 * 2 + 64);
  if (e == cudaSuccess) e = cudaMemsetAsync(dev_buf, 0, L.total, h->stream);
  // He-uniform initial weights (host xorshift), zero biases and moments
  if (e == cudaSuccess) {
    const int np = n_params();
    float* hp = (float*)malloc(sizeof(float) * np);
    uint64_t s = seed * 0x9E3779B97F4A7C15ull + 1;
    int k = 0;
    for (int l = 0; l < 5; l++) {
      const float lim = sqrtf(6.0f / lay_in(l));
      for (int i = 0; i < lay_out(l) * lay_in(l); i++) {
        s ^= s << 13;
        s ^= s >> 7;
        s ^= s << 17;
        hp[k++] = lim * (2.0f * (float)((s >> 11) * (1.0 / 9007199254740992.0)) - 1.0f);
      }
      for (int i = 0; i < lay_out(l); i++) hp[k++] = 0.f;
    }
    k = 0;
    for (int l = 0; l < 5 && e == cudaSuccess; l++) {
      const int nw = lay_out(l) * lay_in(l), nb = lay_out(l);
      e = cudaMemcpyAsync(h->P.w[l], hp + k, 4 * nw, cudaMemcpyHostToDevice, h->stream);
      k += nw;
      if (e == cudaSuccess) e = cudaMemcpyAsync(h->P.b[l], hp + k, 4 * nb, cudaMemcpyHostToDevice, h->stream);
      k += nb;
    }
    float norm[32];
    for (int i = 0; i < 32; i++) norm[i] = (i >= IN && i < 2 * IN) || i >= 2 * IN + OUT ? 1.f : 0.f;
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->P.norm, norm, sizeof(norm), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = pack_all(h);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    free(hp);
  }
  if (e != cudaSuccess) {
    delete h;
    return LBM_IMB_ECUDA;
  }
  *out = h;
  return LBM_IMB_OK;
}

int lbm_imb_mlp_num_params(int* n) {
  if (!n) return LBM_IMB_EINVAL;
  *n = n_params();
  return LBM_IMB_OK;
}

int lbm_imb_mlp_set_params(lbm_imb_mlp_t* h, const float* params) {
  if (!h || !params) return LBM_IMB_EINVAL;
  int k = 0;
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < 5 && e == cudaSuccess; l++) {
    const int nw = lay_out(l) * lay_in(l), nb = lay_out(l);
    e = cudaMemcpyAsync(h->P.w[l], params + k, 4 * nw, cudaMemcpyHostToDevice, h->stream);
    k += nw;
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->P.b[l], params + k, 4 * nb, cudaMemcpyHostToDevice, h->stream);
    k += nb;
  }
  if (e == cudaSuccess) e = pack_all(h);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? LBM_IMB_OK : LBM_IMB_ECUDA;
}

int lbm_imb_mlp_get_params(lbm_imb_mlp_t* h, float* params) {
  if (!h || !params) return LBM_IMB_EINVAL;
  int k = 0;
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < 5 && e == cudaSuccess; l++) {
    const int nw = lay_out(l) * lay_in(l), nb = lay_out(l);
    e = cudaMemcpyAsync(params + k, h->P.w[l], 4 * nw, cudaMemcpyDeviceToHost, h->stream);
    k += nw;
    if (e == cudaSuccess) e = cudaMemcpyAsync(params + k, h->P.b[l], 4 * nb, cudaMemcpyDeviceToHost, h->stream);
    k += nb;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? LBM_IMB_OK : LBM_IMB_ECUDA;
}

int lbm_imb_mlp_set_normalization(lbm_imb_mlp_t* h, const float* x_mean, const float* x_std,
                                  const float* y_mean, const float* y_std) {
  if (!h || !x_mean || !x_std || !y_mean || !y_std) return LBM_IMB_EINVAL;
  float norm[32] = {0};
  for (int i = 0; i < IN; i++) {
    if (!(x_std[i] > 0.f)) return LBM_IMB_EINVAL;
    norm[i] = x_mean[i];
    norm[IN + i] = x_std[i];
  }
  for (int i = 0; i < OUT; i++) {
    if (!(y_std[i] > 0.f)) return LBM_IMB_EINVAL;
    norm[2 * IN + i] = y_mean[i];
    norm[2 * IN + OUT + i] = y_std[i];
  }
  cudaError_t e = cudaMemcpyAsync(h->P.norm, norm, sizeof(norm), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? LBM_IMB_OK : LBM_IMB_ECUDA;
}

int lbm_imb_mlp_predict(lbm_imb_mlp_t* h, const float* x, float* y, int64_t n) {
  if (!h || n < 0 || (n > 0 && (!x || !y))) return LBM_IMB_EINVAL;
  for (int64_t s = 0; s < n; s += (1ll << 30)) {
    const int B = (int)((n - s) < (1ll << 30) ? (n - s) : (1ll << 30));
    if (launch_forward(h, x + s * IN, B, 0, y + s * OUT) != cudaSuccess) return LBM_IMB_ECUDA;
  }
  return read_mlp_err(h);
}

int lbm_imb_mlp_gradients(lbm_imb_mlp_t* h, const float* x, const float* t, int64_t B, float* grads,
                          float* loss) {
  if (!h || !x || !t || B < 1 || B > h->max_batch) return LBM_IMB_EINVAL;
  cudaError_t e = cudaMemsetAsync(h->P.loss, 0, 4, h->stream);
  if (e == cudaSuccess) e = launch_forward(h, x, (int)B, 1, nullptr);
  if (e == cudaSuccess) e = launch_backward(h, t, (int)B);
  if (e == cudaSuccess) e = launch_wgrad(h, (int)B);
  if (e == cudaSuccess && grads) {
    int k = 0;
    for (int l = 0; l < 5 && e == cudaSuccess; l++) {
      const int nw = lay_out(l) * lay_in(l), nb = lay_out(l);
      e = cudaMemcpyAsync(grads + k, h->P.gw[l], 4 * nw, cudaMemcpyDeviceToHost, h->stream);
      k += nw;
      if (e == cudaSuccess) e = cudaMemcpyAsync(grads + k, h->P.gb[l], 4 * nb, cudaMemcpyDeviceToHost, h->stream);
      k += nb;
    }
  }
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, h->P.loss, 4, cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return LBM_IMB_ECUDA;
  return read_mlp_err(h);
}

int lbm_imb_mlp_train_steps(lbm_imb_mlp_t* h, const float* x, const float* t, int64_t n, int64_t batch,
                            int64_t steps, float lr, float* last_loss) {
  if (!h || !x || !t || n < 1 || batch < 1 || batch > h->max_batch || steps < 0 || !(lr > 0.f))
    return LBM_IMB_EINVAL;
  cudaError_t e = cudaSuccess;
  int64_t pos = 0;
  for (int64_t s = 0; s < steps && e == cudaSuccess; s++) {
    int64_t B = batch;
    if (pos + B > n) pos = 0;
    if (B > n) B = n;
    e = cudaMemsetAsync(h->P.loss, 0, 4, h->stream);
    if (e == cudaSuccess) e = launch_forward(h, x + pos * IN, (int)B, 1, nullptr);
    if (e == cudaSuccess) e = launch_backward(h, t + pos * OUT, (int)B);
    if (e == cudaSuccess) e = launch_wgrad(h, (int)B);
    h->adam_t++;
    const float c1 = 1.f - powf(0.9f, (float)h->adam_t), c2 = 1.f - powf(0.999f, (float)h->adam_t);
    for (int l = 0; l < 5 && e == cudaSuccess; l++) {
      const int nw = lay_out(l) * lay_in(l);
      mlp_adam_kernel<<<(nw + 255) / 256, 256, 0, h->stream>>>(h->P, l, lr, c1, c2);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = pack_all(h);
    pos += B;
  }
  if (e == cudaSuccess && last_loss) e = cudaMemcpyAsync(last_loss, h->P.loss, 4, cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return LBM_IMB_ECUDA;
  return read_mlp_err(h);
}

int lbm_imb_mlp_destroy(lbm_imb_mlp_t* h) {
  if (!h) return LBM_IMB_EINVAL;
  delete h;
  return LBM_IMB_OK;
}

int lbm_imb_mlp_probe_gemm(const uint16_t* a_host, const uint16_t* b_host, int N, int K, float* d_host,
                           void* dev_scratch, size_t scratch_bytes, void* stream) {
  if (!a_host || !b_host || !d_host || !dev_scratch) return LBM_IMB_EINVAL;
  if (N < 16 || N > 128 || N % 16 || K < 16 || K > 128 || K % 16) return LBM_IMB_EINVAL;
  const size_t need = 128 * 128 * 2 * 2 + 128 * 128 * 4 + 256;
  if (scratch_bytes < need || ((uintptr_t)dev_scratch) % 256) return LBM_IMB_EINVAL;
  unsigned char* base = static_cast<unsigned char*>(dev_scratch);
  __nv_bfloat16* a = reinterpret_cast<__nv_bfloat16*>(base);
  __nv_bfloat16* b = a + 128 * 128;
  float* d = reinterpret_cast<float*>(b + 128 * 128);
  int* err = reinterpret_cast<int*>(d + 128 * 128);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaFuncSetAttribute(mlp_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       2 * 128 * 128 * 2 + 64);
  if (e == cudaSuccess) e = cudaMemcpyAsync(a, a_host, 2 * 128 * K, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b, b_host, 2 * N * K, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 4, s);
  if (e == cudaSuccess) {
    mlp_probe_kernel<<<1, 128, 2 * 128 * 128 * 2 + 64, s>>>(a, b, N, K, d, err);
    e = cudaGetLastError();
  }
  int bits = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_host, d, 4 * 128 * N, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, err, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return LBM_IMB_ECUDA;
  return bits ? LBM_IMB_ETIMEOUT : LBM_IMB_OK;
}

}  // extern "C"
