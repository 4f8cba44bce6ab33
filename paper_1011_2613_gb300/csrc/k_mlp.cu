// K7: the learned drag closure's network on the 5th-generation tensor cores.
//
// MLP 6 -> 128 -> 128 -> 128 -> 128 -> 3 with ReLU, BF16 operands and FP32
// accumulation.  Every product of a training step runs as tcgen05.mma
// (kind::f16, M = 128, N = 16 or 128, K = 16 per instruction) issued by one
// thread of the CTA, with both operands in shared memory in the canonical
// K-major layout without swizzle (8x8 core matrices of 128 contiguous bytes;
// LBO = stride between core matrices along K, SBO = stride between 8-row
// groups) and the FP32 accumulator in tensor memory:
//   forward   H_l = act(H_{l-1} W_l^T + b_l)           (128-sample tile x W_l)
//   backward  dH_{l-1} = (dH_l W_l) * relu'(H_{l-1})   (128-sample tile x W_l^T)
//   weights   dW_l = dH_l^T H_{l-1}                    (K = the minibatch)
// Completion is signalled through tcgen05.commit on an mbarrier; epilogues
// read the accumulator with tcgen05.ld (32 lanes x 16 columns per
// instruction).  A training step is four launches: forward (keeps the
// activations, zeroes the gradient sums), backward (gradients of the
// pre-activations, bias gradients),
// the weight-gradient products, and Adam fused with the refresh of the BF16
// operand tiles.
//
// Operand staging overlaps the products: the forward and backward kernels
// request every weight tile with bulk copies (cp.async.bulk, one mbarrier
// per tile) at launch and wait for a tile only before its first product;
// the weight-gradient kernel streams its operands through a ring of shared
// memory stages (bulk copies completing on per-stage "full" barriers, the
// products releasing a stage through tcgen05.commit on its "empty" barrier),
// so the copies of later K blocks run under the products of earlier ones.
//
// Every wait on an mbarrier is bounded: after the poll limit the kernel sets
// an error flag, waits (bounded) for its copies and products in flight, frees
// its tensor memory and returns.
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
constexpr int KB = 64;      // samples per K block of the weight-gradient products
constexpr int NSTAGE = 4;   // shared-memory stages of the weight-gradient pipeline
constexpr long long kPollLimit = 1ll << 26;
enum : int { MERR_TIMEOUT = 1 };

// layer shapes (out, in) and padded (N, K) of the forward products
__host__ __device__ constexpr int lay_out(int l) { return l == 4 ? OUT : H; }
__host__ __device__ constexpr int lay_in(int l) { return l == 0 ? IN : H; }
__host__ __device__ constexpr int lay_N(int l) { return l == 4 ? NOUT : H; }
__host__ __device__ constexpr int lay_K(int l) { return l == 0 ? KIN : H; }
// rows (features) of the layer inputs act_l and output gradients dact_l
__host__ __device__ constexpr int act_rows(int l) { return l == 0 ? KIN : H; }
__host__ __device__ constexpr int dact_rows(int l) { return l == 4 ? NOUT : H; }

// --------------------------------------------------------------------------
// canonical K-major layout without swizzle: element (r, k) of an R x K tile
// --------------------------------------------------------------------------
__host__ __device__ __forceinline__ int cm_index(int r, int k, int K) {
  return (((r >> 3) * (K >> 3) + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7);
}

// element (feature r, sample m) of the [feature][sample] arrays the
// weight-gradient products read: 64-sample blocks, each an R x 64 tile in the
// canonical K-major layout (K = samples), stored one after the other so that
// a block is one contiguous bulk copy
__host__ __device__ __forceinline__ size_t tblock_index(int r, int m, int R) {
  return (size_t)(m >> 6) * (size_t)(R * KB) + (size_t)cm_index(r, m & (KB - 1), KB);
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

// make barrier initialisations visible to the async proxy (bulk copies,
// tensor-core commits) before any of them can arrive
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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

// arrive on the barrier expecting `bytes` of bulk-copy data in this phase
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// bulk copy global -> this CTA's shared memory, completing on `bar`
// (addresses 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(static_cast<unsigned long long>(__cvta_generic_to_global(src))), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
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

// D (128 x N) = A (128 x K) * B (N x K)^T, issued by thread 0 (after its
// operand barrier `wbar`, if any, has completed phase 0), waited by all;
// returns false on timeout.  Caller has fenced the operand writes.
__device__ __forceinline__ bool tc_gemm(const __nv_bfloat16* A, const __nv_bfloat16* B, int N, int K,
                                        uint32_t tmem_d, uint64_t* bar, uint32_t& phase,
                                        uint64_t* wbar = nullptr) {
  int issued = 1;
  if (threadIdx.x == 0) {
    issued = wbar == nullptr || mbar_wait(wbar, 0) ? 1 : 0;
    if (issued) {
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
  }
  if (__syncthreads_and(issued) == 0) return false;  // the operands never arrived: nothing issued
  const bool ok = mbar_wait(bar, phase);
  phase ^= 1u;
  tc_fence_after();
  return __syncthreads_and(ok) != 0;  // one verdict for the whole CTA
}

// --------------------------------------------------------------------------
// parameter block (device), see lbm_imb_mlp_* in the header
// --------------------------------------------------------------------------
struct Params {
  // flat parameter vectors in the interface order (W_1, b_1, ..., W_5, b_5):
  // FP32 masters, Adam moments, gradients; w[l], b[l], ... point into them
  float* p;
  float* m;
  float* v;
  float* g;
  float* w[5];
  float* b[5];
  float* gw[5];
  float* gb[5];
  __nv_bfloat16* wt[5];    // BF16 W in [N][K] core-matrix order (forward B operand)
  __nv_bfloat16* wtt[5];   // BF16 W^T in [N=in][K=out] core-matrix order (backward B operand)
  float* norm;             // x_mean[6], x_std[6], y_mean[3], y_std[3]
  // activations of the current minibatch in the [feature][sample] block
  // layout of tblock_index: actT[l] = input of layer l (actT[0] = the
  // normalised x, KIN rows; actT[l] = H_l, H rows), dactT[l] = gradient of
  // layer l's pre-activation output (H rows; NOUT rows for l = 4)
  __nv_bfloat16* actT[5];
  __nv_bfloat16* dactT[5];
  // ReLU masks of H_1..H_4 (mask[l], l = 1..4): bit c of sample m's 128 bits
  // = (BF16 H_l[m][c] > 0), uint4 [B]; read by the backward pass
  uint4* mask[5];
  float* y;                // network output, normalised [B][NOUT]
  float* loss;             // [1]
  int* err;                // [1]
};

// offsets of W_l and b_l in the flat parameter vector
__host__ __device__ constexpr int off_w(int l) {
  return l == 0 ? 0 : off_w(l - 1) + lay_out(l - 1) * lay_in(l - 1) + lay_out(l - 1);
}
__host__ __device__ constexpr int off_b(int l) { return off_w(l) + lay_out(l) * lay_in(l); }
constexpr int kNumParams = off_b(4) + OUT;
static_assert(off_w(1) % 4 == 0 && off_w(2) % 4 == 0 && off_w(3) % 4 == 0 && off_b(1) % 4 == 0,
              "float4 gradient sums need 16-byte aligned weight rows");

// bytes of the BF16 operand tiles
__host__ __device__ constexpr uint32_t tile_bytes(int l) { return (uint32_t)(lay_N(l) * lay_K(l) * 2); }

// shared memory of the forward kernel
struct SmemFwd {
  __nv_bfloat16 w1[H * KIN];
  __nv_bfloat16 w[3][H * H];
  __nv_bfloat16 w5[NOUT * H];
  __nv_bfloat16 a[TILE * H];     // current activation tile (K-major)
  __nv_bfloat16 x[TILE * KIN];   // input tile
  uint64_t wbar[5];              // weight tile l arrived
  uint64_t bar;                  // products done
  uint32_t tmem;
};

// thread 0: one barrier per weight tile, all tiles requested at once
__device__ __forceinline__ void request_tiles(uint64_t* wbar, __nv_bfloat16* const* dst,
                                              __nv_bfloat16* const* src, const uint32_t* bytes, int n) {
  for (int i = 0; i < n; i++) mbar_init(&wbar[i], 1);
  mbar_init_fence();
  for (int i = 0; i < n; i++) {
    mbar_expect_tx(&wbar[i], bytes[i]);
    bulk_g2s(dst[i], src[i], bytes[i], &wbar[i]);
  }
}

// forward pass over tiles of 128 samples; train = 1 keeps the activations
// (actT) and the normalised outputs (y) for the backward pass
__global__ void __launch_bounds__(128) mlp_forward_kernel(Params P, const float* x, int B, int train,
                                                          float* y_out) {
  if (*(volatile const int*)P.err != 0) return;  // a wait already timed out: skip the work
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  SmemFwd& S = *reinterpret_cast<SmemFwd*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5;
  if (train) {  // the step's gradient and loss sums start from zero (the backward pass adds to them)
    for (int i = blockIdx.x * blockDim.x + tid; i < kNumParams; i += gridDim.x * blockDim.x) P.g[i] = 0.f;
    if (blockIdx.x == 0 && tid == 0) *P.loss = 0.f;
  }
  if (tid == 0) {
    __nv_bfloat16* dst[5] = {S.w1, S.w[0], S.w[1], S.w[2], S.w5};
    __nv_bfloat16* src[5] = {P.wt[0], P.wt[1], P.wt[2], P.wt[3], P.wt[4]};
    const uint32_t bytes[5] = {tile_bytes(0), tile_bytes(1), tile_bytes(2), tile_bytes(3), tile_bytes(4)};
    request_tiles(S.wbar, dst, src, bytes, 5);
    mbar_init(&S.bar, 1);
    mbar_init_fence();
  }
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
    // normalised input -> BF16 operand (rows past the batch are zero)
#pragma unroll
    for (int k = 0; k < KIN; k++) {
      float v = 0.f;
      if (k < IN && valid) v = (x[(size_t)row * IN + k] - nm[k]) / nm[IN + k];
      const __nv_bfloat16 bv = __float2bfloat16_rn(v);
      S.x[cm_index(tid, k, KIN)] = bv;
      if (train) P.actT[0][tblock_index(k, row, KIN)] = bv;
    }
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    for (int l = 0; l < 5 && ok; l++) {
      const __nv_bfloat16* A = l == 0 ? S.x : S.a;
      const __nv_bfloat16* Bm = l == 0 ? S.w1 : (l == 4 ? S.w5 : S.w[l - 1]);
      ok = tc_gemm(A, Bm, lay_N(l), lay_K(l), tmem, &S.bar, phase, &S.wbar[l]);
      if (!ok) break;
      // epilogue: this warp's 32 rows
      const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
      const float* bias = P.b[l];
      uint32_t mb0 = 0u, mb1 = 0u, mb2 = 0u, mb3 = 0u;  // ReLU mask words (registers, not an array)
      for (int c0 = 0; c0 < lay_N(l); c0 += 16) {
        float r[16];
        tc_ld16(lane_base + c0, r);
        if (l < 4) {
#pragma unroll
          for (int i = 0; i < 16; i++) {
            const float hv = fmaxf(r[i] + bias[c0 + i], 0.f);
            const __nv_bfloat16 bv = __float2bfloat16_rn(hv);
            S.a[cm_index(tid, c0 + i, H)] = bv;
            if (train) {
              P.actT[l + 1][tblock_index(c0 + i, row, H)] = valid ? bv : __float2bfloat16_rn(0.f);
              const uint32_t bit = __bfloat162float(bv) > 0.f ? 1u << ((c0 + i) & 31) : 0u;
              const int w = (c0 + i) >> 5;
              mb0 |= w == 0 ? bit : 0u;
              mb1 |= w == 1 ? bit : 0u;
              mb2 |= w == 2 ? bit : 0u;
              mb3 |= w == 3 ? bit : 0u;
            }
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
      if (train && l < 4) P.mask[l + 1][row] = make_uint4(mb0, mb1, mb2, mb3);
      proxy_fence();
      tc_fence_before();
      __syncthreads();
    }
  }
  if (!ok && tid == 0) atomicOr(P.err, MERR_TIMEOUT);
  if (tid == 0)  // copies still in flight must land before the CTA's memory is released
    for (int i = 0; i < 5; i++) mbar_wait(&S.wbar[i], 0);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_free(tmem);
}

// backward (data) pass: dY from the loss, then dH_{l-1} = (dH_l W_l) * relu'(H_{l-1});
// writes the pre-activation gradients (BF16, for the weight products) and adds
// this tile's column sums (FP32, before rounding) to the bias gradients
struct SmemBwd {
  __nv_bfloat16 w5t[H * NOUT];   // W5^T: N = 128 (in), K = 16 (out, padded)
  __nv_bfloat16 wt[3][H * H];    // W4^T, W3^T, W2^T
  __nv_bfloat16 d[TILE * H];     // current gradient tile (K-major)
  float colsum[4][H];            // per-warp column sums of the gradient tile
  uint64_t wbar[4];
  uint64_t bar;
  uint32_t tmem;
};

// column sums of one 16-column slice over the warp's 32 samples: a
// butterfly that halves the columns a lane carries at each exchange (16
// shuffles instead of 5 per column); lane L ends with the sum of column
// 8 b4 + 4 b3 + 2 b2 + b1 (b_k the bits of L), written by the even lanes
__device__ __forceinline__ void warp_colsum16(const float (&g)[16], float* out) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  float a[8], b[4], c[2];
  const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4, u2 = lane & 2;
#pragma unroll
  for (int i = 0; i < 8; i++) a[i] = (u16 ? g[8 + i] : g[i]) + __shfl_xor_sync(FULL, u16 ? g[i] : g[8 + i], 16);
#pragma unroll
  for (int i = 0; i < 4; i++) b[i] = (u8 ? a[4 + i] : a[i]) + __shfl_xor_sync(FULL, u8 ? a[i] : a[4 + i], 8);
#pragma unroll
  for (int i = 0; i < 2; i++) c[i] = (u4 ? b[2 + i] : b[i]) + __shfl_xor_sync(FULL, u4 ? b[i] : b[2 + i], 4);
  float d = (u2 ? c[1] : c[0]) + __shfl_xor_sync(FULL, u2 ? c[0] : c[1], 2);
  d += __shfl_xor_sync(FULL, d, 1);
  if ((lane & 1) == 0) out[(u16 ? 8 : 0) + (u8 ? 4 : 0) + (u4 ? 2 : 0) + (u2 ? 1 : 0)] = d;
}

// the CTA's per-warp column sums [4][n] -> atomic adds into gb[n]
__device__ __forceinline__ void flush_colsum(float (*colsum)[H], float* gb, int n) {
  __syncthreads();
  for (int c = threadIdx.x; c < n; c += blockDim.x)
    atomicAdd(gb + c, (colsum[0][c] + colsum[1][c]) + (colsum[2][c] + colsum[3][c]));
  __syncthreads();
}

__global__ void __launch_bounds__(128) mlp_backward_kernel(Params P, const float* tgt, int B) {
  if (*(volatile const int*)P.err != 0) return;  // a wait already timed out: skip the work
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  SmemBwd& S = *reinterpret_cast<SmemBwd*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5;
  // barrier k <-> the product with W_{4-k}^T: k = 0 W5^T (w5t), 1 W4^T, 2 W3^T, 3 W2^T
  if (tid == 0) {
    __nv_bfloat16* dst[4] = {S.w5t, S.wt[0], S.wt[1], S.wt[2]};
    __nv_bfloat16* src[4] = {P.wtt[4], P.wtt[3], P.wtt[2], P.wtt[1]};
    const uint32_t bytes[4] = {tile_bytes(4), tile_bytes(3), tile_bytes(2), tile_bytes(1)};
    request_tiles(S.wbar, dst, src, bytes, 4);
    mbar_init(&S.bar, 1);
    mbar_init_fence();
  }
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
    float g[NOUT];
#pragma unroll
    for (int k = 0; k < NOUT; k++) {
      g[k] = 0.f;
      if (k < OUT && valid) {
        const float th = (tgt[(size_t)row * OUT + k] - nm[2 * IN + k]) / nm[2 * IN + OUT + k];
        const float e = P.y[(size_t)row * NOUT + k] - th;
        lsum += e * e;
        g[k] = scale * e;
      }
      const __nv_bfloat16 bg = __float2bfloat16_rn(g[k]);
      S.d[cm_index(tid, k, NOUT)] = bg;
      P.dactT[4][tblock_index(k, row, NOUT)] = bg;
    }
    warp_colsum16(g, S.colsum[warp]);
    flush_colsum(S.colsum, P.gb[4], OUT);
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    // layers 4..1: product with W_l, then the ReLU mask of H_l's pre-activation
    for (int l = 4; l >= 1 && ok; l--) {
      // B operand of step l is W_l^T (staged: w5t = W_5^T, wt[3 - l] = W_l^T)
      const __nv_bfloat16* Bt = l == 4 ? S.w5t : S.wt[3 - l];
      ok = tc_gemm(S.d, Bt, H, l == 4 ? NOUT : H, tmem, &S.bar, phase, &S.wbar[4 - l]);
      if (!ok) break;
      const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
      const uint4 mk = P.mask[l][row];  // H_l > 0 (rows past the batch: all clear)
      for (int c0 = 0; c0 < H; c0 += 16) {
        float r[16], gl[16];
        tc_ld16(lane_base + c0, r);
        const uint32_t word = c0 < 64 ? (c0 < 32 ? mk.x : mk.y) : (c0 < 96 ? mk.z : mk.w);
        const uint32_t bits = word >> (c0 & 31);
#pragma unroll
        for (int i = 0; i < 16; i++) {
          gl[i] = (valid && ((bits >> i) & 1u)) ? r[i] : 0.f;
          const __nv_bfloat16 bg = __float2bfloat16_rn(gl[i]);
          S.d[cm_index(tid, c0 + i, H)] = bg;
          P.dactT[l - 1][tblock_index(c0 + i, row, H)] = bg;
        }
        warp_colsum16(gl, S.colsum[warp] + c0);
      }
      flush_colsum(S.colsum, P.gb[l - 1], H);
      proxy_fence();
      tc_fence_before();
      __syncthreads();
    }
  }
  // loss (mean squared error of this minibatch)
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, o);
  if ((tid & 31) == 0 && lsum != 0.f) atomicAdd(P.loss, lsum / (float)(B * OUT));
  if (!ok && tid == 0) atomicOr(P.err, MERR_TIMEOUT);
  if (tid == 0)
    for (int i = 0; i < 4; i++) mbar_wait(&S.wbar[i], 0);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_free(tmem);
}

// Weight gradients on the tensor cores.  CTA (l, s) accumulates, for layer l,
// the products over 64-sample blocks s*per .. (s+1)*per - 1 of the minibatch
// in tensor memory and adds its partial sum to gw[l]:
//   l = 0..3: D [out][in] = dactT_l (M = 128) x actT_l^T (N = 16 for l = 0, else 128)
//   l = 4:    D [in][out] = actT_4 (M = 128) x dactT_4^T (N = 16), i.e. dW_5^T
// Thread 0 streams the blocks through NSTAGE shared-memory stages and issues
// the products; stage s is refilled once the products reading it are done.
struct SmemWg {
  __nv_bfloat16 a[NSTAGE][H * KB];
  __nv_bfloat16 b[NSTAGE][H * KB];
  uint64_t full[NSTAGE], empty[NSTAGE], done;
  uint32_t tmem;
  int ok, mma;
};

__global__ void __launch_bounds__(128) mlp_wgrad_kernel(Params P, int nblk_total, int per) {
  if (*(volatile const int*)P.err != 0) return;  // a wait already timed out: skip the work
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  SmemWg& S = *reinterpret_cast<SmemWg*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int l = blockIdx.y;
  const int j0 = blockIdx.x * per;
  const int nblk = min(per, nblk_total - j0);
  if (nblk <= 0) return;  // block-uniform, before any barrier or allocation
  const bool last = l == 4;
  const __nv_bfloat16* Ag = last ? P.actT[4] : P.dactT[l];
  const __nv_bfloat16* Bg = last ? P.dactT[4] : P.actT[l];
  const int N = last ? NOUT : act_rows(l);
  const uint32_t abytes = (uint32_t)(H * KB * 2), bbytes = (uint32_t)(N * KB * 2);
  if (tid == 0) {
    for (int s = 0; s < NSTAGE; s++) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], 1);
    }
    mbar_init(&S.done, 1);
    mbar_init_fence();
    S.ok = 1;
    S.mma = 0;
  }
  if (warp == 0) tmem_alloc(&S.tmem);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem;
  if (tid == 0) {
    int use[NSTAGE];       // use count of the last load issued to each stage
    bool landed[NSTAGE];   // that load has been waited for
    for (int s = 0; s < NSTAGE; s++) {
      use[s] = -1;
      landed[s] = true;
    }
    auto load = [&](int j) {
      const int s = j % NSTAGE;
      mbar_expect_tx(&S.full[s], abytes + bbytes);
      bulk_g2s(S.a[s], Ag + (size_t)(j0 + j) * (H * KB), abytes, &S.full[s]);
      bulk_g2s(S.b[s], Bg + (size_t)(j0 + j) * (N * KB), bbytes, &S.full[s]);
      use[s] = j / NSTAGE;
      landed[s] = false;
    };
    bool ok = true, any_mma = false;
    for (int j = 0; j < nblk && j < NSTAGE; j++) load(j);
    const uint32_t idesc = instr_desc(128, N);
    for (int j = 0; j < nblk && ok; j++) {
      const int s = j % NSTAGE;
      ok = mbar_wait(&S.full[s], (uint32_t)((j / NSTAGE) & 1));
      if (!ok) break;
      landed[s] = true;
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < KB; kk += 16) {
        const uint64_t ad = smem_desc(S.a[s] + (kk >> 3) * 64, KB);
        const uint64_t bd = smem_desc(S.b[s] + (kk >> 3) * 64, KB);
        tc_mma(tmem, ad, bd, idesc, (j > 0 || kk > 0) ? 1 : 0);
      }
      any_mma = true;
      tc_commit(&S.empty[s]);
      // refill the stage the previous block used, once its products are done
      const int jr = j - 1 + NSTAGE;
      if (j >= 1 && jr < nblk) {
        const int sp = (j - 1) % NSTAGE;
        ok = mbar_wait(&S.empty[sp], (uint32_t)(((j - 1) / NSTAGE) & 1));
        if (ok) load(jr);
      }
    }
    if (any_mma) tc_commit(&S.done);  // tracks every product issued
    if (!ok) {
      S.ok = 0;
      for (int s = 0; s < NSTAGE; s++)  // copies in flight land before exit
        if (!landed[s]) mbar_wait(&S.full[s], (uint32_t)(use[s] & 1));
    }
    S.mma = any_mma ? 1 : 0;
    if (!any_mma) S.ok = 0;
  }
  __syncthreads();
  bool ok = S.ok != 0;
  // every thread waits for the products issued (bounded; also on the error path)
  if (S.mma && !mbar_wait(&S.done, 0)) ok = false;
  tc_fence_after();
  if (__syncthreads_and(ok ? 1 : 0)) {
    // epilogue: lane = row of D, 16 columns per load
    const int r = warp * 32 + (tid & 31);
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tc_ld16(lane_base + c0, v);
      if (last) {  // D = dW_5^T: row = input feature r, column = output o
        for (int o = 0; o < OUT; o++) atomicAdd(P.gw[4] + o * H + r, v[o]);
      } else if (l == 0) {  // D = dW_1: row = output r, columns = the 6 inputs
        for (int i = 0; i < IN; i++) atomicAdd(P.gw[0] + r * IN + i, v[i]);
      } else {
        float4* dst = reinterpret_cast<float4*>(P.gw[l] + r * H + c0);
#pragma unroll
        for (int q = 0; q < 4; q++) atomicAdd(dst + q, make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
      }
    }
  } else if (tid == 0) {
    atomicOr(P.err, MERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_free(tmem);
}

// Adam on the flat FP32 masters, one thread per parameter, and the refresh of
// the BF16 operand tiles of every weight (W in [out][in] order for the
// forward products, W^T for the backward ones; the zero padding of the tiles
// is never touched)
__global__ void mlp_adam_kernel(Params P, float lr, float c1, float c2) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kNumParams) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float g = P.g[e];
  const float m = b1 * P.m[e] + (1.f - b1) * g;
  const float v = b2 * P.v[e] + (1.f - b2) * g * g;
  P.m[e] = m;
  P.v[e] = v;
  const float w = P.p[e] - lr * (m / c1) / (sqrtf(v / c2) + eps);
  P.p[e] = w;
  const int ow[5] = {off_w(0), off_w(1), off_w(2), off_w(3), off_w(4)};  // folded at compile time
  int l = 0;
  while (l < 4 && e >= ow[l + 1]) l++;
  const int k = e - ow[l];
  if (k < lay_out(l) * lay_in(l)) {
    const int o = k / lay_in(l), i = k % lay_in(l);
    const __nv_bfloat16 bw = __float2bfloat16_rn(w);
    P.wt[l][cm_index(o, i, lay_K(l))] = bw;
    P.wtt[l][cm_index(i, o, lay_N(l))] = bw;
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
};

namespace {
size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// samples of the per-minibatch arrays: whole 128-sample tiles
int64_t padded_batch(int64_t B) { return (B + TILE - 1) / TILE * TILE; }

// arrays of the parameter block (mlp_sizes lists them in this order):
// p, m, v, g; wt[5]; wtt[5]; norm; actT[5]; dactT[5]; mask[5]; y, loss, err
constexpr int kMlpArrays = 4 + 5 + 5 + 1 + 5 + 5 + 5 + 3;

struct MlpLayout {
  size_t off[kMlpArrays];
  size_t total;
};

// sizes of every array of the parameter block, in a fixed order
void mlp_sizes(int64_t B, size_t* sz, int* n) {
  const size_t Bp = (size_t)padded_batch(B);
  int k = 0;
  auto put = [&](size_t bytes) {  // never writes past kMlpArrays entries
    if (k < kMlpArrays) sz[k] = bytes;
    k++;
  };
  for (int i = 0; i < 4; i++) put((size_t)kNumParams * 4);           // p, m, v, g
  for (int l = 0; l < 5; l++) put((size_t)lay_N(l) * lay_K(l) * 2);  // wt
  for (int l = 0; l < 5; l++) put((size_t)lay_N(l) * lay_K(l) * 2);  // wtt
  put(32 * 4);                                                        // norm
  for (int l = 0; l < 5; l++) put(Bp * act_rows(l) * 2);              // actT
  for (int l = 0; l < 5; l++) put(Bp * dact_rows(l) * 2);             // dactT
  for (int l = 0; l < 5; l++) put(l == 0 ? 16 : Bp * 16);             // mask (l = 1..4)
  put(Bp * NOUT * 4);                                                 // y
  put(16);                                                            // loss
  put(16);                                                            // err
  *n = k;  // == kMlpArrays
}

int mlp_layout(int64_t B, MlpLayout* L) {
  if (B < 1 || B > (1ll << 24)) return LBM_IMB_EINVAL;
  size_t sz[kMlpArrays];
  int n = 0;
  mlp_sizes(B, sz, &n);
  if (n != kMlpArrays) return LBM_IMB_EINVAL;  // the list and kMlpArrays disagree (a build error)
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
  P.p = (float*)(base + L.off[k++]);
  P.m = (float*)(base + L.off[k++]);
  P.v = (float*)(base + L.off[k++]);
  P.g = (float*)(base + L.off[k++]);
  for (int l = 0; l < 5; l++) {
    P.w[l] = P.p + off_w(l);
    P.b[l] = P.p + off_b(l);
    P.gw[l] = P.g + off_w(l);
    P.gb[l] = P.g + off_b(l);
  }
  for (int l = 0; l < 5; l++) P.wt[l] = (__nv_bfloat16*)(base + L.off[k++]);
  for (int l = 0; l < 5; l++) P.wtt[l] = (__nv_bfloat16*)(base + L.off[k++]);
  P.norm = (float*)(base + L.off[k++]);
  for (int l = 0; l < 5; l++) P.actT[l] = (__nv_bfloat16*)(base + L.off[k++]);
  for (int l = 0; l < 5; l++) P.dactT[l] = (__nv_bfloat16*)(base + L.off[k++]);
  for (int l = 0; l < 5; l++) P.mask[l] = (uint4*)(base + L.off[k++]);
  P.y = (float*)(base + L.off[k++]);
  P.loss = (float*)(base + L.off[k++]);
  P.err = (int*)(base + L.off[k++]);
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
int smem_wg() { return (int)sizeof(SmemWg) + 1024; }

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

// weight-gradient products: the minibatch's 64-sample blocks split over
// enough CTAs per layer that the five layers fill about one wave
cudaError_t launch_wgrad(lbm_imb_mlp* h, int B) {
  const int nblk = (int)(padded_batch(B) / KB);
  int splits = h->grid / 5;
  if (splits < 1) splits = 1;
  int per = (nblk + splits - 1) / splits;
  if (per < 2) per = 2 < nblk ? 2 : nblk;  // at least two blocks per CTA where there are two
  const int gx = (nblk + per - 1) / per;
  mlp_wgrad_kernel<<<dim3(gx, 5), 128, smem_wg(), h->stream>>>(h->P, nblk, per);
  return cudaGetLastError();
}

// one training step's products on the minibatch x [B][6], t [B][3]: the
// gradients (flat; the forward pass zeroes them) and the loss
cudaError_t launch_gradients(lbm_imb_mlp* h, const float* x, const float* t, int B) {
  cudaError_t e = launch_forward(h, x, B, 1, nullptr);
  if (e == cudaSuccess) e = launch_backward(h, t, B);
  if (e == cudaSuccess) e = launch_wgrad(h, B);
  return e;
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
    e = cudaFuncSetAttribute(mlp_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_wg());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 128 * 128 * 2 + 64);
  if (e == cudaSuccess) e = cudaMemsetAsync(dev_buf, 0, L.total, h->stream);
  // He-uniform initial weights (host xorshift), zero biases and moments
  if (e == cudaSuccess) {
    float* hp = (float*)malloc(sizeof(float) * kNumParams);
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
    e = cudaMemcpyAsync(h->P.p, hp, sizeof(float) * kNumParams, cudaMemcpyHostToDevice, h->stream);
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
  *n = kNumParams;
  return LBM_IMB_OK;
}

int lbm_imb_mlp_set_params(lbm_imb_mlp_t* h, const float* params) {
  if (!h || !params) return LBM_IMB_EINVAL;
  cudaError_t e = cudaMemcpyAsync(h->P.p, params, sizeof(float) * kNumParams, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = pack_all(h);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? LBM_IMB_OK : LBM_IMB_ECUDA;
}

int lbm_imb_mlp_get_params(lbm_imb_mlp_t* h, float* params) {
  if (!h || !params) return LBM_IMB_EINVAL;
  cudaError_t e = cudaMemcpyAsync(params, h->P.p, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost, h->stream);
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
  cudaError_t e = launch_gradients(h, x, t, (int)B);
  if (e == cudaSuccess && grads)
    e = cudaMemcpyAsync(grads, h->P.g, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost, h->stream);
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
    e = launch_gradients(h, x + pos * IN, t + pos * OUT, (int)B);
    h->adam_t++;
    const float c1 = 1.f - powf(0.9f, (float)h->adam_t), c2 = 1.f - powf(0.999f, (float)h->adam_t);
    if (e == cudaSuccess) {
      mlp_adam_kernel<<<(kNumParams + 255) / 256, 256, 0, h->stream>>>(h->P, lr, c1, c2);
      e = cudaGetLastError();
    }
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
