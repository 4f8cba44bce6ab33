// K2: fused pull-stream + LBGK collision with the Noble-Torczynski immersed
// moving boundary term (Xiong et al., Eq. 1 with beta of Eq. 2 and the
// Omega^S term), body force F_i = 3 w_i rho (c_i . g_f), and the per-particle
// force/torque sums of Eq. (3), reduced over each warp by owner before one
// FP64 atomic per (warp, particle).
//
// Layout: structure of arrays f[q][z][y][pitch], x fastest; one thread per
// node, one 128-thread CTA per row segment, so the 19 pulled loads of a warp
// are 32 consecutive elements each (shifted by c_x) and the stores are
// aligned.  Opposite directions are processed as pairs: f^eq_{+-} = A +- B
// shares A = w rho (1 - 1.5 u.u + 4.5 (c.u)^2) and B = 3 w rho (c.u).
//
// Storage variants: FP64 (FP64 arithmetic, the parity form); FP32 deviation
// g = f - w rho0 (FP32 arithmetic); FP16 deviation stored as g / w (FP32
// arithmetic).  In the deviation variants the particle-side arithmetic of the
// IMB nodes (solid velocity, per-node force and torque, warp sums) is FP32
// as well, read from a per-particle FP32 kinematics record; the per-particle
// force/torque accumulators are FP64 in every variant.
#include "dev_collide.cuh"

namespace lbm {

template <class LAT, int STORE, int MINB>
__global__ void __launch_bounds__(128, MINB) collide_kernel(View v) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = x < v.nx;
  collide_node<LAT, STORE>(v, active ? x : v.nx - 1, blockIdx.y, blockIdx.z, active);
}

// ---------------------------------------------------------------------------
// TMA-pipelined persistent form (reduced-precision storages).  A CTA walks
// row tiles of TX = 128 nodes.  For the tile after the current one, thread 0
// issues 19 bulk copies (cp.async.bulk, completion counted on an mbarrier)
// of the x-range [x0, x0 + TX) of each direction's source row (the opposite
// direction's row of the node itself for bounce-back); the one-node halos at
// x0 - 1 and x0 + TX (periodic in x) are prefetched into registers by 38
// threads.  The CTA meanwhile collides the current tile from the other
// buffer.  Every mbarrier wait is bounded; on timeout the CTA records
// ERR_TIMEOUT, waits (bounded) for its other copy and returns.
// ---------------------------------------------------------------------------
constexpr int TX = 128;

template <int STORE>
struct TmaRow {
  using Elem = typename Storage<STORE>::Elem;
  static constexpr int ES = (int)sizeof(Elem);
  static constexpr int PAD = 16 / ES;              // elements before the interior (16 B)
  static constexpr int STRIDE = TX + 2 * PAD;      // row stride in elements (multiple of 16 B)
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool tma_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_addr(bar);
  for (long long i = 0; i < (1ll << 26); i++) {
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

template <class LAT, int STORE>
__global__ void __launch_bounds__(128) collide_tma_kernel(View v, int ntiles) {
  using S = Storage<STORE>;
  using T = typename S::T;
  using Elem = typename S::Elem;
  using RW = TmaRow<STORE>;
  constexpr int Q = LAT::Q;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Elem* buf0 = reinterpret_cast<Elem*>(smem_raw);
  Elem* buf1 = buf0 + Q * RW::STRIDE;
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ int s_bounce[2][Q];  // direction q of this buffer came from the node itself

  const int nx = v.nx, ny = v.ny, nz = v.nz, pitch = v.pitch;
  const int nxb = (nx + TX - 1) / TX;
  const int tid = threadIdx.x;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // per tile: source rows of every direction, copies and halo prefetch
  auto tile_coords = [&](int t, int& x0, int& y, int& z) {
    const int r = t / nxb;
    x0 = (t % nxb) * TX;
    y = r % ny;
    z = r / ny;
  };
  auto src_row = [&](int q, int y, int z, int& plane_q, int& row, bool& bounce) {
    const int cy = LAT::c(q, 1), cz = LAT::c(q, 2);
    bounce = v.wall_y && ((cy == 1 && y == 0) || (cy == -1 && y == ny - 1));
    if (bounce) {
      plane_q = opp(q);
      row = (z * ny + y) * pitch;
    } else {
      int sy = y - cy, sz = z - cz;
      sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
      sz = sz < 0 ? sz + nz : (sz >= nz ? sz - nz : sz);
      plane_q = q;
      row = (sz * ny + sy) * pitch;
    }
  };
  // warp 0: lane 0 announces the bytes, then lane q copies direction q of
  // tile t into buffer b
  auto issue = [&](int t, int b) {
    int x0, y, z;
    tile_coords(t, x0, y, z);
    const int cnt = min(TX, pitch - x0);  // multiple of 32 elements: 16-byte granular
    const uint32_t bytes = (uint32_t)(cnt * RW::ES);
    Elem* dst = b ? buf1 : buf0;
    if (tid == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&bars[b])),
                   "r"(bytes * Q)
                   : "memory");
    }
    __syncwarp();
    const int q = tid;
    if (q < Q) {
      int pq, row;
      bool bounce;
      src_row(q, y, z, pq, row, bounce);
      s_bounce[b][q] = bounce ? 1 : 0;
      const Elem* src = static_cast<const Elem*>(v.src_q[pq]) + row + x0;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_addr(dst + q * RW::STRIDE + RW::PAD)),
          "l"(src), "r"(bytes), "r"(smem_addr(&bars[b]))
          : "memory");
    }
  };
  // threads 0..2Q-1: halo values of tile t (left halo for c_x = +1, right for c_x = -1)
  auto halo_load = [&](int t, Elem& hv) {
    if (tid >= 2 * Q) return;
    int x0, y, z;
    tile_coords(t, x0, y, z);
    const int q = tid >> 1, side = tid & 1;
    int pq, row;
    bool bounce;
    src_row(q, y, z, pq, row, bounce);
    const int nvalid = min(TX, nx - x0);
    const int hx = side == 0 ? (x0 == 0 ? nx - 1 : x0 - 1) : (x0 + nvalid == nx ? 0 : x0 + nvalid);
    hv = static_cast<const Elem*>(v.src_q[pq])[row + hx];
  };
  auto halo_store = [&](int t, int b, Elem hv) {
    if (tid >= 2 * Q) return;
    int x0, y, z;
    tile_coords(t, x0, y, z);
    const int q = tid >> 1, side = tid & 1;
    const int nvalid = min(TX, nx - x0);
    Elem* dst = (b ? buf1 : buf0) + q * RW::STRIDE + RW::PAD;
    dst[side == 0 ? -1 : nvalid] = hv;
  };

  int t = blockIdx.x;
  if (t >= ntiles) return;
  Elem halo;
  if (tid < 32) issue(t, 0);
  halo_load(t, halo);
  uint32_t phases = 0u;  // bit b: parity of the next completion of buffer b
  for (int it = 0; t < ntiles; it++, t += gridDim.x) {
    const int b = it & 1;
    const int tn = t + gridDim.x;
    Elem halo_next;
    if (tn < ntiles) {
      if (tid < 32) issue(tn, b ^ 1);
      halo_load(tn, halo_next);
    }
    bool ok = tma_wait(&bars[b], (phases >> b) & 1u);
    phases ^= 1u << b;
    if (!__syncthreads_and(ok)) {
      if (tid == 0) {
        atomicOr(v.err, ERR_TIMEOUT);
        if (tn < ntiles) tma_wait(&bars[b ^ 1], (phases >> (b ^ 1)) & 1u);  // our other copy, bounded
      }
      return;
    }
    halo_store(t, b, halo);
    __syncthreads();
    // collide the tile from shared memory
    int x0, y, z;
    tile_coords(t, x0, y, z);
    const int x = x0 + tid;
    const bool active = x < nx;
    const int xx = active ? x : nx - 1;
    const int lx = xx - x0;  // interior index of this node
    const Elem* cur = (b ? buf1 : buf0) + RW::PAD;
    T f[Q];
#pragma unroll
    for (int q = 0; q < Q; q++) {
      const int cx = LAT::c(q, 0);
      const int off = s_bounce[b][q] ? lx : lx - cx;
      // shared memory: a plain load (the __ldg path is for global memory only)
      f[q] = S::load_shared(cur + q * RW::STRIDE, off, LAT::w(q));
    }
    collide_core<LAT, STORE>(v, xx, y, z, active, (z * ny + y) * pitch + xx, f);
    __syncthreads();  // buffer b is free for the tile after next
    halo = halo_next;
  }
}

template <class LAT, int STORE>
static int tma_smem_bytes() {
  using RW = TmaRow<STORE>;
  return 2 * LAT::Q * RW::STRIDE * RW::ES;
}

template <class LAT, int STORE>
static void launch_tma(const View& v, cudaStream_t s) {
  static int grid = 0;
  const int smem = tma_smem_bytes<LAT, STORE>();
  if (grid == 0) {
    int per_sm = 0, dev = 0, sms = 0;
    cudaFuncSetAttribute(collide_tma_kernel<LAT, STORE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, collide_tma_kernel<LAT, STORE>, 128, smem);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    grid = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  }
  const int ntiles = ((v.nx + TX - 1) / TX) * v.ny * v.nz;
  collide_tma_kernel<LAT, STORE><<<grid < ntiles ? grid : ntiles, 128, smem, s>>>(v, ntiles);
}

template <class LAT, int STORE, int MINB>
static void launch_one(const View& v, cudaStream_t s) {
  dim3 grid((v.nx + 127) / 128, v.ny, v.nz);
  collide_kernel<LAT, STORE, MINB><<<grid, 128, 0, s>>>(v);
}

// collide variants (chosen per simulation, see lbm_imb_set_collide_variant):
//   0  one node per thread, 128-thread CTAs, occupancy left to the compiler
//   1  same, register budget for 8 CTAs per SM
//   2  TMA-pipelined persistent form (reduced-precision storages; FP64 uses 0)
template <class LAT, int STORE>
static void dispatch(const View& v, cudaStream_t s) {
  if (v.collide_variant == 1) launch_one<LAT, STORE, 8>(v, s);
  else if (v.collide_variant == 2 && STORE != LBM_IMB_STORE_F64) launch_tma<LAT, STORE>(v, s);
  else launch_one<LAT, STORE, 1>(v, s);
}

void launch_collide(const View& v, cudaStream_t s) {
  if (v.dim == 2) {
    if (v.storage == LBM_IMB_STORE_F64) dispatch<D2Q9, LBM_IMB_STORE_F64>(v, s);
    else if (v.storage == LBM_IMB_STORE_F32DEV) dispatch<D2Q9, LBM_IMB_STORE_F32DEV>(v, s);
    else dispatch<D2Q9, LBM_IMB_STORE_F16DEV>(v, s);
  } else {
    if (v.storage == LBM_IMB_STORE_F64) dispatch<D3Q19, LBM_IMB_STORE_F64>(v, s);
    else if (v.storage == LBM_IMB_STORE_F32DEV) dispatch<D3Q19, LBM_IMB_STORE_F32DEV>(v, s);
    else dispatch<D3Q19, LBM_IMB_STORE_F16DEV>(v, s);
  }
}

}  // namespace lbm
