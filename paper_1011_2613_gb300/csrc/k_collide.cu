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

// Row tiles t = (z * ny + y) * nxb + xt of 128 nodes, walked with a fixed
// stride (the grid size) without divisions in the loop.
struct TileWalk {
  int xt, y, z, dxt, dy, dz, nxb, ny;
  __device__ TileWalk(int t0, int stride, int nxb_, int ny_) : nxb(nxb_), ny(ny_) {
    xt = t0 % nxb;
    y = (t0 / nxb) % ny;
    z = (t0 / nxb) / ny;
    dxt = stride % nxb;
    dy = (stride / nxb) % ny;
    dz = (stride / nxb) / ny;
  }
  __device__ void next() {
    xt += dxt;
    const int c1 = xt >= nxb ? 1 : 0;
    xt -= c1 * nxb;
    y += dy + c1;  // < 2 ny
    const int c2 = y >= ny ? 1 : 0;
    y -= c2 * ny;
    z += dz + c2;
  }
};

// Persistent fused form: a CTA of 4 warps walks row tiles of 128 nodes
// (grid-stride); each warp takes its 32-node segment of the tile, so the 19
// pulled loads of a warp are 32 consecutive elements each (shifted by c_x)
// and the stores are aligned.  Covered nodes go through the warp's queue
// (dynamic shared memory, queue_bytes_per_warp per warp).
template <class LAT, int STORE, int MINB>
__global__ void __launch_bounds__(128, MINB) collide_kernel(View v, int ntiles) {
  extern __shared__ __align__(16) unsigned char smem_q[];
  const int nx = v.nx, nz = v.nz;
  const int lane = threadIdx.x & 31;
  const WarpQueue<STORE> wq = warp_queue<LAT, STORE>(smem_q, threadIdx.x >> 5);
  int cnt = 0;
  (void)ntiles;
  for (TileWalk w(blockIdx.x, gridDim.x, (nx + 127) / 128, v.ny_c); w.z < nz; w.next()) {
    const int x = w.xt * 128 + (int)threadIdx.x;
    const bool active = x < nx;
    fused_node<LAT, STORE>(v, active ? x : nx - 1, v.y0 + w.y, w.z, active, wq, cnt, lane);
  }
  queue_drain<LAT, STORE>(v, wq, cnt, lane);
}

// Split form of the pair storage, plain part: persistent row tiles as in
// form 0; covered nodes are skipped (the rasteriser listed them).
template <class LAT, int STORE>
__global__ void __launch_bounds__(128, 4) collide_plain_kernel(View v, int ntiles) {
  using T = typename Storage<STORE>::T;
  const int nx = v.nx, nz = v.nz;
  (void)ntiles;
  for (TileWalk w(blockIdx.x, gridDim.x, (nx + 127) / 128, v.ny_c); w.z < nz; w.next()) {
    const int x = w.xt * 128 + (int)threadIdx.x;
    const bool active = x < nx;
    const int xx = active ? x : nx - 1, y = v.y0 + w.y;
    const int n = (w.z * v.ny + y) * v.pitch + xx;
    const bool covered = v.own[0][n] >= 0;
    if (__all_sync(0xffffffffu, covered || !active)) continue;  // the whole segment is covered
    T f[LAT::Q];
    pull<LAT, STORE>(v, xx, y, w.z, n, active && !covered, f);  // covered nodes: the covered kernel pulls them
    plain_core<LAT, STORE>(v, n, active && !covered, f);
  }
}

// Split form 9 of the pair storage, plain part: as collide_plain_kernel,
// but the covered nodes are pulled here too, and their populations,
// moments, node offset and first owner slots go to a compact buffer (one
// atomic per warp reserves the entries; layout: float2 [Q + 5][cap], then
// double fraction [cap], int node [cap], int owner 0 [cap], int owner 1
// [cap]), which the covered kernel reads contiguously instead of pulling 19
// strided populations and the slots again.
template <class LAT>
__global__ void __launch_bounds__(128, 5) collide_plain_buf_kernel(View v, int ntiles) {
  constexpr int STORE = LBM_IMB_STORE_DFDEV;
  constexpr int Q = LAT::Q;
  const unsigned FULL = 0xffffffffu;
  const int nx = v.nx, nz = v.nz, lane = threadIdx.x & 31;
  const long long cap = v.cbuf_cap;
  (void)ntiles;
  for (TileWalk w(blockIdx.x, gridDim.x, (nx + 127) / 128, v.ny_c); w.z < nz; w.next()) {
    const int x = w.xt * 128 + (int)threadIdx.x;
    const bool active = x < nx;
    const int xx = active ? x : nx - 1, y = v.y0 + w.y;
    const int n = (w.z * v.ny + y) * v.pitch + xx;
    const int o0 = active ? v.own[0][n] : -1;
    const bool covered = o0 >= 0;
    int o1 = -1;
    double e0 = 0.0;
    if (covered) {  // requested with the pull, consumed only by the covered kernel
      o1 = v.own[1][n];
      e0 = static_cast<const double*>(v.eps[0])[n];
    }
    DF f[Q];
    pull<LAT, STORE>(v, xx, y, w.z, n, active, f);
    // every node of the row gets the plain update stored (the covered
    // kernel overwrites the covered ones later): whole sectors, so the L2
    // writes them back without reading the rest of a sector from DRAM
    const Moments<DF> m = plain_core<LAT, STORE>(v, n, active, f);
    const unsigned b = __ballot_sync(FULL, covered);
    if (b == 0u) continue;
    int base = 0;
    if (lane == 0) base = atomicAdd(v.cov_count, __popc(b));
    base = __shfl_sync(FULL, base, 0);
    if (!covered) continue;
    const long long i = (long long)base + __popc(b & ((1u << lane) - 1u));
    if (i >= cap) {  // more covered nodes than the particles' boxes hold: reported, not stored
      atomicOr(v.err, ERR_OWNERS);
      continue;
    }
    float2* e = v.cbuf;
#pragma unroll
    for (int q = 0; q < Q; q++) e[q * cap + i] = make_float2(f[q].h, f[q].l);
    e[(Q + 0) * cap + i] = make_float2(m.rho.h, m.rho.l);
    e[(Q + 1) * cap + i] = make_float2(m.drho.h, m.drho.l);
    e[(Q + 2) * cap + i] = make_float2(m.ux.h, m.ux.l);
    e[(Q + 3) * cap + i] = make_float2(m.uy.h, m.uy.l);
    e[(Q + 4) * cap + i] = make_float2(m.uz.h, m.uz.l);
    reinterpret_cast<double*>(e + (Q + 5) * cap)[i] = e0;
    int* ei = reinterpret_cast<int*>(reinterpret_cast<double*>(e + (Q + 5) * cap) + cap);
    ei[i] = n;
    ei[cap + i] = o0;
    ei[2 * cap + i] = o1;
  }
}

// Split form 9, covered part: the buffer's entries 32 per warp, the
// immersed-boundary update in pair arithmetic.
template <class LAT>
__global__ void __launch_bounds__(128, 4) collide_covered_buf_kernel(View v) {
  constexpr int STORE = LBM_IMB_STORE_DFDEV;
  constexpr int Q = LAT::Q;
  const long long cap = v.cbuf_cap;
  const int cnt = *v.cov_count;
  const int count = cnt < cap ? cnt : (int)cap;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
  const int row = v.ny * v.pitch;
  const float2* e = v.cbuf;
  const double* ee = reinterpret_cast<const double*>(e + (Q + 5) * cap);
  const int* en = reinterpret_cast<const int*>(ee + cap);
  for (int base = warp * 32; base < count; base += nwarps * 32) {
    const int i = base + lane;
    const bool mine = i < count;
    const long long k = mine ? i : base;
    DF f[Q];
#pragma unroll
    for (int q = 0; q < Q; q++) {
      const float2 a = e[q * cap + k];
      f[q] = DF(a.x, a.y);
    }
    Moments<DF> m;
    float2 a = e[(Q + 0) * cap + k];
    m.rho = DF(a.x, a.y);
    a = e[(Q + 1) * cap + k];
    m.drho = DF(a.x, a.y);
    a = e[(Q + 2) * cap + k];
    m.ux = DF(a.x, a.y);
    a = e[(Q + 3) * cap + k];
    m.uy = DF(a.x, a.y);
    a = e[(Q + 4) * cap + k];
    m.uz = DF(a.x, a.y);
    m.k = k_of<LAT, STORE>(m.ux, m.uy, m.uz);
    const int n = en[k];
    const int z = n / row, r = n - z * row;
    const int y = r / v.pitch, x = r - y * v.pitch;
    imb_core<LAT, STORE, true>(v, x, y, z, n, mine, f, m, SlotHead<double>{en[cap + k], en[2 * cap + k], ee[k]});
  }
}

// Split form of the pair storage, plain part with two nodes per thread
// (form 8): CTA = 128 nodes (64 pairs) of two consecutive rows; one grid
// dimension over (row pair, 128-node x tile), x tiles fastest.
template <class LAT>
__global__ void __launch_bounds__(128, 3) collide_plain_pair_kernel(View v) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rows = v.ny_c * v.nz;
  const int nxt = (v.nx + 127) / 128;  // x tiles fastest (see collide_pair_kernel)
  const int r = (int)(blockIdx.x / nxt) * 2 + (warp >> 1);
  const bool row_ok = r < rows;
  const int rr = row_ok ? r : rows - 1;
  const int x = (int)(blockIdx.x % nxt) * 128 + ((warp & 1) * 32 + lane) * 2;
  plain_pair_node<LAT>(v, x, v.y0 + rr % v.ny_c, rr / v.ny_c, row_ok);
}

// Split form, covered part: each warp takes 32 entries of the covered-node
// list (grouped by particle, so the warp's force sums mostly go to one
// owner), pulls and takes the moments in pair arithmetic, and gives the
// immersed-boundary update in FP64.
template <class LAT>
__global__ void __launch_bounds__(128, 3) collide_covered_kernel(View v) {
  constexpr int STORE = LBM_IMB_STORE_DFDEV;
  constexpr int Q = LAT::Q;
  const int count = *v.cov_count;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
  const int row = v.ny * v.pitch;
  for (int base = warp * 32; base < count; base += nwarps * 32) {
    const int i = base + lane;
    const bool mine = i < count;
    const int n = v.cov_list[mine ? i : base];
    const int z = n / row, r = n - z * row;
    const int y = r / v.pitch, x = r - y * v.pitch;
    DF f[Q];
    pull<LAT, STORE>(v, x, y, z, n, true, f);
    const Moments<DF> md = moments<LAT, STORE>(v, f);
    double g[Q];
#pragma unroll
    for (int q = 0; q < Q; q++) g[q] = df_to_bits(f[q]);
    Moments<double> m;
    m.rho = df_to_bits(md.rho);
    m.drho = df_to_bits(md.drho);
    m.ux = df_to_bits(md.ux);
    m.uy = df_to_bits(md.uy);
    m.uz = df_to_bits(md.uz);
    m.k = k_of<LAT, kDfDevImb>(m.ux, m.uy, m.uz);
    imb_core<LAT, kDfDevImb>(v, x, y, z, n, mine, g, m);
  }
}

// The same covered part in pair arithmetic throughout (form 7): the
// update's FP32-pipe instructions instead of the FP64 pipe.
template <class LAT>
__global__ void __launch_bounds__(128, 3) collide_covered_pair_kernel(View v) {
  constexpr int STORE = LBM_IMB_STORE_DFDEV;
  constexpr int Q = LAT::Q;
  const int count = *v.cov_count;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
  const int row = v.ny * v.pitch;
  for (int base = warp * 32; base < count; base += nwarps * 32) {
    const int i = base + lane;
    const bool mine = i < count;
    const int n = v.cov_list[mine ? i : base];
    const int z = n / row, r = n - z * row;
    const int y = r / v.pitch, x = r - y * v.pitch;
    DF f[Q];
    pull<LAT, STORE>(v, x, y, z, n, true, f);
    const Moments<DF> m = moments<LAT, STORE>(v, f);
    imb_core<LAT, STORE>(v, x, y, z, n, mine, f, m);
  }
}

// CTA-packed form: one CTA per 128-node row tile (no persistence).
template <class LAT, int STORE, int MINB>
__global__ void __launch_bounds__(128, MINB) collide_packed_kernel(View v) {
  extern __shared__ __align__(16) unsigned char smem_p[];
  const int x = blockIdx.x * 128 + threadIdx.x;
  const bool active = x < v.nx;
  packed_node<LAT, STORE>(v, active ? x : v.nx - 1, blockIdx.y, blockIdx.z, active, smem_p);
}

// Two-node form: CTA = 128 nodes (64 pairs) of two consecutive rows; one
// grid dimension over (row pair, 128-node x tile), x tiles fastest
// (reduced-precision storages).
template <class LAT, int STORE, int MINB>
__global__ void __launch_bounds__(128, MINB) collide_pair_kernel(View v) {
  extern __shared__ __align__(16) unsigned char smem_pp[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rows = v.ny * v.nz;
  // x tiles fastest, so that the CTAs of a row pair run side by side and the
  // sector a shifted pull shares with the next tile is still in L2
  const int nxt = (v.nx + 127) / 128;
  const int r = (int)(blockIdx.x / nxt) * 2 + (warp >> 1);
  const bool row_ok = r < rows;
  const int rr = row_ok ? r : rows - 1;
  const int x = (int)(blockIdx.x % nxt) * 128 + ((warp & 1) * 32 + lane) * 2;
  pair_node<LAT, STORE>(v, x, rr % v.ny, rr / v.ny, row_ok, smem_pp);
}

// Software-pipelined persistent form: the populations (and owner word) of
// the CTA's next tile are pulled into registers before the current tile is
// collided, so every warp keeps one tile of loads in flight while it
// computes.
template <class LAT, int STORE, int MINB>
__global__ void __launch_bounds__(128, MINB) collide_prefetch_kernel(View v, int ntiles) {
  using T = typename Storage<STORE>::T;
  extern __shared__ __align__(16) unsigned char smem_q[];
  const int nx = v.nx, ny = v.ny, nz = v.nz, pitch = v.pitch;
  const int lane = threadIdx.x & 31;
  const WarpQueue<STORE> wq = warp_queue<LAT, STORE>(smem_q, threadIdx.x >> 5);
  int cnt = 0;
  (void)ntiles;
  TileWalk w(blockIdx.x, gridDim.x, (nx + 127) / 128, ny);
  if (w.z >= nz) return;
  auto xof = [&](const TileWalk& t, bool& act) {
    const int x = t.xt * 128 + (int)threadIdx.x;
    act = x < nx;
    return act ? x : nx - 1;
  };
  bool act;
  int x = xof(w, act);
  T fn[LAT::Q];
  pull<LAT, STORE>(v, x, w.y, w.z, (w.z * ny + w.y) * pitch + x, act, fn);
  while (w.z < nz) {
    T f[LAT::Q];
#pragma unroll
    for (int q = 0; q < LAT::Q; q++) f[q] = fn[q];
    const int cx = x, cy = w.y, cz = w.z;
    const bool cact = act;
    w.next();
    if (w.z < nz) {
      x = xof(w, act);
      pull<LAT, STORE>(v, x, w.y, w.z, (w.z * ny + w.y) * pitch + x, act, fn);
    }
    fused_core<LAT, STORE>(v, cx, cy, cz, (cz * ny + cy) * pitch + cx, cact, f, wq, cnt, lane);
  }
  queue_drain<LAT, STORE>(v, wq, cnt, lane);
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
  const WarpQueue<STORE> wq = warp_queue<LAT, STORE>(smem_raw + 2 * Q * RW::STRIDE * RW::ES, threadIdx.x >> 5);
  int cnt = 0;

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
      f[q] = S::load_shared(cur + q * RW::STRIDE, off);
    }
    const int n = (z * ny + y) * pitch + xx;
    fused_core<LAT, STORE>(v, xx, y, z, n, active, f, wq, cnt, tid & 31);
    __syncthreads();  // buffer b is free for the tile after next
    halo = halo_next;
  }
  queue_drain<LAT, STORE>(v, wq, cnt, tid & 31);
}

template <class LAT, int STORE>
static int tma_smem_bytes() {
  using RW = TmaRow<STORE>;
  return 2 * LAT::Q * RW::STRIDE * RW::ES + 4 * queue_bytes_per_warp<LAT, STORE>();
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

template <class LAT, int STORE, int MINB, bool PREFETCH>
static void launch_fused(const View& v, cudaStream_t s) {
  static int grid = 0;
  const int smem = 4 * queue_bytes_per_warp<LAT, STORE>();
  const void* k;
  if constexpr (PREFETCH) k = (const void*)collide_prefetch_kernel<LAT, STORE, MINB>;
  else k = (const void*)collide_kernel<LAT, STORE, MINB>;
  if (grid == 0) {
    int per_sm = 0, dev = 0, sms = 0;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 128, smem);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    grid = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  }
  const int ntiles = ((v.nx + 127) / 128) * v.ny_c * v.nz;
  const int g = grid < ntiles ? grid : ntiles;
  if constexpr (PREFETCH) collide_prefetch_kernel<LAT, STORE, MINB><<<g, 128, smem, s>>>(v, ntiles);
  else collide_kernel<LAT, STORE, MINB><<<g, 128, smem, s>>>(v, ntiles);
}

// COVERED: 0 FP64 (form 6), 1 pair arithmetic (form 7), 2 pair arithmetic
// with the plain part two nodes per thread (form 8)
template <class LAT, int STORE, int COVERED>
static void launch_split(const View& v, cudaStream_t s) {
  static int grid_a = 0, grid_b = 0, sms = 0;
  if (grid_a == 0) {
    int per_sm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) sms = 1;
    if constexpr (COVERED == 3)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, collide_plain_buf_kernel<LAT>, 128, 0);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, collide_plain_kernel<LAT, STORE>, 128, 0);
    grid_a = (per_sm > 0 ? per_sm : 1) * sms;
    per_sm = 0;
    if constexpr (COVERED == 3)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, collide_covered_buf_kernel<LAT>, 128, 0);
    else if constexpr (COVERED >= 1)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, collide_covered_pair_kernel<LAT>, 128, 0);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, collide_covered_kernel<LAT>, 128, 0);
    grid_b = (per_sm > 0 ? per_sm : 1) * sms;
  }
  const int ntiles = ((v.nx + 127) / 128) * v.ny_c * v.nz;
  if constexpr (COVERED == 3) {  // covered nodes through the compact buffer
    collide_plain_buf_kernel<LAT><<<grid_a < ntiles ? grid_a : ntiles, 128, 0, s>>>(v, ntiles);
    if (v.cbuf != nullptr) collide_covered_buf_kernel<LAT><<<grid_b, 128, 0, s>>>(v);
    return;
  } else if constexpr (COVERED == 2) {  // the plain part two nodes per thread
    const unsigned grid = (unsigned)(((v.ny_c * v.nz + 1) / 2) * ((v.nx + 127) / 128));
    collide_plain_pair_kernel<LAT><<<grid, 128, 0, s>>>(v);
  } else {
    collide_plain_kernel<LAT, STORE><<<grid_a < ntiles ? grid_a : ntiles, 128, 0, s>>>(v, ntiles);
  }
  if (v.cov_list == nullptr) return;
  if constexpr (COVERED >= 1) collide_covered_pair_kernel<LAT><<<grid_b, 128, 0, s>>>(v);
  else collide_covered_kernel<LAT><<<grid_b, 128, 0, s>>>(v);
}

template <class LAT, int STORE, int MINB>
static void launch_packed(const View& v, cudaStream_t s) {
  const int smem = 2 * queue_bytes_per_warp<LAT, STORE>();
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(collide_packed_kernel<LAT, STORE, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  collide_packed_kernel<LAT, STORE, MINB><<<dim3((v.nx + 127) / 128, v.ny, v.nz), 128, smem, s>>>(v);
}

template <class LAT, int STORE, int MINB>
static void launch_pair(const View& v, cudaStream_t s) {
  if constexpr (STORE == LBM_IMB_STORE_F64) {
    launch_fused<LAT, STORE, 4, false>(v, s);  // two-node form: reduced-precision storages only
  } else {
    const int smem = pair_pack_bytes<LAT, STORE>();
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(collide_pair_kernel<LAT, STORE, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           smem);
      attr = true;
    }
    const unsigned grid = (unsigned)(((v.ny * v.nz + 1) / 2) * ((v.nx + 127) / 128));
    collide_pair_kernel<LAT, STORE, MINB><<<grid, 128, smem, s>>>(v);
  }
}

// collide variants (chosen per simulation, see lbm_imb_set_collide_variant):
//   0  persistent fused form, register budget for 4 CTAs per SM
//   1  same, register budget for 8 CTAs per SM
//   2  TMA-pipelined persistent form (reduced-precision storages; FP64 uses 0)
//   3  persistent fused form, register budget for 6 CTAs per SM
//   4  software-pipelined fused form (next tile pulled ahead), 4 CTAs per SM
//   5  the same, 3 CTAs per SM
//   6  CTA-packed form, one CTA per row tile, register budget for 8 CTAs/SM
//   7  the same, 5 CTAs per SM
//   8  two-node form (paired FP32 arithmetic), 6 CTAs per SM (reduced-
//      precision storages; FP64 uses 0)
//   9  the same, 5 CTAs per SM
template <class LAT, int STORE>
static void dispatch(const View& v, cudaStream_t s) {
  if constexpr (STORE == LBM_IMB_STORE_DFDEV) {
    // the persistent fused forms, with the register budgets the pair
    // arithmetic needs (1 and 3: 2 and 3 CTAs per SM; 4 and 5: the
    // prefetching form at 2 and 3), the TMA-pipelined form (2) and the
    // split forms (plain nodes, then the rasteriser's covered-node list: 6
    // in FP64, 7 in pair arithmetic, 8 as 7 with two plain nodes per thread
    // in paired instructions; 9: the covered nodes' pulled populations and
    // moments passed through a compact buffer instead of the list)
    switch (v.collide_variant) {
      case 1: launch_fused<LAT, STORE, 2, false>(v, s); break;
      case 2: launch_tma<LAT, STORE>(v, s); break;
      case 3: launch_fused<LAT, STORE, 3, false>(v, s); break;
      case 4: launch_fused<LAT, STORE, 2, true>(v, s); break;
      case 5: launch_fused<LAT, STORE, 3, true>(v, s); break;
      case kCollideSplit: launch_split<LAT, STORE, 0>(v, s); break;
      case kCollideSplit + 1: launch_split<LAT, STORE, 1>(v, s); break;
      case kCollideSplit + 2: launch_split<LAT, STORE, 2>(v, s); break;
      case kCollideSplit + 3: launch_split<LAT, STORE, 3>(v, s); break;
      default: launch_fused<LAT, STORE, 4, false>(v, s);
    }
  } else {
    switch (v.collide_variant) {
      case 1: launch_fused<LAT, STORE, 8, false>(v, s); break;
      case 2:
        if (STORE != LBM_IMB_STORE_F64) launch_tma<LAT, STORE>(v, s);
        else launch_fused<LAT, STORE, 4, false>(v, s);
        break;
      case 3: launch_fused<LAT, STORE, 6, false>(v, s); break;
      case 4: launch_fused<LAT, STORE, 4, true>(v, s); break;
      case 5: launch_fused<LAT, STORE, 3, true>(v, s); break;
      case 6: launch_packed<LAT, STORE, 8>(v, s); break;
      case 7: launch_packed<LAT, STORE, 5>(v, s); break;
      case 8: launch_pair<LAT, STORE, 6>(v, s); break;
      case 9: launch_pair<LAT, STORE, 5>(v, s); break;
      default: launch_fused<LAT, STORE, 4, false>(v, s);
    }
  }
}

void launch_collide(const View& v, cudaStream_t s) {
  if (v.dim == 2) {
    if (v.storage == LBM_IMB_STORE_F64) dispatch<D2Q9, LBM_IMB_STORE_F64>(v, s);
    else if (v.storage == LBM_IMB_STORE_DFDEV) dispatch<D2Q9, LBM_IMB_STORE_DFDEV>(v, s);
    else if (v.storage == LBM_IMB_STORE_F32DEV) dispatch<D2Q9, LBM_IMB_STORE_F32DEV>(v, s);
    else dispatch<D2Q9, LBM_IMB_STORE_F16DEV>(v, s);
  } else {
    if (v.storage == LBM_IMB_STORE_F64) dispatch<D3Q19, LBM_IMB_STORE_F64>(v, s);
    else if (v.storage == LBM_IMB_STORE_DFDEV) dispatch<D3Q19, LBM_IMB_STORE_DFDEV>(v, s);
    else if (v.storage == LBM_IMB_STORE_F32DEV) dispatch<D3Q19, LBM_IMB_STORE_F32DEV>(v, s);
    else dispatch<D3Q19, LBM_IMB_STORE_F16DEV>(v, s);
  }
}

}  // namespace lbm
