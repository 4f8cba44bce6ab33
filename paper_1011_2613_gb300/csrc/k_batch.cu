// K5: batched persistent step.  One cooperative launch advances every
// suspension of a batch (independent lattices of uneven sizes and particle
// counts) by one time step; its CTAs loop over shared work lists and meet at
// grid barriers between the phases of the method:
//   A  clear the previous eps footprints, zero the Eq. 3 sums and the bins
//   B  rasterise eps (one CTA per particle); bin the particles
//   C  pull-stream + Eq. 1 collision + Eq. 3 sums (tiles of tile_x x
//      128/tile_x nodes, covered nodes through per-warp queues); DEM
//      contacts
//   D  particle update
// The per-node, per-particle and per-cell work is the same device code as the
// per-step kernels (dev_*.cuh), so each member evolves exactly as it would
// alone (up to the order of the FP64 force atomics).
//
// Grid barrier: arrival counter + generation word in global memory.  Each
// wait spins with __nanosleep and gives up after spin_limit polls: it sets
// ERR_TIMEOUT in the batch error word and the CTA leaves the kernel; the
// other CTAs leave at their own next barrier, so a launch always ends.
#include "dev_collide.cuh"
#include "dev_dem.cuh"
#include "dev_eps.cuh"

namespace lbm {

struct BatchArgs {
  const View* views;    // [nm] member views (device memory)
  int nm;
  const int* part_off;  // [nm+1] prefix sums of particle counts
  const int* tile_off;  // [nm+1] prefix sums of collide tiles
  const int* bin_off;   // [nm+1] prefix sums of DEM bins
  const int* tiles_x;   // [nm] tiles along x per row group
  int tile_x;           // tile width (32, 64 or 128); tile height 128 / tile_x
  RasterSmem cap;       // raster table capacities for the largest radius
  unsigned* bar;        // [2] arrival count, generation
  int* err;             // batch error word
  long long spin_limit; // polls before a barrier wait gives up
  int phantom;          // extra arrivals a barrier waits for (test hook; 0)
};

__device__ __forceinline__ int member_of(const int* off, int nm, int i) {
  int lo = 0, hi = nm - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= i) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// returns false when the wait timed out (the caller must leave the kernel)
__device__ __forceinline__ bool grid_barrier(const BatchArgs& a) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* gen = a.bar + 1;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(a.bar, 1u) + 1u;
    if (arrived == gridDim.x + (unsigned)a.phantom) {
      atomicExch(a.bar, 0u);
      __threadfence();
      atomicAdd(a.bar + 1, 1u);
    } else {
      long long polls = 0;
      while (*gen == g) {
        if (++polls > a.spin_limit) {
          atomicOr(a.err, ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (ok && *(volatile int*)a.err & ERR_TIMEOUT) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

template <class LAT, int STORE, typename TE>
__global__ void __launch_bounds__(128) batch_step_kernel(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int gwarp = blockIdx.x * 4 + (threadIdx.x >> 5), nwarps = gridDim.x * 4;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, nthreads = gridDim.x * blockDim.x;
  const int P = a.part_off[a.nm];
  const int NB = a.bin_off[a.nm];
  const int NT = a.tile_off[a.nm];

  // A: footprints, force sums, bins
  for (int i = gwarp; i < P; i += nwarps) {
    const int m = member_of(a.part_off, a.nm, i);
    eps_clear_particle(a.views[m], i - a.part_off[m], lane, true);
  }
  for (int b = gtid; b < NB; b += nthreads) {
    const int m = member_of(a.bin_off, a.nm, b);
    a.views[m].bin_count[b - a.bin_off[m]] = 0;
  }
  if (!grid_barrier(a)) return;

  // B: eps rasterisation, binning
  for (int i = blockIdx.x; i < P; i += gridDim.x) {
    const int m = member_of(a.part_off, a.nm, i);
    if (a.views[m].eps_method == 1) eps_raster_particle<LAT::DIM, TE, true>(a.views[m], i - a.part_off[m], a.cap, smem);
    else eps_raster_particle<LAT::DIM, TE, false>(a.views[m], i - a.part_off[m], a.cap, smem);
  }
  for (int i = gtid; i < P; i += nthreads) {
    const int m = member_of(a.part_off, a.nm, i);
    dem_bin_particle(a.views[m], i - a.part_off[m]);
  }
  if (!grid_barrier(a)) return;

  // C: collision tiles, contacts.  The member's view is staged in shared
  // memory (the collision reads its per-direction plane pointers per access);
  // each warp's covered-node queue lives in the dynamic shared memory the
  // raster tables used in phase B, and is drained before the member changes.
  __shared__ View sv;
  int cached = -1;
  const int ty = 128 / a.tile_x;
  const WarpQueue<STORE> wq = warp_queue<LAT, STORE>(smem, threadIdx.x >> 5);
  int cnt = 0;
  for (int t = blockIdx.x; t < NT; t += gridDim.x) {
    const int m = member_of(a.tile_off, a.nm, t);
    if (m != cached) {
      if (cached >= 0) queue_drain<LAT, STORE>(sv, wq, cnt, lane);
      __syncthreads();
      const int* from = reinterpret_cast<const int*>(a.views + m);
      int* to = reinterpret_cast<int*>(&sv);
      for (int w = threadIdx.x; w < (int)(sizeof(View) / sizeof(int)); w += blockDim.x) to[w] = from[w];
      __syncthreads();
      cached = m;
    }
    const View& v = sv;
    const int local = t - a.tile_off[m];
    const int tx = a.tiles_x[m];
    const int x = (local % tx) * a.tile_x + threadIdx.x % a.tile_x;
    const int r = (local / tx) * ty + threadIdx.x / a.tile_x;  // row = z * ny + y
    const int rows = v.ny * v.nz;
    const bool active = x < v.nx && r < rows;
    const int rr = r < rows ? r : rows - 1;
    fused_node<LAT, STORE>(v, x < v.nx ? x : v.nx - 1, rr % v.ny, rr / v.ny, active, wq, cnt, lane);
  }
  if (cached >= 0) queue_drain<LAT, STORE>(sv, wq, cnt, lane);
  for (int i = gtid; i < P; i += nthreads) {
    const int m = member_of(a.part_off, a.nm, i);
    dem_contact_particle(a.views[m], i - a.part_off[m]);
  }
  if (!grid_barrier(a)) return;

  // D: particle update
  for (int i = gtid; i < P; i += nthreads) {
    const int m = member_of(a.part_off, a.nm, i);
    dem_integrate_particle(a.views[m], i - a.part_off[m], 1.0);
  }
}

template <class LAT, int STORE, typename TE>
static cudaError_t launch_t(const BatchArgs& a, int grid, int smem, cudaStream_t s) {
  void* args[] = {const_cast<BatchArgs*>(&a)};
  return cudaLaunchCooperativeKernel((const void*)batch_step_kernel<LAT, STORE, TE>, dim3(grid), dim3(128),
                                     args, (size_t)smem, s);
}

template <class LAT, int STORE, typename TE>
static const void* kernel_ptr() {
  return (const void*)batch_step_kernel<LAT, STORE, TE>;
}

static const void* batch_kernel(int dim, int storage) {
  if (dim == 2) {
    if (storage == LBM_IMB_STORE_F64) return kernel_ptr<D2Q9, LBM_IMB_STORE_F64, double>();
    if (storage == LBM_IMB_STORE_F32DEV) return kernel_ptr<D2Q9, LBM_IMB_STORE_F32DEV, float>();
    return kernel_ptr<D2Q9, LBM_IMB_STORE_F16DEV, float>();
  }
  if (storage == LBM_IMB_STORE_F64) return kernel_ptr<D3Q19, LBM_IMB_STORE_F64, double>();
  if (storage == LBM_IMB_STORE_F32DEV) return kernel_ptr<D3Q19, LBM_IMB_STORE_F32DEV, float>();
  return kernel_ptr<D3Q19, LBM_IMB_STORE_F16DEV, float>();
}

// dynamic shared memory the batch kernel needs besides the raster tables
int batch_queue_smem(int dim, int storage) {
  if (dim == 2) {
    if (storage == LBM_IMB_STORE_F64) return 4 * queue_bytes_per_warp<D2Q9, LBM_IMB_STORE_F64>();
    if (storage == LBM_IMB_STORE_F32DEV) return 4 * queue_bytes_per_warp<D2Q9, LBM_IMB_STORE_F32DEV>();
    return 4 * queue_bytes_per_warp<D2Q9, LBM_IMB_STORE_F16DEV>();
  }
  if (storage == LBM_IMB_STORE_F64) return 4 * queue_bytes_per_warp<D3Q19, LBM_IMB_STORE_F64>();
  if (storage == LBM_IMB_STORE_F32DEV) return 4 * queue_bytes_per_warp<D3Q19, LBM_IMB_STORE_F32DEV>();
  return 4 * queue_bytes_per_warp<D3Q19, LBM_IMB_STORE_F16DEV>();
}

// co-resident CTAs of the batch kernel (0 on error)
int batch_max_grid(int dim, int storage, int smem) {
  const void* k = batch_kernel(dim, storage);
  // static shared memory (collision packing, raster tables) comes on top of
  // the dynamic raster tables: always opt in to the dynamic size
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 0;
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 128, (size_t)smem) != cudaSuccess) return 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return per_sm * sms;
}

int batch_sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

cudaError_t launch_batch_step(const View* views, int nm, const int* part_off, const int* tile_off,
                              const int* bin_off, const int* tiles_x, int tile_x, int dim, int storage,
                              double rmax, unsigned* bar, int* err, long long spin_limit, int phantom,
                              int grid, int smem, cudaStream_t s) {
  BatchArgs a;
  a.views = views;
  a.nm = nm;
  a.part_off = part_off;
  a.tile_off = tile_off;
  a.bin_off = bin_off;
  a.tiles_x = tiles_x;
  a.tile_x = tile_x;
  a.cap = raster_caps(dim, rmax);
  a.bar = bar;
  a.err = err;
  a.spin_limit = spin_limit;
  a.phantom = phantom;
  if (dim == 2) {
    if (storage == LBM_IMB_STORE_F64) return launch_t<D2Q9, LBM_IMB_STORE_F64, double>(a, grid, smem, s);
    if (storage == LBM_IMB_STORE_F32DEV) return launch_t<D2Q9, LBM_IMB_STORE_F32DEV, float>(a, grid, smem, s);
    return launch_t<D2Q9, LBM_IMB_STORE_F16DEV, float>(a, grid, smem, s);
  }
  if (storage == LBM_IMB_STORE_F64) return launch_t<D3Q19, LBM_IMB_STORE_F64, double>(a, grid, smem, s);
  if (storage == LBM_IMB_STORE_F32DEV) return launch_t<D3Q19, LBM_IMB_STORE_F32DEV, float>(a, grid, smem, s);
  return launch_t<D3Q19, LBM_IMB_STORE_F16DEV, float>(a, grid, smem, s);
}

}  // namespace lbm
