// K1: solid-fraction rasterisation (the covered area/volume eps of each
// lattice cell, defined in the text after the Omega^S equation of Xiong et
// al.), and the clearing of the previous footprint.
//
// eps of a cell is evaluated exactly.  Reflecting the cell into the positive
// quadrant/octant of the particle frame (splitting it where it straddles a
// coordinate plane through the centre) turns it into boxes [a0,a1]x[b0,b1]
// (x[c0,c1]) with non-negative coordinates; a box is the inclusion-exclusion
// of the "upper corner" function
//   2D: U(a,b)   = area of {X>a, Y>b} inside the disk,
//   3D: P(a,b,c) = volume of {X>a, Y>b, Z>c} inside the ball,
// both in closed form.  Near the rim these corner values are small, so the
// inclusion-exclusion does not cancel large numbers.  P follows from the
// divergence theorem: 3P = R^3 Omega - a A_a - b A_b - c A_c with A_a the flat
// face area on the plane X=a and Omega the solid angle of the spherical face
// (Gauss-Bonnet: three vertex angles and three small-circle arcs).
//
// One CTA per particle: fully covered cells claim their node at once;
// partially covered cells are listed, the corner values they need (each
// shared by up to 8 cells) are computed once from per-axis / per-pair angle
// tables, and every listed cell combines its corners and claims an owner
// slot of its node.  The lists keep the FP64 pipe busy with useful lanes.
#include "dev_eps.cuh"

namespace lbm {

__global__ void __launch_bounds__(128) eps_clear_kernel(View v, bool zero_forces) {
  const int p = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (p < v.np) eps_clear_particle(v, p, threadIdx.x & 31, zero_forces);
}

template <int DIM, typename T, bool TABLE>
__global__ void __launch_bounds__(128) eps_raster_kernel(View v, RasterSmem cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (blockIdx.x < v.np) eps_raster_particle<DIM, T, TABLE>(v, blockIdx.x, cap, smem);
}

// Eq. 6 table: one thread per grid point (see dev_eps.cuh for the grid)
template <int DIM>
__global__ void eps_table_build_kernel(double R, float* tab) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  double off[3] = {0.0, 0.0, 0.0};
  if (DIM == 2) {
    if (id >= kTabR2 * kTabT2) return;
    const int i = id / kTabT2, j = id % kTabT2;
    const double r = (R - 0.70710678118654752440) + i * (1.41421356237309504880 / (kTabR2 - 1));
    const double t = j * (1.0 / (kTabT2 - 1));
    off[0] = r / sqrt(1.0 + t * t);
    off[1] = off[0] * t;
  } else {
    if (id >= kTabR3 * kTabS3 * kTabT3) return;
    const int i = id / (kTabS3 * kTabT3), j = (id / kTabT3) % kTabS3, k = id % kTabT3;
    const double r = (R - 0.86602540378443864676) + i * (1.73205080756887729353 / (kTabR3 - 1));
    const double sv = j * (1.41421356237309504880 / (kTabS3 - 1));
    const double t = k * (1.0 / (kTabT3 - 1));
    off[0] = r / sqrt(1.0 + sv * sv);
    off[1] = off[0] * sv / sqrt(1.0 + t * t);
    off[2] = off[1] * t;
  }
  tab[id] = (float)exact_cell_fraction(DIM, R, off);
}

long long eps_table_entries(int dim) {
  return dim == 2 ? (long long)kTabR2 * kTabT2 : (long long)kTabR3 * kTabS3 * kTabT3;
}

void eps_table_geometry(int dim, double R, float* lo_r, float* h_r, float* h_s, float* h_t) {
  if (dim == 2) {
    *lo_r = (float)(R - sqrt(2.0) / 2.0);
    *h_r = (float)(sqrt(2.0) / (kTabR2 - 1));
    *h_s = 0.f;
    *h_t = (float)(1.0 / (kTabT2 - 1));
  } else {
    *lo_r = (float)(R - sqrt(3.0) / 2.0);
    *h_r = (float)(sqrt(3.0) / (kTabR3 - 1));
    *h_s = (float)(sqrt(2.0) / (kTabS3 - 1));
    *h_t = (float)(1.0 / (kTabT3 - 1));
  }
}

cudaError_t launch_eps_table_build(int dim, double R, float* tab, cudaStream_t s) {
  const long long n = eps_table_entries(dim);
  const int grid = (int)((n + 255) / 256);
  if (dim == 2) eps_table_build_kernel<2><<<grid, 256, 0, s>>>(R, tab);
  else eps_table_build_kernel<3><<<grid, 256, 0, s>>>(R, tab);
  return cudaGetLastError();
}

int eps_raster_smem_bytes(int dim, int storage, double rmax) {
  const int esz = fp64_eps(storage) ? 8 : 4;
  // the covered-node list region only for the storage whose split form uses it
  const long long list = storage == LBM_IMB_STORE_DFDEV ? 0 : raster_list_bytes(dim, rmax);
  const long long bytes = raster_bytes(dim, esz, rmax) - list;
  if (bytes > 200 * 1024) return -1;
  return (int)bytes;
}

// the Eq. 6 table form keeps only the covered-node flags (pair storage)
int eps_table_raster_smem_bytes(int dim, int storage, double rmax) {
  if (storage != LBM_IMB_STORE_DFDEV) return 0;
  const long long bytes = raster_list_bytes(dim, rmax);
  return bytes > 200 * 1024 ? -1 : (int)bytes;
}

void launch_eps_clear(const View& v, bool zero_forces, cudaStream_t s) {
  if (v.np <= 0) return;
  eps_clear_kernel<<<(v.np + 3) / 4, 128, 0, s>>>(v, zero_forces);
}

template <int DIM, typename T>
static void raster_t(const View& v, const RasterSmem cap, int smem_bytes, cudaStream_t s) {
  if (v.eps_method == 1)  // no tables; the covered-node list only when it is built
    eps_raster_kernel<DIM, T, true><<<v.np, 128, v.cov_list ? (int)raster_list_bytes(DIM, v.rmax_bins) : 0, s>>>(
        v, cap);
  else eps_raster_kernel<DIM, T, false><<<v.np, 128, smem_bytes, s>>>(v, cap);
}

void launch_eps_raster(const View& v, int smem_bytes, cudaStream_t s) {
  if (v.np <= 0) return;
  const RasterSmem cap = raster_caps(v.dim, v.rmax_bins);
  // the pair storage rasterises in pair arithmetic (FP32 pipe), the FP64
  // storage in FP64, the others in FP32
  if (v.dim == 2) {
    if (v.storage == LBM_IMB_STORE_DFDEV) raster_t<2, DF>(v, cap, smem_bytes, s);
    else if (fp64_eps(v.storage)) raster_t<2, double>(v, cap, smem_bytes, s);
    else raster_t<2, float>(v, cap, smem_bytes, s);
  } else {
    if (v.storage == LBM_IMB_STORE_DFDEV) raster_t<3, DF>(v, cap, smem_bytes, s);
    else if (fp64_eps(v.storage)) raster_t<3, double>(v, cap, smem_bytes, s);
    else raster_t<3, float>(v, cap, smem_bytes, s);
  }
}

// opt in to large dynamic shared memory (called at handle creation)
template <bool TABLE>
static bool set_attrs_t(int bytes) {
  const int a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  return cudaFuncSetAttribute(eps_raster_kernel<2, DF, TABLE>, (cudaFuncAttribute)a, bytes) == cudaSuccess &&
         cudaFuncSetAttribute(eps_raster_kernel<3, DF, TABLE>, (cudaFuncAttribute)a, bytes) == cudaSuccess &&
         cudaFuncSetAttribute(eps_raster_kernel<2, double, TABLE>, (cudaFuncAttribute)a, bytes) == cudaSuccess &&
         cudaFuncSetAttribute(eps_raster_kernel<2, float, TABLE>, (cudaFuncAttribute)a, bytes) == cudaSuccess &&
         cudaFuncSetAttribute(eps_raster_kernel<3, double, TABLE>, (cudaFuncAttribute)a, bytes) == cudaSuccess &&
         cudaFuncSetAttribute(eps_raster_kernel<3, float, TABLE>, (cudaFuncAttribute)a, bytes) == cudaSuccess;
}

// the attribute only grows (handles with larger particles may coexist); the
// kernels' static shared memory counts against the same 227 KB, so it is set
// for every rasterising handle, not only above 48 KB of dynamic memory
int eps_raster_set_attrs(int bytes) {
  static int granted = 0;
  if (bytes <= granted) return 0;
  if (!(set_attrs_t<false>(bytes) && set_attrs_t<true>(bytes))) return -1;
  granted = bytes;
  return 0;
}

__global__ void atan2_probe_kernel(const double* y, const double* x, double* fast, double* ref, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  fast[i] = atan2_q1(y[i], x[i]);
  ref[i] = atan2(y[i], x[i]);
}

}  // namespace lbm

extern "C" int lbm_imb_probe_atan2q1(const double* y, const double* x, double* fast, double* ref, int64_t n,
                                     void* stream) {
  if (!y || !x || !fast || !ref || n < 0) return LBM_IMB_EINVAL;
  if (n == 0) return LBM_IMB_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  lbm::atan2_probe_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(y, x, fast, ref, (long long)n);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return LBM_IMB_ECUDA;
  return LBM_IMB_OK;
}
