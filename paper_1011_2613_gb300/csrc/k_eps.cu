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

template <int DIM, typename T>
__global__ void __launch_bounds__(128) eps_raster_kernel(View v, RasterSmem cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (blockIdx.x < v.np) eps_raster_particle<DIM, T>(v, blockIdx.x, cap, smem);
}

int eps_raster_smem_bytes(int dim, int storage, double rmax) {
  const int esz = storage == LBM_IMB_STORE_F64 ? 8 : 4;
  const long long bytes = raster_bytes(dim, esz, rmax);
  if (bytes > 200 * 1024) return -1;
  return (int)bytes;
}

void launch_eps_clear(const View& v, bool zero_forces, cudaStream_t s) {
  if (v.np <= 0) return;
  eps_clear_kernel<<<(v.np + 3) / 4, 128, 0, s>>>(v, zero_forces);
}

void launch_eps_raster(const View& v, int smem_bytes, cudaStream_t s) {
  if (v.np <= 0) return;
  const RasterSmem cap = raster_caps(v.dim, v.rmax_bins);
  if (v.dim == 2) {
    if (v.storage == LBM_IMB_STORE_F64)
      eps_raster_kernel<2, double><<<v.np, 128, smem_bytes, s>>>(v, cap);
    else
      eps_raster_kernel<2, float><<<v.np, 128, smem_bytes, s>>>(v, cap);
  } else {
    if (v.storage == LBM_IMB_STORE_F64)
      eps_raster_kernel<3, double><<<v.np, 128, smem_bytes, s>>>(v, cap);
    else
      eps_raster_kernel<3, float><<<v.np, 128, smem_bytes, s>>>(v, cap);
  }
}

// opt in to large dynamic shared memory (called at handle creation)
int eps_raster_set_attrs(int bytes) {
  cudaError_t e1 = cudaFuncSetAttribute(eps_raster_kernel<2, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaError_t e2 = cudaFuncSetAttribute(eps_raster_kernel<2, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaError_t e3 = cudaFuncSetAttribute(eps_raster_kernel<3, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaError_t e4 = cudaFuncSetAttribute(eps_raster_kernel<3, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return (e1 == cudaSuccess && e2 == cudaSuccess && e3 == cudaSuccess && e4 == cudaSuccess) ? 0 : -1;
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
