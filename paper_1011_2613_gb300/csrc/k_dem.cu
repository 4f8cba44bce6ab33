// K3: DEM particle update (Xiong et al., Eqs. 4-5: frictionless linear
// spring-dashpot contacts) with a per-step cell list (or Verlet lists
// rebuilt on demand, dem_skin > 0), and the symplectic
// Euler integration of the particles under the hydrodynamic force/torque of
// Eq. (3), the contact force and gravity.
//
// Cell list: bins of side >= 2 R_max, a fixed capacity of kBinCap particles
// each (overflow raises LBM_IMB_EBIN).  One thread per particle scans the
// 3^d neighbouring bins, keeps its contacts, and sums them in ascending
// partner id so the contact force does not depend on the order particles
// entered a bin.  The device functions live in dev_dem.cuh.
#include "dev_dem.cuh"

namespace lbm {

__global__ void dem_zero_bins_kernel(int* count, int nbins) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nbins) count[i] = 0;
}

__global__ void dem_bin_kernel(View v) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < v.np) dem_bin_particle(v, p);
}

__global__ void dem_contact_kernel(View v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < v.np) dem_contact_particle(v, i);
}

__global__ void dem_integrate_kernel(View v, double dt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.np) return;
  dem_integrate_particle(v, i, dt);
  if (v.dem_skin > 0.0) dem_verlet_check_particle(v, i);
}

// Verlet path: the bins and lists are rebuilt only while the device flag is
// set (the launches stay in the captured graph and return at once otherwise)
__global__ void dem_vl_zero_bins_kernel(View v, int nbins) {
  if (*(volatile int*)v.vl_flag == 0) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nbins) v.bin_count[i] = 0;
}

__global__ void dem_vl_bin_kernel(View v) {
  if (*(volatile int*)v.vl_flag == 0) return;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < v.np) dem_bin_particle(v, p);
}

__global__ void dem_vl_build_kernel(View v) {
  if (*(volatile int*)v.vl_flag == 0) return;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < v.np) dem_verlet_build_particle(v, p);
}

__global__ void dem_vl_done_kernel(View v) {
  if (*v.vl_flag != 0) {
    *v.vl_flag = 0;
    *v.vl_builds += 1;
  }
}

__global__ void dem_vl_contact_kernel(View v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < v.np) dem_verlet_contact_particle(v, i);
}

void launch_dem_contacts(const View& v, cudaStream_t s) {
  if (v.np <= 0) return;
  const int nbins = v.nb[0] * v.nb[1] * v.nb[2];
  const int T = 128;
  if (v.dem_skin > 0.0) {
    dem_vl_zero_bins_kernel<<<(nbins + 255) / 256, 256, 0, s>>>(v, nbins);
    dem_vl_bin_kernel<<<(v.np + T - 1) / T, T, 0, s>>>(v);
    dem_vl_build_kernel<<<(v.np + T - 1) / T, T, 0, s>>>(v);
    dem_vl_done_kernel<<<1, 1, 0, s>>>(v);
    dem_vl_contact_kernel<<<(v.np + T - 1) / T, T, 0, s>>>(v);
    return;
  }
  dem_zero_bins_kernel<<<(nbins + 255) / 256, 256, 0, s>>>(v.bin_count, nbins);
  dem_bin_kernel<<<(v.np + T - 1) / T, T, 0, s>>>(v);
  dem_contact_kernel<<<(v.np + T - 1) / T, T, 0, s>>>(v);
}

void launch_dem(const View& v, cudaStream_t s) {
  if (v.np <= 0) return;
  const int T = 128;
  const double dt = 1.0 / v.substeps;
  for (int k = 0; k < v.substeps; k++) {
    launch_dem_contacts(v, s);
    dem_integrate_kernel<<<(v.np + T - 1) / T, T, 0, s>>>(v, dt);
  }
}

// bins of side >= 2 rmax along each axis of the domain (1 bin on an axis
// shorter than that); returns 0, or a negative status
int dem_bin_geometry(int dim, const int* ext, int wall_y, double rmax, int nb[3], double bsz[3]) {
  for (int d = 0; d < 3; d++) {
    nb[d] = 1;
    bsz[d] = (double)ext[d];
    if (d < dim && rmax > 0.0) {
      const bool periodic = !(d == 1 && wall_y);
      if (periodic && ext[d] < 2.0 * rmax + 2.0) return LBM_IMB_EUNSUPPORTED;
      int n = (int)floor(ext[d] / (2.0 * rmax));
      if (n < 1) n = 1;
      nb[d] = n;
      bsz[d] = (double)ext[d] / n;
    }
  }
  return 0;
}

}  // namespace lbm
