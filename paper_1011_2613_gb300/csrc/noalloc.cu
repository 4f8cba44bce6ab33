// lbm_imb_dem_forces_static: the DEM contact-force entry point for callers
// that cannot allocate device memory.  Its bins live in a file-scope device
// array of fixed size instead of a caller workspace; nothing is allocated on
// any call.
#include <math.h>
#include <string.h>

#include <mutex>

#include "lbm_internal.cuh"

namespace {

// Fixed scratch capacity (8 MiB): error word, per-particle bin index and the
// cell-list bins.  Every device that loads the library holds this array
// until the process exits.
constexpr size_t kStaticScratchBytes = 8u << 20;
__device__ __align__(256) unsigned char g_dem_scratch[kStaticScratchBytes];

// The array's name is only a host-side stand-in; its device address is looked
// up once per device (with that device current) and cached here.
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

int scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_IMB_ECUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_dem_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return LBM_IMB_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return LBM_IMB_OK;
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" int lbm_imb_dem_forces_static(int32_t dim, const int32_t* extent, int32_t wall_y, int64_t n,
                                         double rmax, const double* pos, const double* vel,
                                         const double* radius, const double* mass, double k_n,
                                         double restitution, double* fc, void* stream) {
  // the checks of lbm_imb_dem_forces, in its order: with n = 0 there is
  // nothing to do and no layout to check
  if (n > 0 && (!pos || !vel || !radius || !mass || !fc)) return LBM_IMB_EINVAL;
  if (!(k_n >= 0.0) || !(restitution > 0.0 && restitution <= 1.0)) return LBM_IMB_EINVAL;
  if (n == 0) return LBM_IMB_OK;
  if ((dim != 2 && dim != 3) || !extent || n < 0 || n > (1ll << 30) || !(rmax > 0.0)) return LBM_IMB_EINVAL;
  if (wall_y != 0 && wall_y != 1) return LBM_IMB_EINVAL;
  int ext[3] = {extent[0], extent[1], dim == 3 ? extent[2] : 1};
  for (int d = 0; d < 3; d++)
    if (ext[d] < 1) return LBM_IMB_EINVAL;
  int nb[3];
  double bsz[3];
  int st = lbm::dem_bin_geometry(dim, ext, wall_y, rmax, nb, bsz);
  if (st) return st;
  const size_t nbins = (size_t)nb[0] * nb[1] * nb[2];
  const size_t off_err = 0;
  const size_t off_binof = up256(16);
  const size_t off_count = off_binof + up256((size_t)(n > 0 ? n : 1) * 4);
  const size_t off_slot = off_count + up256(nbins * 4);
  const size_t total = off_slot + up256(nbins * lbm::kBinCap * 4);
  if (total > kStaticScratchBytes) return LBM_IMB_EUNSUPPORTED;  // beyond the fixed scratch
  void* scratch = nullptr;
  st = scratch_address(&scratch);
  if (st) return st;
  unsigned char* base = static_cast<unsigned char*>(scratch);
  lbm::View v;
  memset(&v, 0, sizeof(v));
  v.dim = dim;
  v.nx = ext[0];
  v.ny = ext[1];
  v.nz = ext[2];
  v.wall_y = wall_y;
  v.np = (int)n;
  v.pos = const_cast<double*>(pos);
  v.vel = const_cast<double*>(vel);
  v.rad = const_cast<double*>(radius);
  v.mass = const_cast<double*>(mass);
  v.fc = fc;
  v.err = reinterpret_cast<int*>(base + off_err);
  v.bin_of = reinterpret_cast<int*>(base + off_binof);
  v.bin_count = reinterpret_cast<int*>(base + off_count);
  v.bin_slot = reinterpret_cast<int*>(base + off_slot);
  for (int d = 0; d < 3; d++) {
    v.nb[d] = nb[d];
    v.bsz[d] = bsz[d];
  }
  v.rmax_bins = rmax;
  v.kn = k_n;
  const double le = log(restitution);
  v.ln_e = le;
  v.dem_den = M_PI * M_PI + le * le;
  v.substeps = 1;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: the error word is cleared
  // here and the bin counts by the first kernel of launch_dem_contacts
  cudaError_t e = cudaMemsetAsync(v.err, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    lbm::launch_dem_contacts(v, s);
    e = cudaGetLastError();
  }
  int bits = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, v.err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return LBM_IMB_ECUDA;
  return lbm::status_of_err_bits(bits);
}
