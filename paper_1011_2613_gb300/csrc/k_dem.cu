// K3: DEM particle update (Xiong et al., Eqs. 4-5: frictionless linear
// spring-dashpot contacts) with a per-step cell list, and the symplectic
// Euler integration of the particles under the hydrodynamic force/torque of
// Eq. (3), the contact force and gravity.
//
// Cell list: bins of side >= 2 R_max, a fixed capacity of kBinCap particles
// each (overflow raises LBM_IMB_EBIN).  One thread per particle scans the
// 3^d neighbouring bins, keeps its contacts, and sums them in ascending
// partner id so the contact force does not depend on the order particles
// entered a bin.  This file is compiled without FMA contraction so that the
// per-pair arithmetic is the plain IEEE sequence.
#include "lbm_internal.cuh"

namespace lbm {

constexpr int kMaxContacts = 24;

__global__ void dem_zero_bins_kernel(int* count, int nbins) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nbins) count[i] = 0;
}

__device__ __forceinline__ int bin_coord(double x, int d, const View& v) {
  // domain starts at -1/2 on a wall axis, at 0 (wrapped positions) otherwise
  const double origin = (d == 1 && v.wall_y) ? -0.5 : 0.0;
  int b = (int)floor((x - origin) / v.bsz[d]);
  if (b < 0) b = 0;
  if (b >= v.nb[d]) b = v.nb[d] - 1;
  return b;
}

__global__ void dem_bin_kernel(View v) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= v.np) return;
  int b[3] = {0, 0, 0};
  for (int d = 0; d < v.dim; d++) b[d] = bin_coord(v.pos[3 * p + d], d, v);
  const int bin = (b[2] * v.nb[1] + b[1]) * v.nb[0] + b[0];
  v.bin_of[p] = bin;
  if (v.rad[p] > v.rmax_bins) atomicOr(v.err, ERR_BIN);  // bins too small for it
  const int slot = atomicAdd(v.bin_count + bin, 1);
  if (slot < kBinCap) v.bin_slot[bin * kBinCap + slot] = p;
  else atomicOr(v.err, ERR_BIN);
}

__device__ __forceinline__ double wrap_delta(double d, int n) {
  const double L = (double)n;
  if (d > 0.5 * L) d -= L;
  else if (d < -0.5 * L) d += L;
  return d;
}

__global__ void dem_contact_kernel(View v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.np) return;
  const int dim = v.dim;
  double pi_[3], vi[3];
  for (int d = 0; d < 3; d++) {
    pi_[d] = v.pos[3 * i + d];
    vi[d] = v.vel[3 * i + d];
  }
  const double Ri = v.rad[i], mi = v.mass[i];
  int bc[3] = {0, 0, 0};
  for (int d = 0; d < dim; d++) bc[d] = bin_coord(pi_[d], d, v);

  int cj[kMaxContacts];
  double cf[kMaxContacts][3];
  int nc = 0;
  bool overflow = false;

  // distinct neighbouring bins per axis
  int nbr[3][3], nn[3];
  for (int d = 0; d < 3; d++) {
    nn[d] = 0;
    if (d >= dim) { nbr[d][nn[d]++] = 0; continue; }
    const bool periodic = !(d == 1 && v.wall_y);
    for (int o = -1; o <= 1; o++) {
      int b = bc[d] + o;
      if (periodic) b = ((b % v.nb[d]) + v.nb[d]) % v.nb[d];
      else if (b < 0 || b >= v.nb[d]) continue;
      bool dup = false;
      for (int k = 0; k < nn[d]; k++) dup |= nbr[d][k] == b;
      if (!dup) nbr[d][nn[d]++] = b;
    }
  }
  for (int a = 0; a < nn[0]; a++)
    for (int b = 0; b < nn[1]; b++)
      for (int c = 0; c < nn[2]; c++) {
        const int bin = (nbr[2][c] * v.nb[1] + nbr[1][b]) * v.nb[0] + nbr[0][a];
        int cnt = v.bin_count[bin];
        if (cnt > kBinCap) cnt = kBinCap;
        for (int s = 0; s < cnt; s++) {
          const int j = v.bin_slot[bin * kBinCap + s];
          if (j == i) continue;
          double r[3], d2 = 0.0;
          for (int d = 0; d < 3; d++) {
            r[d] = pi_[d] - v.pos[3 * j + d];
            if (d < dim && !(d == 1 && v.wall_y)) r[d] = wrap_delta(r[d], d == 0 ? v.nx : (d == 1 ? v.ny : v.nz));
            if (d >= dim) r[d] = 0.0;
            d2 += r[d] * r[d];
          }
          const double dist = sqrt(d2);
          const double xi = Ri + v.rad[j] - dist;
          if (!(xi > 0.0) || dist == 0.0) continue;
          const double n0 = r[0] / dist, n1 = r[1] / dist, n2 = r[2] / dist;
          const double vr = (vi[0] - v.vel[3 * j]) * n0 + (vi[1] - v.vel[3 * j + 1]) * n1 +
                            (vi[2] - v.vel[3 * j + 2]) * n2;
          const double mj = v.mass[j];
          const double ms = mi * mj / (mi + mj);
          const double eta = -2.0 * v.ln_e * sqrt(ms * v.kn / v.dem_den);
          if (nc < kMaxContacts) {
            cj[nc] = j;
            cf[nc][0] = v.kn * xi * n0 - eta * vr * n0;
            cf[nc][1] = v.kn * xi * n1 - eta * vr * n1;
            cf[nc][2] = v.kn * xi * n2 - eta * vr * n2;
            nc++;
          } else {
            overflow = true;
          }
        }
      }
  if (overflow) atomicOr(v.err, ERR_BIN);
  // sum in ascending partner id
  for (int a = 1; a < nc; a++) {
    const int kj = cj[a];
    const double k0 = cf[a][0], k1 = cf[a][1], k2 = cf[a][2];
    int b = a - 1;
    while (b >= 0 && cj[b] > kj) {
      cj[b + 1] = cj[b];
      cf[b + 1][0] = cf[b][0];
      cf[b + 1][1] = cf[b][1];
      cf[b + 1][2] = cf[b][2];
      b--;
    }
    cj[b + 1] = kj;
    cf[b + 1][0] = k0;
    cf[b + 1][1] = k1;
    cf[b + 1][2] = k2;
  }
  double F[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < nc; a++) {
    F[0] += cf[a][0];
    F[1] += cf[a][1];
    F[2] += cf[a][2];
  }
  if (v.wall_y) {
    // walls at y = -1/2 (normal +y) and y = ny - 1/2 (normal -y), m* = m_i
    const double eta = -2.0 * v.ln_e * sqrt(mi * v.kn / v.dem_den);
    const double xb = Ri - (pi_[1] + 0.5);
    if (xb > 0.0) F[1] += v.kn * xb - eta * vi[1];
    const double xt = Ri - (((double)v.ny - 0.5) - pi_[1]);
    if (xt > 0.0) F[1] += -(v.kn * xt - eta * (-vi[1]));
  }
  v.fc[3 * i] = F[0];
  v.fc[3 * i + 1] = F[1];
  v.fc[3 * i + 2] = F[2];
}

__global__ void dem_integrate_kernel(View v, double dt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.np) return;
  const double m = v.mass[i];
  for (int d = 0; d < v.dim; d++) {
    const double a = (v.ff[3 * i + d] + v.fc[3 * i + d] + m * v.gs[d]) / m;
    double vel = v.vel[3 * i + d] + a * dt;
    double x = v.pos[3 * i + d] + vel * dt;
    if (!(d == 1 && v.wall_y)) {
      const double L = (double)(d == 0 ? v.nx : (d == 1 ? v.ny : v.nz));
      if (x >= L) x -= L;
      else if (x < 0.0) x += L;
    }
    v.vel[3 * i + d] = vel;
    v.pos[3 * i + d] = x;
  }
  const double I = v.inertia[i];
  for (int d = 0; d < 3; d++) v.omg[3 * i + d] += v.tf[3 * i + d] / I * dt;
}

void launch_dem_contacts(const View& v, cudaStream_t s) {
  if (v.np <= 0) return;
  const int nbins = v.nb[0] * v.nb[1] * v.nb[2];
  const int T = 128;
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
