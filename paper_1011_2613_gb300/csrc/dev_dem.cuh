// DEM device functions (Xiong et al., Eqs. 4-5; symplectic Euler update),
// shared by the per-step kernels and the batched persistent kernel.  The
// multiply-add sequences are written with __dmul_rn / __dadd_rn / __dsub_rn,
// which the compiler never fuses into FMAs, so the contact and integration
// arithmetic is the plain IEEE sequence under any -fmad setting.
#pragma once
#include "lbm_internal.cuh"

namespace lbm {

constexpr int kMaxContacts = 24;

__device__ __forceinline__ int dem_bin_coord(double x, int d, const View& v) {
  // domain starts at -1/2 on a wall axis, at 0 (wrapped positions) otherwise
  const double origin = (d == 1 && v.wall_y) ? -0.5 : 0.0;
  int b = (int)floor((x - origin) / v.bsz[d]);
  if (b < 0) b = 0;
  if (b >= v.nb[d]) b = v.nb[d] - 1;
  return b;
}

__device__ __forceinline__ void dem_bin_particle(const View& v, int p) {
  // a non-finite (or runaway) centre is reported and left out of the bins,
  // so no other particle meets it; its own contact scan finds nothing
  bool bad = false;
  for (int d = 0; d < v.dim; d++) bad |= !(fabs(v.pos[3 * p + d]) <= kPosLimit);
  if (bad) {
    v.bin_of[p] = -1;
    atomicOr(v.err, ERR_NONFINITE);
    return;
  }
  int b[3] = {0, 0, 0};
  for (int d = 0; d < v.dim; d++) b[d] = dem_bin_coord(v.pos[3 * p + d], d, v);
  const int bin = (b[2] * v.nb[1] + b[1]) * v.nb[0] + b[0];
  v.bin_of[p] = bin;
  if (v.rad[p] > v.rmax_bins) atomicOr(v.err, ERR_BIN);  // bins too small for it
  const int slot = atomicAdd(v.bin_count + bin, 1);
  if (slot < kBinCap) v.bin_slot[bin * kBinCap + slot] = p;
  else atomicOr(v.err, ERR_BIN);
}

__device__ __forceinline__ double dem_wrap_delta(double d, int n) {
  const double L = (double)n;
  if (d > 0.5 * L) d -= L;
  else if (d < -0.5 * L) d += L;
  return d;
}

// contact force on i from j (Eqs. 4-5 as read): false when they do not touch
__device__ __forceinline__ bool dem_pair_force(const View& v, const int i, const int j, const double* pi_,
                                               const double* vi, const double Ri, const double mi, double* f) {
  const int dim = v.dim;
  double r[3], d2 = 0.0;
  for (int d = 0; d < 3; d++) {
    r[d] = pi_[d] - v.pos[3 * j + d];
    if (d < dim && !(d == 1 && v.wall_y)) r[d] = dem_wrap_delta(r[d], d == 0 ? v.nx : (d == 1 ? v.ny : v.nz));
    if (d >= dim) r[d] = 0.0;
    d2 = __dadd_rn(d2, __dmul_rn(r[d], r[d]));
  }
  const double dist = sqrt(d2);
  const double xi = Ri + v.rad[j] - dist;
  if (!(xi > 0.0) || dist == 0.0) return false;
  const double n0 = r[0] / dist, n1 = r[1] / dist, n2 = r[2] / dist;
  double vr = __dmul_rn(vi[0] - v.vel[3 * j], n0);
  vr = __dadd_rn(vr, __dmul_rn(vi[1] - v.vel[3 * j + 1], n1));
  vr = __dadd_rn(vr, __dmul_rn(vi[2] - v.vel[3 * j + 2], n2));
  const double mj = v.mass[j];
  const double ms = mi * mj / (mi + mj);
  const double eta = -2.0 * v.ln_e * sqrt(ms * v.kn / v.dem_den);
  const double kx = __dmul_rn(v.kn, xi), ev = __dmul_rn(eta, vr);
  f[0] = __dsub_rn(__dmul_rn(kx, n0), __dmul_rn(ev, n0));
  f[1] = __dsub_rn(__dmul_rn(kx, n1), __dmul_rn(ev, n1));
  f[2] = __dsub_rn(__dmul_rn(kx, n2), __dmul_rn(ev, n2));
  return true;
}

// wall contacts (walls at y = -1/2, normal +y, and y = ny - 1/2, normal -y; m* = m_i)
__device__ __forceinline__ void dem_wall_force(const View& v, const double* pi_, const double* vi, const double Ri,
                                               const double mi, double* F) {
  if (!v.wall_y) return;
  const double eta = -2.0 * v.ln_e * sqrt(mi * v.kn / v.dem_den);
  const double xb = Ri - (pi_[1] + 0.5);
  if (xb > 0.0) F[1] = __dadd_rn(F[1], __dsub_rn(__dmul_rn(v.kn, xb), __dmul_rn(eta, vi[1])));
  const double xt = Ri - (((double)v.ny - 0.5) - pi_[1]);
  if (xt > 0.0) F[1] = __dadd_rn(F[1], -__dsub_rn(__dmul_rn(v.kn, xt), __dmul_rn(eta, -vi[1])));
}

__device__ __forceinline__ void dem_contact_particle(const View& v, int i) {
  const int dim = v.dim;
  double pi_[3], vi[3];
  for (int d = 0; d < 3; d++) {
    pi_[d] = v.pos[3 * i + d];
    vi[d] = v.vel[3 * i + d];
  }
  const double Ri = v.rad[i], mi = v.mass[i];
  int bc[3] = {0, 0, 0};
  for (int d = 0; d < dim; d++) bc[d] = dem_bin_coord(pi_[d], d, v);

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
          double fj[3];
          if (!dem_pair_force(v, i, j, pi_, vi, Ri, mi, fj)) continue;
          if (nc < kMaxContacts) {
            cj[nc] = j;
            cf[nc][0] = fj[0];
            cf[nc][1] = fj[1];
            cf[nc][2] = fj[2];
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
  dem_wall_force(v, pi_, vi, Ri, mi, F);
  v.fc[3 * i] = F[0];
  v.fc[3 * i + 1] = F[1];
  v.fc[3 * i + 2] = F[2];
}

// ---------------------------------------------------------------------------
// Verlet neighbour lists (dem_skin > 0).  A build (only while the device
// flag asks for one) lists, for particle i, the partners j closer than
// R_i + R_j + skin, found in the bins of side >= 2 R_max + skin, in ascending
// id, and remembers i's position.  The contact pass then visits only the
// list, in that order, with the contact arithmetic of the cell-list path,
// so the summed force is bitwise the same as long as no pair outside the
// list touches: guaranteed while no particle has moved more than skin/2
// since the build, which the integration checks after every update (it sets
// the flag for the next pass).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void dem_verlet_build_particle(const View& v, const int i) {
  const int dim = v.dim;
  double pi_[3];
  for (int d = 0; d < 3; d++) pi_[d] = v.pos[3 * i + d];
  const double Ri = v.rad[i];
  int bc[3] = {0, 0, 0};
  for (int d = 0; d < dim; d++) bc[d] = dem_bin_coord(pi_[d], d, v);
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
  int* list = v.vl_nbr + (size_t)i * kVerletCap;
  int cnt = 0;
  bool overflow = false;
  for (int a = 0; a < nn[0]; a++)
    for (int b = 0; b < nn[1]; b++)
      for (int c = 0; c < nn[2]; c++) {
        const int bin = (nbr[2][c] * v.nb[1] + nbr[1][b]) * v.nb[0] + nbr[0][a];
        int bcnt = v.bin_count[bin];
        if (bcnt > kBinCap) bcnt = kBinCap;
        for (int s = 0; s < bcnt; s++) {
          const int j = v.bin_slot[bin * kBinCap + s];
          if (j == i) continue;
          double d2 = 0.0;
          for (int d = 0; d < dim; d++) {
            double r = pi_[d] - v.pos[3 * j + d];
            if (!(d == 1 && v.wall_y)) r = dem_wrap_delta(r, d == 0 ? v.nx : (d == 1 ? v.ny : v.nz));
            d2 += r * r;
          }
          const double reach = Ri + v.rad[j] + v.dem_skin;
          if (d2 >= reach * reach) continue;
          if (cnt < kVerletCap) {
            int k = cnt++;  // insert in ascending id
            while (k > 0 && list[k - 1] > j) {
              list[k] = list[k - 1];
              k--;
            }
            list[k] = j;
          } else {
            overflow = true;
          }
        }
      }
  if (overflow) atomicOr(v.err, ERR_BIN);
  v.vl_count[i] = cnt;
  for (int d = 0; d < 3; d++) v.vl_ref[3 * i + d] = pi_[d];
}

__device__ __forceinline__ void dem_verlet_contact_particle(const View& v, const int i) {
  double pi_[3], vi[3];
  for (int d = 0; d < 3; d++) {
    pi_[d] = v.pos[3 * i + d];
    vi[d] = v.vel[3 * i + d];
  }
  const double Ri = v.rad[i], mi = v.mass[i];
  const int* list = v.vl_nbr + (size_t)i * kVerletCap;
  const int cnt = v.vl_count[i];
  double F[3] = {0.0, 0.0, 0.0};
  int nc = 0;
  for (int k = 0; k < cnt; k++) {
    double fj[3];
    if (!dem_pair_force(v, i, list[k], pi_, vi, Ri, mi, fj)) continue;
    if (nc++ >= kMaxContacts) continue;  // the cell-list path keeps the first kMaxContacts too
    F[0] += fj[0];
    F[1] += fj[1];
    F[2] += fj[2];
  }
  if (nc > kMaxContacts) atomicOr(v.err, ERR_BIN);
  dem_wall_force(v, pi_, vi, Ri, mi, F);
  v.fc[3 * i] = F[0];
  v.fc[3 * i + 1] = F[1];
  v.fc[3 * i + 2] = F[2];
}

// after an update: has particle i moved more than skin/2 since the build?
__device__ __forceinline__ void dem_verlet_check_particle(const View& v, const int i) {
  double d2 = 0.0;
  for (int d = 0; d < v.dim; d++) {
    double r = v.pos[3 * i + d] - v.vl_ref[3 * i + d];
    if (!(d == 1 && v.wall_y)) r = dem_wrap_delta(r, d == 0 ? v.nx : (d == 1 ? v.ny : v.nz));
    d2 += r * r;
  }
  if (4.0 * d2 > v.dem_skin * v.dem_skin) atomicExch(v.vl_flag, 1);
}

__device__ __forceinline__ void dem_integrate_particle(const View& v, int i, double dt) {
  const double m = v.mass[i];
  for (int d = 0; d < v.dim; d++) {
    const double a = __dadd_rn(__dadd_rn(v.ff[3 * i + d], v.fc[3 * i + d]), __dmul_rn(m, v.gs[d])) / m;
    const double vel = __dadd_rn(v.vel[3 * i + d], __dmul_rn(a, dt));
    double x = __dadd_rn(v.pos[3 * i + d], __dmul_rn(vel, dt));
    if (!(d == 1 && v.wall_y)) {
      const double L = (double)(d == 0 ? v.nx : (d == 1 ? v.ny : v.nz));
      if (x >= L) x -= L;
      else if (x < 0.0) x += L;
    }
    v.vel[3 * i + d] = vel;
    v.pos[3 * i + d] = x;
  }
  const double I = v.inertia[i];
  bool bad = false;
  for (int d = 0; d < 3; d++) {
    const double w = __dadd_rn(v.omg[3 * i + d], __dmul_rn(v.tf[3 * i + d] / I, dt));
    v.omg[3 * i + d] = w;
    bad |= !isfinite(w) || !isfinite(v.vel[3 * i + d]) || !(fabs(v.pos[3 * i + d]) <= kPosLimit);
  }
  if (bad) atomicOr(v.err, ERR_NONFINITE);  // reported; the state is left as computed
}

}  // namespace lbm
