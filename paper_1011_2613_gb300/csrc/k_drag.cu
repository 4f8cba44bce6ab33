// K8: per-particle drag samples for the learned closure.  One CTA per
// particle scans the nodes at distance (R, R + shell] from the centre and
// forms the local solid fraction, the (1 - eps)-weighted fluid velocity and
// from them the slip velocity and Reynolds number; the target is the
// particle's resolved hydrodynamic force (Eq. 3) over the Stokes scale.
#include <math.h>

#include "lbm_internal.cuh"

namespace lbm {

__global__ void __launch_bounds__(128) drag_samples_kernel(View v, const double* __restrict__ u,
                                                           const double* __restrict__ eps, double shell,
                                                           float* feats, float* target) {
  const int p = blockIdx.x;
  if (p >= v.np) return;
  const int dim = v.dim;
  const double R = v.rad[p];
  const double Ro = R + shell;
  double c[3];
  int lo[3] = {0, 0, 0}, ne[3] = {1, 1, 1};
  for (int d = 0; d < 3; d++) c[d] = v.pos[3 * p + d];
  for (int d = 0; d < dim; d++) {
    lo[d] = (int)ceil(c[d] - Ro);
    ne[d] = (int)floor(c[d] + Ro) - lo[d] + 1;
  }
  const long long N = (long long)v.nx * v.ny * v.nz;
  double se = 0.0, cnt = 0.0, w = 0.0, su[3] = {0.0, 0.0, 0.0};
  const int total = ne[0] * ne[1] * ne[2];
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int idx[3] = {lo[0] + t % ne[0], lo[1] + (t / ne[0]) % ne[1], lo[2] + t / (ne[0] * ne[1])};
    double d2 = 0.0;
    int node[3];
    bool skip = false;
    const int ext[3] = {v.nx, v.ny, v.nz};
    for (int d = 0; d < 3; d++) {
      node[d] = idx[d];
      if (d >= dim) continue;
      double r = (double)idx[d] - c[d];
      const bool periodic = !(d == 1 && v.wall_y);
      if (periodic) {
        node[d] = ((idx[d] % ext[d]) + ext[d]) % ext[d];
      } else if (idx[d] < 0 || idx[d] >= ext[d]) {
        skip = true;
      }
      d2 += r * r;
    }
    if (skip || !(d2 > R * R) || d2 > Ro * Ro) continue;
    const long long n = ((long long)node[2] * v.ny + node[1]) * v.nx + node[0];
    const double e = eps[n];
    se += e;
    cnt += 1.0;
    w += 1.0 - e;
    for (int d = 0; d < dim; d++) su[d] += (1.0 - e) * u[d * N + n];
  }
  // block sums
  __shared__ double red[6][4];
  double vals[6] = {se, cnt, w, su[0], su[1], su[2]};
  for (int k = 0; k < 6; k++) {
    double x = vals[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double tot[6];
  for (int k = 0; k < 6; k++) tot[k] = red[k][0] + red[k][1] + red[k][2] + red[k][3];
  const double phi = tot[1] > 0.0 ? tot[0] / tot[1] : 0.0;
  double slip[3] = {0.0, 0.0, 0.0};
  for (int d = 0; d < dim; d++) slip[d] = (tot[2] > 0.0 ? tot[3 + d] / tot[2] : 0.0) - v.vel[3 * p + d];
  const double nu = (v.tau - 0.5) / 3.0;
  const double smag = sqrt(slip[0] * slip[0] + slip[1] * slip[1] + slip[2] * slip[2]);
  const double vol = dim == 3 ? (4.0 / 3.0) * M_PI * R * R * R : M_PI * R * R;
  const double scale = dim == 3 ? 6.0 * M_PI * v.rho0 * nu * R : 4.0 * M_PI * v.rho0 * nu;
  float* f = feats + 6 * (size_t)p;
  f[0] = (float)phi;
  f[1] = (float)slip[0];
  f[2] = (float)slip[1];
  f[3] = (float)slip[2];
  f[4] = (float)(smag * 2.0 * R / nu);
  f[5] = (float)(v.mass[p] / vol / v.rho0);
  for (int d = 0; d < 3; d++) target[3 * (size_t)p + d] = (float)(v.ff[3 * p + d] / scale);
}

void launch_drag_samples(const View& v, const double* u, const double* eps, double shell, float* feats,
                         float* target, cudaStream_t s) {
  if (v.np <= 0) return;
  drag_samples_kernel<<<v.np, 128, 0, s>>>(v, u, eps, shell, feats, target);
}

}  // namespace lbm
