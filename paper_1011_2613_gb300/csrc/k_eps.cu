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
// One CTA per particle builds the table of corner values its partially
// covered cells need (each corner is shared by up to 8 cells), then every
// cell combines its corners and claims an owner slot of its node.
#include <math.h>

#include "lbm_internal.cuh"

namespace lbm {

template <typename T>
__device__ __forceinline__ T kPi() { return T(3.14159265358979323846); }

// area of {X > a, Y > b} inside the disk of radius R centred at 0; a, b >= 0
template <typename T>
__device__ __forceinline__ T upper_quadrant_area(T a, T b, T R) {
  const T R2 = R * R;
  if (a * a + b * b >= R2) return T(0);
  const T sa = sqrt((R - a) * (R + a));  // Y of the disk boundary at X = a
  const T sb = sqrt((R - b) * (R + b));  // X of the disk boundary at Y = b
  // angle of the arc from (sb, b) to (a, sa)
  const T th = atan2(sb * sa - a * b, b * sa + a * sb);
  return T(0.5) * R2 * th - T(0.5) * (b * sb + a * sa) + a * b;
}

// volume of {X > a, Y > b, Z > c} inside the ball of radius R; a, b, c >= 0
template <typename T>
__device__ __forceinline__ T upper_octant_volume(T a, T b, T c, T R) {
  const T R2 = R * R;
  if (a * a + b * b + c * c >= R2) return T(0);
  // third coordinate of the sphere on the three edge lines of the corner
  const T zab = sqrt(R2 - a * a - b * b);
  const T zac = sqrt(R2 - a * a - c * c);
  const T zbc = sqrt(R2 - b * b - c * c);
  // arc angles of the three flat faces (circles of radius sqrt(R^2 - k^2))
  const T tha = atan2(zac * zab - b * c, b * zac + c * zab);
  const T thb = atan2(zbc * zab - a * c, a * zbc + c * zab);
  const T thc = atan2(zbc * zac - a * b, a * zbc + b * zac);
  // solid angle: interior vertex angles minus pi minus the geodesic
  // curvature integrals of the three small-circle arcs
  const T om = atan2(R * zab, a * b) + atan2(R * zac, a * c) +
               atan2(R * zbc, b * c) - kPi<T>() -
               (a * tha + b * thb + c * thc) / R;
  const T Aa = T(0.5) * (R2 - a * a) * tha - T(0.5) * (b * zab + c * zac) + b * c;
  const T Ab = T(0.5) * (R2 - b * b) * thb - T(0.5) * (a * zab + c * zbc) + a * c;
  const T Ac = T(0.5) * (R2 - c * c) * thc - T(0.5) * (a * zac + b * zbc) + a * b;
  return (R2 * R * om - a * Aa - b * Ab - c * Ac) / T(3);
}

// --------------------------------------------------------------------------
// clear the previous footprint (all owner slots) and zero the force sums
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(128) eps_clear_kernel(View v, bool zero_forces) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = blockIdx.x * 4 + warp;
  if (p >= v.np) return;
  const int* box = v.lo + 6 * p;
  const int lx = box[0], ly = box[1], lz = box[2];
  const int ex = box[3], ey = box[4], ez = box[5];
  const int total = ex * ey * ez;
  for (int t = lane; t < total; t += 32) {
    int i = lx + t % ex;
    int j = ly + (t / ex) % ey;
    int k = lz + t / (ex * ey);
    if (v.wall_y) {
      if (j < 0 || j >= v.ny) continue;
    } else {
      j = ((j % v.ny) + v.ny) % v.ny;
    }
    i = ((i % v.nx) + v.nx) % v.nx;
    k = ((k % v.nz) + v.nz) % v.nz;
    const long long n = ((long long)k * v.ny + j) * v.pitch + i;
#pragma unroll
    for (int s = 0; s < kMaxOwners; s++) v.own[s][n] = -1;
  }
  if (zero_forces && lane < 3) {
    v.ff[3 * p + lane] = 0.0;
    v.tf[3 * p + lane] = 0.0;
  }
}

// --------------------------------------------------------------------------
// rasterise one particle per CTA
// --------------------------------------------------------------------------
template <int DIM, typename T>
__global__ void __launch_bounds__(128) eps_raster_kernel(View v, int tab_cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int p = blockIdx.x;
  if (p >= v.np) return;
  const double R64 = v.rad[p];
  const T R = T(R64);
  double c[3] = {v.pos[3 * p], v.pos[3 * p + 1], v.pos[3 * p + 2]};
  int lo[3] = {0, 0, 0}, ne[3] = {1, 1, 1};
#pragma unroll
  for (int d = 0; d < DIM; d++) {
    lo[d] = (int)ceil(c[d] - R64 - 0.5);
    ne[d] = (int)floor(c[d] + R64 + 0.5) - lo[d] + 1;
  }
  // table dims: ne+1 boundaries plus one "zero" entry per axis
  const int tx = ne[0] + 2, ty = ne[1] + 2, tz = DIM == 3 ? ne[2] + 2 : 1;
  const int tsize = tx * ty * tz;
  if (tsize > tab_cap || ne[0] > 62 || ne[1] > 62 || ne[2] > 62) {  // radius beyond the launch's table capacity
    if (threadIdx.x == 0) atomicOr(v.err, ERR_OWNERS);
    return;
  }
  T* tab = reinterpret_cast<T*>(smem);
  unsigned char* need = smem + sizeof(T) * tab_cap;
  __shared__ T bnd[3][64];  // boundary offsets (cell edges minus centre)
  if (threadIdx.x == 0) {
    for (int d = 0; d < 3; d++) {
      v.lo[6 * p + d] = lo[d];
      v.lo[6 * p + 3 + d] = ne[d];
    }
  }
  for (int t = threadIdx.x; t < 3 * 64; t += blockDim.x) {
    const int d = t / 64, i = t % 64;
    bnd[d][i] = (d < DIM && i <= ne[d]) ? T(((double)(lo[d] + i) - 0.5) - c[d]) : T(0);
  }
  for (int t = threadIdx.x; t < tsize; t += blockDim.x) need[t] = 0;
  __syncthreads();

  const int ncell = ne[0] * ne[1] * ne[2];
  const T R2 = R * R;

  // per-axis decomposition of cell i into (lower, upper) table indices of
  // boxes in the positive half-axis; returns the number of boxes (1 or 2)
  auto decompose = [&](int d, int i, int (&lo_i)[2], int (&hi_i)[2]) -> int {
    const T bl = bnd[d][i], bh = bnd[d][i + 1];
    const int zero = ne[d] + 1;
    if (bl >= T(0)) { lo_i[0] = i; hi_i[0] = i + 1; return 1; }
    if (bh <= T(0)) { lo_i[0] = i + 1; hi_i[0] = i; return 1; }
    lo_i[0] = zero; hi_i[0] = i;
    lo_i[1] = zero; hi_i[1] = i + 1;
    return 2;
  };
  // 0: empty, 1: full, 2: partial
  auto classify = [&](int ci, int cj, int ck) -> int {
    T near2 = T(0), far2 = T(0);
    const int idx[3] = {ci, cj, ck};
#pragma unroll
    for (int d = 0; d < DIM; d++) {
      const T bl = bnd[d][idx[d]], bh = bnd[d][idx[d] + 1];
      const T nd = bl > T(0) ? bl : (bh < T(0) ? -bh : T(0));
      const T fd = fabs(bl) > fabs(bh) ? fabs(bl) : fabs(bh);
      near2 += nd * nd;
      far2 += fd * fd;
    }
    if (near2 >= R2) return 0;
    if (far2 <= R2) return 1;
    return 2;
  };

  // pass 1: mark the corner values that partially covered cells need
  for (int t = threadIdx.x; t < ncell; t += blockDim.x) {
    const int ci = t % ne[0], cj = (t / ne[0]) % ne[1], ck = t / (ne[0] * ne[1]);
    if (classify(ci, cj, ck) != 2) continue;
    int al[2], ah[2], bl[2], bh[2], cl[2] = {0, 0}, ch[2] = {0, 0};
    const int na = decompose(0, ci, al, ah);
    const int nb = decompose(1, cj, bl, bh);
    const int nc = DIM == 3 ? decompose(2, ck, cl, ch) : 1;
    for (int ia = 0; ia < na; ia++)
      for (int ib = 0; ib < nb; ib++)
        for (int ic = 0; ic < nc; ic++) {
          const int xs[2] = {al[ia], ah[ia]}, ys[2] = {bl[ib], bh[ib]}, zs[2] = {cl[ic], ch[ic]};
          for (int s = 0; s < (DIM == 3 ? 8 : 4); s++)
            need[(zs[(s >> 2) & 1] * ty + ys[(s >> 1) & 1]) * tx + xs[s & 1]] = 1;
        }
  }
  __syncthreads();
  // pass 2: corner values
  for (int t = threadIdx.x; t < tsize; t += blockDim.x) {
    if (!need[t]) continue;
    const int i = t % tx, j = (t / tx) % ty, k = t / (tx * ty);
    const T a = i <= ne[0] ? fabs(bnd[0][i]) : T(0);
    const T b = j <= ne[1] ? fabs(bnd[1][j]) : T(0);
    if (DIM == 2) {
      tab[t] = upper_quadrant_area<T>(a, b, R);
    } else {
      const T cc = k <= ne[2] ? fabs(bnd[2][k]) : T(0);
      tab[t] = upper_octant_volume<T>(a, b, cc, R);
    }
  }
  __syncthreads();
  // pass 3: cells
  for (int t = threadIdx.x; t < ncell; t += blockDim.x) {
    const int ci = t % ne[0], cj = (t / ne[0]) % ne[1], ck = t / (ne[0] * ne[1]);
    const int cls = classify(ci, cj, ck);
    if (cls == 0) continue;
    T e = T(1);
    if (cls == 2) {
      int al[2], ah[2], bl[2], bh[2], cl[2] = {0, 0}, ch[2] = {0, 0};
      const int na = decompose(0, ci, al, ah);
      const int nb = decompose(1, cj, bl, bh);
      const int nc = DIM == 3 ? decompose(2, ck, cl, ch) : 1;
      T sum = T(0);
      for (int ia = 0; ia < na; ia++)
        for (int ib = 0; ib < nb; ib++)
          for (int ic = 0; ic < nc; ic++) {
            const int xs[2] = {al[ia], ah[ia]}, ys[2] = {bl[ib], bh[ib]}, zs[2] = {cl[ic], ch[ic]};
            for (int s = 0; s < (DIM == 3 ? 8 : 4); s++) {
              const int sx = s & 1, sy = (s >> 1) & 1, sz = (s >> 2) & 1;
              const T val = tab[(zs[sz] * ty + ys[sy]) * tx + xs[sx]];
              sum += ((sx + sy + sz) & 1) ? -val : val;
            }
          }
      e = sum < T(0) ? T(0) : (sum > T(1) ? T(1) : sum);
      if (!(e > T(0))) continue;
    }
    // node of this cell
    int i = lo[0] + ci, j = lo[1] + cj, k = lo[2] + ck;
    if (v.wall_y) {
      if (j < 0 || j >= v.ny) continue;
    } else {
      j = ((j % v.ny) + v.ny) % v.ny;
    }
    i = ((i % v.nx) + v.nx) % v.nx;
    k = ((k % v.nz) + v.nz) % v.nz;
    const long long n = ((long long)k * v.ny + j) * v.pitch + i;
    bool claimed = false;
#pragma unroll
    for (int s = 0; s < kMaxOwners; s++) {
      if (atomicCAS(&v.own[s][n], -1, p) == -1) {
        static_cast<T*>(v.eps[s])[n] = e;
        claimed = true;
        break;
      }
    }
    if (!claimed) atomicOr(v.err, ERR_OWNERS);
  }
}

int eps_raster_smem_bytes(int dim, int storage, double rmax) {
  const int nmax = (int)(2.0 * rmax) + 3;
  long long entries = 1;
  for (int d = 0; d < dim; d++) entries *= (nmax + 2);
  const int esz = storage == LBM_IMB_STORE_F64 ? 8 : 4;
  long long bytes = entries * (esz + 1);
  bytes = (bytes + 15) & ~15LL;
  if (bytes > 200 * 1024) return -1;
  return (int)bytes;
}

void launch_eps_clear(const View& v, bool zero_forces, cudaStream_t s) {
  if (v.np <= 0) return;
  eps_clear_kernel<<<(v.np + 3) / 4, 128, 0, s>>>(v, zero_forces);
}

void launch_eps_raster(const View& v, int smem_bytes, cudaStream_t s) {
  if (v.np <= 0) return;
  const int esz = v.storage == LBM_IMB_STORE_F64 ? 8 : 4;
  const int cap = smem_bytes / (esz + 1);
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

}  // namespace lbm
