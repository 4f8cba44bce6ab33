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
// arithmetic).  Force and torque accumulate in FP64 in every variant.
#include "lbm_internal.cuh"

namespace lbm {

template <int STORE>
struct Storage;
template <>
struct Storage<LBM_IMB_STORE_F64> {
  using T = double;
  using E = double;  // eps slot element
  static constexpr bool DEV = false;
  __device__ static __forceinline__ T load(const void* p, long long i, double) {
    return __ldg(static_cast<const double*>(p) + i);
  }
  __device__ static __forceinline__ void store(void* p, long long i, T v, double) {
    static_cast<double*>(p)[i] = v;
  }
};
template <>
struct Storage<LBM_IMB_STORE_F32DEV> {
  using T = float;
  using E = float;
  static constexpr bool DEV = true;
  __device__ static __forceinline__ T load(const void* p, long long i, double) {
    return __ldg(static_cast<const float*>(p) + i);
  }
  __device__ static __forceinline__ void store(void* p, long long i, T v, double) {
    static_cast<float*>(p)[i] = v;
  }
};
template <>
struct Storage<LBM_IMB_STORE_F16DEV> {
  using T = float;
  using E = float;
  static constexpr bool DEV = true;
  // stored value = g / w (keeps the diagonal deviations out of subnormals)
  __device__ static __forceinline__ T load(const void* p, long long i, double w) {
    return __half2float(__ldg(static_cast<const __half*>(p) + i)) * float(w);
  }
  __device__ static __forceinline__ void store(void* p, long long i, T v, double w) {
    static_cast<__half*>(p)[i] = __float2half_rn(v * float(1.0 / w));
  }
};

// Segmented suffix sum over runs of equal keys in a warp; the first lane of
// each run adds the run total to the particle's force/torque.
__device__ __forceinline__ void warp_reduce_to_particles(int key, double (&val)[6], double* ff,
                                                         double* tf) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int next = __shfl_down_sync(FULL, key, 1);
  const int prev = __shfl_up_sync(FULL, key, 1);
  const unsigned tails = __ballot_sync(FULL, lane == 31 || next != key);
  const int run_end = __ffs(tails & (FULL << lane)) - 1;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
    for (int k = 0; k < 6; k++) {
      const double t = __shfl_down_sync(FULL, val[k], d);
      if (lane + d <= run_end) val[k] += t;
    }
  }
  const bool head = lane == 0 || prev != key;
  if (head && key >= 0) {
#pragma unroll
    for (int k = 0; k < 3; k++) {
      if (val[k] != 0.0) atomicAdd(ff + 3 * key + k, val[k]);
      if (val[3 + k] != 0.0) atomicAdd(tf + 3 * key + k, val[3 + k]);
    }
  }
}

// c . u built from the non-zero components only (after unrolling the
// direction loop the branches fold, and no 0*u term survives)
template <typename T>
__device__ __forceinline__ T cdot(int cx, int cy, int cz, T ux, T uy, T uz) {
  T r = T(0);
  bool have = false;
  if (cx != 0) { r = cx > 0 ? ux : -ux; have = true; }
  if (cy != 0) { const T t = cy > 0 ? uy : -uy; r = have ? r + t : t; have = true; }
  if (cz != 0) { const T t = cz > 0 ? uz : -uz; r = have ? r + t : t; have = true; }
  return r;
}

// feq_q = A +- B for the pair (q, q+1):  A = w rho (1 - 1.5 u.u + 4.5 cu^2)
// (+ w drho in deviation form, without the w rho0 rest part)
template <bool DEV, typename T>
__device__ __forceinline__ T pair_A(T w, T wr, T drho, T usq15, T cu) {
  if constexpr (DEV) return w * drho + wr * (T(4.5) * cu * cu - usq15);
  else return wr * ((T(1) - usq15) + T(4.5) * cu * cu);
}

__device__ __forceinline__ double min_image(double d, int n, bool periodic) {
  if (!periodic) return d;
  const double L = (double)n;
  if (d > 0.5 * L) d -= L;
  else if (d < -0.5 * L) d += L;
  return d;
}

template <class LAT, int STORE>
__global__ void __launch_bounds__(128) collide_kernel(View v) {
  using S = Storage<STORE>;
  using T = typename S::T;
  using E = typename S::E;
  constexpr int Q = LAT::Q;
  constexpr bool D3 = LAT::DIM == 3;

  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  const int z = blockIdx.z;
  const bool active = x < v.nx;
  const int xx = active ? x : v.nx - 1;  // inactive lanes stay in bounds
  const int nx = v.nx, ny = v.ny, nz = v.nz;
  const int xm = xx == 0 ? nx - 1 : xx - 1, xp = xx == nx - 1 ? 0 : xx + 1;
  const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
  const long long pitch = v.pitch, plane = v.plane;
  const long long n = ((long long)z * ny + y) * pitch + xx;

  // ---- pull streaming (halfway bounce-back at y walls) ----
  T f[Q];
#pragma unroll
  for (int q = 0; q < Q; q++) {
    const int cx = LAT::c(q, 0), cy = LAT::c(q, 1), cz = LAT::c(q, 2);
    const int sx = cx == 1 ? xm : (cx == -1 ? xp : xx);
    const int sy = cy == 1 ? ym : (cy == -1 ? yp : y);
    const int sz = cz == 1 ? zm : (cz == -1 ? zp : z);
    const bool bounce = v.wall_y && ((cy == 1 && y == 0) || (cy == -1 && y == ny - 1));
    if (bounce)
      f[q] = S::load(v.fsrc, opp(q) * plane + n, LAT::w(opp(q)));
    else
      f[q] = S::load(v.fsrc, q * plane + ((long long)sz * ny + sy) * pitch + sx, LAT::w(q));
  }

  // ---- moments ----
  T s0 = T(0), jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
  for (int q = 0; q < Q; q++) {
    s0 += f[q];
    if (LAT::c(q, 0) == 1) jx += f[q];
    if (LAT::c(q, 0) == -1) jx -= f[q];
    if (LAT::c(q, 1) == 1) jy += f[q];
    if (LAT::c(q, 1) == -1) jy -= f[q];
    if (D3 && LAT::c(q, 2) == 1) jz += f[q];
    if (D3 && LAT::c(q, 2) == -1) jz -= f[q];
  }
  const T drho = S::DEV ? s0 : T(0);                 // deviation of density
  const T rho = S::DEV ? T(v.rho0) + s0 : s0;        // density
  const T irho = T(1) / rho;
  const T ux = jx * irho, uy = jy * irho, uz = jz * irho;
  const T usq15 = T(1.5) * (ux * ux + uy * uy + uz * uz);
  const T om = T(v.omega);

  // ---- owners of this node (ascending particle id) ----
  int own[kMaxOwners];
  E eown[kMaxOwners];
  int no = 0;
  if (active) {
#pragma unroll
    for (int s = 0; s < kMaxOwners; s++) {
      if (s == no) {
        const int o = v.own[s][n];
        if (o >= 0) {
          own[s] = o;
          eown[s] = static_cast<const E*>(v.eps[s])[n];
          no = s + 1;
        }
      }
    }
  }
  const unsigned FULL = 0xffffffffu;
  const bool warp_has_solid = __any_sync(FULL, no > 0);

  T out[Q];
  if (!warp_has_solid) {
    // ---------------- plain LBGK ----------------
    {
      const T w0r = T(LAT::w(0)) * rho;
      const T feq0 = pair_A<S::DEV, T>(T(LAT::w(0)), w0r, drho, usq15, T(0));
      out[0] = f[0] - om * (f[0] - feq0);
    }
#pragma unroll
    for (int q = 1; q < Q; q += 2) {
      const int cx = LAT::c(q, 0), cy = LAT::c(q, 1), cz = LAT::c(q, 2);
      const T cu = cdot<T>(cx, cy, cz, ux, uy, uz);
      const T wr = T(LAT::w(q)) * rho;
      const T A = pair_A<S::DEV, T>(T(LAT::w(q)), wr, drho, usq15, cu);
      const T B = (T(3) * wr) * cu;
      const T fr = T(v.fq[q]) * rho;
      out[q] = f[q] - om * (f[q] - (A + B)) + fr;
      out[q + 1] = f[q + 1] - om * (f[q + 1] - (A - B)) - fr;
    }
  } else {
    // ---------------- NT immersed moving boundary ----------------
    // sort owners by id
#pragma unroll
    for (int a = 1; a < kMaxOwners; a++) {
      if (a < no) {
        int k = own[a];
        E ek = eown[a];
        int b = a - 1;
        while (b >= 0 && own[b] > k) {
          own[b + 1] = own[b];
          eown[b + 1] = eown[b];
          b--;
        }
        own[b + 1] = k;
        eown[b + 1] = ek;
      }
    }
    double esum = 0.0;
    double vs[3] = {0.0, 0.0, 0.0};
    double rk[kMaxOwners][3];
    for (int k = 0; k < no; k++) {
      const int p = own[k];
      const double r0 = min_image((double)xx - v.pos[3 * p], nx, true);
      const double r1 = min_image((double)y - v.pos[3 * p + 1], ny, !v.wall_y);
      const double r2 = D3 ? min_image((double)z - v.pos[3 * p + 2], nz, true) : 0.0;
      rk[k][0] = r0;
      rk[k][1] = r1;
      rk[k][2] = r2;
      const double* w = v.omg + 3 * p;
      const double* vp = v.vel + 3 * p;
      const double V0 = vp[0] + (w[1] * r2 - w[2] * r1);
      const double V1 = vp[1] + (w[2] * r0 - w[0] * r2);
      const double V2 = vp[2] + (w[0] * r1 - w[1] * r0);
      const double e = (double)eown[k];
      esum += e;
      vs[0] += e * V0;
      vs[1] += e * V1;
      vs[2] += e * V2;
    }
    T beta = T(0), VSx = T(0), VSy = T(0), VSz = T(0);
    if (no > 0 && esum > 0.0) {
      VSx = T(vs[0] / esum);
      VSy = T(vs[1] / esum);
      VSz = T(vs[2] / esum);
      const T eps = esum < 1.0 ? T(esum) : T(1);
      const T th = T(v.tau) - T(0.5);
      beta = eps * th / ((T(1) - eps) + th);  // Eq. (2)
    }
    const T omb = (T(1) - beta) * om;
    const T vsq15 = T(1.5) * (VSx * VSx + VSy * VSy + VSz * VSz);
    T mx = T(0), my = T(0), mz = T(0);
    {
      const T w0r = T(LAT::w(0)) * rho;
      const T feq0 = pair_A<S::DEV, T>(T(LAT::w(0)), w0r, drho, usq15, T(0));
      const T feqS0 = pair_A<S::DEV, T>(T(LAT::w(0)), w0r, drho, vsq15, T(0));
      const T Om0 = feqS0 - feq0;  // f_0 - f_0 cancels
      out[0] = f[0] - omb * (f[0] - feq0) + beta * Om0;
    }
#pragma unroll
    for (int q = 1; q < Q; q += 2) {
      const int cx = LAT::c(q, 0), cy = LAT::c(q, 1), cz = LAT::c(q, 2);
      const T wr = T(LAT::w(q)) * rho;
      const T cu = cdot<T>(cx, cy, cz, ux, uy, uz);
      const T A = pair_A<S::DEV, T>(T(LAT::w(q)), wr, drho, usq15, cu);
      const T B = (T(3) * wr) * cu;
      const T cv = cdot<T>(cx, cy, cz, VSx, VSy, VSz);
      const T AS = pair_A<S::DEV, T>(T(LAT::w(q)), wr, drho, vsq15, cv);
      const T BS = (T(3) * wr) * cv;
      // Omega^S_q = f_{-q} - f_q + feq_q(rho, V_S) - feq_{-q}(rho, u)
      const T Omp = f[q + 1] - f[q] + (AS + BS) - (A - B);
      const T Omm = f[q] - f[q + 1] + (AS - BS) - (A + B);
      const T fr = T(v.fq[q]) * rho;
      out[q] = f[q] - omb * (f[q] - (A + B)) + beta * Omp + fr;
      out[q + 1] = f[q + 1] - omb * (f[q + 1] - (A - B)) + beta * Omm - fr;
      const T dm = Omp - Omm;  // c_{q+1} = -c_q
      if (cx) mx += T(cx) * dm;
      if (cy) my += T(cy) * dm;
      if (cz) mz += T(cz) * dm;
    }
    // momentum given to the fluid m = beta sum_i Omega_i^S c_i; the force on
    // the particles is -m, split by covered fraction (Eq. 3 and reading)
    const double m0 = (double)(beta * mx), m1 = (double)(beta * my), m2 = (double)(beta * mz);
    double val[6] = {0, 0, 0, 0, 0, 0};
    int key = -1;
    for (int k = 0; k < no; k++) {
      const double a = (double)eown[k] / esum;
      const double p0 = a * m0, p1 = a * m1, p2 = a * m2;
      const double F0 = -p0, F1 = -p1, F2 = -p2;
      const double T0 = -(rk[k][1] * p2 - rk[k][2] * p1);
      const double T1 = -(rk[k][2] * p0 - rk[k][0] * p2);
      const double T2 = -(rk[k][0] * p1 - rk[k][1] * p0);
      if (k == 0) {
        key = own[0];
        val[0] = F0; val[1] = F1; val[2] = F2;
        val[3] = T0; val[4] = T1; val[5] = T2;
      } else {
        const int p = own[k];
        atomicAdd(v.ff + 3 * p, F0);
        atomicAdd(v.ff + 3 * p + 1, F1);
        if (D3) atomicAdd(v.ff + 3 * p + 2, F2);
        if (D3) {
          atomicAdd(v.tf + 3 * p, T0);
          atomicAdd(v.tf + 3 * p + 1, T1);
        }
        atomicAdd(v.tf + 3 * p + 2, T2);
      }
    }
    if (!(esum > 0.0)) key = -1;
    warp_reduce_to_particles(key, val, v.ff, v.tf);
  }

  if (active) {
#pragma unroll
    for (int q = 0; q < Q; q++) S::store(v.fdst, q * plane + n, out[q], LAT::w(q));
  }
}

template <class LAT, int STORE>
static void launch_one(const View& v, cudaStream_t s) {
  dim3 grid((v.nx + 127) / 128, v.ny, v.nz);
  collide_kernel<LAT, STORE><<<grid, 128, 0, s>>>(v);
}

void launch_collide(const View& v, cudaStream_t s) {
  if (v.dim == 2) {
    if (v.storage == LBM_IMB_STORE_F64) launch_one<D2Q9, LBM_IMB_STORE_F64>(v, s);
    else if (v.storage == LBM_IMB_STORE_F32DEV) launch_one<D2Q9, LBM_IMB_STORE_F32DEV>(v, s);
    else launch_one<D2Q9, LBM_IMB_STORE_F16DEV>(v, s);
  } else {
    if (v.storage == LBM_IMB_STORE_F64) launch_one<D3Q19, LBM_IMB_STORE_F64>(v, s);
    else if (v.storage == LBM_IMB_STORE_F32DEV) launch_one<D3Q19, LBM_IMB_STORE_F32DEV>(v, s);
    else launch_one<D3Q19, LBM_IMB_STORE_F16DEV>(v, s);
  }
}

}  // namespace lbm
