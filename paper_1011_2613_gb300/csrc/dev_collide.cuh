// K2 device code: fused pull-stream + LBGK collision with the
// Noble-Torczynski immersed moving boundary term, shared by the per-step
// kernel (k_collide.cu) and the batched persistent kernel (k_batch.cu).
#pragma once
#include "lbm_internal.cuh"

namespace lbm {

template <int STORE>
struct Storage;
template <>
struct Storage<LBM_IMB_STORE_F64> {
  using Elem = double;
  using T = double;
  using E = double;  // eps slot element
  static constexpr bool DEV = false;
  __device__ static __forceinline__ T load(const Elem* p, int i, double) { return __ldg(p + i); }
  __device__ static __forceinline__ T load_shared(const Elem* p, int i, double) { return p[i]; }
  __device__ static __forceinline__ void store(Elem* p, int i, T v, double) { p[i] = v; }
};
template <>
struct Storage<LBM_IMB_STORE_F32DEV> {
  using Elem = float;
  using T = float;
  using E = float;
  static constexpr bool DEV = true;
  __device__ static __forceinline__ T load(const Elem* p, int i, double) { return __ldg(p + i); }
  __device__ static __forceinline__ T load_shared(const Elem* p, int i, double) { return p[i]; }
  __device__ static __forceinline__ void store(Elem* p, int i, T v, double) { p[i] = v; }
};
template <>
struct Storage<LBM_IMB_STORE_F16DEV> {
  using Elem = __half;
  using T = float;
  using E = float;
  static constexpr bool DEV = true;
  // stored value = g / w (keeps the diagonal deviations out of subnormals)
  __device__ static __forceinline__ T load(const Elem* p, int i, double w) {
    return __half2float(__ldg(p + i)) * float(w);
  }
  __device__ static __forceinline__ T load_shared(const Elem* p, int i, double w) {
    return __half2float(p[i]) * float(w);
  }
  __device__ static __forceinline__ void store(Elem* p, int i, T v, double w) {
    p[i] = __float2half_rn(v * float(1.0 / w));
  }
};

// Sum the per-node force/torque contributions of a warp by particle (key)
// and add them to the FP64 per-particle accumulators.
template <typename PT>
__device__ __forceinline__ void warp_reduce_to_particles(int key, PT (&val)[6], double* ff, double* tf) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned owned = __ballot_sync(FULL, key >= 0);
  if (owned == 0u) return;
  const int k0 = __shfl_sync(FULL, key, __ffs(owned) - 1);
  if (__all_sync(FULL, key < 0 || key == k0)) {
    // one particle covers all owned lanes: butterfly sum, one lane commits
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
#pragma unroll
      for (int k = 0; k < 6; k++) val[k] += __shfl_xor_sync(FULL, val[k], d);
    }
    if (lane < 6) {
      PT x = val[0];
#pragma unroll
      for (int k = 1; k < 6; k++) x = lane == k ? val[k] : x;
      if (x != PT(0)) atomicAdd((lane < 3 ? ff + 3 * k0 + lane : tf + 3 * k0 + lane - 3), (double)x);
    }
    return;
  }
  // several particles: segmented suffix sums over runs of equal keys; the
  // first lane of each run commits its run
  const int next = __shfl_down_sync(FULL, key, 1);
  const int prev = __shfl_up_sync(FULL, key, 1);
  const unsigned tails = __ballot_sync(FULL, lane == 31 || next != key);
  const int run_end = __ffs(tails & (FULL << lane)) - 1;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
    for (int k = 0; k < 6; k++) {
      const PT t = __shfl_down_sync(FULL, val[k], d);
      if (lane + d <= run_end) val[k] += t;
    }
  }
  const bool head = lane == 0 || prev != key;
  if (head && key >= 0) {
#pragma unroll
    for (int k = 0; k < 3; k++) {
      if (val[k] != PT(0)) atomicAdd(ff + 3 * key + k, (double)val[k]);
      if (val[3 + k] != PT(0)) atomicAdd(tf + 3 * key + k, (double)val[3 + k]);
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

template <bool DEV, typename T>
__device__ __forceinline__ T fq_of(const View& v, int q) {
  if constexpr (DEV) return v.fq_f[q];
  else return v.fq[q];
}

__device__ __forceinline__ float min_image_f(float d, int n, bool periodic) {
  if (!periodic) return d;
  const float L = (float)n;
  if (d > 0.5f * L) d -= L;
  else if (d < -0.5f * L) d += L;
  return d;
}

__device__ __forceinline__ double min_image(double d, int n, bool periodic) {
  if (!periodic) return d;
  const double L = (double)n;
  if (d > 0.5 * L) d -= L;
  else if (d < -0.5 * L) d += L;
  return d;
}

// One node per thread of the fused pull-stream + collision; the whole CTA
// (128 threads, 4 full warps) calls it together.  Lanes outside the lattice
// pass active = false with in-range coordinates.  Node offsets within a
// population plane are 32-bit (the library rejects planes of 2^31 nodes or
// more).
//
// Every thread computes the plain BGK update and stores it unless its node
// is covered.  Covered nodes are then packed into the first lanes of the CTA
// through shared memory (f - f^eq, rho, u per node), so the immersed-boundary
// work runs on full warps; it adds the correction
//   f*_i - f*_i(plain) = beta (omega (f_i - f^eq_i) + Omega^S_i),
//   Omega^S_i = (f - f^eq)_{-i} - (f - f^eq)_i + f^eq_i(rho, V_S) - f^eq_i(rho, u)
// (Eq. 1 with the Omega^S term rearranged) and the Eq. 3 force/torque.
// The collision of one node from its pulled populations f (see collide_node).
template <class LAT, int STORE>
__device__ __forceinline__ void collide_core(const View& v, const int xx, const int y, const int z,
                                             const bool active, const int n,
                                             typename Storage<STORE>::T (&f)[LAT::Q]) {
  using S = Storage<STORE>;
  using T = typename S::T;
  using E = typename S::E;
  using Elem = typename S::Elem;
  constexpr int Q = LAT::Q;
  constexpr int NP = (Q - 1) / 2;  // opposite pairs
  constexpr bool D3 = LAT::DIM == 3;
  constexpr int NS = Q + 5;        // packed state: f - f^eq, rho, drho, u
  const int nx = v.nx, ny = v.ny, nz = v.nz;
  (void)nx;
  (void)ny;
  (void)nz;
  T rho0p, om, tau_t;
  if constexpr (S::DEV) {
    rho0p = v.rho0_f;
    om = v.omega_f;
    tau_t = v.tau_f;
  } else {
    rho0p = T(0);
    om = v.omega;
    tau_t = v.tau;
  }
  // ---- owners of this node (slot s+1 is read only where slot s is taken) ----
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

  // ---- moments ----
  T s0 = f[0], jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
  for (int q = 1; q < Q; q++) {
    s0 += f[q];
    if (LAT::c(q, 0) == 1) jx += f[q];
    if (LAT::c(q, 0) == -1) jx -= f[q];
    if (LAT::c(q, 1) == 1) jy += f[q];
    if (LAT::c(q, 1) == -1) jy -= f[q];
    if (D3 && LAT::c(q, 2) == 1) jz += f[q];
    if (D3 && LAT::c(q, 2) == -1) jz -= f[q];
  }
  const T drho = S::DEV ? s0 : T(0);        // deviation of density
  const T rho = S::DEV ? rho0p + s0 : s0;   // density
  const T irho = T(1) / rho;
  const T ux = jx * irho, uy = jy * irho, uz = jz * irho;
  const T usq15 = T(1.5) * (ux * ux + uy * uy + uz * uz);

  // ---- plain BGK; f becomes f - f^eq ----
  T out[Q];
  {
    const T a = pair_A<S::DEV, T>(T(LAT::w(0)), T(LAT::w(0)) * rho, drho, usq15, T(0));
    f[0] -= a;
    out[0] = (f[0] + a) - om * f[0];
  }
#pragma unroll
  for (int k = 0; k < NP; k++) {
    const int q = 2 * k + 1;
    const int cx = LAT::c(q, 0), cy = LAT::c(q, 1), cz = LAT::c(q, 2);
    const T cu = cdot<T>(cx, cy, cz, ux, uy, uz);
    const T wr = T(LAT::w(q)) * rho;
    const T a = pair_A<S::DEV, T>(T(LAT::w(q)), wr, drho, usq15, cu);
    const T b = (T(3) * wr) * cu;
    const T fr = fq_of<S::DEV, T>(v, q) * rho;
    const T fp = f[q], fm = f[q + 1];
    f[q] = fp - (a + b);
    f[q + 1] = fm - (a - b);
    out[q] = fp - om * f[q] + fr;
    out[q + 1] = fm - om * f[q + 1] - fr;
  }
  if (active && no == 0) {
#pragma unroll
    for (int q = 0; q < Q; q++) S::store(static_cast<Elem*>(v.dst_q[q]), n, out[q], LAT::w(q));
  }

  // ---- pack the covered nodes of the CTA ----
  __shared__ T s_st[NS][128];
  __shared__ int s_n[128], s_xyz[128], s_no[128], s_own[kMaxOwners][128];
  __shared__ E s_e[kMaxOwners][128];
  __shared__ int s_cnt[4];
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned covered = __ballot_sync(FULL, no > 0);
  __syncthreads();  // the previous call's packed state has been consumed
  if (lane == 0) s_cnt[warp] = __popc(covered);
  __syncthreads();
  int base = 0, total = 0;
#pragma unroll
  for (int w = 0; w < 4; w++) {
    base += w < warp ? s_cnt[w] : 0;
    total += s_cnt[w];
  }
  if (no > 0) {
    const int slot = base + __popc(covered & ((1u << lane) - 1u));
#pragma unroll
    for (int q = 0; q < Q; q++) s_st[q][slot] = f[q];
    s_st[Q][slot] = rho;
    s_st[Q + 1][slot] = drho;
    s_st[Q + 2][slot] = ux;
    s_st[Q + 3][slot] = uy;
    s_st[Q + 4][slot] = uz;
    s_n[slot] = n;
    s_xyz[slot] = xx | (y << 16);  // x, y < 65536
    s_no[slot] = no | (z << 8);
#pragma unroll
    for (int s = 0; s < kMaxOwners; s++) {
      s_own[s][slot] = s < no ? own[s] : -1;
      s_e[s][slot] = s < no ? eown[s] : E(0);
    }
  }
  __syncthreads();
  if (threadIdx.x >= ((total + 31) & ~31)) return;  // whole warps beyond the packed nodes

  // ---------------- NT immersed moving boundary on packed nodes ----------------
  const int slot = threadIdx.x;
  const bool mine = slot < total;
  const int ps = mine ? slot : 0;
  const int cn = s_n[ps];
  const int cx_ = s_xyz[ps] & 0xffff, cy_ = s_xyz[ps] >> 16, cz_ = s_no[ps] >> 8;
  no = mine ? (s_no[ps] & 0xff) : 0;
#pragma unroll
  for (int s = 0; s < kMaxOwners; s++) {
    own[s] = s_own[s][ps];
    eown[s] = s_e[s][ps];
  }
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
  T g[Q];
#pragma unroll
  for (int q = 0; q < Q; q++) g[q] = s_st[q][ps];
  const T crho = s_st[Q][ps], cdrho = s_st[Q + 1][ps];
  const T cux = s_st[Q + 2][ps], cuy = s_st[Q + 3][ps], cuz = s_st[Q + 4][ps];
  const T cusq15 = T(1.5) * (cux * cux + cuy * cuy + cuz * cuz);
  {
    // solid velocity at the node; particle arithmetic in FP64 for FP64
    // storage, in FP32 (from the per-particle FP32 kinematics record)
    // otherwise
    using PT = typename S::T;
    PT esum = PT(0), vs0 = PT(0), vs1 = PT(0), vs2 = PT(0);
    PT rk[kMaxOwners][3];
    PT V1x = PT(0), V1y = PT(0), V1z = PT(0);
    for (int k = 0; k < no; k++) {
      const int p = own[k];
      PT r0, r1, r2, V0, Vy, V2;
      if constexpr (S::DEV) {
        const float4* kp = reinterpret_cast<const float4*>(v.kin) + 4 * p;
        const float4 fr = __ldg(kp);
        const int4 ir = __ldg(reinterpret_cast<const int4*>(kp) + 1);
        const float4 vp = __ldg(kp + 2);
        const float4 wp = __ldg(kp + 3);
        r0 = min_image_f(float(cx_ - ir.x) - fr.x, nx, true);
        r1 = min_image_f(float(cy_ - ir.y) - fr.y, ny, !v.wall_y);
        r2 = D3 ? min_image_f(float(cz_ - ir.z) - fr.z, nz, true) : 0.f;
        V0 = vp.x + (wp.y * r2 - wp.z * r1);
        Vy = vp.y + (wp.z * r0 - wp.x * r2);
        V2 = vp.z + (wp.x * r1 - wp.y * r0);
      } else {
        r0 = min_image((double)cx_ - v.pos[3 * p], nx, true);
        r1 = min_image((double)cy_ - v.pos[3 * p + 1], ny, !v.wall_y);
        r2 = D3 ? min_image((double)cz_ - v.pos[3 * p + 2], nz, true) : 0.0;
        const double* w = v.omg + 3 * p;
        const double* vp = v.vel + 3 * p;
        V0 = vp[0] + (w[1] * r2 - w[2] * r1);
        Vy = vp[1] + (w[2] * r0 - w[0] * r2);
        V2 = vp[2] + (w[0] * r1 - w[1] * r0);
      }
      rk[k][0] = r0;
      rk[k][1] = r1;
      rk[k][2] = r2;
      const PT e = (PT)eown[k];
      if (k == 0) {
        V1x = V0;
        V1y = Vy;
        V1z = V2;
      }
      esum += e;
      vs0 += e * V0;
      vs1 += e * Vy;
      vs2 += e * V2;
    }
    T beta = T(0), VSx = T(0), VSy = T(0), VSz = T(0);
    PT inv_esum = PT(1);
    if (no == 1) {
      VSx = T(V1x);  // one owner: V_S is its velocity, the split factor 1
      VSy = T(V1y);
      VSz = T(V1z);
    } else if (no > 1) {
      inv_esum = PT(1) / esum;
      VSx = T(vs0 * inv_esum);
      VSy = T(vs1 * inv_esum);
      VSz = T(vs2 * inv_esum);
    }
    if (no > 0 && esum > PT(0)) {
      const T eps = esum < PT(1) ? T(esum) : T(1);
      const T th = tau_t - T(0.5);
      beta = eps * th / ((T(1) - eps) + th);  // Eq. (2)
    }
    const T vsq15 = T(1.5) * (VSx * VSx + VSy * VSy + VSz * VSz);
    T mx = T(0), my = T(0), mz = T(0);
    T res[Q];
    {
      const T w0r = T(LAT::w(0)) * crho;
      const T a = pair_A<S::DEV, T>(T(LAT::w(0)), w0r, cdrho, cusq15, T(0));
      const T AS0 = pair_A<S::DEV, T>(T(LAT::w(0)), w0r, cdrho, vsq15, T(0));
      const T Om0 = AS0 - a;  // f_0 - f_0 cancels
      res[0] = (g[0] + a) - om * g[0] + beta * (om * g[0] + Om0);
    }
#pragma unroll
    for (int k = 0; k < NP; k++) {
      const int q = 2 * k + 1;
      const int cx = LAT::c(q, 0), cy = LAT::c(q, 1), cz = LAT::c(q, 2);
      const T wr = T(LAT::w(q)) * crho;
      const T cu = cdot<T>(cx, cy, cz, cux, cuy, cuz);
      const T a = pair_A<S::DEV, T>(T(LAT::w(q)), wr, cdrho, cusq15, cu);
      const T b = (T(3) * wr) * cu;
      const T cv = cdot<T>(cx, cy, cz, VSx, VSy, VSz);
      const T AS = pair_A<S::DEV, T>(T(LAT::w(q)), wr, cdrho, vsq15, cv);
      const T BS = (T(3) * wr) * cv;
      const T fr = fq_of<S::DEV, T>(v, q) * crho;
      // Omega^S_q = f_{-q} - f_q + feq_q(rho, V_S) - feq_{-q}(rho, u)
      const T dA = AS - a;
      const T Omp = (g[q + 1] - g[q]) + (dA + (BS - b));
      const T Omm = (g[q] - g[q + 1]) + (dA - (BS - b));
      res[q] = (g[q] + (a + b)) - om * g[q] + fr + beta * (om * g[q] + Omp);
      res[q + 1] = (g[q + 1] + (a - b)) - om * g[q + 1] - fr + beta * (om * g[q + 1] + Omm);
      const T dm = Omp - Omm;  // c_{q+1} = -c_q
      if (cx) mx += T(cx) * dm;
      if (cy) my += T(cy) * dm;
      if (cz) mz += T(cz) * dm;
    }
    if (mine) {
#pragma unroll
      for (int q = 0; q < Q; q++) S::store(static_cast<Elem*>(v.dst_q[q]), cn, res[q], LAT::w(q));
    }
    // momentum given to the fluid m = beta sum_i Omega_i^S c_i; the force on
    // the particles is -m, split by covered fraction (Eq. 3 and reading)
    const PT m0 = PT(beta * mx), m1 = PT(beta * my), m2 = PT(beta * mz);
    PT val[6] = {PT(0), PT(0), PT(0), PT(0), PT(0), PT(0)};
    int key = -1;
    for (int k = 0; k < no; k++) {
      const PT a = no == 1 ? PT(1) : PT(eown[k]) * inv_esum;
      const PT p0 = a * m0, p1 = a * m1, p2 = a * m2;
      const PT F0 = -p0, F1 = -p1, F2 = -p2;
      const PT T0 = -(rk[k][1] * p2 - rk[k][2] * p1);
      const PT T1 = -(rk[k][2] * p0 - rk[k][0] * p2);
      const PT T2 = -(rk[k][0] * p1 - rk[k][1] * p0);
      if (k == 0) {
        key = own[0];
        val[0] = F0; val[1] = F1; val[2] = F2;
        val[3] = T0; val[4] = T1; val[5] = T2;
      } else {
        const int p = own[k];
        atomicAdd(v.ff + 3 * p, (double)F0);
        atomicAdd(v.ff + 3 * p + 1, (double)F1);
        if (D3) atomicAdd(v.ff + 3 * p + 2, (double)F2);
        if (D3) {
          atomicAdd(v.tf + 3 * p, (double)T0);
          atomicAdd(v.tf + 3 * p + 1, (double)T1);
        }
        atomicAdd(v.tf + 3 * p + 2, (double)T2);
      }
    }
    if (!(esum > PT(0))) key = -1;
    warp_reduce_to_particles<PT>(key, val, v.ff, v.tf);
}

}

template <class LAT, int STORE>
__device__ __forceinline__ void collide_node(const View& v, const int xx, const int y, const int z,
                                             const bool active) {
  using S = Storage<STORE>;
  using T = typename S::T;
  using Elem = typename S::Elem;
  constexpr int Q = LAT::Q;
  const int nx = v.nx, ny = v.ny, nz = v.nz, pitch = v.pitch;
  const int xm = xx == 0 ? nx - 1 : xx - 1, xp = xx == nx - 1 ? 0 : xx + 1;
  const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
  const int n = (z * ny + y) * pitch + xx;
  // ---- pull streaming; rows are whole warps, so the wall test is uniform ----
  const int ry[3] = {y * pitch, ym * pitch, yp * pitch};
  const int rz[3] = {z * ny * pitch, zm * ny * pitch, zp * ny * pitch};
  T f[Q];
  const bool wall_row = v.wall_y && (y == 0 || y == ny - 1);
  if (!wall_row) {
#pragma unroll
    for (int q = 0; q < Q; q++) {
      const int cx = LAT::c(q, 0), cy = LAT::c(q, 1), cz = LAT::c(q, 2);
      const int sx = cx == 1 ? xm : (cx == -1 ? xp : xx);
      const int idx = rz[cz == 0 ? 0 : (cz == 1 ? 1 : 2)] + ry[cy == 0 ? 0 : (cy == 1 ? 1 : 2)] + sx;
      f[q] = S::load(static_cast<const Elem*>(v.src_q[q]), idx, LAT::w(q));
    }
  } else {
#pragma unroll
    for (int q = 0; q < Q; q++) {
      const int cx = LAT::c(q, 0), cy = LAT::c(q, 1), cz = LAT::c(q, 2);
      const int sx = cx == 1 ? xm : (cx == -1 ? xp : xx);
      const int idx = rz[cz == 0 ? 0 : (cz == 1 ? 1 : 2)] + ry[cy == 0 ? 0 : (cy == 1 ? 1 : 2)] + sx;
      const bool bounce = (cy == 1 && y == 0) || (cy == -1 && y == ny - 1);
      if (bounce)  // halfway bounce-back: the opposite population of this node
        f[q] = S::load(static_cast<const Elem*>(v.src_q[opp(q)]), n, LAT::w(opp(q)));
      else
        f[q] = S::load(static_cast<const Elem*>(v.src_q[q]), idx, LAT::w(q));
    }
  }

  collide_core<LAT, STORE>(v, xx, y, z, active, n, f);
}

}  // namespace lbm
