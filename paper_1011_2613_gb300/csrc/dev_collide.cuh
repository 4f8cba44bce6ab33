// K2 device code: fused pull-stream + LBGK collision with the
// Noble-Torczynski immersed moving boundary term, shared by the per-step
// kernel (k_collide.cu) and the batched persistent kernel (k_batch.cu).
#pragma once
#include <type_traits>

#include "dev_df.cuh"
#include "lbm_internal.cuh"

namespace lbm {

template <int STORE>
struct Storage;
// load/store move the stored form; SCALED storages hold g_q / w_q (the
// collision then works on h_q = g_q / w_q and never multiplies by w_q except
// in the density and momentum sums)
template <>
struct Storage<LBM_IMB_STORE_F64> {
  using Elem = double;
  using T = double;
  using E = double;  // eps slot element
  static constexpr bool DEV = false;
  static constexpr bool SCALED = false;
  __device__ static __forceinline__ T load(const Elem* p, int i) { return __ldg(p + i); }
  __device__ static __forceinline__ T load_shared(const Elem* p, int i) { return p[i]; }
  __device__ static __forceinline__ void store(Elem* p, int i, T v) { p[i] = v; }
  __device__ static __forceinline__ void store2(Elem* p, Elem* r, int i, T a, T b) {
    p[i] = a;
    r[i] = b;
  }
};
template <>
struct Storage<LBM_IMB_STORE_F32DEV> {
  using Elem = float;
  using T = float;
  using E = float;
  static constexpr bool DEV = true;
  static constexpr bool SCALED = false;
  __device__ static __forceinline__ T load(const Elem* p, int i) { return __ldg(p + i); }
  __device__ static __forceinline__ T load_shared(const Elem* p, int i) { return p[i]; }
  __device__ static __forceinline__ void store(Elem* p, int i, T v) { p[i] = v; }
  __device__ static __forceinline__ void store2(Elem* p, Elem* r, int i, T a, T b) {
    p[i] = a;
    r[i] = b;
  }
};
template <>
struct Storage<LBM_IMB_STORE_F16DEV> {
  using Elem = __half;
  using T = float;
  using E = float;
  static constexpr bool DEV = true;
  // stored value h = g / w (keeps the diagonal deviations out of subnormals)
  static constexpr bool SCALED = true;
  __device__ static __forceinline__ T load(const Elem* p, int i) { return __half2float(__ldg(p + i)); }
  __device__ static __forceinline__ T load_shared(const Elem* p, int i) { return __half2float(p[i]); }
  __device__ static __forceinline__ void store(Elem* p, int i, T v) { p[i] = __float2half_rn(v); }
  // two values converted by one paired instruction
  __device__ static __forceinline__ void store2(Elem* p, Elem* r, int i, T a, T b) {
    const __half2 h = __floats2half2_rn(a, b);
    p[i] = __low2half(h);
    r[i] = __high2half(h);
  }
};

// deviation g = f - w rho0 stored as an unevaluated FP32 pair (h, l) and
// collided in pair arithmetic (dev_df.cuh): FP64 accuracy on f with the
// arithmetic on the FP32 pipe; a store renormalises the pair
template <>
struct Storage<LBM_IMB_STORE_DFDEV> {
  using Elem = float2;
  using T = DF;
  using E = double;
  static constexpr bool DEV = true;
  static constexpr bool SCALED = false;
  __device__ static __forceinline__ T load(const Elem* p, int i) {
    const float2 w = __ldg(p + i);
    return DF(w.x, w.y);
  }
  __device__ static __forceinline__ T load_shared(const Elem* p, int i) { return DF(p[i].x, p[i].y); }
  __device__ static __forceinline__ void store(Elem* p, int i, T v) {
    const DF r = df_norm(v);
    p[i] = make_float2(r.h, r.l);
  }
  __device__ static __forceinline__ void store2(Elem* p, Elem* r, int i, T a, T b) {
    store(p, i, a);
    store(r, i, b);
  }
};

// FP64 arithmetic on the deviation of the pair storage: the covered-node
// update runs on the FP64 pipe while the plain updates of other warps use
// the FP32 pipe (internal id, not a storage of the C ABI); pairs <-> FP64 by
// integer bit operations
constexpr int kDfDevImb = 16;
template <>
struct Storage<kDfDevImb> {
  using Elem = float2;
  using T = double;
  using E = double;
  static constexpr bool DEV = true;
  static constexpr bool SCALED = false;
  __device__ static __forceinline__ T load(const Elem* p, int i) {
    const float2 w = __ldg(p + i);
    return df_to_bits(DF(w.x, w.y));
  }
  __device__ static __forceinline__ T load_shared(const Elem* p, int i) { return df_to_bits(DF(p[i].x, p[i].y)); }
  __device__ static __forceinline__ void store(Elem* p, int i, T v) {
    const DF r = df_from_bits(v);
    p[i] = make_float2(r.h, r.l);
  }
  __device__ static __forceinline__ void store2(Elem* p, Elem* r, int i, T a, T b) {
    store(p, i, a);
    store(r, i, b);
  }
};

// the pair storage's plain update of two adjacent nodes at once in paired
// FP32 instructions (DF2; internal id, not a storage of the C ABI): the
// arithmetic type only; the two-node kernel does its own loads and stores
constexpr int kDfDevPair = 17;
template <>
struct Storage<kDfDevPair> {
  using Elem = float2;
  using T = DF2;
  using E = double;
  static constexpr bool DEV = true;
  static constexpr bool SCALED = false;
};

// a per-simulation constant in the arithmetic type of the storage
template <int STORE>
__device__ __forceinline__ typename Storage<STORE>::T pick(const double d, const float f, const float (&p)[2]) {
  if constexpr (STORE == LBM_IMB_STORE_F64 || STORE == kDfDevImb) return d;
  else if constexpr (STORE == LBM_IMB_STORE_DFDEV) return DF(p[0], p[1]);
  else if constexpr (STORE == kDfDevPair) return DF2(DF(p[0], p[1]));
  else return f;
}

// warp shuffles and the FP64 value of each arithmetic type
__device__ __forceinline__ float shfl_xor(const float a, const int d) { return __shfl_xor_sync(0xffffffffu, a, d); }
__device__ __forceinline__ double shfl_xor(const double a, const int d) { return __shfl_xor_sync(0xffffffffu, a, d); }
__device__ __forceinline__ float shfl_down(const float a, const int d) { return __shfl_down_sync(0xffffffffu, a, d); }
__device__ __forceinline__ double shfl_down(const double a, const int d) {
  return __shfl_down_sync(0xffffffffu, a, d);
}
__device__ __forceinline__ double to_double(const float a) { return (double)a; }
__device__ __forceinline__ double to_double(const double a) { return a; }
__device__ __forceinline__ double to_double(const DF a) { return df_to_bits(a); }
// a stored covered fraction in the particle-side arithmetic type
template <typename PT, typename E>
__device__ __forceinline__ PT to_pt(const E a) {
  return (PT)a;
}
template <>
__device__ __forceinline__ DF to_pt<DF, double>(const double a) {
  return df_from_bits(a);
}

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
      for (int k = 0; k < 6; k++) val[k] += shfl_xor(val[k], d);
    }
    if (lane < 6) {
      PT x = val[0];
#pragma unroll
      for (int k = 1; k < 6; k++) x = lane == k ? val[k] : x;
      if (x != PT(0)) atomicAdd((lane < 3 ? ff + 3 * k0 + lane : tf + 3 * k0 + lane - 3), to_double(x));
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
      const PT t = shfl_down(val[k], d);
      if (lane + d <= run_end) val[k] += t;
    }
  }
  const bool head = lane == 0 || prev != key;
  if (head && key >= 0) {
#pragma unroll
    for (int k = 0; k < 3; k++) {
      if (val[k] != PT(0)) atomicAdd(ff + 3 * key + k, to_double(val[k]));
      if (val[3 + k] != PT(0)) atomicAdd(tf + 3 * key + k, to_double(val[3 + k]));
    }
  }
}

// Two FP32 values processed together by the paired instructions of this
// GPU (FADD2 / FMUL2 / FFMA2): the arithmetic type of the two-node forms.
struct F2 {
  float2 v;
  __device__ __forceinline__ F2() {}
  __device__ __forceinline__ F2(float s) : v(make_float2(s, s)) {}
  __device__ __forceinline__ F2(double s) : v(make_float2((float)s, (float)s)) {}
  __device__ __forceinline__ F2(int s) : v(make_float2((float)s, (float)s)) {}
  __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
  // found by argument-dependent lookup only (does not hide ::fma)
  friend __device__ __forceinline__ F2 fma(const F2 a, const F2 b, const F2 c) {
    F2 r;
    r.v = __ffma2_rn(a.v, b.v, c.v);
    return r;
  }
};
__device__ __forceinline__ F2 operator+(const F2 a, const F2 b) {
  F2 r;
  r.v = __fadd2_rn(a.v, b.v);
  return r;
}
__device__ __forceinline__ F2 operator*(const F2 a, const F2 b) {
  F2 r;
  r.v = __fmul2_rn(a.v, b.v);
  return r;
}
__device__ __forceinline__ F2 operator-(const F2 a) { return a * F2(-1.f); }  // exact
__device__ __forceinline__ F2 operator-(const F2 a, const F2 b) { return fma(b, F2(-1.f), a); }  // one rounding

__device__ __forceinline__ float rcp(const float x) { return __frcp_rn(x); }
// 1 / x (x > 0, normal): the hardware's approximate reciprocal refined by
// two Newton-Raphson steps r <- r + r (1 - x r), within an ulp or two of the
// rounded quotient at four FP64 operations
__device__ __forceinline__ double rcp(const double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  r = fma(r, fma(-x, r, 1.0), r);
  return fma(r, fma(-x, r, 1.0), r);
}
__device__ __forceinline__ F2 rcp(const F2 x) { return F2(__frcp_rn(x.v.x), __frcp_rn(x.v.y)); }

// a / b: FP64 through the Newton reciprocal above, other types as written
template <typename T>
__device__ __forceinline__ T quot(const T a, const T b) {
  if constexpr (std::is_same<T, double>::value) return a * rcp(b);
  else return a / b;
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

template <int STORE>
__device__ __forceinline__ typename Storage<STORE>::T fq_of(const View& v, int q) {
  return pick<STORE>(v.fq[q], v.fq_f[q], v.fq_df[q]);
}

template <int STORE>
__device__ __forceinline__ typename Storage<STORE>::T cg3_of(const View& v, int q) {
  return pick<STORE>(v.cg3[q], v.cg3_f[q], v.cg3_df[q]);
}

// j_a += c_a (w) m for one opposite pair; the first non-zero term assigns
// (after unrolling, `have` and the branches fold)
template <bool SCALED, typename T>
__device__ __forceinline__ void axis_acc(T& j, bool& have, int c, T wq, T m) {
  if (c == 0) return;
  if (SCALED) {
    const T cw = c > 0 ? wq : -wq;
    j = have ? fma(cw, m, j) : cw * m;
  } else {
    j = have ? (c > 0 ? j + m : j - m) : (c > 0 ? m : -m);
  }
  have = true;
}

__device__ __forceinline__ float min_image_f(float d, int n, bool periodic) {
  if (!periodic) return d;
  const float L = (float)n;
  if (d > 0.5f * L) d -= L;
  else if (d < -0.5f * L) d += L;
  return d;
}

__device__ __forceinline__ DF min_image_df(DF d, int n, bool periodic) {
  if (!periodic) return d;
  const float L = (float)n;
  if (d.h > 0.5f * L) d = d - DF(L);
  else if (d.h < -0.5f * L) d = d + DF(L);
  return d;
}

__device__ __forceinline__ double min_image(double d, int n, bool periodic) {
  if (!periodic) return d;
  const double L = (double)n;
  if (d > 0.5 * L) d -= L;
  else if (d < -0.5 * L) d += L;
  return d;
}

// ---------------------------------------------------------------------------
// Pull streaming of one node: f_q(x) = f_q(x - c_q) of the source lattice,
// or the halfway bounce-back f_q(x) = f_{-q}(x) where x - c_q lies beyond a
// wall in y.  Node offsets within a population plane are 32-bit (the library
// rejects planes of 2^31 nodes or more).  Lanes with load = false read
// nothing (their f is zero).
// ---------------------------------------------------------------------------
template <class LAT, int STORE>
__device__ __forceinline__ void pull(const View& v, const int xx, const int y, const int z, const int n,
                                     const bool load, typename Storage<STORE>::T (&f)[LAT::Q]) {
  using S = Storage<STORE>;
  using T = typename S::T;
  using Elem = typename S::Elem;
  constexpr int Q = LAT::Q;
  const int nx = v.nx, ny = v.ny, nz = v.nz, pitch = v.pitch;
  const int xm = xx == 0 ? nx - 1 : xx - 1, xp = xx == nx - 1 ? 0 : xx + 1;
  const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
  const int ry[3] = {y * pitch, ym * pitch, yp * pitch};
  const int rz[3] = {z * ny * pitch, zm * ny * pitch, zp * ny * pitch};
  const bool wlo = v.wall_lo && y == v.y0, whi = v.wall_hi && y == v.y0 + v.ny_c - 1;
  if (!(wlo || whi)) {  // rows are whole warps: the test is warp-uniform in the row kernel
#pragma unroll
    for (int q = 0; q < Q; q++) {
      const int cx = LAT::c(q, 0), cy = LAT::c(q, 1), cz = LAT::c(q, 2);
      const int sx = cx == 1 ? xm : (cx == -1 ? xp : xx);
      const int idx = rz[cz == 0 ? 0 : (cz == 1 ? 1 : 2)] + ry[cy == 0 ? 0 : (cy == 1 ? 1 : 2)] + sx;
      f[q] = load ? S::load(static_cast<const Elem*>(v.src_q[q]), idx) : T(0);
    }
  } else {
#pragma unroll
    for (int q = 0; q < Q; q++) {
      const int cx = LAT::c(q, 0), cy = LAT::c(q, 1), cz = LAT::c(q, 2);
      const int sx = cx == 1 ? xm : (cx == -1 ? xp : xx);
      const int idx = rz[cz == 0 ? 0 : (cz == 1 ? 1 : 2)] + ry[cy == 0 ? 0 : (cy == 1 ? 1 : 2)] + sx;
      const bool bounce = (cy == 1 && wlo) || (cy == -1 && whi);
      if (bounce)  // halfway bounce-back: the opposite population of this node
        f[q] = load ? S::load(static_cast<const Elem*>(v.src_q[opp(q)]), n) : T(0);
      else
        f[q] = load ? S::load(static_cast<const Elem*>(v.src_q[q]), idx) : T(0);
    }
  }
}

// Velocities are carried scaled, u_s = sqrt(4.5) u, so that in
//   f^eq_i = w rho (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u)
//          = w rho (1 + sqrt(2) c.u_s + (c.u_s)^2 - u_s.u_s / 3)
// the square needs no extra factor.
constexpr double kSqrt45 = 2.12132034355964257320;  // sqrt(4.5)
constexpr double kSqrt2 = 1.41421356237309504880;

// Density deviation, density and scaled velocity of a node from the sums and
// differences of its opposite pairs (SCALED: f holds h = g / w, so the sums
// carry the weights).  k is the velocity term of the bracket above:
// 1 - u_s.u_s / 3 for full populations, -u_s.u_s / 3 in deviation form.
template <typename T>
struct Moments {
  T drho, rho, ux, uy, uz, k;
};

template <class LAT, int STORE, class T = typename Storage<STORE>::T>
__device__ __forceinline__ T k_of(const T ux, const T uy, const T uz) {
  const T usq = LAT::DIM == 3 ? fma(ux, ux, fma(uy, uy, uz * uz)) : fma(ux, ux, uy * uy);
  return Storage<STORE>::DEV ? usq * T(-1.0 / 3.0) : fma(usq, T(-1.0 / 3.0), T(1));
}

template <class LAT, int STORE, class T = typename Storage<STORE>::T>
__device__ __forceinline__ Moments<T> moments(const View& v, const T (&f)[LAT::Q]) {
  using S = Storage<STORE>;
  constexpr int NP = (LAT::Q - 1) / 2;
  constexpr bool D3 = LAT::DIM == 3;
  T s0 = S::SCALED ? T(LAT::w(0)) * f[0] : f[0];
  T jx = T(0), jy = T(0), jz = T(0);
  bool hx = false, hy = false, hz = false;
#pragma unroll
  for (int k = 0; k < NP; k++) {
    const int q = 2 * k + 1;
    const T wq = T(LAT::w(q));
    const T p = f[q] + f[q + 1], m = f[q] - f[q + 1];
    s0 = S::SCALED ? fma(wq, p, s0) : s0 + p;
    axis_acc<S::SCALED>(jx, hx, LAT::c(q, 0), wq, m);
    axis_acc<S::SCALED>(jy, hy, LAT::c(q, 1), wq, m);
    if (D3) axis_acc<S::SCALED>(jz, hz, LAT::c(q, 2), wq, m);
  }
  Moments<T> r;
  r.drho = S::DEV ? s0 : T(0);
  r.rho = S::DEV ? pick<STORE>(v.rho0, v.rho0_f, v.rho0_df) + s0 : s0;
  const T is = T(kSqrt45) * rcp(r.rho);
  r.ux = jx * is;
  r.uy = jy * is;
  r.uz = D3 ? jz * is : T(0);
  r.k = k_of<LAT, STORE, T>(r.ux, r.uy, r.uz);
  return r;
}

// Plain BGK in the stored form: out_i = (1 - omega) f_i + omega f^eq_i + F_i.
// For the pair (q, q+1 = -q), omega f^eq + F is A + B and A - B with
//   A = omega W (k + (c.u_s)^2)            (+ omega w drho in deviation form)
//   B = W (sqrt(2) omega c.u_s + 3 c.g_f),  W = w rho
// (w = 1 in the scaled form).  The weight products fold per weight class.
template <class LAT, int STORE, class T = typename Storage<STORE>::T>
__device__ __forceinline__ void bgk(const View& v, const Moments<T>& m, const T (&f)[LAT::Q], T (&out)[LAT::Q]) {
  using S = Storage<STORE>;
  constexpr int NP = (LAT::Q - 1) / 2;
  const T om = pick<STORE>(v.omega, v.omega_f, v.omega_df);
  const T omc = pick<STORE>(v.omc, v.omc_f, v.omc_df);
  const T omb = T(kSqrt2) * om;
  auto A_of = [&](T wq, T t) -> T {
    const T ow = om * (S::SCALED ? T(1) : wq);
    if constexpr (S::DEV) return fma(ow * m.rho, t, ow * m.drho);
    else return (ow * m.rho) * t;
  };
  out[0] = fma(omc, f[0], A_of(T(LAT::w(0)), m.k));
#pragma unroll
  for (int k = 0; k < NP; k++) {
    const int q = 2 * k + 1;
    const T wq = T(LAT::w(q));
    const T cu = cdot<T>(LAT::c(q, 0), LAT::c(q, 1), LAT::c(q, 2), m.ux, m.uy, m.uz);
    const T A = A_of(wq, fma(cu, cu, m.k));
    const T B = ((S::SCALED ? T(1) : wq) * m.rho) * fma(omb, cu, cg3_of<STORE>(v, q));
    out[q] = fma(omc, f[q], A + B);
    out[q + 1] = fma(omc, f[q + 1], A - B);
  }
}

// Plain update of a node whose pulled populations are f; stored where go.
// Returns the moments (the immersed-boundary update reuses them).
template <class LAT, int STORE>
__device__ __forceinline__ Moments<typename Storage<STORE>::T> plain_core(
    const View& v, const int n, const bool go, const typename Storage<STORE>::T (&f)[LAT::Q]) {
  using S = Storage<STORE>;
  using T = typename S::T;
  using Elem = typename S::Elem;
  constexpr int NP = (LAT::Q - 1) / 2;
  const Moments<T> m = moments<LAT, STORE>(v, f);
  T out[LAT::Q];
  bgk<LAT, STORE>(v, m, f, out);
  if (go) {
    S::store(static_cast<Elem*>(v.dst_q[0]), n, out[0]);
#pragma unroll
    for (int k = 0; k < NP; k++)
      S::store2(static_cast<Elem*>(v.dst_q[2 * k + 1]), static_cast<Elem*>(v.dst_q[2 * k + 2]), n, out[2 * k + 1],
                out[2 * k + 2]);
  }
  return m;
}

// Particle kinematics for the solid velocity: FP64 position, velocity and
// spin (FP64 storage), or the FP32 record (nearest node as int, offset,
// velocity, spin) for the reduced-precision storages.
template <typename PT>
struct Kin {
  PT c[3], vel[3], w[3];  // centre (FP64) or offset from ic (FP32)
  int ic[3];
};

template <int STORE>
__device__ __forceinline__ Kin<typename Storage<STORE>::T> load_kin(const View& v, const int q) {
  Kin<typename Storage<STORE>::T> k;
  if constexpr (STORE == LBM_IMB_STORE_DFDEV) {
    // 32-float record: high parts, nearest node, then the low parts
    const float4* kp = reinterpret_cast<const float4*>(v.kin) + 8 * q;
    const float4 fr = __ldg(kp), vp = __ldg(kp + 2), wp = __ldg(kp + 3);
    const int4 ir = __ldg(reinterpret_cast<const int4*>(kp) + 1);
    const float4 frl = __ldg(kp + 4), vpl = __ldg(kp + 6), wpl = __ldg(kp + 7);
    k.c[0] = DF(fr.x, frl.x); k.c[1] = DF(fr.y, frl.y); k.c[2] = DF(fr.z, frl.z);
    k.ic[0] = ir.x; k.ic[1] = ir.y; k.ic[2] = ir.z;
    k.vel[0] = DF(vp.x, vpl.x); k.vel[1] = DF(vp.y, vpl.y); k.vel[2] = DF(vp.z, vpl.z);
    k.w[0] = DF(wp.x, wpl.x); k.w[1] = DF(wp.y, wpl.y); k.w[2] = DF(wp.z, wpl.z);
  } else if constexpr (std::is_same<typename Storage<STORE>::T, float>::value) {
    const float4* kp = reinterpret_cast<const float4*>(v.kin) + 4 * q;
    const float4 fr = __ldg(kp);
    const int4 ir = __ldg(reinterpret_cast<const int4*>(kp) + 1);
    const float4 vp = __ldg(kp + 2);
    const float4 wp = __ldg(kp + 3);
    k.c[0] = fr.x; k.c[1] = fr.y; k.c[2] = fr.z;
    k.ic[0] = ir.x; k.ic[1] = ir.y; k.ic[2] = ir.z;
    k.vel[0] = vp.x; k.vel[1] = vp.y; k.vel[2] = vp.z;
    k.w[0] = wp.x; k.w[1] = wp.y; k.w[2] = wp.z;
  } else {
#pragma unroll
    for (int d = 0; d < 3; d++) {
      k.c[d] = v.pos[3 * q + d];
      k.vel[d] = v.vel[3 * q + d];
      k.w[d] = v.omg[3 * q + d];
      k.ic[d] = 0;
    }
  }
  return k;
}

// node position relative to the particle (minimum image; y is the local row,
// global row y + ygo) and the rigid-body velocity V = v + w x r there
template <bool D3, typename PT>
__device__ __forceinline__ void node_rel(const View& v, const Kin<PT>& k, const int x, const int y, const int z,
                                         PT (&r)[3], PT (&V)[3]) {
  if constexpr (std::is_same<PT, DF>::value) {
    r[0] = min_image_df(DF(float(x - k.ic[0])) - k.c[0], v.nx, true);
    r[1] = min_image_df(DF(float(y + v.ygo - k.ic[1])) - k.c[1], v.ny_glob, !v.wall_y);
    r[2] = D3 ? min_image_df(DF(float(z - k.ic[2])) - k.c[2], v.nz, true) : DF(0.f);
  } else if constexpr (sizeof(PT) == 4) {
    r[0] = min_image_f(float(x - k.ic[0]) - k.c[0], v.nx, true);
    r[1] = min_image_f(float(y + v.ygo - k.ic[1]) - k.c[1], v.ny_glob, !v.wall_y);
    r[2] = D3 ? min_image_f(float(z - k.ic[2]) - k.c[2], v.nz, true) : 0.f;
  } else {
    r[0] = min_image((double)x - k.c[0], v.nx, true);
    r[1] = min_image((double)(y + v.ygo) - k.c[1], v.ny_glob, !v.wall_y);
    r[2] = D3 ? min_image((double)z - k.c[2], v.nz, true) : 0.0;
  }
  V[0] = k.vel[0] + (k.w[1] * r[2] - k.w[2] * r[1]);
  V[1] = k.vel[1] + (k.w[2] * r[0] - k.w[0] * r[2]);
  V[2] = k.vel[2] + (k.w[0] * r[1] - k.w[1] * r[0]);
}

// ---------------------------------------------------------------------------
// Immersed-boundary update of one covered node: Eq. (1) with beta of Eq. (2)
// and the solid term
//   Omega^S_i = (f - f^eq)_{-i} - (f - f^eq)_i + f^eq_i(rho, V_S) - f^eq_i(rho, u),
// written as a correction of the plain update,
//   f*_i = f*_i(plain) + beta (omega (f_i - f^eq_i) + Omega^S_i),
// and the Eq. (3) force/torque on each owner (-beta sum_i Omega^S_i c_i split
// by covered fraction): the first owner's share is summed over the warp by
// owner (warp_reduce_to_particles), the others go to their FP64
// accumulators directly.  f: the node's pulled populations (stored form).
// The whole warp calls it; lanes with mine = false do the arithmetic on a
// valid node and write nothing.
// ---------------------------------------------------------------------------
// the first two owner slots and first covered fraction of a node, when a
// caller has them already (HEAD = true)
template <typename E>
struct SlotHead {
  int o0, o1;
  E e0;
};

template <class LAT, int STORE, bool HEAD = false>
__device__ __forceinline__ void imb_core(const View& v, const int xx, const int y, const int z, const int n,
                                         const bool mine, typename Storage<STORE>::T (&f)[LAT::Q],
                                         const Moments<typename Storage<STORE>::T>& m,
                                         const SlotHead<typename Storage<STORE>::E> head = {}) {
  using S = Storage<STORE>;
  using T = typename S::T;
  using E = typename S::E;
  using Elem = typename S::Elem;
  using PT = T;  // particle-side arithmetic: FP64 for FP64 storage, FP32 otherwise
  constexpr int Q = LAT::Q;
  constexpr int NP = (Q - 1) / 2;
  constexpr bool D3 = LAT::DIM == 3;
  constexpr int K = kMaxOwners;
  const T om = pick<STORE>(v.omega, v.omega_f, v.omega_df);
  const T tau_t = pick<STORE>(v.tau, v.tau_f, v.tau_df);

  // owners, sorted by id with empty slots last, so that V_S sums in particle
  // order.  Slots fill in order, so the taken ones are a prefix: slots 0 and
  // 1 are read at once, and the rest (and the fractions past the first) only
  // where the second slot is taken, so that the usual node with one owner
  // touches two of the eight slot arrays.
  int own[K];
  E eo[K];
  int no = 0;
  {
    const int o0 = HEAD ? head.o0 : v.own[0][n], o1 = HEAD ? head.o1 : v.own[1][n];
    const E e0 = HEAD ? head.e0 : static_cast<const E*>(v.eps[0])[n];
    own[0] = o0 >= 0 ? o0 : 0x7fffffff;
    eo[0] = o0 >= 0 ? e0 : E(0);
    no = o0 >= 0 ? 1 : 0;
#pragma unroll
    for (int s = 1; s < K; s++) {
      own[s] = 0x7fffffff;
      eo[s] = E(0);
    }
    if (o1 >= 0) {
      own[1] = o1;
      eo[1] = static_cast<const E*>(v.eps[1])[n];
      no = 2;
#pragma unroll
      for (int s = 2; s < K; s++) {
        const int o = v.own[s][n];
        if (o < 0) break;
        own[s] = o;
        eo[s] = static_cast<const E*>(v.eps[s])[n];
        no = s + 1;
      }
    }
  }
  auto cswap = [&](int a, int b) {
    if (own[a] > own[b]) {
      const int t = own[a];
      own[a] = own[b];
      own[b] = t;
      const E te = eo[a];
      eo[a] = eo[b];
      eo[b] = te;
    }
  };
  static_assert(K == 4, "sorting network for four owner slots");
  cswap(0, 1);
  cswap(2, 3);
  cswap(0, 2);
  cswap(1, 3);
  cswap(1, 2);

  if constexpr (S::SCALED) {
#pragma unroll
    for (int q = 0; q < Q; q++) f[q] *= T(LAT::w(q));  // g = h w
  }

  // solid velocity at the node, position relative to each owner
  PT esum = PT(0), vs0 = PT(0), vs1 = PT(0), vs2 = PT(0);
  PT rk[K][3];
  PT V1x = PT(0), V1y = PT(0), V1z = PT(0);
#pragma unroll
  for (int k = 0; k < K; k++) {
    rk[k][0] = rk[k][1] = rk[k][2] = PT(0);
    if (k < no) {
      const int q = own[k];
      const Kin<PT> kq = load_kin<STORE>(v, q);
      PT V[3];
      node_rel<D3>(v, kq, xx, y, z, rk[k], V);
      const PT e = to_pt<PT>(eo[k]);
      if (k == 0) {
        V1x = V[0];
        V1y = V[1];
        V1z = V[2];
      }
      esum += e;
      vs0 += e * V[0];
      vs1 += e * V[1];
      vs2 += e * V[2];
    }
  }
  T beta = T(0), VSx = T(0), VSy = T(0), VSz = T(0);
  PT inv_esum = PT(1);
  if (no == 1) {
    VSx = T(V1x);  // one owner: V_S is its velocity, the split factor 1
    VSy = T(V1y);
    VSz = T(V1z);
  } else if (no > 1) {
    inv_esum = quot(PT(1), esum);
    VSx = T(vs0 * inv_esum);
    VSy = T(vs1 * inv_esum);
    VSz = T(vs2 * inv_esum);
  }
  if (no > 0 && esum > PT(0)) {
    const T eps = esum < PT(1) ? T(esum) : T(1);
    const T th = tau_t - T(0.5);
    beta = quot(eps * th, (T(1) - eps) + th);  // Eq. (2)
  }

  // update, with f (deviation form for DEV storages, unscaled) and the
  // pair parts of f^eq(rho, u) = A +- B, f^eq(rho, V_S) = AS +- BS:
  //   g = f - f^eq,  D = g_{-q} - g_q,  dA = AS - A,  dB = BS - B,
  //   Omega^S_q = D + dA + dB,  Omega^S_{-q} = dA - (D + dB),
  //   f*_q = f_q + F_q + (beta - 1) omega g_q + beta Omega^S_q
  // with A = W (k + (c.u_s)^2) (+ w drho), B = sqrt(2) W c.u_s, W = w rho.
  const T rho = m.rho;
  const T vx = T(kSqrt45) * VSx, vy = T(kSqrt45) * VSy, vz = T(kSqrt45) * VSz;
  const T dk = k_of<LAT, STORE>(vx, vy, vz) - m.k;
  const T cfac = (beta - T(1)) * om;
  T mx = T(0), my = T(0), mz = T(0);
  T res[Q];
  {
    const T W0 = T(LAT::w(0)) * rho;
    const T A0 = S::DEV ? fma(W0, m.k, T(LAT::w(0)) * m.drho) : W0 * m.k;
    res[0] = fma(beta, W0 * dk, fma(cfac, f[0] - A0, f[0]));  // Omega^S_0 = dA_0
  }
#pragma unroll
  for (int k = 0; k < NP; k++) {
    const int q = 2 * k + 1;
    const int cx = LAT::c(q, 0), cy = LAT::c(q, 1), cz = LAT::c(q, 2);
    const T wq = T(LAT::w(q));
    const T W = wq * rho, Wb = (T(kSqrt2) * wq) * rho;
    const T cu = cdot<T>(cx, cy, cz, m.ux, m.uy, m.uz);
    const T cv = cdot<T>(cx, cy, cz, vx, vy, vz);
    const T t = fma(cu, cu, m.k);
    const T A = S::DEV ? fma(W, t, wq * m.drho) : W * t;
    const T B = Wb * cu;
    const T gp = f[q] - (A + B), gm = f[q + 1] - (A - B);
    const T dA = W * fma(cv, cv, fma(-cu, cu, dk));
    const T E = (gm - gp) + Wb * (cv - cu);  // D + dB
    const T Fq = fq_of<STORE>(v, q) * rho;
    res[q] = fma(beta, E + dA, fma(cfac, gp, f[q] + Fq));
    res[q + 1] = fma(beta, dA - E, fma(cfac, gm, f[q + 1] - Fq));
    // Omega^S_q - Omega^S_{-q} = 2 E, and c_{q+1} = -c_q
    if (cx) mx += cx > 0 ? E : -E;
    if (cy) my += cy > 0 ? E : -E;
    if (cz) mz += cz > 0 ? E : -E;
  }
  if (mine) {
#pragma unroll
    for (int q = 0; q < Q; q++)
      S::store(static_cast<Elem*>(v.dst_q[q]), n, S::SCALED ? res[q] * T(1.0 / LAT::w(q)) : res[q]);
  }

  // momentum given to the fluid m = beta sum_i Omega_i^S c_i; the force on
  // the particles is -m, split by covered fraction (Eq. 3 and reading)
  const T b2 = T(2) * beta;
  const PT m0 = PT(b2 * mx), m1 = PT(b2 * my), m2 = PT(b2 * mz);
  const bool any = mine && esum > PT(0);
  PT val[6] = {PT(0), PT(0), PT(0), PT(0), PT(0), PT(0)};
#pragma unroll
  for (int k = 0; k < K; k++) {
    if (any && k < no) {
      const PT a = no == 1 ? PT(1) : to_pt<PT>(eo[k]) * inv_esum;
      const PT p0 = a * m0, p1 = a * m1, p2 = a * m2;
      const PT F0 = -p0, F1 = -p1, F2 = -p2;
      const PT T0 = -(rk[k][1] * p2 - rk[k][2] * p1);
      const PT T1 = -(rk[k][2] * p0 - rk[k][0] * p2);
      const PT T2 = -(rk[k][0] * p1 - rk[k][1] * p0);
      if (k == 0) {
        val[0] = F0; val[1] = F1; val[2] = F2;
        val[3] = T0; val[4] = T1; val[5] = T2;
      } else {
        const int q = own[k];
        atomicAdd(v.ff + 3 * q, to_double(F0));
        atomicAdd(v.ff + 3 * q + 1, to_double(F1));
        if (D3) atomicAdd(v.ff + 3 * q + 2, to_double(F2));
        if (D3) {
          atomicAdd(v.tf + 3 * q, to_double(T0));
          atomicAdd(v.tf + 3 * q + 1, to_double(T1));
        }
        atomicAdd(v.tf + 3 * q + 2, to_double(T2));
      }
    }
  }
  warp_reduce_to_particles<PT>(any ? own[0] : -1, val, v.ff, v.tf);
}

// ---------------------------------------------------------------------------
// Fused collision with a per-warp queue of covered nodes.  A warp takes row
// segments of 32 nodes one after another: every node gets the plain BGK
// update from its pulled populations (stored unless covered); the covered
// nodes' populations and coordinates are appended to the warp's queue in
// shared memory, and whenever 32 are queued the warp gives them the
// immersed-boundary update with all lanes busy.  Only __syncwarp is used:
// the warps of a CTA never wait for one another.
// ---------------------------------------------------------------------------
constexpr int kQueueCap = 64;  // 31 left over + 32 new at most

template <int STORE>
struct WarpQueue {
  typename Storage<STORE>::T* f;  // [Q + 5][kQueueCap] populations (stored form), rho, drho, u_s
  int* n;                          // [kQueueCap] node offset
  int* xy;                         // [kQueueCap] x | y << 16
  int* z;                          // [kQueueCap]
};

template <class LAT, int STORE>
__host__ __device__ constexpr int queue_bytes_per_warp() {
  return kQueueCap * ((LAT::Q + 5) * (int)sizeof(typename Storage<STORE>::T) + 3 * 4);
}

template <class LAT, int STORE>
__device__ __forceinline__ WarpQueue<STORE> warp_queue(unsigned char* base, const int warp) {
  using T = typename Storage<STORE>::T;
  unsigned char* b = base + warp * queue_bytes_per_warp<LAT, STORE>();
  WarpQueue<STORE> w;
  w.f = reinterpret_cast<T*>(b);
  w.n = reinterpret_cast<int*>(b + kQueueCap * (LAT::Q + 5) * sizeof(T));
  w.xy = w.n + kQueueCap;
  w.z = w.xy + kQueueCap;
  return w;
}

// immersed-boundary update of the first count (<= 32) queued nodes
template <class LAT, int STORE>
__device__ __forceinline__ void queue_flush(const View& v, const WarpQueue<STORE>& wq, const int count,
                                            const int lane) {
  using T = typename Storage<STORE>::T;
  const bool mine = lane < count;
  const int s = mine ? lane : 0;
  constexpr int Q = LAT::Q;
  T f[Q];
#pragma unroll
  for (int q = 0; q < Q; q++) f[q] = wq.f[q * kQueueCap + s];
  Moments<T> m;
  m.rho = wq.f[Q * kQueueCap + s];
  m.drho = wq.f[(Q + 1) * kQueueCap + s];
  m.ux = wq.f[(Q + 2) * kQueueCap + s];
  m.uy = wq.f[(Q + 3) * kQueueCap + s];
  m.uz = wq.f[(Q + 4) * kQueueCap + s];
  m.k = k_of<LAT, STORE>(m.ux, m.uy, m.uz);
  const int xy = wq.xy[s];
  imb_core<LAT, STORE>(v, xy & 0xffff, xy >> 16, wq.z[s], wq.n[s], mine, f, m);
}

// covered nodes of the double-FP32 storage: one out-of-line copy of an FP64
// update (the pair arithmetic of this update is long and instruction-cache
// bound; on the FP64 pipe it overlaps the FP32 work of the plain updates)
template <class LAT, int STORE>
__device__ __noinline__ void queue_flush_call(const View& v, const WarpQueue<STORE>& wq, const int count,
                                              const int lane) {
  if constexpr (STORE == LBM_IMB_STORE_DFDEV) {
    // queued pairs -> FP64, then the FP64 immersed-boundary update
    const bool mine = lane < count;
    const int s = mine ? lane : 0;
    constexpr int Q = LAT::Q;
    double f[Q];
#pragma unroll
    for (int q = 0; q < Q; q++) f[q] = df_to_bits(wq.f[q * kQueueCap + s]);
    Moments<double> m;
    m.rho = df_to_bits(wq.f[Q * kQueueCap + s]);
    m.drho = df_to_bits(wq.f[(Q + 1) * kQueueCap + s]);
    m.ux = df_to_bits(wq.f[(Q + 2) * kQueueCap + s]);
    m.uy = df_to_bits(wq.f[(Q + 3) * kQueueCap + s]);
    m.uz = df_to_bits(wq.f[(Q + 4) * kQueueCap + s]);
    m.k = k_of<LAT, kDfDevImb>(m.ux, m.uy, m.uz);
    const int xy = wq.xy[s];
    imb_core<LAT, kDfDevImb>(v, xy & 0xffff, xy >> 16, wq.z[s], wq.n[s], mine, f, m);
  } else {
    queue_flush<LAT, STORE>(v, wq, count, lane);
  }
}
template <class LAT, int STORE>
__device__ __forceinline__ void flush_queue(const View& v, const WarpQueue<STORE>& wq, const int count,
                                            const int lane) {
  if constexpr (STORE == LBM_IMB_STORE_DFDEV) queue_flush_call<LAT, STORE>(v, wq, count, lane);
  else queue_flush<LAT, STORE>(v, wq, count, lane);
}

// One lane's node of the warp's row segment, populations f already pulled;
// cnt is the warp's queue length (warp-uniform).
template <class LAT, int STORE>
__device__ __forceinline__ void fused_core(const View& v, const int xx, const int y, const int z, const int n,
                                           const bool active, typename Storage<STORE>::T (&f)[LAT::Q],
                                           const WarpQueue<STORE>& wq, int& cnt, const int lane) {
  const unsigned FULL = 0xffffffffu;
  constexpr int Q = LAT::Q;
  const bool covered = active && v.own[0][n] >= 0;
  const Moments<typename Storage<STORE>::T> m = plain_core<LAT, STORE>(v, n, active && !covered, f);
  const unsigned b = __ballot_sync(FULL, covered);
  if (b == 0u) return;
  if (covered) {
    const int pos = cnt + __popc(b & ((1u << lane) - 1u));
#pragma unroll
    for (int q = 0; q < Q; q++) wq.f[q * kQueueCap + pos] = f[q];
    wq.f[Q * kQueueCap + pos] = m.rho;
    wq.f[(Q + 1) * kQueueCap + pos] = m.drho;
    wq.f[(Q + 2) * kQueueCap + pos] = m.ux;
    wq.f[(Q + 3) * kQueueCap + pos] = m.uy;
    wq.f[(Q + 4) * kQueueCap + pos] = m.uz;
    wq.n[pos] = n;
    wq.xy[pos] = xx | (y << 16);  // x, y < 65536
    wq.z[pos] = z;
  }
  cnt += __popc(b);
  __syncwarp();
  if (cnt >= 32) {
    flush_queue<LAT, STORE>(v, wq, 32, lane);
    __syncwarp();
    if (lane < cnt - 32) {
#pragma unroll
      for (int q = 0; q < Q + 5; q++) wq.f[q * kQueueCap + lane] = wq.f[q * kQueueCap + 32 + lane];
      wq.n[lane] = wq.n[32 + lane];
      wq.xy[lane] = wq.xy[32 + lane];
      wq.z[lane] = wq.z[32 + lane];
    }
    cnt -= 32;
    __syncwarp();
  }
}

// the same with the populations pulled from global memory
template <class LAT, int STORE>
__device__ __forceinline__ void fused_node(const View& v, const int xx, const int y, const int z, const bool active,
                                           const WarpQueue<STORE>& wq, int& cnt, const int lane) {
  using T = typename Storage<STORE>::T;
  const int n = (z * v.ny + y) * v.pitch + xx;
  T f[LAT::Q];
  pull<LAT, STORE>(v, xx, y, z, n, active, f);
  fused_core<LAT, STORE>(v, xx, y, z, n, active, f, wq, cnt, lane);
}

// CTA-packed form (non-persistent): every lane of a 128-node row tile gets
// the plain update; the tile's covered nodes are packed into the first lanes
// through shared memory (two CTA barriers) and updated by full warps.
// smem: queue_bytes_per_warp * 2 bytes (128 packed entries).
template <class LAT, int STORE>
__device__ __forceinline__ void packed_node(const View& v, const int xx, const int y, const int z, const bool active,
                                            unsigned char* smem) {
  using T = typename Storage<STORE>::T;
  constexpr int Q = LAT::Q;
  constexpr int CAP = 128;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* sf = reinterpret_cast<T*>(smem);  // [Q + 5][CAP]
  int* sn = reinterpret_cast<int*>(sf + (Q + 5) * CAP);
  int* sxy = sn + CAP;
  int* sz = sxy + CAP;
  __shared__ int s_cnt[4];
  const int n = (z * v.ny + y) * v.pitch + xx;
  T f[Q];
  pull<LAT, STORE>(v, xx, y, z, n, active, f);
  const bool covered = active && v.own[0][n] >= 0;
  const Moments<T> m = plain_core<LAT, STORE>(v, n, active && !covered, f);
  const unsigned b = __ballot_sync(FULL, covered);
  __syncthreads();  // the previous tile's packed state has been consumed
  if (lane == 0) s_cnt[warp] = __popc(b);
  __syncthreads();
  int base = 0, total = 0;
#pragma unroll
  for (int w = 0; w < 4; w++) {
    base += w < warp ? s_cnt[w] : 0;
    total += s_cnt[w];
  }
  if (total == 0) return;
  if (covered) {
    const int pos = base + __popc(b & ((1u << lane) - 1u));
#pragma unroll
    for (int q = 0; q < Q; q++) sf[q * CAP + pos] = f[q];
    sf[Q * CAP + pos] = m.rho;
    sf[(Q + 1) * CAP + pos] = m.drho;
    sf[(Q + 2) * CAP + pos] = m.ux;
    sf[(Q + 3) * CAP + pos] = m.uy;
    sf[(Q + 4) * CAP + pos] = m.uz;
    sn[pos] = n;
    sxy[pos] = xx | (y << 16);
    sz[pos] = z;
  }
  __syncthreads();
  if ((int)threadIdx.x >= ((total + 31) & ~31)) return;  // whole warps beyond the packed nodes
  const bool mine = (int)threadIdx.x < total;
  const int s = mine ? (int)threadIdx.x : 0;
  T g[Q];
#pragma unroll
  for (int q = 0; q < Q; q++) g[q] = sf[q * CAP + s];
  Moments<T> mm;
  mm.rho = sf[Q * CAP + s];
  mm.drho = sf[(Q + 1) * CAP + s];
  mm.ux = sf[(Q + 2) * CAP + s];
  mm.uy = sf[(Q + 3) * CAP + s];
  mm.uz = sf[(Q + 4) * CAP + s];
  mm.k = k_of<LAT, STORE>(mm.ux, mm.uy, mm.uz);
  imb_core<LAT, STORE>(v, sxy[s] & 0xffff, sxy[s] >> 16, sz[s], sn[s], mine, g, mm);
}

// ---------------------------------------------------------------------------
// Two-node form (reduced-precision storages).  A thread takes the adjacent
// nodes x, x+1 (x even) of a row: directions with c_x = 0 come as one
// aligned two-element load, the others as two element loads; the moments and
// the BGK update of both nodes run as paired FP32 arithmetic (F2); stores
// are aligned pairs.  A CTA covers 128 nodes of two rows; its covered nodes
// are packed into the first lanes through shared memory and get the
// immersed-boundary update one node per thread (their plain values, stored
// first, are overwritten after the CTA barrier).
// smem: pair_pack_bytes<LAT, STORE>() bytes.
// ---------------------------------------------------------------------------
template <int STORE>
struct PairIO;
template <>
struct PairIO<LBM_IMB_STORE_F32DEV> {
  __device__ static __forceinline__ float2 load2(const float* p, int i) {
    return __ldg(reinterpret_cast<const float2*>(p + i));
  }
  __device__ static __forceinline__ float load1(const float* p, int i) { return __ldg(p + i); }
  __device__ static __forceinline__ void store2(float* p, int i, float2 v) {
    *reinterpret_cast<float2*>(p + i) = v;
  }
  __device__ static __forceinline__ void store1(float* p, int i, float a) { p[i] = a; }
};
template <>
struct PairIO<LBM_IMB_STORE_F16DEV> {
  __device__ static __forceinline__ float2 load2(const __half* p, int i) {
    return __half22float2(__ldg(reinterpret_cast<const __half2*>(p + i)));
  }
  __device__ static __forceinline__ float load1(const __half* p, int i) { return __half2float(__ldg(p + i)); }
  __device__ static __forceinline__ void store2(__half* p, int i, float2 v) {
    *reinterpret_cast<__half2*>(p + i) = __floats2half2_rn(v.x, v.y);
  }
  __device__ static __forceinline__ void store1(__half* p, int i, float a) { p[i] = __float2half_rn(a); }
};

template <class LAT, int STORE>
__host__ __device__ constexpr int pair_pack_bytes() {
  return 256 * ((LAT::Q + 5) * 4 + 3 * 4);
}

// pull of the node pair (x, x+1) of row (y, z); n = offset of node x (even)
template <class LAT, int STORE>
__device__ __forceinline__ void pull_pair(const View& v, const int x, const int y, const int z, const int n,
                                          F2 (&f)[LAT::Q]) {
  using IO = PairIO<STORE>;
  using Elem = typename Storage<STORE>::Elem;
  constexpr int Q = LAT::Q;
  const int nx = v.nx, ny = v.ny, nz = v.nz, pitch = v.pitch;
  const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
  const int ry[3] = {y * pitch, ym * pitch, yp * pitch};
  const int rz[3] = {z * ny * pitch, zm * ny * pitch, zp * ny * pitch};
  // x sources of the two nodes for c_x = +1 (left) and c_x = -1 (right)
  const int l0 = x == 0 ? nx - 1 : x - 1, l1 = x;
  const int r0 = x + 1 < nx ? x + 1 : 0, r1 = x + 2 < nx ? x + 2 : (x + 2 == nx ? 0 : 1);
  const bool wlo = v.wall_lo && y == v.y0, whi = v.wall_hi && y == v.y0 + v.ny_c - 1;
#pragma unroll
  for (int q = 0; q < Q; q++) {
    const int cx = LAT::c(q, 0), cy = LAT::c(q, 1), cz = LAT::c(q, 2);
    const int row = rz[cz == 0 ? 0 : (cz == 1 ? 1 : 2)] + ry[cy == 0 ? 0 : (cy == 1 ? 1 : 2)];
    const bool bounce = (cy == 1 && wlo) || (cy == -1 && whi);
    if (bounce) {  // halfway bounce-back: the opposite populations of the pair itself
      const float2 w = IO::load2(static_cast<const Elem*>(v.src_q[opp(q)]), n);
      f[q] = F2(w.x, w.y);
    } else {
      const Elem* src = static_cast<const Elem*>(v.src_q[q]);
      if (cx == 0) {
        const float2 w = IO::load2(src, row + x);
        f[q] = F2(w.x, w.y);
      } else {
        const int s0 = cx == 1 ? l0 : r0, s1 = cx == 1 ? l1 : r1;
        f[q] = F2(IO::load1(src, row + s0), IO::load1(src, row + s1));
      }
    }
  }
}

template <class LAT, int STORE>
__device__ __forceinline__ void pair_node(const View& v, const int x, const int y, const int z, const bool row_ok,
                                          unsigned char* smem) {
  using S = Storage<STORE>;
  using IO = PairIO<STORE>;
  using Elem = typename S::Elem;
  constexpr int Q = LAT::Q;
  constexpr int NP = (Q - 1) / 2;
  constexpr int CAP = 256;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* sf = reinterpret_cast<float*>(smem);  // [Q + 5][CAP]
  int* sn = reinterpret_cast<int*>(sf + (Q + 5) * CAP);
  int* sxy = sn + CAP;
  int* sz = sxy + CAP;
  __shared__ int s_cnt[4];
  const int nx = v.nx;
  const bool a0 = row_ok && x < nx, a1 = row_ok && x + 1 < nx;
  const int xc = a0 ? x : ((nx - 1) & ~1);  // a valid even node for idle lanes
  const int n = (z * v.ny + y) * v.pitch + xc;
  const int2 o = *reinterpret_cast<const int2*>(v.own[0] + n);
  const bool c0 = a0 && o.x >= 0, c1 = a1 && o.y >= 0;
  F2 f[Q];
  pull_pair<LAT, STORE>(v, xc, y, z, n, f);
  const Moments<F2> m = moments<LAT, STORE, F2>(v, f);
  F2 out[Q];
  bgk<LAT, STORE, F2>(v, m, f, out);
  if (a1) {
#pragma unroll
    for (int q = 0; q < Q; q++) IO::store2(static_cast<Elem*>(v.dst_q[q]), n, out[q].v);
  } else if (a0) {
#pragma unroll
    for (int q = 0; q < Q; q++) IO::store1(static_cast<Elem*>(v.dst_q[q]), n, out[q].v.x);
  }
  // pack the covered nodes of the CTA
  const unsigned b0 = __ballot_sync(FULL, c0), b1 = __ballot_sync(FULL, c1);
  if (lane == 0) s_cnt[warp] = __popc(b0) + __popc(b1);
  __syncthreads();
  int base = 0, total = 0;
#pragma unroll
  for (int w = 0; w < 4; w++) {
    base += w < warp ? s_cnt[w] : 0;
    total += s_cnt[w];
  }
  if (total == 0) return;
  const unsigned lt = (1u << lane) - 1u;
  int pos = base + __popc(b0 & lt) + __popc(b1 & lt);
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const bool ch = h == 0 ? c0 : c1;
    if (ch) {
#pragma unroll
      for (int q = 0; q < Q; q++) sf[q * CAP + pos] = h == 0 ? f[q].v.x : f[q].v.y;
      sf[Q * CAP + pos] = h == 0 ? m.rho.v.x : m.rho.v.y;
      sf[(Q + 1) * CAP + pos] = h == 0 ? m.drho.v.x : m.drho.v.y;
      sf[(Q + 2) * CAP + pos] = h == 0 ? m.ux.v.x : m.ux.v.y;
      sf[(Q + 3) * CAP + pos] = h == 0 ? m.uy.v.x : m.uy.v.y;
      sf[(Q + 4) * CAP + pos] = h == 0 ? m.uz.v.x : m.uz.v.y;
      sn[pos] = n + h;
      sxy[pos] = (xc + h) | (y << 16);  // x, y < 65536
      sz[pos] = z;
      pos++;
    }
  }
  __syncthreads();
  for (int b = 0; b < total; b += 128) {
    if (b + warp * 32 >= total) break;  // whole warps beyond the packed nodes
    const int i = b + (int)threadIdx.x;
    const bool mine = i < total;
    const int s = mine ? i : b;
    float g[Q];
#pragma unroll
    for (int q = 0; q < Q; q++) g[q] = sf[q * CAP + s];
    Moments<float> mm;
    mm.rho = sf[Q * CAP + s];
    mm.drho = sf[(Q + 1) * CAP + s];
    mm.ux = sf[(Q + 2) * CAP + s];
    mm.uy = sf[(Q + 3) * CAP + s];
    mm.uz = sf[(Q + 4) * CAP + s];
    mm.k = k_of<LAT, STORE, float>(mm.ux, mm.uy, mm.uz);
    imb_core<LAT, STORE>(v, sxy[s] & 0xffff, sxy[s] >> 16, sz[s], sn[s], mine, g, mm);
  }
  (void)NP;
}

// ---------------------------------------------------------------------------
// Plain part of the pair storage's split form, two adjacent nodes x, x+1 (x
// even) per thread in paired FP32 instructions (DF2): directions with
// c_x = 0 come as one aligned 16-byte load of both nodes' pairs, the others
// as two 8-byte loads; the moments and BGK of both nodes run side by side
// (bitwise the single-node results); uncovered nodes are pulled and stored
// (aligned 16 bytes when both are), covered ones are left to the covered
// kernel.
// ---------------------------------------------------------------------------
template <class LAT>
__device__ __forceinline__ void plain_pair_node(const View& v, const int x, const int y, const int z,
                                                const bool row_ok) {
  constexpr int Q = LAT::Q;
  constexpr int NP = (Q - 1) / 2;
  constexpr int ST = kDfDevPair;
  const int nx = v.nx, ny = v.ny, nz = v.nz, pitch = v.pitch;
  const bool a0 = row_ok && x < nx, a1 = row_ok && x + 1 < nx;
  const int xc = a0 ? x : ((nx - 1) & ~1);  // a valid even node for idle lanes
  const int n = (z * ny + y) * pitch + xc;
  const int2 o = *reinterpret_cast<const int2*>(v.own[0] + n);
  const bool s0 = a0 && o.x < 0, s1 = a1 && o.y < 0;  // stored here (not covered)
  if (!__any_sync(0xffffffffu, s0 || s1)) return;     // the whole warp's nodes are covered (or idle)
  const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
  const int ry[3] = {y * pitch, ym * pitch, yp * pitch};
  const int rz[3] = {z * ny * pitch, zm * ny * pitch, zp * ny * pitch};
  const int l0 = xc == 0 ? nx - 1 : xc - 1, l1 = xc;
  const int r0 = xc + 1 < nx ? xc + 1 : 0, r1 = xc + 2 < nx ? xc + 2 : (xc + 2 == nx ? 0 : 1);
  const bool wlo = v.wall_lo && y == v.y0, whi = v.wall_hi && y == v.y0 + v.ny_c - 1;
  DF2 f[Q];
#pragma unroll
  for (int q = 0; q < Q; q++) {
    const int cx = LAT::c(q, 0), cy = LAT::c(q, 1), cz = LAT::c(q, 2);
    const int row = rz[cz == 0 ? 0 : (cz == 1 ? 1 : 2)] + ry[cy == 0 ? 0 : (cy == 1 ? 1 : 2)];
    const bool bounce = (cy == 1 && wlo) || (cy == -1 && whi);
    // only the nodes stored here are pulled (the covered kernel pulls the
    // others); both as one aligned 16-byte load where the sources are adjacent
    const float2* src = static_cast<const float2*>(v.src_q[bounce ? opp(q) : q]);
    const bool adj = bounce || cx == 0;  // halfway bounce-back: the pair's own opposite populations
    const int i0 = bounce ? n : row + (cx == 0 ? xc : (cx == 1 ? l0 : r0));
    const int i1 = bounce ? n + 1 : row + (cx == 0 ? xc + 1 : (cx == 1 ? l1 : r1));
    float2 e0 = make_float2(0.f, 0.f), e1 = make_float2(0.f, 0.f);
    if (adj && s0 && s1) {
      const float4 w = __ldg(reinterpret_cast<const float4*>(src + i0));
      e0 = make_float2(w.x, w.y);
      e1 = make_float2(w.z, w.w);
    } else {
      if (s0) e0 = __ldg(src + i0);
      if (s1) e1 = __ldg(src + i1);
    }
    f[q] = DF2(make_float2(e0.x, e1.x), make_float2(e0.y, e1.y));
  }
  const Moments<DF2> m = moments<LAT, ST>(v, f);
  DF2 out[Q];
  bgk<LAT, ST>(v, m, f, out);
#pragma unroll
  for (int q = 0; q < Q; q++) {
    const DF2 r = df_norm(out[q]);
    float2* dst = static_cast<float2*>(v.dst_q[q]) + n;
    if (s0 && s1) {
      *reinterpret_cast<float4*>(dst) = make_float4(r.h.x, r.l.x, r.h.y, r.l.y);
    } else {
      if (s0) dst[0] = make_float2(r.h.x, r.l.x);
      if (s1) dst[1] = make_float2(r.h.y, r.l.y);
    }
  }
  (void)NP;
}

// drain a warp's queue (at the end of its segments)
template <class LAT, int STORE>
__device__ __forceinline__ void queue_drain(const View& v, const WarpQueue<STORE>& wq, int& cnt, const int lane) {
  if (cnt > 0) flush_queue<LAT, STORE>(v, wq, cnt, lane);
  cnt = 0;
  __syncwarp();
}

}  // namespace lbm
