// K1 device code: solid-fraction rasterisation and footprint clearing,
// shared by the per-step kernels (k_eps.cu) and the batched persistent
// kernel (k_batch.cu).
#pragma once
#include <math.h>

#include <type_traits>

#include "dev_df.cuh"
#include "lbm_internal.cuh"

namespace lbm {

// Division of small non-negative ints (t < 2^16) by a per-particle divisor
// d < 2^16 by one high multiply: q = floor(t * (floor((2^32 - 1)/d) + 1) /
// 2^32) is exact there (the error of the scaled reciprocal is below t/2^32
// < 1/d).  One integer division per divisor instead of one per index.
struct FastDiv {
  unsigned d, m;
  __device__ __forceinline__ explicit FastDiv(int dd) : d((unsigned)dd), m(dd > 1 ? 0xFFFFFFFFu / (unsigned)dd + 1u : 0u) {}
  __device__ __forceinline__ int div(int t) const { return d > 1 ? (int)__umulhi((unsigned)t, m) : t; }
};

// t = i + ex (j + ey k) -> (i, j, k)
struct FastDiv3 {
  FastDiv a, b;
  __device__ __forceinline__ FastDiv3(int ex, int ey) : a(ex), b(ex * ey) {}
  __device__ __forceinline__ void split(int t, int& i, int& j, int& k) const {
    k = b.div(t);
    const int r = t - k * (int)b.d;
    j = a.div(r);
    i = r - j * (int)a.d;
  }
};

// periodic index into [0, n) for boxes reaching at most one period outside
__device__ __forceinline__ int wrap_idx(int i, const int n) {
  if (i < 0) i += n;
  else if (i >= n) i -= n;
  if ((unsigned)i >= (unsigned)n) i = ((i % n) + n) % n;  // lattices smaller than a particle box
  return i;
}

// --------------------------------------------------------------------------
// clear the previous footprint (the taken owner slots) and zero the force sums
// --------------------------------------------------------------------------
// one warp per particle
// whether rows ly .. ly + ey - 1 of the whole lattice include one of this
// slab's computed rows (always, for a whole lattice)
__device__ __forceinline__ bool rows_meet_slab(const View& v, const int ly, const int ey) {
  if (v.ny_c == v.ny_glob) return true;
  for (int r = 0; r < ey; r++) {
    int j = ly + r;
    if (v.wall_y) {
      if (j < 0 || j >= v.ny_glob) continue;
    } else {
      j = wrap_idx(j, v.ny_glob);
    }
    j -= v.ygo;
    if (j >= v.y0 && j < v.y0 + v.ny_c) return true;
  }
  return false;
}

__device__ __forceinline__ void eps_clear_particle(const View& v, const int p, const int lane,
                                                   const bool zero_forces) {
  if (p == 0 && lane == 0 && v.cov_count != nullptr) *v.cov_count = 0;  // the list is rebuilt by the raster
  const int* box = v.lo + 6 * p;
  const int lx = box[0], ly = box[1], lz = box[2];
  const int ex = box[3], ey = box[4], ez = box[5];
  const int total = rows_meet_slab(v, ly, ey) ? ex * ey * ez : 0;
  const FastDiv3 fd(ex, ey);
  for (int t = lane; t < total; t += 32) {
    int ci, cj, ck;
    fd.split(t, ci, cj, ck);
    int i = lx + ci, j = ly + cj, k = lz + ck;
    if (v.wall_y) {
      if (j < 0 || j >= v.ny_glob) continue;
    } else {
      j = wrap_idx(j, v.ny_glob);
    }
    j -= v.ygo;  // local row; only this slab's computed rows
    if (j < v.y0 || j >= v.y0 + v.ny_c) continue;
    i = wrap_idx(i, v.nx);
    k = wrap_idx(k, v.nz);
    const long long n = ((long long)k * v.ny + j) * v.pitch + i;
    // taken slots form a prefix: stop at the first free one (concurrent
    // clears of overlapping boxes only ever write -1, so the order of their
    // reads and writes does not matter)
    for (int s = 0; s < kMaxOwners; s++) {
      if (v.own[s][n] < 0) break;
      v.own[s][n] = -1;
    }
  }
  // FP32 kinematics record of the particle for the reduced-precision
  // collision: position split into the nearest node (int) and the offset
  // from it (float), velocity and spin (float)
  if (v.kin != nullptr && v.storage == LBM_IMB_STORE_DFDEV) {
    // 32-float record for the double-FP32 collision: high parts of the
    // offset, velocity and spin, the nearest node, then the low parts
    const int d = lane & 3, part = lane >> 2;
    float* rec = v.kin + 32 * p;
    const int src = part & 3;
    const bool low = part >= 4;
    float out = 0.f;
    if (d < 3 && part != 5) {
      if (src == 1) {
        reinterpret_cast<int*>(rec)[lane] = (int)floor(v.pos[3 * p + d] + 0.5);
      } else {
        const double x = src == 0 ? v.pos[3 * p + d] - floor(v.pos[3 * p + d] + 0.5)
                                  : (src == 2 ? v.vel[3 * p + d] : v.omg[3 * p + d]);
        const float xh = (float)x;
        out = low ? (float)(x - (double)xh) : xh;
      }
    }
    if (!(d < 3 && src == 1 && !low)) rec[lane] = out;
  } else if (v.kin != nullptr && lane < 16) {
    const int d = lane & 3, part = lane >> 2;
    float* rec = v.kin + 16 * p;
    if (d == 3) {
      rec[lane] = 0.f;
    } else if (part == 0 || part == 1) {
      const double x = v.pos[3 * p + d];
      const double xi = floor(x + 0.5);
      if (part == 0) rec[lane] = (float)(x - xi);
      else reinterpret_cast<int*>(rec)[lane] = (int)xi;
    } else if (part == 2) {
      rec[lane] = (float)v.vel[3 * p + d];
    } else {
      rec[lane] = (float)v.omg[3 * p + d];
    }
  }
  if (zero_forces && lane < 3) {
    v.ff[3 * p + lane] = 0.0;
    v.tf[3 * p + lane] = 0.0;
  }
}

// --------------------------------------------------------------------------
// rasterise one particle per CTA
//
// Corner values come from small tables: with s(v) = sqrt(R^2 - v^2) and
// psi(v) = atan2(s(v), v) per axis value v, the disk corner area is
//   U(a,b) = R^2/2 (psi(a) + psi(b) - pi/2) - (a s(a) + b s(b))/2 + a b.
// For the ball every angle of the Gauss-Bonnet form depends on two of the
// three coordinates: for a pair (u,v) with z = sqrt(R^2 - u^2 - v^2) the
// vertex angle alpha = atan2(R z, u v) and the polar angles phi_u =
// atan2(z, u), phi_v = atan2(z, v) give the three face arcs
//   th_a = phi_b(ab) + phi_c(ac) - pi/2   (and cyclically),
// the solid angle Omega = alpha_ab + alpha_ac + alpha_bc - pi
//   - (a th_a + b th_b + c th_c)/R, the faces
//   A_a = (R^2 - a^2) th_a / 2 - (b z_ab + c z_ac)/2 + b c,
// and P = (R^3 Omega - a A_a - b A_b - c A_c)/3.
// --------------------------------------------------------------------------
struct RasterSmem {
  int tab_cap, pair_cap, cell_cap;
};

// bytes of the tables before the covered-node flags (the flags, one byte
// per cell, come last; the table form keeps only the flags)
__host__ __device__ inline int raster_list_offset(const RasterSmem c, int esz) {
  const long long b = (long long)c.tab_cap * esz + 12LL * c.pair_cap * esz + (long long)c.tab_cap * 4 +
                      (long long)c.cell_cap * 4 + c.tab_cap;
  return (int)((b + 15) & ~15LL);
}


template <typename T>
__device__ __forceinline__ int classify_cell(const T (*bnd)[64], const float (*bndf)[64], const int idx[3],
                                             int dim, const T R2, float R2f) {
  // exact decision in T; the FP64 instantiation first tries FP32 copies of
  // the offsets with a relative margin that cannot flip a decision
  if (sizeof(T) == 8) {
    float n2 = 0.f, f2 = 0.f;
    for (int d = 0; d < dim; d++) {
      const float bl = bndf[d][idx[d]], bh = bndf[d][idx[d] + 1];
      const float nd = bl > 0.f ? bl : (bh < 0.f ? -bh : 0.f);
      const float fd = fmaxf(fabsf(bl), fabsf(bh));
      n2 += nd * nd;
      f2 += fd * fd;
    }
    if (n2 >= R2f * 1.0001f) return 0;
    if (f2 <= R2f * 0.9999f) return 1;
  }
  T near2 = T(0), far2 = T(0);
  for (int d = 0; d < dim; d++) {
    const T bl = bnd[d][idx[d]], bh = bnd[d][idx[d] + 1];
    const T nd = bl > T(0) ? bl : (bh < T(0) ? -bh : T(0));
    const T fd = fabs(bl) > fabs(bh) ? fabs(bl) : fabs(bh);
    near2 += nd * nd;
    far2 += fd * fd;
  }
  if (near2 >= R2) return 0;
  if (far2 <= R2) return 1;
  return 2;
}

// per-axis decomposition of cell i into (lower, upper) value indices of boxes
// on the non-negative half-axis; returns the number of boxes (1 or 2).  Only
// signs are tested, so the FP32 copies of the offsets serve every element
// type (the conversion keeps the sign and zero; offsets are multiples of the
// centre's ulp, far above FP32's smallest number)
template <typename T>
__device__ __forceinline__ int split_axis(const T* b, int i, int zero, int (&lo_i)[2], int (&hi_i)[2]) {
  const T bl = b[i], bh = b[i + 1];
  if (bl >= T(0)) { lo_i[0] = i; hi_i[0] = i + 1; return 1; }
  if (bh <= T(0)) { lo_i[0] = i + 1; hi_i[0] = i; return 1; }
  lo_i[0] = zero; hi_i[0] = i;
  lo_i[1] = zero; hi_i[1] = i + 1;
  return 2;
}

// atan(k/16), k = 0..16 (round to nearest); the FP32-pair copy for the
// rasteriser of the pair storage
constexpr double kAtanK16[17] = {
    0.0, 0.06241880999595735, 0.12435499454676144, 0.18534794999569476,
    0.24497866312686414, 0.3028848683749714, 0.35877067027057225, 0.4124104415973873,
    0.4636476090008061, 0.5123894603107377, 0.5585993153435624, 0.6022873461349642,
    0.6435011087932844, 0.6823165548747481, 0.7188299996216245, 0.7531512809621944,
    0.7853981633974483};
__constant__ double kAtanTab[17] = {
    kAtanK16[0], kAtanK16[1], kAtanK16[2], kAtanK16[3], kAtanK16[4], kAtanK16[5], kAtanK16[6], kAtanK16[7], kAtanK16[8], kAtanK16[9], kAtanK16[10], kAtanK16[11], kAtanK16[12], kAtanK16[13], kAtanK16[14], kAtanK16[15], kAtanK16[16]};
__constant__ DF kAtanTabDF[17] = {
    DF(kAtanK16[0]), DF(kAtanK16[1]), DF(kAtanK16[2]), DF(kAtanK16[3]), DF(kAtanK16[4]), DF(kAtanK16[5]), DF(kAtanK16[6]), DF(kAtanK16[7]), DF(kAtanK16[8]), DF(kAtanK16[9]), DF(kAtanK16[10]), DF(kAtanK16[11]), DF(kAtanK16[12]), DF(kAtanK16[13]), DF(kAtanK16[14]), DF(kAtanK16[15]), DF(kAtanK16[16])};

// atan2(y, x) for y, x >= 0, not both zero (all angles of the exact-volume
// formulas lie in the first quadrant).  Method: with t = min/max <= 1 and
// c = k/16 the nearest table point, the arctangent addition formula gives
// atan(t) = atan(c) + atan(t'), t' = (t - c)/(1 + t c) = (n - c d)/(d + c n),
// |t'| <= 1/32 (slightly more if k is off by one); atan(t') is its Taylor
// series through t'^11 (truncation below 1e-17 relative).  y > x uses
// pi/2 - atan(x/y).  One reciprocal (approximation + two Newton steps)
// instead of two divisions plus range logic.
__device__ __forceinline__ double atan2_q1(const double y, const double x) {
  const bool sw = y > x;
  const double num = sw ? x : y, den = sw ? y : x;
  int k = __float2int_rn(16.f * __fdividef((float)num, (float)den));
  k = k < 0 ? 0 : (k > 16 ? 16 : k);
  const double c = (double)k * 0.0625;
  // t' = (n - c d) * (1 / (d + c n)): the hardware's approximate reciprocal
  // refined by two Newton-Raphson steps r <- r + r (1 - q r) (the relative
  // error squares at each step); q >= d > 0
  const double q = fma(c, num, den);
  double rq;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(rq) : "d"(q));
  rq = fma(rq, fma(-q, rq, 1.0), rq);
  rq = fma(rq, fma(-q, rq, 1.0), rq);
  const double tp = fma(-c, den, num) * rq;
  const double s = tp * tp;
  double p = fma(s, -1.0 / 11.0, 1.0 / 9.0);
  p = fma(s, p, -1.0 / 7.0);
  p = fma(s, p, 1.0 / 5.0);
  p = fma(s, p, -1.0 / 3.0);
  p = fma(s * tp, p, tp);
  const double r = kAtanTab[k] + p;
  return sw ? 1.57079632679489661923 - r : r;
}
__device__ __forceinline__ float atan2_q1(const float y, const float x) { return atan2f(y, x); }
// the same method in pair arithmetic (the pair storage's rasteriser): one
// pair reciprocal, the series' terms from t'^7 on in FP32 (below 2^-48 of the
// result), the rest in pairs
__device__ __forceinline__ DF atan2_q1(const DF y, const DF x) {
  const bool sw = y > x;
  const DF num = sw ? x : y, den = sw ? y : x;
  int k = __float2int_rn(16.f * __fdividef(num.h, den.h));
  k = k < 0 ? 0 : (k > 16 ? 16 : k);
  const float c = (float)k * 0.0625f;
  const DF tp = (num - den * c) * rcp(den + num * c);
  const DF s = tp * tp;
  const float sf = s.h;
  const float tail = __fmaf_rn(sf, __fmaf_rn(sf, -1.f / 11.f, 1.f / 9.f), -1.f / 7.f);
  DF u = DF(0.2) + s * tail;
  u = DF(-1.0 / 3.0) + s * u;
  const DF r = kAtanTabDF[k] + (tp + (tp * s) * u);
  return sw ? DF(1.57079632679489661923) - r : r;
}

// conversions of the rasteriser's element type
__device__ __forceinline__ float to_f32(const double x) { return (float)x; }
__device__ __forceinline__ float to_f32(const float x) { return x; }
__device__ __forceinline__ float to_f32(const DF x) { return x.h; }
template <typename T>
__device__ __forceinline__ T from_f64(const double x) {
  if constexpr (std::is_same<T, DF>::value) return df_from_bits(x);
  else return (T)x;
}
// a covered fraction into its slot (FP64 slots for the pair storage)
template <typename T>
__device__ __forceinline__ void store_eps(void* slot, const long long n, const T e) {
  if constexpr (std::is_same<T, DF>::value) static_cast<double*>(slot)[n] = df_to_bits(e);
  else static_cast<T*>(slot)[n] = e;
}

// --------------------------------------------------------------------------
// Exact fraction of one cell, without tables (builds the Eq. 6 table).
// corner_area(R, u, v): area of the disk inside {X >= u, Y >= v}, u, v >= 0;
// corner_volume(R, a, b, c): volume of the ball inside {X >= a, Y >= b,
// Z >= c} (the closed forms of the rasteriser, evaluated directly).
// --------------------------------------------------------------------------
__device__ __forceinline__ double corner_area(const double R, const double u, const double v) {
  if (u * u + v * v >= R * R) return 0.0;
  const double su = sqrt((R - u) * (R + u)), sv = sqrt((R - v) * (R + v));
  const double hpi = 1.57079632679489661923;
  return 0.5 * R * R * (atan2_q1(su, u) + atan2_q1(sv, v) - hpi) - 0.5 * (u * su + v * sv) + u * v;
}

__device__ __forceinline__ double corner_volume(const double R, const double a, const double b, const double c) {
  const double R2 = R * R;
  if ((a * a + b * b) + c * c >= R2) return 0.0;
  const double hpi = 1.57079632679489661923;
  const double zab = sqrt((R2 - a * a) - b * b), zac = sqrt((R2 - a * a) - c * c);
  const double zbc = sqrt((R2 - b * b) - c * c);
  const double tha = atan2_q1(zab, b) + atan2_q1(zac, c) - hpi;
  const double thb = atan2_q1(zab, a) + atan2_q1(zbc, c) - hpi;
  const double thc = atan2_q1(zac, a) + atan2_q1(zbc, b) - hpi;
  const double om = atan2_q1(R * zab, a * b) + atan2_q1(R * zac, a * c) + atan2_q1(R * zbc, b * c) -
                    2.0 * hpi - (a * tha + b * thb + c * thc) / R;
  const double Aa = 0.5 * (R2 - a * a) * tha - 0.5 * (b * zab + c * zac) + b * c;
  const double Ab = 0.5 * (R2 - b * b) * thb - 0.5 * (a * zab + c * zbc) + a * c;
  const double Ac = 0.5 * (R2 - c * c) * thc - 0.5 * (a * zac + b * zbc) + a * b;
  return (R2 * R * om - a * Aa - b * Ab - c * Ac) / 3.0;
}

// covered fraction of the unit cell centred at offset off from the centre:
// each axis interval is reflected onto the non-negative half-axis (split at
// 0 when it straddles it) and the box volume is the alternating sum of the
// corner functions over its 2^dim corners
__device__ __forceinline__ double exact_cell_fraction(const int dim, const double R, const double* off) {
  double lo[3][2], hi[3][2];
  int np[3] = {1, 1, 1};
  for (int d = 0; d < 3; d++) {
    const double l = off[d] - 0.5, h = off[d] + 0.5;
    if (d >= dim) { lo[d][0] = 0.0; hi[d][0] = 0.0; continue; }
    if (l >= 0.0) { lo[d][0] = l; hi[d][0] = h; }
    else if (h <= 0.0) { lo[d][0] = -h; hi[d][0] = -l; }
    else { lo[d][0] = 0.0; hi[d][0] = -l; lo[d][1] = 0.0; hi[d][1] = h; np[d] = 2; }
  }
  double sum = 0.0;
  for (int ia = 0; ia < np[0]; ia++)
    for (int ib = 0; ib < np[1]; ib++)
      for (int ic = 0; ic < (dim == 3 ? np[2] : 1); ic++)
        for (int s = 0; s < (dim == 3 ? 8 : 4); s++) {
          const int sx = s & 1, sy = (s >> 1) & 1, sz = (s >> 2) & 1;
          const double x = sx ? hi[0][ia] : lo[0][ia], y = sy ? hi[1][ib] : lo[1][ib];
          const double vv = dim == 3 ? corner_volume(R, x, y, sz ? hi[2][ic] : lo[2][ic]) : corner_area(R, x, y);
          sum += ((sx + sy + sz) & 1) ? -vv : vv;
        }
  return sum;
}

// --------------------------------------------------------------------------
// Eq. 6: covered fraction from a table over the cell's offset from the
// centre, for one particle radius R.  With the sorted offsets a >= b (>= c)
// >= 0 the table runs over
//   2D: r = |(a,b)| in [R - sqrt(2)/2, R + sqrt(2)/2] (kTabR2 points),
//       t = b/a in [0, 1] (kTabT2 points);
//   3D: r = |(a,b,c)| in [R - sqrt(3)/2, R + sqrt(3)/2] (kTabR3), s = |(b,c)|/a
//       in [0, sqrt(2)] (kTabS3), t = c/b in [0, 1] (kTabT3),
// entries = exact fractions at the grid points (FP32), and a cell takes the
// (bi/tri)linear interpolation, every FP32 operation rounded on its own (no
// contraction), so that any IEEE implementation of these steps gives the
// same value.  Only cells that meet the surface use the table; cells inside
// take 1 and cells outside 0 as in the exact rasteriser.
// --------------------------------------------------------------------------
constexpr int kTabR2 = 256, kTabT2 = 128;
constexpr int kTabR3 = 96, kTabS3 = 64, kTabT3 = 48;

__device__ __forceinline__ float tab_lerp(const float x, const float y, const float w) {
  return __fadd_rn(__fmul_rn(__fsub_rn(1.f, w), x), __fmul_rn(w, y));
}

// index and weight of coordinate x on a grid lo + i h, i = 0..n-1
__device__ __forceinline__ float tab_coord(const float x, const float lo, const float h, const int n, int& i) {
  float f = __fdiv_rn(__fsub_rn(x, lo), h);
  f = fminf(fmaxf(f, 0.f), (float)(n - 1));
  int k = (int)f;
  k = k > n - 2 ? n - 2 : k;
  i = k;
  return __fsub_rn(f, (float)k);
}

// off: the cell centre's offset from the particle centre, each component
// computed in FP64 and rounded to FP32
template <int DIM>
__device__ __forceinline__ float eps_table_lookup(const View& v, const float* off) {
  float a = fabsf(off[0]), b = fabsf(off[1]), c = DIM == 3 ? fabsf(off[2]) : 0.f;
  float t0;
  if (a < b) { t0 = a; a = b; b = t0; }
  if (DIM == 3) {
    if (b < c) { t0 = b; b = c; c = t0; }
    if (a < b) { t0 = a; a = b; b = t0; }
  }
  const float* T = v.eps_tab;
  if (DIM == 2) {
    const float r = __fsqrt_rn(__fadd_rn(__fmul_rn(a, a), __fmul_rn(b, b)));
    const float t = a > 0.f ? __fdiv_rn(b, a) : 0.f;
    int i, j;
    const float wr = tab_coord(r, v.tab_lo_r, v.tab_h_r, kTabR2, i);
    const float wt = tab_coord(t, 0.f, v.tab_h_t, kTabT2, j);
    const float* q = T + i * kTabT2 + j;
    return tab_lerp(tab_lerp(q[0], q[1], wt), tab_lerp(q[kTabT2], q[kTabT2 + 1], wt), wr);
  }
  const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(a, a), __fmul_rn(b, b)), __fmul_rn(c, c));
  const float r = __fsqrt_rn(r2);
  const float s = a > 0.f ? __fdiv_rn(__fsqrt_rn(__fadd_rn(__fmul_rn(b, b), __fmul_rn(c, c))), a) : 0.f;
  const float t = b > 0.f ? __fdiv_rn(c, b) : 0.f;
  int i, j, k;
  const float wr = tab_coord(r, v.tab_lo_r, v.tab_h_r, kTabR3, i);
  const float ws = tab_coord(s, 0.f, v.tab_h_s, kTabS3, j);
  const float wt = tab_coord(t, 0.f, v.tab_h_t, kTabT3, k);
  const float* q = T + (i * kTabS3 + j) * kTabT3 + k;
  const int dj = kTabT3, di = kTabS3 * kTabT3;
  const float c0 = tab_lerp(tab_lerp(q[0], q[1], wt), tab_lerp(q[dj], q[dj + 1], wt), ws);
  const float c1 = tab_lerp(tab_lerp(q[di], q[di + 1], wt), tab_lerp(q[di + dj], q[di + dj + 1], wt), ws);
  return tab_lerp(c0, c1, wr);
}

// one CTA per particle (block-uniform p); smem = dynamic shared memory of the
// size raster_bytes gives
template <int DIM, typename T, bool TABLE = false>
__device__ __forceinline__ void eps_raster_particle(const View& v, const int p, const RasterSmem cap,
                                                    unsigned char* smem) {
  __syncthreads();  // the block may still be reading the previous particle's tables
  const double R64 = v.rad[p];
  const T R = from_f64<T>(R64);
  const double c[3] = {v.pos[3 * p], v.pos[3 * p + 1], v.pos[3 * p + 2]};
  int lo[3] = {0, 0, 0}, ne[3] = {1, 1, 1};
  // a non-finite (or runaway) centre is reported and the particle covers no
  // cell: its box is recorded empty so the next clear walks nothing, and no
  // index is formed from it (block-uniform)
  bool bad = false;
#pragma unroll
  for (int d = 0; d < DIM; d++) bad |= !(fabs(c[d]) <= kPosLimit);
  if (bad) {
    if (threadIdx.x == 0) {
      for (int d = 0; d < 6; d++) v.lo[6 * p + d] = 0;
      atomicOr(v.err, ERR_NONFINITE);
    }
    return;
  }
#pragma unroll
  for (int d = 0; d < DIM; d++) {
    lo[d] = (int)ceil(c[d] - R64 - 0.5);
    ne[d] = (int)floor(c[d] + R64 + 0.5) - lo[d] + 1;
  }
  // value lists per axis: |cell boundary - centre| (ne+1 of them), then 0
  const int tx = ne[0] + 2, ty = ne[1] + 2, tz = DIM == 3 ? ne[2] + 2 : 1;
  const int tsize = tx * ty * tz;
  const int ncell = ne[0] * ne[1] * ne[2];
  if (tsize > cap.tab_cap || ncell > cap.cell_cap || ne[0] > 62 || ne[1] > 62 || ne[2] > 62 ||
      (DIM == 3 && (tx * ty > cap.pair_cap || tx * tz > cap.pair_cap || ty * tz > cap.pair_cap))) {
    if (threadIdx.x == 0) atomicOr(v.err, ERR_OWNERS);  // radius beyond the launch's capacity
    return;
  }
  T* tab = reinterpret_cast<T*>(smem);
  T* pr = tab + cap.tab_cap;                          // 3D: 3 pair tables x 4 values
  int* clist = reinterpret_cast<int*>(pr + 12 * cap.pair_cap);
  int* cells = clist + cap.tab_cap;
  unsigned char* need = reinterpret_cast<unsigned char*>(cells + cap.cell_cap);
  __shared__ T bnd[3][64];  // signed boundary offsets
  __shared__ float bndf[3][64];
  __shared__ T val[3][64];  // value lists
  __shared__ T kax[3][64];  // 3D: v (3 R^2 - v^2) / 2 of every axis value v
  __shared__ T ax_s[2][64], ax_psi[2][64];  // 2D per-axis tables
  __shared__ float offc[TABLE ? 3 : 1][64];  // table: cell-centre offsets (FP64 difference, FP32)
  __shared__ int n_part, n_need, n_pin, cov_base, cov_wsum[4];
  // nodes whose first owner slot this particle claims (split collision):
  // one flag per cell of the box, compacted in box order (x fastest, then
  // y, then z) at the end, so that the list holds each particle's nodes in
  // row order and consecutive entries are mostly adjacent in memory
  const bool want_list = v.cov_list != nullptr && split_form(v.collide_variant);
  unsigned char* s_flag = smem + (TABLE ? 0 : raster_list_offset(cap, (int)sizeof(T)));
  const double R2 = R64 * R64;
  const float R2f = (float)R2;
  const T R2t = from_f64<T>(R2);

  if (threadIdx.x == 0) {
    for (int d = 0; d < 3; d++) {
      v.lo[6 * p + d] = lo[d];
      v.lo[6 * p + 3 + d] = ne[d];
    }
    n_part = 0;
    n_need = 0;
    n_pin = 0;
  }
  if (!rows_meet_slab(v, lo[1], ne[1])) return;  // another slab's particle (block-uniform)
  for (int t = threadIdx.x; t < 3 * 64; t += blockDim.x) {
    const int d = t / 64, i = t % 64;
    const T b = (d < DIM && i <= ne[d]) ? from_f64<T>(((double)(lo[d] + i) - 0.5) - c[d]) : T(0);
    bnd[d][i] = b;
    bndf[d][i] = to_f32(b);
    if constexpr (TABLE) offc[d][i] = (d < DIM && i < ne[d]) ? (float)((double)(lo[d] + i) - c[d]) : 0.f;
    val[d][i] = (d < DIM && i <= ne[d]) ? fabs(b) : T(0);
    if (DIM == 3) kax[d][i] = T(0.5) * val[d][i] * (T(3) * R * R - val[d][i] * val[d][i]);
  }
  if constexpr (!TABLE)
    for (int t = threadIdx.x; t < tsize; t += blockDim.x) need[t] = 0;
  if (want_list)
    for (int t = threadIdx.x; t < ncell; t += blockDim.x) s_flag[t] = 0;
  __syncthreads();

  // pass 1: full cells claim their node at once; partial cells are listed
  // and mark the corner values they combine
  // node offset of box cell (ci, cj, ck); false if the cell is not a node of
  // this lattice (beyond a wall, or outside this slab's computed rows)
  auto node_of = [&](int ci, int cj, int ck, long long& n) -> bool {
    int i = lo[0] + ci, j = lo[1] + cj, k = lo[2] + ck;
    if (v.wall_y) {
      if (j < 0 || j >= v.ny_glob) return false;
    } else {
      j = wrap_idx(j, v.ny_glob);
    }
    j -= v.ygo;  // local row; only this slab's computed rows
    if (j < v.y0 || j >= v.y0 + v.ny_c) return false;
    i = wrap_idx(i, v.nx);
    k = wrap_idx(k, v.nz);
    n = ((long long)k * v.ny + j) * v.pitch + i;
    return true;
  };
  auto claim = [&](int ci, int cj, int ck, T e) {
    long long n;
    if (!node_of(ci, cj, ck, n)) return;
#pragma unroll
    for (int s = 0; s < kMaxOwners; s++) {
      if (atomicCAS(&v.own[s][n], -1, p) == -1) {
        store_eps<T>(v.eps[s], n, e);
        if (s == 0 && want_list) s_flag[(ck * ne[1] + cj) * ne[0] + ci] = 1;
        return;
      }
    }
    atomicOr(v.err, ERR_OWNERS);
  };
  // the flagged cells in box order: a block scan of per-thread counts over
  // contiguous cell ranges, one reservation per particle in the global list
  auto flush_list = [&]() {
    if (!want_list) return;
    __syncthreads();
    const int per = (ncell + (int)blockDim.x - 1) / (int)blockDim.x;
    const int t0 = min((int)threadIdx.x * per, ncell), t1 = min(t0 + per, ncell);
    int c = 0;
    for (int t = t0; t < t1; t++) c += s_flag[t];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) cov_wsum[wid] = incl;
    __syncthreads();
    int wbase = 0, total = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
      wbase += w < wid ? cov_wsum[w] : 0;
      total += cov_wsum[w];
    }
    if (threadIdx.x == 0) cov_base = total > 0 ? atomicAdd(v.cov_count, total) : 0;
    __syncthreads();
    int o = cov_base + wbase + incl - c;
    for (int t = t0; t < t1; t++) {
      if (!s_flag[t]) continue;
      const int ci = t % ne[0], cj = (t / ne[0]) % ne[1], ck = t / (ne[0] * ne[1]);
      long long n = 0;
      node_of(ci, cj, ck, n);
      v.cov_list[o++] = (int)n;
    }
  };
  const FastDiv3 cdiv(ne[0], ne[1]);
  for (int t = threadIdx.x; t < ncell; t += blockDim.x) {
    int idx[3];
    cdiv.split(t, idx[0], idx[1], idx[2]);
    const int cls = classify_cell<T>(bnd, bndf, idx, DIM, R2t, R2f);
    if (cls == 0) continue;
    if (cls == 1) {
      claim(idx[0], idx[1], idx[2], T(1));
      continue;
    }
    if constexpr (TABLE) {  // Eq. 6
      float off[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int d = 0; d < DIM; d++) off[d] = offc[d][idx[d]];
      const float e = eps_table_lookup<DIM>(v, off);
      const float ec = e < 0.f ? 0.f : (e > 1.f ? 1.f : e);
      if (ec > 0.f) claim(idx[0], idx[1], idx[2], T(ec));
      continue;
    }
    cells[atomicAdd(&n_part, 1)] = idx[0] | (idx[1] << 8) | (idx[2] << 16);  // ne <= 62
    int al[2], ah[2], bl[2], bh[2], cl[2] = {0, 0}, ch[2] = {0, 0};
    const int na = split_axis<float>(bndf[0], idx[0], ne[0] + 1, al, ah);
    const int nb = split_axis<float>(bndf[1], idx[1], ne[1] + 1, bl, bh);
    const int nc = DIM == 3 ? split_axis<float>(bndf[2], idx[2], ne[2] + 1, cl, ch) : 1;
    for (int ia = 0; ia < na; ia++)
      for (int ib = 0; ib < nb; ib++)
        for (int ic = 0; ic < nc; ic++) {
          const int xs[2] = {al[ia], ah[ia]}, ys[2] = {bl[ib], bh[ib]}, zs[2] = {cl[ic], ch[ic]};
          for (int s = 0; s < (DIM == 3 ? 8 : 4); s++)
            need[(zs[(s >> 2) & 1] * ty + ys[(s >> 1) & 1]) * tx + xs[s & 1]] = 1;
        }
  }
  if constexpr (TABLE) {
    flush_list();
    return;
  }
  // per-axis (2D) or per-pair (3D) angle tables
  const T hpi = T(1.57079632679489661923);
  if (DIM == 2) {
    for (int t = threadIdx.x; t < tx + ty; t += blockDim.x) {
      const int d = t < tx ? 0 : 1, i = t < tx ? t : t - tx;
      const T u = val[d][i];
      const T su = u < R ? sqrt((R - u) * (R + u)) : T(0);
      ax_s[d][i] = su;
      ax_psi[d][i] = atan2_q1(su, u);
    }
  } else {
    // entries whose edge line meets the ball are listed first (the list
    // shares the corner list's space, built later) and then evaluated by
    // consecutive threads, so that no lane idles through the square root
    // and arctangents of its neighbours; the others are the limit z -> 0
    // of the angles, zero
    const int axes[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    const int n01 = tx * ty, n02 = tx * tz, n12 = ty * tz;
    const FastDiv dx(tx), dy(ty);
    auto pair_entry = [&](const int t, int& g, int& r, T& u, T& w) -> T {
      g = t < n01 ? 0 : (t < n01 + n02 ? 1 : 2);
      r = t - (g == 0 ? 0 : (g == 1 ? n01 : n01 + n02));
      const FastDiv& dv = g == 2 ? dy : dx;
      const int j = dv.div(r), i = r - j * (int)dv.d;
      u = val[axes[g][0]][i];
      w = val[axes[g][1]][j];
      return (R * R - u * u) - w * w;
    };
    for (int t = threadIdx.x; t < n01 + n02 + n12; t += blockDim.x) {
      int g, r;
      T u, w;
      if (pair_entry(t, g, r, u, w) > T(0)) {
        clist[atomicAdd(&n_pin, 1)] = t;
      } else {
        T* e = pr + 4 * (g * cap.pair_cap + r);
        e[0] = e[1] = e[2] = e[3] = T(0);
      }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < n_pin; q += blockDim.x) {
      int g, r;
      T u, w;
      const T z = sqrt(pair_entry(clist[q], g, r, u, w));
      T* e = pr + 4 * (g * cap.pair_cap + r);
      e[0] = (u * w) * z;
      e[1] = atan2_q1(R * z, u * w);
      e[2] = atan2_q1(z, u);
      e[3] = atan2_q1(z, w);
    }
  }
  __syncthreads();
  // needed corners inside the ball are listed (the others are zero), so
  // that the closed forms below run on consecutive threads
  const FastDiv3 tdiv(tx, ty);
  auto corner_inside = [&](const int t) -> bool {
    int i, j, k;
    tdiv.split(t, i, j, k);
    const T a = val[0][i], b = val[1][j];
    if (DIM == 2) return a * a + b * b < R * R;
    const T cc = val[2][k];
    return (a * a + b * b) + cc * cc < R * R;
  };
  for (int t = threadIdx.x; t < tsize; t += blockDim.x) {
    if (!need[t]) continue;
    if (corner_inside(t)) clist[atomicAdd(&n_need, 1)] = t;
    else tab[t] = T(0);
  }
  __syncthreads();

  // pass 2: the needed corner values.  3D: with the face angles
  // th_a = s_a - pi/2 (s_a the sum of the two vertex angles on the face
  // X = a), the solid angle Omega = sum(alpha) - pi - (a th_a + b th_b +
  // c th_c) / R and the face areas A_a = (R^2 - a^2) th_a / 2 -
  // (b z_ab + c z_ac) / 2 + b c, the divergence form 3P = R^3 Omega -
  // a A_a - b A_b - c A_c collects to
  //   3P = R^3 (sum(alpha) - pi) - sum_d k_d th_d + sum_pairs u v z_uv - 3abc,
  // k_d = v_d (3R^2 - v_d^2) / 2 per axis value, u v z_uv per pair entry.
  const T R3 = R * R * R;
  const T piR3 = T(3.14159265358979323846) * R3;
  for (int q = threadIdx.x; q < n_need; q += blockDim.x) {
    const int t = clist[q];
    int i, j, k;
    tdiv.split(t, i, j, k);
    const T a = val[0][i], b = val[1][j];
    T out;
    if (DIM == 2) {
      out = T(0.5) * R * R * (ax_psi[0][i] + ax_psi[1][j] - hpi) -
            T(0.5) * (a * ax_s[0][i] + b * ax_s[1][j]) + a * b;
    } else {
      const T cc = val[2][k];
      const T* ab = pr + 4 * (0 * cap.pair_cap + j * tx + i);
      const T* ac = pr + 4 * (1 * cap.pair_cap + k * tx + i);
      const T* bc = pr + 4 * (2 * cap.pair_cap + k * ty + j);
      const T ka = kax[0][i], kb = kax[1][j], kc = kax[2][k];
      T t3 = fma(R3, (ab[1] + ac[1]) + bc[1], -piR3);
      t3 = fma(-ka, ab[3] + ac[3], t3);
      t3 = fma(-kb, ab[2] + bc[3], t3);
      t3 = fma(-kc, ac[2] + bc[2], t3);
      t3 = fma(hpi, (ka + kb) + kc, t3);
      t3 += (ab[0] + ac[0]) + bc[0];
      t3 = fma(T(-3) * (a * b), cc, t3);
      out = t3 * T(1.0 / 3.0);
    }
    tab[t] = out;
  }
  __syncthreads();

  // pass 3: partially covered cells
  for (int q = threadIdx.x; q < n_part; q += blockDim.x) {
    const int t = cells[q];
    const int idx[3] = {t & 0xff, (t >> 8) & 0xff, t >> 16};
    int al[2], ah[2], bl[2], bh[2], cl[2] = {0, 0}, ch[2] = {0, 0};
    const int na = split_axis<float>(bndf[0], idx[0], ne[0] + 1, al, ah);
    const int nb = split_axis<float>(bndf[1], idx[1], ne[1] + 1, bl, bh);
    const int nc = DIM == 3 ? split_axis<float>(bndf[2], idx[2], ne[2] + 1, cl, ch) : 1;
    T sum = T(0);
    for (int ia = 0; ia < na; ia++)
      for (int ib = 0; ib < nb; ib++)
        for (int ic = 0; ic < nc; ic++) {
          const int xs[2] = {al[ia], ah[ia]}, ys[2] = {bl[ib], bh[ib]}, zs[2] = {cl[ic], ch[ic]};
          for (int s = 0; s < (DIM == 3 ? 8 : 4); s++) {
            const int sx = s & 1, sy = (s >> 1) & 1, sz = (s >> 2) & 1;
            const T vv = tab[(zs[sz] * ty + ys[sy]) * tx + xs[sx]];
            sum += ((sx + sy + sz) & 1) ? -vv : vv;
          }
        }
    const T e = sum < T(0) ? T(0) : (sum > T(1) ? T(1) : sum);
    if (e > T(0)) claim(idx[0], idx[1], idx[2], e);
  }
  flush_list();
}

static inline RasterSmem raster_caps(int dim, double rmax) {
  const int nmax = (int)(2.0 * rmax) + 3;
  const int t = nmax + 2;
  RasterSmem c;
  c.tab_cap = dim == 3 ? t * t * t : t * t;
  c.pair_cap = dim == 3 ? t * t : 0;
  c.cell_cap = dim == 3 ? nmax * nmax * nmax : nmax * nmax;
  return c;
}

// the covered-node flags: one byte per cell of the box
static inline long long raster_list_bytes(int dim, double rmax) {
  return ((long long)raster_caps(dim, rmax).cell_cap + 15) & ~15LL;
}

static inline long long raster_bytes(int dim, int esz, double rmax) {
  const RasterSmem c = raster_caps(dim, rmax);
  return (long long)raster_list_offset(c, esz) + raster_list_bytes(dim, rmax);
}

}  // namespace lbm
