// Double-FP32 arithmetic for the FP64-accuracy collision and rasteriser of
// the pair storage, on the FP32 pipe.
//
// A value is the unevaluated sum h + l of two FP32 numbers with |l| about
// half an FP32 ulp of h (a few ulps between renormalisations, see
// LBM_DF_LAZY): 48 significant bits.  The operations are the
// error-free transformations of the double-double literature written for
// FP32 pairs: Knuth's TwoSum, Dekker's Fast2Sum, and the exact product error
// through FMA (Dekker 1971; Hida, Li and Bailey, "Algorithms for quad-double
// precision floating point arithmetic", 2001).  Every step uses the _rn
// intrinsics, so the compiler neither contracts nor reorders them.
//
// Why: GB300 issues FP32 at 64 times its FP64 rate.  The collision works on
// the deviation g = f - w rho0 (|g| is 1e-2 w or less), stored as such a
// pair, so 48 bits of g are more than the 53 bits of f: the update is as
// accurate as the FP64 update of f while no FP64 instruction runs.  The
// FP64 <-> pair conversions (covered fractions, and the collision forms that
// update covered nodes in FP64) are integer bit operations.
#pragma once
#include <cuda_runtime.h>

#ifndef LBM_DF_LAZY
#define LBM_DF_LAZY 1
#endif

namespace lbm {

struct DF {
  float h, l;
  __device__ __forceinline__ DF() {}
  __host__ __device__ __forceinline__ constexpr DF(float a, float b) : h(a), l(b) {}
  __device__ __forceinline__ DF(float a) : h(a), l(0.f) {}
  __device__ __forceinline__ DF(int a) : h((float)a), l(0.f) {}
  // compile-time constants (folded by the compiler; at run time this would
  // use the FP64 pipe, so run-time doubles go through df_from_bits)
  __host__ __device__ __forceinline__ constexpr explicit DF(double d)
      : h((float)d), l((float)(d - (double)(float)d)) {}
  // a b + c with one normalisation; found by argument-dependent lookup only
  // (does not hide ::fma for other types)
  friend __device__ __forceinline__ DF fma(const DF a, const DF b, const DF c) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    const float s = __fadd_rn(p, c.h);
    const float bb = __fsub_rn(s, p);
    float t = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(c.h, bb));
    t = __fadd_rn(t, __fadd_rn(e, c.l));
#if LBM_DF_LAZY
    return DF(s, t);
#else
    const float r = __fadd_rn(s, t);
    return DF(r, __fsub_rn(t, __fsub_rn(r, s)));
#endif
  }
  // |a| and sqrt(a) (a >= 0): found by argument-dependent lookup only
  friend __device__ __forceinline__ DF fabs(const DF a) { return a.h < 0.f ? DF(-a.h, -a.l) : a; }
  // FP32 root of h refined by one Newton step in pair arithmetic (Karp and
  // Markstein): s = s0 + (a - s0^2) / (2 s0), the residual a - s0^2 exact
  // through the FMA product error
  friend __device__ __forceinline__ DF sqrt(const DF x) {
    // normalised first: after a cancellation l may hold much of the value,
    // and the FP32 seed must be close to the whole value
    const float xs = __fadd_rn(x.h, x.l);
    const DF a(xs, __fsub_rn(x.l, __fsub_rn(xs, x.h)));
    if (!(a.h > 0.f)) return DF(0.f, 0.f);
    const float s0 = __fsqrt_rn(a.h);
    const float p = __fmul_rn(s0, s0);
    const float e = __fmaf_rn(s0, s0, -p);
    const float res = __fadd_rn(__fsub_rn(__fsub_rn(a.h, p), e), a.l);  // a - s0^2 (a.h - p is exact)
    const float corr = __fmul_rn(res, __fmul_rn(0.5f, __frcp_rn(s0)));
    const float hs = __fadd_rn(s0, corr);
    return DF(hs, __fsub_rn(corr, __fsub_rn(hs, s0)));
  }
};

__device__ __forceinline__ DF fast_two_sum(const float a, const float b) {
  const float s = __fadd_rn(a, b);
  return DF(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// with LBM_DF_LAZY the sums and products skip the final Fast2Sum: l may
// grow to a few ulps of h (the value is still h + l); stores, reciprocals and
// comparisons normalise first
__device__ __forceinline__ DF df_norm(const DF a) {
#if LBM_DF_LAZY
  return fast_two_sum(a.h, a.l);
#else
  return a;
#endif
}

__device__ __forceinline__ DF operator+(const DF a, const DF b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));  // TwoSum error
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
#if LBM_DF_LAZY
  return DF(s, e);
#else
  return fast_two_sum(s, e);
#endif
}
__device__ __forceinline__ DF operator-(const DF a) { return DF(-a.h, -a.l); }
__device__ __forceinline__ DF operator-(const DF a, const DF b) { return a + (-b); }

__device__ __forceinline__ DF operator*(const DF a, const DF b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);  // exact product error
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
#if LBM_DF_LAZY
  return DF(p, e);
#else
  return fast_two_sum(p, e);
#endif
}
__device__ __forceinline__ DF operator*(const DF a, const float b) {
  const float p = __fmul_rn(a.h, b);
  float e = __fmaf_rn(a.h, b, -p);
  e = __fmaf_rn(a.l, b, e);
#if LBM_DF_LAZY
  return DF(p, e);
#else
  return fast_two_sum(p, e);
#endif
}

// 1 / a: FP32 reciprocal of h refined by one Newton step in pair arithmetic
__device__ __forceinline__ DF rcp(const DF x) {
  const DF a = df_norm(x);
  const float r = __frcp_rn(a.h);
  float t = __fmaf_rn(-a.h, r, 1.f);  // 1 - h r, exact
  t = __fmaf_rn(-a.l, r, t);
  return fast_two_sum(r, __fmul_rn(r, t));
}
__device__ __forceinline__ DF operator/(const DF a, const DF b) { return a * rcp(b); }

__device__ __forceinline__ DF& operator+=(DF& a, const DF b) { return a = a + b; }
__device__ __forceinline__ DF& operator-=(DF& a, const DF b) { return a = a - b; }
__device__ __forceinline__ DF& operator*=(DF& a, const DF b) { return a = a * b; }

__device__ __forceinline__ bool operator<(const DF x, const DF y) {
  const DF a = df_norm(x), b = df_norm(y);
  return a.h < b.h || (a.h == b.h && a.l < b.l);
}
__device__ __forceinline__ bool operator>(const DF a, const DF b) { return b < a; }
__device__ __forceinline__ bool operator>=(const DF a, const DF b) { return !(a < b); }
__device__ __forceinline__ bool operator<=(const DF a, const DF b) { return !(b < a); }
__device__ __forceinline__ bool operator==(const DF x, const DF y) {
  const DF a = df_norm(x), b = df_norm(y);
  return a.h == b.h && a.l == b.l;
}
__device__ __forceinline__ bool operator!=(const DF a, const DF b) { return !(a == b); }

__device__ __forceinline__ DF shfl_xor(const DF a, const int d) {
  return DF(__shfl_xor_sync(0xffffffffu, a.h, d), __shfl_xor_sync(0xffffffffu, a.l, d));
}
__device__ __forceinline__ DF shfl_down(const DF a, const int d) {
  return DF(__shfl_down_sync(0xffffffffu, a.h, d), __shfl_down_sync(0xffffffffu, a.l, d));
}

// FP64 -> pair with integer operations: h = the significand truncated to 24
// bits, l = the remaining 29 bits (rounded to 24 bits, 2^-48 of the value);
// |d| < 2^-126 gives 0, |d| < 2^-74 drops l, non-finite gives NaN.
__device__ __forceinline__ DF df_from_bits(const double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sgn = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  const unsigned hb = sgn | ((unsigned)(e - 896) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const float scale = __uint_as_float((unsigned)(e >= 949 ? e - 948 : 0) << 23);  // 2^(e-1075), or 0
  const float l = __uint_as_float(__float_as_uint(__fmul_rn(__uint2float_rn(lo & 0x1fffffffu), scale)) | sgn);
  if (e < 897) return DF(0.f, 0.f);
  if (e > 1150) return DF(__uint_as_float(0x7fc00000u), 0.f);
  return DF(__uint_as_float(hb), l);
}

// pair -> FP64 with integer operations: h converted exactly, then l added as
// an integer number of FP64 ulps of h (rounded to nearest), which is the
// correctly rounded h + l for |l| <= ulp32(h) / 2; below a power of two the
// ulp halves.  |h| < 2^-74 drops l; zero or subnormal h gives a signed zero.
__device__ __forceinline__ double df_to_bits(const DF xx) {
  const DF x = df_norm(xx);
  const unsigned H = __float_as_uint(x.h);
  const int eh = (int)((H >> 23) & 0xffu);
  const unsigned mh = H & 0x7fffffu;
  const unsigned long long hi_bits =
      ((unsigned long long)((H & 0x80000000u) | ((unsigned)(eh + 896) << 20) | (mh >> 3)) << 32) |
      ((unsigned long long)(mh & 7u) << 29);
  const bool opp = ((__float_as_uint(x.l) ^ H) & 0x80000000u) != 0u;
  const int sc = 306 - eh + ((mh == 0u && opp) ? 1 : 0);  // biased exponent of 2^(179 - eh (+1))
  const float scale = __uint_as_float((unsigned)(sc < 254 ? sc : 254) << 23);
  const long long K = eh >= 53 ? (long long)__float2int_rn(__fmul_rn(fabsf(x.l), scale)) : 0LL;
  unsigned long long bits = opp ? hi_bits - (unsigned long long)K : hi_bits + (unsigned long long)K;
  if (eh == 0) bits = (unsigned long long)(H & 0x80000000u) << 32;
  if (eh == 255) bits = 0x7ff8000000000000ull;
  return __longlong_as_double((long long)bits);
}

// Two pair values (the same node quantity of two adjacent nodes) processed
// together by the paired FP32 instructions of this GPU (FADD2 / FMUL2 /
// FFMA2): every step of the pair operations above, lane by lane, each
// rounded on its own, so DF2 gives bitwise the results of two DF
// computations.  Subtraction is a fused multiply-add by -1 (one rounding,
// the same value as the subtraction).
struct DF2 {
  float2 h, l;
  __device__ __forceinline__ DF2() {}
  __device__ __forceinline__ DF2(float2 a, float2 b) : h(a), l(b) {}
  __device__ __forceinline__ DF2(const DF a) : h(make_float2(a.h, a.h)), l(make_float2(a.l, a.l)) {}
  __device__ __forceinline__ DF2(int a) : h(make_float2((float)a, (float)a)), l(make_float2(0.f, 0.f)) {}
  __device__ __forceinline__ explicit DF2(double d) : DF2(DF(d)) {}
  __device__ __forceinline__ DF lo() const { return DF(h.x, l.x); }
  __device__ __forceinline__ DF hi() const { return DF(h.y, l.y); }
  friend __device__ DF2 df2_fma(const DF2 a, const DF2 b, const DF2 c);
  friend __device__ __forceinline__ DF2 fma(const DF2 a, const DF2 b, const DF2 c) { return df2_fma(a, b, c); }
};

__device__ __forceinline__ float2 f2_sub(const float2 a, const float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 f2_neg(const float2 a) { return __fmul2_rn(a, make_float2(-1.f, -1.f)); }

__device__ __forceinline__ DF2 fast_two_sum2(const float2 a, const float2 b) {
  const float2 s = __fadd2_rn(a, b);
  return DF2(s, f2_sub(b, f2_sub(s, a)));
}

__device__ __forceinline__ DF2 df_norm(const DF2 a) {
#if LBM_DF_LAZY
  return fast_two_sum2(a.h, a.l);
#else
  return a;
#endif
}

__device__ __forceinline__ DF2 operator+(const DF2 a, const DF2 b) {
  const float2 s = __fadd2_rn(a.h, b.h);
  const float2 bb = f2_sub(s, a.h);
  float2 e = __fadd2_rn(f2_sub(a.h, f2_sub(s, bb)), f2_sub(b.h, bb));
  e = __fadd2_rn(e, __fadd2_rn(a.l, b.l));
#if LBM_DF_LAZY
  return DF2(s, e);
#else
  return fast_two_sum2(s, e);
#endif
}
__device__ __forceinline__ DF2 operator-(const DF2 a) { return DF2(f2_neg(a.h), f2_neg(a.l)); }
__device__ __forceinline__ DF2 operator-(const DF2 a, const DF2 b) { return a + (-b); }

__device__ __forceinline__ DF2 operator*(const DF2 a, const DF2 b) {
  const float2 p = __fmul2_rn(a.h, b.h);
  float2 e = __ffma2_rn(a.h, b.h, f2_neg(p));
  e = __ffma2_rn(a.h, b.l, e);
  e = __ffma2_rn(a.l, b.h, e);
#if LBM_DF_LAZY
  return DF2(p, e);
#else
  return fast_two_sum2(p, e);
#endif
}

// a b + c with one normalisation: found by argument-dependent lookup only,
// through the friend declaration in DF2 (does not hide ::fma for other types)
__device__ __forceinline__ DF2 df2_fma(const DF2 a, const DF2 b, const DF2 c) {
  const float2 p = __fmul2_rn(a.h, b.h);
  float2 e = __ffma2_rn(a.h, b.h, f2_neg(p));
  e = __ffma2_rn(a.h, b.l, e);
  e = __ffma2_rn(a.l, b.h, e);
  const float2 s = __fadd2_rn(p, c.h);
  const float2 bb = f2_sub(s, p);
  float2 t = __fadd2_rn(f2_sub(p, f2_sub(s, bb)), f2_sub(c.h, bb));
  t = __fadd2_rn(t, __fadd2_rn(e, c.l));
#if LBM_DF_LAZY
  return DF2(s, t);
#else
  const float2 r = __fadd2_rn(s, t);
  return DF2(r, f2_sub(t, f2_sub(r, s)));
#endif
}

// 1 / a lane by lane (the hardware reciprocal has no paired form)
__device__ __forceinline__ DF2 rcp(const DF2 x) {
  const DF2 a = df_norm(x);
  const float2 r = make_float2(__frcp_rn(a.h.x), __frcp_rn(a.h.y));
  float2 t = __ffma2_rn(f2_neg(a.h), r, make_float2(1.f, 1.f));  // 1 - h r, exact
  t = __ffma2_rn(f2_neg(a.l), r, t);
  return fast_two_sum2(r, __fmul2_rn(r, t));
}

}  // namespace lbm
