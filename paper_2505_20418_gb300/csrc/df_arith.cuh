// Double-float arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum h + l of two floats. Sums and products are
// built from error-free transformations: Knuth's TwoSum (a + b = s + e
// exactly, any order of magnitude), Dekker's Fast2Sum (the same when |a| >=
// |b|) and the FMA-based exact product (a b = p + e with e = fma(a, b, -p)).
// Products drop the lo x lo term and round the cross terms once, so a chain
// of a few operations keeps ~46 bits (relative error ~1e-14): far beyond what
// the FP64 parity bar of the forces (1e-10) needs, at a fraction of the cost
// of the FP64 pipe on GB300 (2 FP64 operations per clock per SM against 128
// FP32 lanes; an FP64 warp instruction occupies the pipe 16 cycles).
//
// The explicit __f*_rn intrinsics keep the compiler from contracting or
// reassociating the compensation terms.
#pragma once

namespace maze {

struct dfl {
  float h, l;
};

__device__ __forceinline__ dfl df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

// |a| >= |b| (or a == 0)
__device__ __forceinline__ dfl df_fast_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dfl df_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return df_fast_sum(p, e);
}

__device__ __forceinline__ dfl df_sqr(dfl a) {
  const float p = __fmul_rn(a.h, a.h);
  float e = __fmaf_rn(a.h, a.h, -p);
  e = __fmaf_rn(__fadd_rn(a.h, a.h), a.l, e);
  return df_fast_sum(p, e);
}

// a + b (the "sloppy" sum: exact TwoSum of the hi parts, the lo parts added
// once; loses accuracy only when a and b nearly cancel, which the callers'
// terms do not at the precision asked of them)
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  const dfl s = df_two_sum(a.h, b.h);
  return df_fast_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}

__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.h, -a.l}; }

// a < b for normalised pairs
__device__ __forceinline__ bool df_less(dfl a, dfl b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }

// exp(x) by Tang's table-driven method (P. T. P. Tang, ACM TOMS 15, 1989)
// carried out in double-float: x = (64 m + j) ln2/64 + t with |t| <= ln2/128,
// exp(x) = 2^m 2^(j/64) e^t. tab[j] = 2^(j/64) as (hi, lo). ln2/64 is split
// in three floats, the first with 11 significant bits so that n C1 is exact
// for |n| < 2^13 (|x| < 88); e^t - 1 = t + t^2/2 + t^3/6 + t^4/24 + t^5/120
// (the remainder t^6/720 is below 4e-17), its first two terms in
// double-float, the rest in FP32 (their size keeps them below 1e-15 of the
// result); 2^m is set in the exponent field. |x| >= 87 returns 0 (x < 0) or
// infinity; below x = -70 the lo part falls into FP32's subnormal range and
// the result keeps fewer bits (the pair kernel's arguments stay above -30).
__device__ __forceinline__ dfl df_exp(dfl x, const float2* __restrict__ tab) {
  if (fabsf(x.h) >= 87.f) return {x.h < 0.f ? 0.f : __int_as_float(0x7f800000), 0.f};
  const float kd = __fmaf_rn(x.h, 0x1.715476p+6f, 0x1.8p23f);   // 64/ln2, then round to an integer
  const int k = __float_as_int(kd) - 0x4b400000;                // (the low bits of 1.5 2^23 + n)
  const float kf = __fsub_rn(kd, 0x1.8p23f);
  const float u = __fmaf_rn(-kf, 0x1.62cp-7f, x.h);              // exact
  const dfl v = df_two_prod(kf, 0x1.217f7ep-18f);
  const dfl th = df_two_sum(u, -v.h);
  const dfl tx = df_two_sum(th.h, x.l);                          // (x.l reaches 2^-18 for |x| < 128)
  const float tl = __fmaf_rn(-kf, -0x1.c610cap-43f, __fadd_rn(__fsub_rn(th.l, v.l), tx.l));
  const dfl t = df_fast_sum(tx.h, tl);
  // e^t - 1
  const dfl q = df_two_prod(t.h, t.h);
  const float ql = __fmaf_rn(__fadd_rn(t.h, t.h), t.l, q.l);
  float c = __fmaf_rn(t.h, 1.f / 120.f, 1.f / 24.f);
  c = __fmaf_rn(t.h, c, 1.f / 6.f);
  const float h3 = __fmul_rn(__fmul_rn(q.h, c), t.h);          // t^3/6 + t^4/24 + t^5/120
  const dfl p0 = df_fast_sum(t.h, __fmul_rn(0.5f, q.h));
  const float pl = __fadd_rn(p0.l, __fadd_rn(t.l, __fmaf_rn(0.5f, ql, h3)));
  // 2^(j/64) (1 + p)
  const float2 T = __ldg(tab + (k & 63));
  const dfl w = df_two_prod(T.x, p0.h);
  const dfl R = df_fast_sum(T.x, w.h);
  const float Rl = __fadd_rn(R.l, __fadd_rn(w.l, __fmaf_rn(T.x, pl, __fmaf_rn(T.y, p0.h, T.y))));
  const float s = __int_as_float(((k >> 6) + 127) << 23);
  return {__fmul_rn(R.h, s), __fmul_rn(Rl, s)};
}

}  // namespace maze
