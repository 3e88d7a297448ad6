// boys_ds.cuh -- double-single ("float-float") arithmetic and the FP64-accurate
// Boys function / primitive prologue of the mixed-precision path.
//
// GB300 executes FP64 at 1/62 of the FP32 rate (measured), and the
// per-primitive-quartet prologue (argument, prefactor, Boys function, erfc
// difference) is the bulk of the FP64 work.  The mixed path therefore carries
// these quantities as unevaluated sums hi + lo of two FP32 numbers (about 44
// significant bits after rounding errors), with error-free transformations
// built from the FP32 pipe: Knuth's TwoSum, Dekker's Fast-TwoSum and the FMA
// form of TwoProduct.  Terms of a Taylor series that are below 1e-4 of the sum
// are evaluated in plain FP32.  The Boys values agree with the FP64 evaluator
// to about 1e-12 relative (tested).  All additions and multiplications inside
// the transformations use explicit round-to-nearest intrinsics so the
// compiler cannot contract them into FMAs.
#pragma once
#include <cuda_runtime.h>

#include "eri_common.cuh"

namespace hfx {

struct ds {
  float hi, lo;
};

__device__ __forceinline__ ds ds_from_double(double d) {
  const float h = __double2float_rn(d);
  return {h, __double2float_rn(d - (double)h)};
}

// Knuth TwoSum: s + e == a + b exactly.
__device__ __forceinline__ ds two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// Dekker Fast-TwoSum (|a| >= |b|).
__device__ __forceinline__ ds fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ds ds_add(ds x, ds y) {
  const ds s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ ds ds_sub(ds x, ds y) { return ds_add(x, {-y.hi, -y.lo}); }

// Products are left unnormalised: (p, e) with p the FP32 product of the high
// parts and e the rest, |e| within a few ulp of p.  Every operation here
// reads such a pair correctly (the next product drops only the lo * lo term,
// the next sum renormalises), so the final renormalisation of a product is
// left out.
__device__ __forceinline__ ds ds_mul(ds x, ds y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return {p, e};
}

__device__ __forceinline__ ds ds_mulf(ds x, float f) {
  const float p = __fmul_rn(x.hi, f);
  float e = __fmaf_rn(x.hi, f, -p);
  e = __fmaf_rn(x.lo, f, e);
  return {p, e};
}

__device__ __forceinline__ ds ds_addf(ds x, float f) {
  const ds s = two_sum(x.hi, f);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, x.lo));
}

// 1/x: FP32 seed, one Newton-Raphson step r + r (1 - x r) in double-single.
__device__ __forceinline__ ds ds_rcp(ds x) {
  const float r = __frcp_rn(x.hi);
  const ds e = ds_addf(ds_mulf({-x.hi, -x.lo}, r), 1.0f);  // 1 - x r
  return ds_addf(ds_mulf(e, r), r);
}

// 1/sqrt(x): FP32 seed, one Newton step y + y (1 - x y^2) / 2 in double-single.
__device__ __forceinline__ ds ds_rsqrt(ds x) {
  const float y = rsqrtf(x.hi);
  const ds xy2 = ds_mulf(ds_mulf(x, y), y);
  const ds e = ds_addf({-xy2.hi, -xy2.lo}, 1.0f);  // 1 - x y^2
  return ds_addf(ds_mulf(e, 0.5f * y), y);
}

// Double-single Boys table: the FP64 Taylor tables (eri_common.cuh) split into
// hi/lo floats, tabds[((L * kBoysNT + k) * 8 + j) * 2 + {0,1}].
// Reciprocals 1/(2m+1), m = 0..8, as double-single constants.
__device__ __forceinline__ ds inv_odd(int m) {
  // hi = fl(1/(2m+1)), lo = fl(1/(2m+1) - hi), precomputed
  const float hi[9] = {1.000000000e+00f, 3.333333433e-01f, 2.000000030e-01f, 1.428571492e-01f, 1.111111119e-01f,
                       9.090909362e-02f, 7.692307979e-02f, 6.666667014e-02f, 5.882352963e-02f};
  const float lo[9] = {0.0f, -9.934107759e-09f, -2.980232283e-09f, -6.386212004e-09f, -8.278422947e-10f,
                       -2.709302116e-09f, -2.865607973e-09f, -3.476937627e-09f, -2.191347243e-10f};
  return {hi[m], lo[m]};
}

// F_0..F_L at T (double-single).  T < 60: Taylor expansion of F_L about the
// nearest grid point T_k (|x| = |T_k - T| <= 1/32; terms j = 3..6 in FP32,
// at most 5e-6 of the sum, j = 0..2 in double-single), exp(-T) = exp(-T_k)
// exp(x) (terms x^3.. in FP32), downward recursion
// F_m = (2T F_{m+1} + exp(-T)) / (2m+1).
// T >= 60: F_0 = sqrt(pi)/2 T^{-1/2}, F_{m+1} = F_m (2m+1) / (2T).
template <int L>
__device__ __forceinline__ void boys_ds(const float* __restrict__ tab, ds T, ds* F) {
  if (T.hi < (float)kBoysTmax) {
    const int it = __float2int_rn(T.hi * 16.0f);
#ifdef HFX_CHECKED
    if (!HFX_IN(it, kBoysNT, "boys_ds grid", L)) return;
#endif
    const float Tk = (float)it * 0.0625f;
    const ds xs = two_sum(Tk, -T.hi);
    const ds x = fast_two_sum(xs.hi, __fadd_rn(xs.lo, -T.lo));
    const float4* r4 = reinterpret_cast<const float4*>(tab + ((size_t)L * kBoysNT + it) * 16);
    const float4 q01 = __ldg(r4), q23 = __ldg(r4 + 1), q45 = __ldg(r4 + 2), q6e = __ldg(r4 + 3);
    // c_j = (hi, lo): c0 = q01.x,y  c1 = q01.z,w  c2 = q23.x,y  c3 = q23.z,w  c4 = q45.x,y  c5 = q45.z,w
    //                 c6 = q6e.x,y  exp(-T_k) = q6e.z,w
    float r = fmaf(q6e.x, x.hi, q45.z);
    r = fmaf(r, x.hi, q45.x);
    r = fmaf(r, x.hi, q23.z);
    ds f = ds_add(ds_mulf(x, r), {q23.x, q23.y});
    f = ds_add(ds_mul(f, x), {q01.z, q01.w});
    f = ds_add(ds_mul(f, x), {q01.x, q01.y});
    F[L] = f;
    if (L > 0) {
      // exp(x) = 1 + x (1 + x (1/2 + x t)),  t = 1/6 + x/24 + x^2/120 + x^3/720 + x^4/5040 (FP32)
      float t = fmaf(x.hi, 1.0f / 5040.0f, 1.0f / 720.0f);
      t = fmaf(t, x.hi, 1.0f / 120.0f);
      t = fmaf(t, x.hi, 1.0f / 24.0f);
      t = fmaf(t, x.hi, 1.0f / 6.0f);
      ds e = ds_addf(ds_mulf(x, t), 0.5f);
      e = ds_addf(ds_mul(e, x), 1.0f);
      e = ds_addf(ds_mul(e, x), 1.0f);
      const ds ex = ds_mul(e, {q6e.z, q6e.w});
      const ds t2 = {2.0f * T.hi, 2.0f * T.lo};
#pragma unroll
      for (int m = L - 1; m >= 0; --m) F[m] = ds_mul(ds_add(ds_mul(t2, F[m + 1]), ex), inv_odd(m));
    }
  } else {
    const ds y = ds_rsqrt(T);
    F[0] = ds_mul(y, {8.862269521e-01f, -2.662319964e-08f});  // sqrt(pi)/2
    const ds h = ds_mulf(ds_mul(y, y), 0.5f);  // 1/(2T)
#pragma unroll
    for (int m = 0; m < L; ++m) F[m + 1] = ds_mulf(ds_mul(F[m], h), (float)(2 * m + 1));
  }
}

// Primitive-quartet prologue of the mixed path, FP64-accurate in
// double-single: T = rho |PQ|^2 from double-single P, Q, p, q; the Boys
// function(s); the erfc difference F_m(T) - f^{m+1/2} F_m(f T) taken before
// rounding; then G_m = pref * D_m, with the prefactor
// 2 pi^{5/2} K_ab K_cd / (p q sqrt(p+q)) also in double-single, rounded to
// FP32 once (w2 = omega^2 as a double-single pair formed once per launch;
// K_ab c_a c_b / p were formed in FP64 when the pairs were built and are read
// as FP32).  Also returns FP32 1/(p+q) and PQ.
template <int L>
__device__ __forceinline__ void prologue_ds(const float* __restrict__ tab, int kernel, ds w2,
                                            const PrimPair& pb, const PrimPair& pk, float* G, float& inv_s,
                                            float* PQf) {
  const ds p = {pb.pf, pb.plo}, q = {pk.pf, pk.plo};
  const ds s = ds_add(p, q);
  const ds ys = ds_rsqrt(s);    // (p+q)^{-1/2}, for the prefactor
  const ds rs = ds_mul(ys, ys);  // 1/(p+q)
  const ds rho = ds_mul(ds_mul(p, q), rs);
  ds pq2 = {0.f, 0.f};
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    const ds d0 = two_sum(pb.Phi[x], -pk.Phi[x]);
    const ds d = fast_two_sum(d0.hi, __fadd_rn(d0.lo, __fsub_rn(pb.Plo[x], pk.Plo[x])));
    PQf[x] = d.hi;
    pq2 = ds_add(pq2, ds_mul(d, d));
  }
  const ds T = ds_mul(rho, pq2);
  inv_s = __fadd_rn(rs.hi, rs.lo);  // rounded once (rs is an unnormalised product)
  // prefactor 2 pi^{5/2} K_ab K_cd / sqrt(p+q) in double-single, so that G_m
  // is the FP32 rounding of an accurate product (an FP32 product with an
  // approximate reciprocal square root would carry the same small relative
  // error into every integral)
  const ds pref = ds_mulf(ds_mulf(ds_mul({3.498683548e+01f, 1.175513376e-06f}, ys), pb.kpf), pk.kpf);
  ds F[L + 1];
  if (kernel != kErf) {
    boys_ds<L>(tab, T, F);
    if (kernel == kCoulomb) {
#pragma unroll
      for (int m = 0; m <= L; ++m) {
        const ds g = ds_mul(pref, F[m]);
        G[m] = g.hi + g.lo;
      }
      return;
    }
  }
  // f = w^2 / (w^2 + rho): f^{1/2} = w^2 (w^2 (w^2 + rho))^{-1/2}, f = (f^{1/2})^2
  const ds c0 = ds_mul(w2, ds_rsqrt(ds_mul(w2, ds_add(w2, rho))));
  const ds f = ds_mul(c0, c0);
  ds Fw[L + 1];
  boys_ds<L>(tab, ds_mul(f, T), Fw);
  ds c = c0;  // f^{1/2}, then f^{m+1/2}
#pragma unroll
  for (int m = 0; m <= L; ++m) {
    const ds cw = ds_mul(c, Fw[m]);
    const ds d = (kernel == kErfc) ? ds_sub(F[m], cw) : cw;
    const ds g = ds_mul(pref, d);
    G[m] = g.hi + g.lo;
    c = ds_mul(c, f);
  }
}

}  // namespace hfx
