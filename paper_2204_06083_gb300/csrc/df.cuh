// Double-float arithmetic on the FP32 pipe.
//
// A double-float (DF) value is the unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi) / 2: about 48 significant bits, against 53 for
// FP64, from FP32 instructions only.  GB300 issues FP64 FMAs, adds and
// float <-> double conversions at under 2 lanes per clock per SM against about
// 116 for FP32 FMAs, so an outer Krylov iteration kept in DF runs at memory
// speed where the same iteration in FP64 is bound by the FP64 pipe.
//
// The building blocks are the error-free transformations of the
// double-double literature, written here for FP32: Knuth's TwoSum (s + e =
// a + b exactly, any magnitudes), Dekker's FastTwoSum (the same when |a| >=
// |b|) and the exact product p + e = a b from one FMA.  Every operation uses
// the _rn intrinsics, which the compiler never contracts into FMAs or
// reassociates: a contracted a * b + c would break the exactness the
// transformations rely on.  The compound operations (DF + DF with both
// components' errors carried, DF x DF) follow the standard double-double
// constructions (Dekker 1971; Hida, Li and Bailey 2001).
//
// The functions are __host__ __device__ so that a plain C++ build can check
// them against exact rational arithmetic on the CPU.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define DF_FN __host__ __device__ __forceinline__
#else
#include <cmath>
#define DF_FN inline
#endif

namespace ebk {

struct DF {
  float hi, lo;
};

#if defined(__CUDA_ARCH__)
DF_FN float df_fadd(float a, float b) { return __fadd_rn(a, b); }
DF_FN float df_fsub(float a, float b) { return __fsub_rn(a, b); }
DF_FN float df_fmul(float a, float b) { return __fmul_rn(a, b); }
DF_FN float df_ffma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
#else
// host build (checks): compiled without FP contraction
DF_FN float df_fadd(float a, float b) { return a + b; }
DF_FN float df_fsub(float a, float b) { return a - b; }
DF_FN float df_fmul(float a, float b) { return a * b; }
DF_FN float df_ffma(float a, float b, float c) { return std::fma(a, b, c); }
#endif

// s + e = a + b exactly (Knuth)
DF_FN void two_sum(float a, float b, float& s, float& e) {
  s = df_fadd(a, b);
  const float bv = df_fsub(s, a);
  const float av = df_fsub(s, bv);
  e = df_fadd(df_fsub(a, av), df_fsub(b, bv));
}

// s + e = a + b exactly when |a| >= |b| or a = 0 (Dekker)
DF_FN void fast_two_sum(float a, float b, float& s, float& e) {
  s = df_fadd(a, b);
  e = df_fsub(b, df_fsub(s, a));
}

// p + e = a b exactly (barring underflow)
DF_FN void two_prod(float a, float b, float& p, float& e) {
  p = df_fmul(a, b);
  e = df_ffma(a, b, -p);
}

DF_FN DF df_make(float v) { return DF{v, 0.0f}; }
DF_FN DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }

// a + b with the rounding errors of both components carried (accurate under
// cancellation)
DF_FN DF df_add(DF a, DF b) {
  float s, e, t, f;
  two_sum(a.hi, b.hi, s, e);
  two_sum(a.lo, b.lo, t, f);
  e = df_fadd(e, t);
  fast_two_sum(s, e, s, e);
  e = df_fadd(e, f);
  fast_two_sum(s, e, s, e);
  return DF{s, e};
}
DF_FN DF df_sub(DF a, DF b) { return df_add(a, df_neg(b)); }

// a + b with the low parts added in FP32 (two fewer error-free steps than
// df_add): accurate to about 2^-48 (|a| + |b|), so for sums that do not cancel
// (the p and q recurrences, x += alpha p, accumulations)
DF_FN DF df_add_fast(DF a, DF b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = df_fadd(e, df_fadd(a.lo, b.lo));
  fast_two_sum(s, e, s, e);
  return DF{s, e};
}

// s += a b for DF a, b: the exact product of the high parts (FMA), the cross
// terms in FP32, one TwoSum into s and a renormalisation
DF_FN void df_acc_prod(DF& s, DF a, DF b) {
  const float p = df_fmul(a.hi, b.hi);
  float pe = df_ffma(a.hi, b.hi, -p);
  pe = df_ffma(a.hi, b.lo, pe);
  pe = df_ffma(a.lo, b.hi, pe);
  float t, e;
  two_sum(s.hi, p, t, e);
  e = df_fadd(e, df_fadd(s.lo, pe));
  fast_two_sum(t, e, s.hi, s.lo);
}
// s += a b for DF a and FP32 b
DF_FN void df_acc_prod_f(DF& s, DF a, float b) {
  const float p = df_fmul(a.hi, b);
  float pe = df_ffma(a.hi, b, -p);
  pe = df_ffma(a.lo, b, pe);
  float t, e;
  two_sum(s.hi, p, t, e);
  e = df_fadd(e, df_fadd(s.lo, pe));
  fast_two_sum(t, e, s.hi, s.lo);
}

// Cascaded summation of FP32 values (Ogita, Rump and Oishi's Sum2): the
// running FP32 sum s with the exact error of every addition (TwoSum)
// collected in c; df_sum2_end gives (s + c) as a DF.  Accurate to about
// 2^-48 of the sum of magnitudes.
struct Sum2 {
  float s, c;
};
DF_FN Sum2 sum2_start(float v) { return Sum2{v, 0.0f}; }
DF_FN void sum2_add(Sum2& a, float v) {
  float e;
  two_sum(a.s, v, a.s, e);
  a.c = df_fadd(a.c, e);
}

// p - (a.s + a.c) for an exact product p + pe (two_prod), as a DF: the
// stencil value D_k z_k - sum of the neighbour values
DF_FN DF df_prod_minus_sum2(float p, float pe, const Sum2& a) {
  float t, e;
  two_sum(p, -a.s, t, e);
  e = df_fadd(e, df_fsub(pe, a.c));
  fast_two_sum(t, e, t, e);
  return DF{t, e};
}

// a + b for an FP32 b
DF_FN DF df_add_f(DF a, float b) {
  float s, e;
  two_sum(a.hi, b, s, e);
  e = df_fadd(e, a.lo);
  fast_two_sum(s, e, s, e);
  return DF{s, e};
}

// a b
DF_FN DF df_mul(DF a, DF b) {
  float p, e;
  two_prod(a.hi, b.hi, p, e);
  e = df_ffma(a.hi, b.lo, e);
  e = df_ffma(a.lo, b.hi, e);
  fast_two_sum(p, e, p, e);
  return DF{p, e};
}

// a b for an FP32 b
DF_FN DF df_mul_f(DF a, float b) {
  float p, e;
  two_prod(a.hi, b, p, e);
  e = df_ffma(a.lo, b, e);
  fast_two_sum(p, e, p, e);
  return DF{p, e};
}

// a b for two FP32 numbers (exact)
DF_FN DF df_prod(float a, float b) {
  float p, e;
  two_prod(a, b, p, e);
  return DF{p, e};
}

// the DF nearest to an FP64 value (two FP64 roundings), and back
DF_FN DF df_from_double(double v) {
  const float hi = (float)v;
  return DF{hi, (float)(v - (double)hi)};
}
DF_FN double df_to_double(DF a) { return (double)a.hi + (double)a.lo; }

}  // namespace ebk

#if defined(__CUDACC__)
namespace ebk {
// Sum of v over the CTA in DF (xor shuffles -- df_add is commutative bit for
// bit, so every lane of a warp holds the same sum -- then the warps in order);
// thread 0 holds the result.  sm: blockDim.x / 32 slots.
__device__ __forceinline__ DF df_block_sum_df(DF v, DF* sm) {
  for (int o = 16; o > 0; o >>= 1) {
    const DF w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = df_add(v, w);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sm[w] = v;
  __syncthreads();
  DF s{0.0f, 0.0f};
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s = df_add(s, sm[i]);
  return s;
}
// the same rounded to FP64 (thread 0)
__device__ __forceinline__ double df_block_sum(DF v, DF* sm) { return df_to_double(df_block_sum_df(v, sm)); }

// reduction partials of the DF iteration: a DF in the 8 bytes of a slot of
// the partials array (of doubles)
__device__ __forceinline__ void df_part_store(double* part, int64_t i, DF v) {
  reinterpret_cast<float2*>(part)[i] = make_float2(v.hi, v.lo);
}
__device__ __forceinline__ DF df_part_load(const double* part, int64_t i) {
  const float2 t = reinterpret_cast<const float2*>(part)[i];
  return DF{t.x, t.y};
}
// sum of n DF partials in a fixed order, the same in every CTA, in DF on the
// FP32 pipe and rounded to FP64 once; thread 0 holds the result
__device__ __forceinline__ double df_sum_parts(const double* part, int n, DF* sm) {
  DF a{0.0f, 0.0f};
  for (int i = threadIdx.x; i < n; i += blockDim.x) a = df_add(a, df_part_load(part, i));
  return df_block_sum(a, sm);
}

// the DF pair (node, node + 1) of a DF vector stored in a buffer of doubles
// (element i at bytes 8 i .. 8 i + 7: hi, lo); node even
__device__ __forceinline__ void df_ld2(const double* v, int32_t node, DF& a, DF& b) {
  const float4 t = __ldg(reinterpret_cast<const float4*>(v + node));
  a = DF{t.x, t.y};
  b = DF{t.z, t.w};
}
__device__ __forceinline__ void df_ld2_rw(const double* v, int32_t node, DF& a, DF& b) {
  const float4 t = *reinterpret_cast<const float4*>(v + node);
  a = DF{t.x, t.y};
  b = DF{t.z, t.w};
}
__device__ __forceinline__ void df_st2(double* v, int32_t node, DF a, DF b) {
  *reinterpret_cast<float4*>(v + node) = make_float4(a.hi, a.lo, b.hi, b.lo);
}
}  // namespace ebk
#endif
