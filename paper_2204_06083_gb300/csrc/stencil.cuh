// The EB stencil at computational points: eq. 3 with beta = 1 and the
// line-by-line diagonal of Sec. 2.1.  (sigma I + A) x at CP k is
//   (D_k x_k - sum over CP neighbours x_j) / h^2 + sigma x_k,
// D_k = 2 dim at interior CPs (code 0x80) and sum_s c_s at cut CPs (read from
// diag).  The code byte's low six bits mark BP neighbours, whose values are
// never used (the caller's entries off the CPs are ignored).
//
// Pair form: one thread evaluates two x-adjacent nodes.  All loads of the
// pair's stencil are issued at once, predicated on indices only (never on a
// loaded value); the code bytes then select which neighbours enter the sum.
// Only cut CPs (a few per cent) make a dependent load, of their D_k.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "tiles.cuh"

namespace ebk {

constexpr uint32_t CODE_CP_BIT = 0x80;  // the CP bit of a node code byte

template <class T>
struct AccOf {
  using type = float;
};
template <>
struct AccOf<double> {
  using type = double;
};

template <class A>
struct Two {
  A x, y;
};

// load policies: read-only path (data not written during the launch) and the
// L2-coherent path (data written by other CTAs earlier in the same launch)
struct LdRO {
  __device__ __forceinline__ static double ld(const double* p) { return __ldg(p); }
  __device__ __forceinline__ static float ld(const float* p) { return __ldg(p); }
  __device__ __forceinline__ static float ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
  __device__ __forceinline__ static Two<double> ld2(const double* p) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    return {v.x, v.y};
  }
  __device__ __forceinline__ static Two<float> ld2(const float* p) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return {v.x, v.y};
  }
  __device__ __forceinline__ static Two<float> ld2(const __nv_bfloat16* p) {
    const float2 v = __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(p)));
    return {v.x, v.y};
  }
};
struct LdCG {
  __device__ __forceinline__ static double ld(const double* p) { return __ldcg(p); }
  __device__ __forceinline__ static float ld(const float* p) { return __ldcg(p); }
  __device__ __forceinline__ static Two<double> ld2(const double* p) {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
    return {v.x, v.y};
  }
  __device__ __forceinline__ static Two<float> ld2(const float* p) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return {v.x, v.y};
  }
};

__device__ __forceinline__ void st_val(double* p, double v) { *p = v; }
__device__ __forceinline__ void st_val(float* p, float v) { *p = v; }
__device__ __forceinline__ void st_val(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void st2(double* p, double a, double b) { *reinterpret_cast<double2*>(p) = make_double2(a, b); }
__device__ __forceinline__ void st2(float* p, float a, float b) { *reinterpret_cast<float2*>(p) = make_float2(a, b); }
__device__ __forceinline__ void st2(__nv_bfloat16* p, float a, float b) {
  *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
}

__device__ __forceinline__ Two<double> ld2d(const double* p) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  return {v.x, v.y};
}

// D_k x_k - sum of the CP-neighbour values, for the pair (node, node + 1).
// nn = number of grid nodes (even); the pair's codes c0, c1 are given.  diag
// is the FP64 D_k array for FP64 kernels and its FP32 copy for the others, so
// that FP32 kernels run no FP64 instruction (GB300's FP64 pipe is narrow).
template <int DIM, class L, class T, class DT>
__device__ __forceinline__ void stencil_pair(const T* __restrict__ x, int32_t node, int32_t nn, uint32_t c0,
                                             uint32_t c1, const DT* __restrict__ diag, int32_t sy, int32_t sz,
                                             Two<typename AccOf<T>::type>& xc, Two<typename AccOf<T>::type>& core) {
  using A = typename AccOf<T>::type;
  const Two<A> z{0, 0};
  xc = L::ld2(x + node);
  const A left = node > 0 ? L::ld(x + node - 1) : (A)0;
  const A right = node + 2 < nn ? L::ld(x + node + 2) : (A)0;
  const Two<A> dn = node >= sy ? L::ld2(x + node - sy) : z;
  const Two<A> up = node + sy < nn ? L::ld2(x + node + sy) : z;
  Two<A> bk = z, fr = z;
  if (DIM == 3) {
    bk = node >= sz ? L::ld2(x + node - sz) : z;
    fr = node + sz < nn ? L::ld2(x + node + sz) : z;
  }
  A s0 = ((c0 & 1) ? (A)0 : left) + ((c0 & 2) ? (A)0 : xc.y);
  A s1 = ((c1 & 1) ? (A)0 : xc.x) + ((c1 & 2) ? (A)0 : right);
  s0 += ((c0 & 4) ? (A)0 : dn.x) + ((c0 & 8) ? (A)0 : up.x);
  s1 += ((c1 & 4) ? (A)0 : dn.y) + ((c1 & 8) ? (A)0 : up.y);
  if (DIM == 3) {
    s0 += ((c0 & 16) ? (A)0 : bk.x) + ((c0 & 32) ? (A)0 : fr.x);
    s1 += ((c1 & 16) ? (A)0 : bk.y) + ((c1 & 32) ? (A)0 : fr.y);
  }
  const A D0 = (c0 & 0x7F) ? (A)__ldg(diag + node) : (A)(2 * DIM);
  const A D1 = (c1 & 0x7F) ? (A)__ldg(diag + node + 1) : (A)(2 * DIM);
  core.x = D0 * xc.x - s0;
  core.y = D1 * xc.y - s1;
}

// The same with a variable coefficient (eq. 3): each CP neighbour enters with
// the beta of the half point between it and the node, and D_k = sum_s beta_s
// c_s is read at every CP.  bt[a] holds beta at node + h/2 e_a.
template <int DIM, class L, class T, class DT>
__device__ __forceinline__ void stencil_pair_beta(const T* __restrict__ x, int32_t node, int32_t nn, uint32_t c0,
                                                  uint32_t c1, const DT* __restrict__ diag, int32_t sy, int32_t sz,
                                                  const DT* const* bt, Two<typename AccOf<T>::type>& xc,
                                                  Two<typename AccOf<T>::type>& core) {
  using A = typename AccOf<T>::type;
  const Two<A> z{0, 0};
  xc = L::ld2(x + node);
  const A left = node > 0 ? L::ld(x + node - 1) : (A)0;
  const A right = node + 2 < nn ? L::ld(x + node + 2) : (A)0;
  const Two<A> dn = node >= sy ? L::ld2(x + node - sy) : z;
  const Two<A> up = node + sy < nn ? L::ld2(x + node + sy) : z;
  const DT* bx = bt[0];
  const DT* by = bt[1];
  const A wl = node > 0 ? (A)__ldg(bx + node - 1) : (A)0;
  const A wm = (A)__ldg(bx + node);
  const A wr = node + 2 < nn ? (A)__ldg(bx + node + 1) : (A)0;
  const Two<A> wd = node >= sy ? Two<A>{(A)__ldg(by + node - sy), (A)__ldg(by + node - sy + 1)} : z;
  const Two<A> wu{(A)__ldg(by + node), (A)__ldg(by + node + 1)};
  A s0 = ((c0 & 1) ? (A)0 : wl * left) + ((c0 & 2) ? (A)0 : wm * xc.y);
  A s1 = ((c1 & 1) ? (A)0 : wm * xc.x) + ((c1 & 2) ? (A)0 : wr * right);
  s0 += ((c0 & 4) ? (A)0 : wd.x * dn.x) + ((c0 & 8) ? (A)0 : wu.x * up.x);
  s1 += ((c1 & 4) ? (A)0 : wd.y * dn.y) + ((c1 & 8) ? (A)0 : wu.y * up.y);
  if (DIM == 3) {
    const DT* bz = bt[2];
    const Two<A> bk = node >= sz ? L::ld2(x + node - sz) : z;
    const Two<A> fr = node + sz < nn ? L::ld2(x + node + sz) : z;
    const Two<A> wb = node >= sz ? Two<A>{(A)__ldg(bz + node - sz), (A)__ldg(bz + node - sz + 1)} : z;
    const Two<A> wf{(A)__ldg(bz + node), (A)__ldg(bz + node + 1)};
    s0 += ((c0 & 16) ? (A)0 : wb.x * bk.x) + ((c0 & 32) ? (A)0 : wf.x * fr.x);
    s1 += ((c1 & 16) ? (A)0 : wb.y * bk.y) + ((c1 & 32) ? (A)0 : wf.y * fr.y);
  }
  const A D0 = (c0 & CODE_CP_BIT) ? (A)__ldg(diag + node) : (A)0;
  const A D1 = (c1 & CODE_CP_BIT) ? (A)__ldg(diag + node + 1) : (A)0;
  core.x = D0 * xc.x - s0;
  core.y = D1 * xc.y - s1;
}

__device__ __forceinline__ const double* const* beta_ptrs(const TileView& tv, const double*) { return tv.beta64; }
__device__ __forceinline__ const float* const* beta_ptrs(const TileView& tv, const float*) { return tv.beta32; }

// stencil_pair on a tile view; DIM carrying DIM_VB selects, at compile time,
// the variable-coefficient form with the view's beta (kernels of beta = 1 keep
// their registers and instructions)
template <int DIM, class L, class T, class DT>
__device__ __forceinline__ void stencil_tv(const TileView& tv, const T* __restrict__ x, int32_t node, uint32_t c0,
                                           uint32_t c1, const DT* __restrict__ diag,
                                           Two<typename AccOf<T>::type>& xc, Two<typename AccOf<T>::type>& core) {
  if constexpr ((DIM & DIM_VB) != 0)
    stencil_pair_beta<dim_of(DIM), L>(x, node, tv.nn, c0, c1, diag, tv.sy, tv.sz, beta_ptrs(tv, diag), xc, core);
  else
    stencil_pair<dim_of(DIM), L>(x, node, tv.nn, c0, c1, diag, tv.sy, tv.sz, xc, core);
}

// the two code bytes of a pair
__device__ __forceinline__ void ld_codes(const uint8_t* __restrict__ code, int32_t node, uint32_t& c0, uint32_t& c1) {
  const uint32_t v = __ldg(reinterpret_cast<const unsigned short*>(code + node));
  c0 = v & 0xFFu;
  c1 = v >> 8;
}

// 1 / (sigma + D_k / h^2)
__device__ __forceinline__ double inv_diag(uint32_t c, const double* __restrict__ diag, int32_t node, double inv_h2,
                                           double sigma, double dinv_interior) {
  return (c & 0x7F) ? 1.0 / (sigma + __ldg(diag + node) * inv_h2) : dinv_interior;
}

}  // namespace ebk
