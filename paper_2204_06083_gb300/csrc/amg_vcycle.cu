// V-cycle of the smoothed-aggregation hierarchy (AMG preconditioner of
// Algorithm 1 step 4), in FP64, or in FP32 or BF16 storage with FP32
// arithmetic.
//
// Level 0 is matrix free on the grid (stencil.cuh), swept over the node pairs
// that hold a CP (EB_SWEEP); coarser levels use CSR.
// Smoother: Chebyshev polynomial of degree k for D^-1 A on [rho/30, 1.1 rho],
// one sweep before and one after the coarse correction; the first sweep
// starts from x = 0 and needs no operator apply.  The coarsest level is solved
// by its FP64 explicit inverse.  With FP32 / BF16 storage the right-hand side
// is rounded on entry and the result is widened to FP64 on exit (the last
// smoothing step writes FP64 directly); the outer PCG (eb_solve.cu) then uses
// the flexible (Polak-Ribiere) beta.  BF16 storage: level vectors and the
// values of A_l, P_l, R_l and D_l^-1 in bfloat16, every sum in FP32; the
// level-0 diagonal stays FP32.
#include "amg_internal.cuh"
#include "df.cuh"
#include "stencil.cuh"
#include "tma.cuh"

#include <algorithm>
#include <cmath>
#include <type_traits>

namespace ebk {

template <class V>
struct CsrV {
  int64_t n;
  const int32_t* rp;
  const int32_t* ci;
  const V* v;
};

// operator constants in the arithmetic type of the kernel
template <class A>
struct GOp {
  A inv_h2, sigma, dinv_int;
};

template <class A, class DT>
__device__ __forceinline__ A inv_diag_t(uint32_t c, const DT* __restrict__ diag, int32_t node, const GOp<A>& o) {
  if (!(c & 0x7F)) return o.dinv_int;
  return (A)1 / (o.sigma + (A)__ldg(diag + node) * o.inv_h2);
}

// per-tile shift of a batched view (unit spacing, sigma_g per geometry)
__device__ __forceinline__ GOp<float> tile_op(const TileView& tv, int64_t tt, GOp<float> o) {
  if (tv.tshift32) {
    const float2 t = __ldg(tv.tshift32 + tt);
    o.sigma = t.x;
    o.dinv_int = t.y;
  }
  return o;
}
__device__ __forceinline__ GOp<double> tile_op(const TileView& tv, int64_t tt, GOp<double> o) {
  if (tv.tshift64) {
    const double2 t = __ldg(tv.tshift64 + tt);
    o.sigma = t.x;
    o.dinv_int = t.y;
  }
  return o;
}

__device__ __forceinline__ void st2o(double* p, double a, double b) { st2(p, a, b); }
__device__ __forceinline__ void st2o(float* p, float a, float b) { st2(p, a, b); }
__device__ __forceinline__ void st2o(__nv_bfloat16* p, float a, float b) { st2(p, a, b); }

// conversions between the storage type and the arithmetic types
template <class To, class From>
__device__ __forceinline__ To cvt(From v) {
  return static_cast<To>(v);
}
template <>
__device__ __forceinline__ float cvt<float, __nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
template <>
__device__ __forceinline__ double cvt<double, __nv_bfloat16>(__nv_bfloat16 v) {
  return (double)__bfloat162float(v);
}
template <>
__device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16, float>(float v) {
  return __float2bfloat16_rn(v);
}
template <>
__device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16, double>(double v) {
  return __double2bfloat16(v);
}

// the operator constants at item tt_ of EB_SWEEP: per tile for a batched view
template <int DIM, class A>
__device__ __forceinline__ GOp<A> sweep_op(const TileView& tv, int64_t tt, const GOp<A>& o) {
  if constexpr ((DIM & DIM_LIST) != 0) return o;
  else return tile_op(tv, tt, o);
}

// the view without its CP pair list: EB_SWEEP then visits every pair of the
// active tiles
inline TileView tiles_only(TileView tv) {
  tv.pair_node = nullptr;
  tv.npairs = 0;
  return tv;
}

// level 0 ----------------------------------------------------------------
// b_out = (V) r; x = d = D^-1 b / theta.  RDF: r is a double-float vector
// (the DF outer iteration), of which the V-cycle takes the FP32 high part.
template <int DIM, class V, bool RDF = false>
__global__ void __launch_bounds__(TILE_NODES) k_g_cheb_first(TileView tv, const uint8_t* __restrict__ code,
                                                             const typename DiagOf<V>::type* __restrict__ diag,
                                                             GOp<typename AccOf<V>::type> o,
                                                             const double* __restrict__ r, V* __restrict__ b_out,
                                                             V* __restrict__ x, V* __restrict__ d,
                                                             typename AccOf<V>::type theta) {
  using A = typename AccOf<V>::type;
  EB_SWEEP(DIM, tv, node) {
    const GOp<A> ot = sweep_op<DIM>(tv, tt_, o);
    uint32_t c0, c1;
    ld_codes(code, node, c0, c1);
    A r0, r1;
    if constexpr (RDF) {
      DF a, b;
      df_ld2(r, node, a, b);
      r0 = (A)a.hi;
      r1 = (A)b.hi;
    } else {
      const Two<double> rv = LdRO::ld2(r + node);
      r0 = (A)rv.x;
      r1 = (A)rv.y;
    }
    const A b0 = (c0 & CODE_CP) ? r0 : (A)0, b1 = (c1 & CODE_CP) ? r1 : (A)0;
    if (b_out) st2o(b_out + node, b0, b1);
    const A v0 = (c0 & CODE_CP) ? inv_diag_t<A>(c0, diag, node, ot) * b0 / theta : (A)0;
    const A v1 = (c1 & CODE_CP) ? inv_diag_t<A>(c1, diag, node + 1, ot) * b1 / theta : (A)0;
    st2o(x + node, v0, v1);
    st2o(d + node, v0, v1);
  }
}

// The PCG's x += alpha h2 p, r -= alpha q, r'r (and, flexible, r'zold)
// partials (k_update_xr, same
// grid, same pair list and order: the same values and partials) followed, per
// node pair, by k_g_cheb_first on the new r: b_out = (V) r; x = d = D^-1 b /
// theta.  It runs over the CP pairs only (single grids): the entries of pairs
// without a CP are never read at a CP.
template <int DIM, class V>
__global__ void __launch_bounds__(TILE_NODES) k_update_first(PairList pl, PcgUpdate u, const uint8_t* __restrict__ code,
                                                             const typename DiagOf<V>::type* __restrict__ diag,
                                                             GOp<typename AccOf<V>::type> o, V* __restrict__ b_out,
                                                             V* __restrict__ x0, V* __restrict__ d,
                                                             typename AccOf<V>::type theta) {
  using A = typename AccOf<V>::type;
  __shared__ double sm[32];
  __shared__ double s_alpha;
  if (cta_done(u.sc)) {
    if (threadIdx.x == 0) u.rr_part[blockIdx.x] = 0.0;
    return;
  }
  const double alpha = pcg_alpha(u.sc, u.pq_part, u.nblk, sm, &s_alpha);
  const double ax = alpha * u.h2;  // q holds h^2 (sigma I + A) p
  double srr = 0.0, srzo = 0.0;
  EB_LIST_LOOP(pl, node) {
    const Two<double> rv = ld2d(u.r + node), qv = LdRO::ld2(u.q + node), pv = LdRO::ld2(u.p + node),
                      xv = ld2d(u.x + node);
    const double r0 = rv.x - alpha * qv.x, r1 = rv.y - alpha * qv.y;
    st2(u.x + node, xv.x + ax * pv.x, xv.y + ax * pv.y);
    st2(u.r + node, r0, r1);
    srr += r0 * r0 + r1 * r1;
    if (u.rzo_part) {
      const Two<double> zv = LdRO::ld2(u.z + node);
      srzo += r0 * zv.x + r1 * zv.y;
    }
    const GOp<A>& ot = o;
    uint32_t c0, c1;
    ld_codes(code, node, c0, c1);
    const A b0 = (c0 & CODE_CP) ? (A)r0 : (A)0, b1 = (c1 & CODE_CP) ? (A)r1 : (A)0;
    if (b_out) st2o(b_out + node, b0, b1);
    const A v0 = (c0 & CODE_CP) ? inv_diag_t<A>(c0, diag, node, ot) * b0 / theta : (A)0;
    const A v1 = (c1 & CODE_CP) ? inv_diag_t<A>(c1, diag, node + 1, ot) * b1 / theta : (A)0;
    st2o(x0 + node, v0, v1);
    st2o(d + node, v0, v1);
  }
  if (u.rzo_part) {
    const double t = block_sum(srzo, sm);
    if (threadIdx.x == 0) u.rzo_part[blockIdx.x] = t;
  }
  const double t = block_sum(srr, sm);
  if (threadIdx.x == 0) u.rr_part[blockIdx.x] = t;
}

// k_update_first for the DF outer iteration: x, r, p, q are double-float
// vectors (DF pairs in the buffers of doubles), z the FP32 output of the
// V-cycle, the reduction partials DF.  x += (alpha h2) p, r -= alpha q in DF,
// the r'r and r'zold partials summed in DF; the V-cycle's first step then
// takes the FP32 high part of the new r (x = d = D^-1 b (1 / theta)).
// one pair's inputs of k_update_first_df
struct UfIn {
  DF r0, r1, q0, q1, p0, p1, xa, xb;
  float2 zv;
  uint32_t c0, c1;
};

__device__ __forceinline__ void uf_load(UfIn& in, const PcgUpdate& u, const uint8_t* code, int32_t node) {
  df_ld2_rw(u.r, node, in.r0, in.r1);
  df_ld2(u.q, node, in.q0, in.q1);
  df_ld2(u.p, node, in.p0, in.p1);
  df_ld2_rw(u.x, node, in.xa, in.xb);
  in.zv = u.rzo_part ? __ldg(reinterpret_cast<const float2*>(reinterpret_cast<const float*>(u.z) + node))
                     : make_float2(0.0f, 0.0f);
  ld_codes(code, node, in.c0, in.c1);
}

// k_update_first for the DF outer iteration: x, r, p, q are double-float
// vectors (DF pairs in the buffers of doubles), z the FP32 output of the
// V-cycle, the reduction partials DF.  x += (alpha h2) p, r -= alpha q in DF,
// the r'r and r'zold partials summed in DF; the V-cycle's first step then
// takes the FP32 high part of the new r (x = d = D^-1 b (1 / theta)).  A
// thread's first pair is loaded before the partial sums that give alpha.
template <int DIM, class V>
__global__ void __launch_bounds__(TILE_NODES) k_update_first_df(PairList pl, PcgUpdate u, const uint8_t* __restrict__ code,
                                                                const typename DiagOf<V>::type* __restrict__ diag,
                                                                GOp<float> o, V* __restrict__ b_out,
                                                                V* __restrict__ x0, V* __restrict__ d,
                                                                float inv_theta) {
  __shared__ DF dsm[32];
  __shared__ DF s_a[2];
  if (cta_done(u.sc)) {
    if (threadIdx.x == 0) {
      df_part_store(u.rr_part, blockIdx.x, DF{0.0f, 0.0f});
      if (u.rzo_part) df_part_store(u.rzo_part, blockIdx.x, DF{0.0f, 0.0f});
    }
    return;
  }
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  UfIn in;
  int32_t node = li < pl.n ? __ldg(pl.node + li) : 0;
  if (li < pl.n) uf_load(in, u, code, node);
  // alpha from the DF p'q partials (FP64 scalars), split into DF once per CTA
  const double pq = df_sum_parts(u.pq_part, u.nblk, dsm);
  if (threadIdx.x == 0) {
    const double alpha = pcg_alpha_from(u.sc, pq);
    s_a[0] = df_from_double(alpha);
    s_a[1] = df_from_double(alpha * u.h2);
  }
  __syncthreads();
  const DF a_df = s_a[0], ax_df = s_a[1];
  DF srr{0.0f, 0.0f}, srzo{0.0f, 0.0f};
  while (li < pl.n) {
    const int64_t ln = li + step;
    const int32_t nnode = ln < pl.n ? __ldg(pl.node + ln) : 0;
    // the residual update cancels by design: the accurate DF sum
    const DF r0 = df_sub(in.r0, df_mul(a_df, in.q0)), r1 = df_sub(in.r1, df_mul(a_df, in.q1));
    df_st2(u.x, node, df_add_fast(in.xa, df_mul(ax_df, in.p0)), df_add_fast(in.xb, df_mul(ax_df, in.p1)));
    df_st2(u.r, node, r0, r1);
    df_acc_prod(srr, r0, r0);
    df_acc_prod(srr, r1, r1);
    if (u.rzo_part) {
      df_acc_prod_f(srzo, r0, in.zv.x);
      df_acc_prod_f(srzo, r1, in.zv.y);
    }
    const uint32_t c0 = in.c0, c1 = in.c1;
    const float b0 = (c0 & CODE_CP) ? r0.hi : 0.0f, b1 = (c1 & CODE_CP) ? r1.hi : 0.0f;
    if (b_out) st2o(b_out + node, b0, b1);
    const float v0 = (c0 & CODE_CP) ? inv_diag_t<float>(c0, diag, node, o) * b0 * inv_theta : 0.0f;
    const float v1 = (c1 & CODE_CP) ? inv_diag_t<float>(c1, diag, node + 1, o) * b1 * inv_theta : 0.0f;
    st2o(x0 + node, v0, v1);
    st2o(d + node, v0, v1);
    if (ln < pl.n) uf_load(in, u, code, nnode);
    li = ln;
    node = nnode;
  }
  if (u.rzo_part) {
    const DF t = df_block_sum_df(srzo, dsm);
    if (threadIdx.x == 0) df_part_store(u.rzo_part, blockIdx.x, t);
  }
  const DF t = df_block_sum_df(srr, dsm);
  if (threadIdx.x == 0) df_part_store(u.rr_part, blockIdx.x, t);
}

// res = D^-1 (b - A x); d = c1 d + c2 res; xo = x + d   (xo may be FP64).
// DOT = 1 (xo FP64, the V-cycle's output z): also the CTA's partial r.z,
// summed over its node pairs in loop order exactly as the PCG's own dot kernel
// does; DOT = 2 (xo FP32, r a double-float vector): the same partial summed
// and stored in DF.
template <int DIM, class V, class O, int DOT = 0>
__global__ void __launch_bounds__(TILE_NODES) k_g_cheb_step(TileView tv, const uint8_t* __restrict__ code,
                                                            const typename DiagOf<V>::type* __restrict__ diag,
                                                            GOp<typename AccOf<V>::type> o,
                                                            const V* __restrict__ b, const V* __restrict__ x,
                                                            O* __restrict__ xo, V* __restrict__ d,
                                                            typename AccOf<V>::type c1, typename AccOf<V>::type c2,
                                                            const double* __restrict__ r64 = nullptr,
                                                            double* __restrict__ part = nullptr) {
  using A = typename AccOf<V>::type;
  double srz = 0.0;
  DF srz_df{0.0f, 0.0f};
  EB_SWEEP(DIM, tv, node) {
    const GOp<A> ot = sweep_op<DIM>(tv, tt_, o);
    uint32_t k0, k1;
    ld_codes(code, node, k0, k1);
    Two<A> xc, core;
    stencil_tv<DIM, LdRO>(tv, x, node, k0, k1, diag, xc, core);
    const Two<A> bv = LdRO::ld2(b + node);
    Two<A> dv{0, 0};
    if (c1 != (A)0) {
      const Two<A> t = LdRO::ld2(d + node);
      dv = t;
    }
    const A res0 = inv_diag_t<A>(k0, diag, node, ot) * (bv.x - (core.x * ot.inv_h2 + ot.sigma * xc.x));
    const A res1 = inv_diag_t<A>(k1, diag, node + 1, ot) * (bv.y - (core.y * ot.inv_h2 + ot.sigma * xc.y));
    const A d0 = (k0 & CODE_CP) ? c1 * dv.x + c2 * res0 : (A)0;
    const A d1 = (k1 & CODE_CP) ? c1 * dv.y + c2 * res1 : (A)0;
    st2o(d + node, d0, d1);
    const A z0 = (k0 & CODE_CP) ? xc.x + d0 : (A)0, z1 = (k1 & CODE_CP) ? xc.y + d1 : (A)0;
    st2(xo + node, z0, z1);
    if constexpr (DOT == 1) {
      const Two<double> rv = LdRO::ld2(r64 + node);
      srz += rv.x * (double)z0 + rv.y * (double)z1;
    } else if constexpr (DOT == 2) {
      DF ra, rb;
      df_ld2(r64, node, ra, rb);
      df_acc_prod_f(srz_df, ra, (float)z0);
      df_acc_prod_f(srz_df, rb, (float)z1);
    }
  }
  if constexpr (DOT == 1) {
    __shared__ double sm[32];
    const double a = block_sum(srz, sm);
    if (threadIdx.x == 0) part[blockIdx.x] = a;
  } else if constexpr (DOT == 2) {
    __shared__ DF dsm[32];
    const DF a = df_block_sum_df(srz_df, dsm);
    if (threadIdx.x == 0) df_part_store(part, blockIdx.x, a);
  }
}

// Level-0 Chebyshev step on a tile view without a pair list (batched grids,
// 2D, FP32 storage), fed by tensor copies: per listed tile, one copy of the
// x box with its halo (tx + 8 x ty + 2 nodes from (x0 - 4, y0 - 1): the
// 16-byte aligned start left of the tile), and copies of the tile's b, d and
// code boxes, into a ring of TS_STAGES shared-memory stages; one thread of
// warp 4 issues them ahead while warps 0-3 (one node pair each) compute the
// step from shared memory and store d and x' directly.  The arithmetic is
// k_g_cheb_step's, operation for operation, so the results are the same bit
// for bit; copies beyond the grid read zeros, where that kernel reads zeros
// or values the node codes mask out.  Every wait is bounded: a wait that gives
// up raises a shared abort flag, every role leaves its loop, *err is set, and
// the copies in flight land (bounded wait) before the CTA ends.
constexpr int TS_STAGES = 4;
constexpr int TS_THREADS = 160;  // warps 0-3 compute, warp 4 copies
constexpr uint32_t TS_SPIN = 1u << 22;

struct TsMeta {
  int32_t base, lim;
  float sigma, dinv;
};

// shared-memory layout of one stage for tiles of tx x ty (x, b, d, code; 128-byte aligned)
struct TsLayout {
  int tx, ty, xw;  // xw = tx + 8: the x box width
  uint32_t off_b, off_d, off_c, stage;
  __host__ __device__ static uint32_t up128(uint32_t v) { return (v + 127u) & ~127u; }
  __host__ __device__ TsLayout(int tx_, int ty_) : tx(tx_), ty(ty_), xw(tx_ + 8) {
    off_b = up128((uint32_t)(xw * (ty + 2) * 4));
    off_d = off_b + up128((uint32_t)(tx * ty * 4));
    off_c = off_d + up128((uint32_t)(tx * ty * 4));
    stage = off_c + up128((uint32_t)(tx * ty));
  }
};

__device__ __forceinline__ bool ts_wait(uint32_t bar, uint32_t parity, volatile int* abort) {
  for (uint32_t it = 0; it < TS_SPIN; ++it) {
    uint32_t ok = 0;
    asm volatile(
        "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 63) == 63 && *abort) return false;
  }
  *abort = 1;
  return false;
}

__device__ __forceinline__ void ts_copy2d(uint32_t dst, const CUtensorMap* map, int cx, int cy, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(cx), "r"(cy), "r"(bar)
      : "memory");
}

__global__ void __launch_bounds__(TS_THREADS) k_g_cheb_step_tma(
    const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap bmap,
    const __grid_constant__ CUtensorMap dmap, const __grid_constant__ CUtensorMap cmap, TileView tv, int tx, int ty,
    const float* __restrict__ diag, GOp<float> o, float* __restrict__ xo, float* __restrict__ d, float c1, float c2,
    int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char ts_smem[];
  const TsLayout L(tx, ty);
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(ts_smem);
  unsigned char* tail = ts_smem + TS_STAGES * L.stage;
  TsMeta* meta = reinterpret_cast<TsMeta*>(tail);
  const uint32_t bars = sbase + TS_STAGES * L.stage + TS_STAGES * (uint32_t)sizeof(TsMeta);  // 8-byte aligned
  volatile int* abort = reinterpret_cast<volatile int*>(tail + TS_STAGES * sizeof(TsMeta) + 16 * TS_STAGES);
  auto full = [&](int st) { return bars + 8 * st; };
  auto empty = [&](int st) { return bars + 8 * (TS_STAGES + st); };
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool rd = c1 != 0.0f;
  if (tid == 0) {
    for (int st = 0; st < TS_STAGES; ++st) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full(st)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(empty(st)));  // one arrive per compute warp
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  const int64_t njob = tv.ntiles > (int64_t)blockIdx.x ? (tv.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int32_t S = tv.sy;
  if (warp == 4) {
    if (lane == 0) {
      const uint32_t bytes = (uint32_t)(L.xw * (ty + 2) * 4 + tx * ty * 4 * (rd ? 2 : 1) + tx * ty);
      int64_t k = 0;
      for (; k < njob; ++k) {
        const int st = (int)(k % TS_STAGES);
        const uint32_t u = (uint32_t)(k / TS_STAGES);
        if (u > 0 && !ts_wait(empty(st), (u - 1) & 1u, abort)) break;
        const int64_t tt = blockIdx.x + k * gridDim.x;
        const int32_t base = __ldg(tv.base + tt);
        const float2 sh = tv.tshift32 ? __ldg(tv.tshift32 + tt) : make_float2(o.sigma, o.dinv_int);
        meta[st] = TsMeta{base, __ldg(tv.lim + tt), sh.x, sh.y};
        const int x0 = base % S, y0 = base / S;
        const uint32_t sa = sbase + st * L.stage;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(full(st)), "r"(bytes) : "memory");
        ts_copy2d(sa, &xmap, x0 - 4, y0 - 1, full(st));
        ts_copy2d(sa + L.off_b, &bmap, x0, y0, full(st));
        if (rd) ts_copy2d(sa + L.off_d, &dmap, x0, y0, full(st));
        ts_copy2d(sa + L.off_c, &cmap, x0, y0, full(st));
      }
      // copies still in flight (an aborted run) land before the CTA ends
      for (int64_t q = k > TS_STAGES ? k - TS_STAGES : 0; q < k; ++q) {
        volatile int never = 0;
        ts_wait(full((int)(q % TS_STAGES)), (uint32_t)(q / TS_STAGES) & 1u, &never);
      }
    }
  } else {
    const int hp = tx >> 1;  // pairs per tile row
    const int px = tid % hp, ly = tid / hp;
    for (int64_t k = 0; k < njob; ++k) {
      const int st = (int)(k % TS_STAGES);
      const bool okw = ts_wait(full(st), (uint32_t)(k / TS_STAGES) & 1u, abort);
      if (!__all_sync(0xffffffffu, okw)) {
        *abort = 1;
        break;
      }
      const TsMeta m = meta[st];
      const unsigned char* sp = ts_smem + st * L.stage;
      const float* sx = reinterpret_cast<const float*>(sp);
      const float* sb = reinterpret_cast<const float*>(sp + L.off_b);
      const float* sd = reinterpret_cast<const float*>(sp + L.off_d);
      const uint8_t* sc = sp + L.off_c;
      if (2 * px < (m.lim & 0xFF) && ly < ((m.lim >> 8) & 0xFF)) {
        const int32_t node = m.base + 2 * px + ly * S;
        GOp<float> ot = o;
        ot.sigma = m.sigma;
        ot.dinv_int = m.dinv;
        const uint32_t k0 = sc[ly * tx + 2 * px], k1 = sc[ly * tx + 2 * px + 1];
        const int row = (ly + 1) * L.xw + 4 + 2 * px;  // the pair's first node in the x box
        const Two<float> xc{sx[row], sx[row + 1]};
        const float left = sx[row - 1], right = sx[row + 2];
        const Two<float> dn{sx[row - L.xw], sx[row - L.xw + 1]}, up{sx[row + L.xw], sx[row + L.xw + 1]};
        // stencil_pair's sums, in its order
        float s0 = ((k0 & 1) ? 0.0f : left) + ((k0 & 2) ? 0.0f : xc.y);
        float s1 = ((k1 & 1) ? 0.0f : xc.x) + ((k1 & 2) ? 0.0f : right);
        s0 += ((k0 & 4) ? 0.0f : dn.x) + ((k0 & 8) ? 0.0f : up.x);
        s1 += ((k1 & 4) ? 0.0f : dn.y) + ((k1 & 8) ? 0.0f : up.y);
        const float D0 = (k0 & 0x7F) ? __ldg(diag + node) : 4.0f;
        const float D1 = (k1 & 0x7F) ? __ldg(diag + node + 1) : 4.0f;
        const Two<float> core{D0 * xc.x - s0, D1 * xc.y - s1};
        const int bi = ly * tx + 2 * px;
        const Two<float> bv{sb[bi], sb[bi + 1]};
        const Two<float> dv = rd ? Two<float>{sd[bi], sd[bi + 1]} : Two<float>{0.0f, 0.0f};
        const float res0 = inv_diag_t<float>(k0, diag, node, ot) * (bv.x - (core.x * ot.inv_h2 + ot.sigma * xc.x));
        const float res1 = inv_diag_t<float>(k1, diag, node + 1, ot) * (bv.y - (core.y * ot.inv_h2 + ot.sigma * xc.y));
        const float d0 = (k0 & CODE_CP) ? c1 * dv.x + c2 * res0 : 0.0f;
        const float d1 = (k1 & CODE_CP) ? c1 * dv.y + c2 * res1 : 0.0f;
        st2(d + node, d0, d1);
        st2(xo + node, (k0 & CODE_CP) ? xc.x + d0 : 0.0f, (k1 & CODE_CP) ? xc.y + d1 : 0.0f);
      }
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(empty(st)) : "memory");
    }
  }
  __syncthreads();
  if (tid == 0 && *abort) atomicExch(err, 1);
}

template <int DIM, class V>
__global__ void __launch_bounds__(TILE_NODES) k_g_resid(TileView tv, const uint8_t* __restrict__ code,
                                                        const typename DiagOf<V>::type* __restrict__ diag,
                                                        GOp<typename AccOf<V>::type> o,
                                                        const V* __restrict__ b, const V* __restrict__ x,
                                                        V* __restrict__ r) {
  using A = typename AccOf<V>::type;
  EB_SWEEP(DIM, tv, node) {
    const GOp<A> ot = sweep_op<DIM>(tv, tt_, o);
    uint32_t c0, c1;
    ld_codes(code, node, c0, c1);
    Two<A> xc, core;
    stencil_tv<DIM, LdRO>(tv, x, node, c0, c1, diag, xc, core);
    const Two<A> bv = LdRO::ld2(b + node);
    st2o(r + node, (c0 & CODE_CP) ? bv.x - (core.x * ot.inv_h2 + ot.sigma * xc.x) : (A)0,
         (c1 & CODE_CP) ? bv.y - (core.y * ot.inv_h2 + ot.sigma * xc.y) : (A)0);
  }
}

// CSR kernels: a group of G lanes (G = 1..32, chosen per matrix from its mean
// row length) owns one row; lane g sums entries g, g+G, ... and the group
// reduces by xor-shuffles in a fixed order (deterministic).
template <int G, class A>
__device__ __forceinline__ A group_reduce(A s) {
  for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, G);
  return s;
}

// Lane g's part of sum_e v[e] x[col[e]] over entries beg..end-1 of a row:
// entries g, g+G, g+2G, ... summed in that order.  The column indices and
// values of CSR_UNROLL entries are loaded before their x gathers, so a row
// costs two dependent memory round trips per CSR_UNROLL * G entries instead of
// two per G; the summation order, hence the rounding, is that of the plain
// loop.
constexpr int CSR_UNROLL = 8;
template <int G, class V, class X>
__device__ __forceinline__ typename AccOf<V>::type csr_dot(const int32_t* __restrict__ col, const V* __restrict__ v,
                                                           const X* x, int32_t beg, int32_t end, int g) {
  using A = typename AccOf<V>::type;
  A s = 0;
  for (int32_t e0 = beg + g; e0 < end; e0 += CSR_UNROLL * G) {
    int32_t c[CSR_UNROLL];
    A w[CSR_UNROLL];
#pragma unroll
    for (int u = 0; u < CSR_UNROLL; ++u) {
      const int32_t e = e0 + u * G;
      c[u] = e < end ? __ldg(col + e) : -1;
      w[u] = e < end ? cvt<A>(v[e]) : (A)0;
    }
#pragma unroll
    for (int u = 0; u < CSR_UNROLL; ++u)
      if (c[u] >= 0) s += w[u] * cvt<A>(x[c[u]]);
  }
  return s;
}

// The first Chebyshev step of a coarse level, x = d = D^-1 b / theta, done by
// the restriction that produces its b (the values of a separate first-step
// launch: the same expression on the stored b); dinv == nullptr: not done.
template <class V>
struct CoarseFirst {
  const V* dinv = nullptr;
  V* x = nullptr;
  V* d = nullptr;
  typename AccOf<V>::type theta = 1;
};

template <class V>
__device__ __forceinline__ void store_restricted(V* out, int64_t i, typename AccOf<V>::type s, const CoarseFirst<V>& f) {
  using A = typename AccOf<V>::type;
  const V b = cvt<V>(s);
  out[i] = b;
  if (f.dinv) {
    const V v = cvt<V>(cvt<A>(f.dinv[i]) * cvt<A>(b) / f.theta);
    f.x[i] = v;
    f.d[i] = v;
  }
}

// out = R r with R's columns given as grid nodes
template <int G, class V>
__global__ void k_restrict0(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ node_col,
                            const V* __restrict__ v, const V* __restrict__ r, V* __restrict__ out, CoarseFirst<V> f) {
  using A = typename AccOf<V>::type;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = t / G;
  const int g = (int)(t % G);
  A s = 0;
  if (i < n) s = csr_dot<G>(node_col, v, r, rp[i], rp[i + 1], g);
  s = group_reduce<G>(s);
  if (i < n && g == 0) store_restricted(out, i, s, f);
}

// x[node(i)] += sum_c P_ic e_c over the CPs i
template <int G, class V>
__global__ void k_prolong0(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const V* __restrict__ v, const int32_t* __restrict__ cp_node, const V* __restrict__ e,
                           V* __restrict__ x) {
  using A = typename AccOf<V>::type;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = t / G;
  const int g = (int)(t % G);
  A s = 0;
  if (i < n) s = csr_dot<G>(ci, v, e, rp[i], rp[i + 1], g);
  s = group_reduce<G>(s);
  if (i < n && g == 0) {
    const int32_t node = cp_node[i];
    x[node] = cvt<V>(cvt<A>(x[node]) + s);
  }
}

// matrix-free level-0 transfers ----------------------------------------------
// t_j = e[agg(j)] sc[agg(j)] (the tentative prolongation at CP node j)
template <class V, class SC>
__device__ __forceinline__ typename AccOf<V>::type t_at(const int32_t* __restrict__ agg_node, const SC* __restrict__ sc,
                                                       const V* __restrict__ e, int32_t j) {
  using A = typename AccOf<V>::type;
  const int32_t c = __ldg(agg_node + j);
  return cvt<A>(e[c]) * (A)__ldg(sc + c);
}

// x_i += t_i - omega D_ii^-1 (A t)_i at the CPs (P = (I - omega D^-1 A) P_hat)
template <int DIM, class V, class SC>
__global__ void __launch_bounds__(TILE_NODES) k_prolong_mf(TileView tv, const uint8_t* __restrict__ code,
                                                           const typename DiagOf<V>::type* __restrict__ diag,
                                                           GOp<typename AccOf<V>::type> o,
                                                           typename AccOf<V>::type omega,
                                                           const int32_t* __restrict__ agg_node,
                                                           const SC* __restrict__ sc, const V* __restrict__ e,
                                                           V* __restrict__ x) {
  using A = typename AccOf<V>::type;
  const int32_t st[3] = {1, tv.sy, tv.sz};
  EB_SWEEP(DIM, tv, node) {
    uint32_t c0, c1;
    ld_codes(code, node, c0, c1);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t c = h ? c1 : c0;
      const int32_t i = node + h;
      if (!(c & CODE_CP)) continue;
      const A ti = t_at(agg_node, sc, e, i);
      A sum = 0;
#pragma unroll
      for (int sdir = 0; sdir < 2 * dim_of(DIM); ++sdir)
        if (!(c & (1u << sdir))) {
          const int32_t j = i + ((sdir & 1) ? st[sdir >> 1] : -st[sdir >> 1]);
          const A tj = t_at(agg_node, sc, e, j);
          // variable beta: each neighbour weighted by the beta of its half point
          if constexpr ((DIM & DIM_VB) != 0)
            sum += (A)__ldg(beta_ptrs(tv, diag)[sdir >> 1] + ((sdir & 1) ? i : j)) * tj;
          else
            sum += tj;
        }
      const A D = (c & 0x7F) ? (A)__ldg(diag + i) : (A)(2 * dim_of(DIM));
      const A at = (o.sigma + D * o.inv_h2) * ti - o.inv_h2 * sum;
      x[i] = cvt<V>(cvt<A>(x[i]) + ti - omega * inv_diag_t<A>(c, diag, i, o) * at);
    }
  }
}

// compact levels -----------------------------------------------------------
template <int G, class V>
__device__ __forceinline__ typename AccOf<V>::type csr_row(const CsrV<V>& M, const V* x, int64_t i, int g) {
  using A = typename AccOf<V>::type;
  A s = 0;
  if (i < M.n) s = csr_dot<G>(M.ci, M.v, x, M.rp[i], M.rp[i + 1], g);
  return group_reduce<G>(s);
}

// the row's own values are loaded first, alongside the row pointers
template <int G, class V>
__global__ void k_c_cheb_step(CsrV<V> M, const V* dinv, const V* b, const V* x, V* xo, V* d,
                              typename AccOf<V>::type c1, typename AccOf<V>::type c2) {
  using A = typename AccOf<V>::type;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = t / G;
  const int g = (int)(t % G);
  A di = 0, bi = 0, dd = 0, xi = 0;
  if (i < M.n && g == 0) {
    di = cvt<A>(dinv[i]);
    bi = cvt<A>(b[i]);
    if (c1 != (A)0) dd = cvt<A>(d[i]);
    xi = cvt<A>(x[i]);
  }
  const A ax = csr_row<G>(M, x, i, g);
  if (i >= M.n || g != 0) return;
  const A res = di * (bi - ax);
  const A dv = (c1 == (A)0 ? (A)0 : c1 * dd) + c2 * res;
  d[i] = cvt<V>(dv);
  xo[i] = cvt<V>(xi + dv);
}

template <int G, class V>
__global__ void k_c_resid(CsrV<V> M, const V* b, const V* x, V* r) {
  using A = typename AccOf<V>::type;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = t / G;
  const int g = (int)(t % G);
  const A ax = csr_row<G>(M, x, i, g);
  if (i < M.n && g == 0) r[i] = cvt<V>(cvt<A>(b[i]) - ax);
}

// y = M x (the restriction of the compact levels), with the coarse level's
// first smoothing step when f.dinv is set
template <int G, class V>
__global__ void k_c_spmv(CsrV<V> M, const V* x, V* y, CoarseFirst<V> f) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = t / G;
  const int g = (int)(t % G);
  const auto s = csr_row<G>(M, x, i, g);
  if (i < M.n && g == 0) store_restricted(y, i, s, f);
}

template <int G, class V>
__global__ void k_c_prolong_add(CsrV<V> P, const V* e, V* x) {
  using A = typename AccOf<V>::type;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = t / G;
  const int g = (int)(t % G);
  const A s = csr_row<G>(P, e, i, g);
  if (i < P.n && g == 0) x[i] = cvt<V>(cvt<A>(x[i]) + s);
}

// group width for a CSR matrix: the largest power of two G <= 32 with
// G * epl <= its mean row length (epl: entries per lane, tuned per solver)
inline int group_width(int64_t nnz, int64_t n, int epl) {
  const double avg = n > 0 ? (double)nnz / (double)n : 1.0;
  int g = 1;
  while (g < 32 && 2 * g * epl <= avg) g *= 2;
  return g;
}

#define EB_GROUP_LAUNCH(G, kernel, V, rows, s, ...)                                               \
  do {                                                                                           \
    const unsigned nb_ = blocks_for((int64_t)(rows) * (G), 256);                                 \
    switch (G) {                                                                                 \
      case 1: kernel<1, V><<<nb_, 256, 0, s>>>(__VA_ARGS__); break;                              \
      case 2: kernel<2, V><<<nb_, 256, 0, s>>>(__VA_ARGS__); break;                              \
      case 4: kernel<4, V><<<nb_, 256, 0, s>>>(__VA_ARGS__); break;                              \
      case 8: kernel<8, V><<<nb_, 256, 0, s>>>(__VA_ARGS__); break;                              \
      case 16: kernel<16, V><<<nb_, 256, 0, s>>>(__VA_ARGS__); break;                            \
      default: kernel<32, V><<<nb_, 256, 0, s>>>(__VA_ARGS__); break;                            \
    }                                                                                            \
  } while (0)

// x = M b with M the FP64 inverse (row-major); one warp per row
template <class V>
__global__ void k_dense_gemv(const double* __restrict__ M, int64_t n, const V* __restrict__ b, V* __restrict__ x) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  double s = 0.0;
  for (int64_t j = lane; j < n; j += 32) s += M[row * n + j] * cvt<double>(b[j]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) x[row] = cvt<V>(s);
}

template <class V>
__global__ void k_gather_cp(int64_t n, const int32_t* cp_node, const double* g, V* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = cvt<V>(g[cp_node[i]]);
}

template <class V>
__global__ void k_scatter_cp(int64_t n, const int32_t* cp_node, const V* in, double* g) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) g[cp_node[i]] = cvt<double>(in[i]);
}

__global__ void k_to_f32(int64_t n, const double* a, float* b) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

__global__ void k_to_bf16(int64_t n, const double* a, __nv_bfloat16* b) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __double2bfloat16(a[i]);
}

// ------------------------------------------------------------------ host
struct ChebCoef {
  double theta, c1[9], c2[9];
  int deg;
};

static ChebCoef cheb_coef(double rho, int deg) {
  ChebCoef c{};
  const double lo = rho / 30.0, hi = 1.1 * rho;
  c.theta = 0.5 * (hi + lo);
  const double delta = 0.5 * (hi - lo);
  const double sigma = c.theta / delta;
  double r0 = 1.0 / sigma;
  c.deg = deg;
  c.c1[0] = 0.0;
  c.c2[0] = 1.0 / c.theta;
  for (int k = 1; k < deg; ++k) {
    const double r1 = 1.0 / (2.0 * sigma - r0);
    c.c1[k] = r1 * r0;
    c.c2[k] = 2.0 * r1 / delta;
    r0 = r1;
  }
  return c;
}

template <class V>
struct LevelView;
template <>
struct LevelView<double> {
  static VecSet<double>& vec(Level& L) { return L.v64; }
  static VecSet<double>& grid(Hierarchy& H) { return H.g64; }
  static CsrV<double> A(const Level& L) { return {L.A.n, L.A.rp, L.A.ci, L.A.v}; }
  static CsrV<double> P(const Level& L) { return {L.P.n, L.P.rp, L.P.ci, L.P.v}; }
  static CsrV<double> R(const Level& L) { return {L.R.n, L.R.rp, L.R.ci, L.R.v}; }
  static const double* dinv(const Level& L) { return L.dinv; }
};
template <>
struct LevelView<float> {
  static VecSet<float>& vec(Level& L) { return L.v32; }
  static VecSet<float>& grid(Hierarchy& H) { return H.g32; }
  static CsrV<float> A(const Level& L) { return {L.A.n, L.A.rp, L.A.ci, L.A32}; }
  static CsrV<float> P(const Level& L) { return {L.P.n, L.P.rp, L.P.ci, L.P32}; }
  static CsrV<float> R(const Level& L) { return {L.R.n, L.R.rp, L.R.ci, L.R32}; }
  static const float* dinv(const Level& L) { return L.dinv32; }
};

template <>
struct LevelView<__nv_bfloat16> {
  static VecSet<__nv_bfloat16>& vec(Level& L) { return L.v16; }
  static VecSet<__nv_bfloat16>& grid(Hierarchy& H) { return H.g16; }
  static CsrV<__nv_bfloat16> A(const Level& L) { return {L.A.n, L.A.rp, L.A.ci, L.A16}; }
  static CsrV<__nv_bfloat16> P(const Level& L) { return {L.P.n, L.P.rp, L.P.ci, L.P16}; }
  static CsrV<__nv_bfloat16> R(const Level& L) { return {L.R.n, L.R.rp, L.R.ci, L.R16}; }
  static const __nv_bfloat16* dinv(const Level& L) { return L.dinv16; }
};

// the first-step outputs for compact level l, or none if l is the coarsest
// (its dense solve replaces smoothing)
template <class V>
static CoarseFirst<V> coarse_first(Solver& S, size_t l) {
  using LV = LevelView<V>;
  Hierarchy& H = *S.H;
  CoarseFirst<V> f;
  if (l + 1 >= H.L.size()) return f;
  Level& L = H.L[l];
  VecSet<V>& v = LV::vec(L);
  f.dinv = LV::dinv(L);
  f.x = v.x;
  f.d = v.d;
  f.theta = (typename AccOf<V>::type)cheb_coef(L.rho, S.opts.cheb_degree).theta;
  return f;
}

// Cycle from compact level l down; the restriction into l already did its
// first smoothing step (coarse_first) unless warm: then the cycle starts from
// the level's current x (the second coarse-grid cycle of a W-cycle) and runs
// all its pre-smoothing steps.  With opts.cycle = 2 every coarse-grid
// correction is two cycles of the coarser level (W-cycle).
template <class V>
static void vcycle_compact(Solver& S, size_t l, cudaStream_t s, bool warm = false) {
  using LV = LevelView<V>;
  Hierarchy& H = *S.H;
  Level& L = H.L[l];
  VecSet<V>& v = LV::vec(L);
  const int64_t n = L.A.n;
  if (l + 1 == H.L.size()) {
    S.nlaunch += 1;
    k_dense_gemv<V><<<blocks_for(n * 32, 256), 256, 0, s>>>(H.coarse_inv, n, v.b, v.x);
    return;
  }
  const ChebCoef cc = cheb_coef(L.rho, S.opts.cheb_degree);
  S.nlaunch += 2 + 2 * cc.deg + (warm ? 1 : 0);  // pre steps, residual, restriction, prolongation, deg steps
  const CsrV<V> A = LV::A(L);
  const int e = S.csr_epl;
  const int gA = group_width(L.A.nnz, L.A.n, e), gP = group_width(L.P.nnz, L.P.n, e),
            gR = group_width(L.R.nnz, L.R.n, e);
  const bool mark = l == 1;  // level-1 smoother launches are timed with PROF_LEVEL1
  for (int k = warm ? 0 : 1; k < cc.deg; ++k) {
    if (mark) S.prof_mark(s, true, PROF_LEVEL1);
    EB_GROUP_LAUNCH(gA, k_c_cheb_step, V, n, s, A, LV::dinv(L), v.b, v.x, v.x2, v.d, cc.c1[k], cc.c2[k]);
    if (mark) S.prof_mark(s, false, PROF_LEVEL1);
    std::swap(v.x, v.x2);
  }
  EB_GROUP_LAUNCH(gA, k_c_resid, V, n, s, A, v.b, v.x, v.r);
  Level& C = H.L[l + 1];
  VecSet<V>& cv = LV::vec(C);
  EB_GROUP_LAUNCH(gR, k_c_spmv, V, C.A.n, s, LV::R(L), v.r, cv.b, coarse_first<V>(S, l + 1));
  vcycle_compact<V>(S, l + 1, s);
  if (S.opts.cycle == 2 && l + 2 < H.L.size()) vcycle_compact<V>(S, l + 1, s, true);
  EB_GROUP_LAUNCH(gP, k_c_prolong_add, V, n, s, LV::P(L), cv.x, v.x);
  for (int k = 0; k < cc.deg; ++k) {
    if (mark) S.prof_mark(s, true, PROF_LEVEL1);
    EB_GROUP_LAUNCH(gA, k_c_cheb_step, V, n, s, A, LV::dinv(L), v.b, v.x, v.x2, v.d, cc.c1[k], cc.c2[k]);
    if (mark) S.prof_mark(s, false, PROF_LEVEL1);
    std::swap(v.x, v.x2);
  }
}

// tensor map of a 2D grid array (S columns x R rows, element size es) with boxes of bw x bh
static CUtensorMap ts_map(const void* p, CUtensorMapDataType dt, int es, int64_t S, int64_t R, int bw, int bh) {
  CUtensorMap m;
  const cuuint64_t dims[2] = {(cuuint64_t)S, (cuuint64_t)R};
  const cuuint64_t strides[1] = {(cuuint64_t)(S * es)};
  const cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult rc = tensor_map_encoder()(&m, dt, 2, const_cast<void*>(p), dims, strides, box, estr,
                                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  EB_REQUIRE(rc == CUDA_SUCCESS, EB_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)rc) + ")");
  return m;
}

// whether the tensor-copy step applies to this view: 2D tiles without a pair
// list, tiles 16 to 128 nodes wide (16-byte aligned code boxes, boxes of at
// most 256), rows a multiple of 16 nodes (16-byte row pitch of the codes)
static bool ts_eligible(const Solver& S, const EBHandle& eb) {
  const TileView tv = eb.tv();
  const int tx = 1 << tv.bx;
  return S.l0_tma && eb.g.dim == 2 && !tv.pair_node && tv.ntiles > 0 && tx >= 16 && tx <= 128 && tv.sy % 16 == 0 &&
         (int64_t)eb.g.num_nodes % tv.sy == 0;
}

// one level-0 Chebyshev step through k_g_cheb_step_tma (FP32 storage)
static void ts_step(Solver& S, const EBHandle& eb, const GOp<float>& o, const float* b, const float* x, float* xo,
                    float* d, float c1, float c2, cudaStream_t s) {
  const TileView tv = eb.tv();
  const int tx = 1 << tv.bx, ty = 1 << tv.by;
  const int64_t Sx = tv.sy, R = (int64_t)eb.g.num_nodes / Sx;
  const CUtensorMap xm = ts_map(x, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, Sx, R, tx + 8, ty + 2);
  const CUtensorMap bm = ts_map(b, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, Sx, R, tx, ty);
  const CUtensorMap dm = ts_map(d, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, Sx, R, tx, ty);
  const CUtensorMap cm = ts_map(eb.code, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, Sx, R, tx, ty);
  const TsLayout L(tx, ty);
  const size_t smem = TS_STAGES * (size_t)L.stage + TS_STAGES * sizeof(TsMeta) + 16 * TS_STAGES + 16;
  if (!S.dev_err) S.dev_err = dalloc<int>(1, s);
  static size_t smem_set = 0;
  if (smem > 48 * 1024 && smem > smem_set) {
    EB_CUDA(cudaFuncSetAttribute(k_g_cheb_step_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    smem_set = smem;
  }
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tv.ntiles, (int64_t)num_sms() * 8));
  k_g_cheb_step_tma<<<grid, TS_THREADS, smem, s>>>(xm, bm, dm, cm, tv, tx, ty, diag_of<float>(eb), o, xo, d, c1, c2,
                                                   S.dev_err);
}

template <class V, int DIM>
static int vcycle_grid(Solver& S, const double* r, double* z, cudaStream_t s, const VcycleDot* dot, bool first_done) {
  using LV = LevelView<V>;
  Hierarchy& H = *S.H;
  const EBHandle& eb = *S.eb;
  const Geometry& G = eb.g;
  Level& L0 = H.L[0];
  if (H.L.size() == 1) {  // single level: the dense inverse acts on the CP vector
    VecSet<V>& v = LV::vec(L0);
    const int64_t n = L0.A.n;
    EB_CUDA(cudaMemsetAsync(z, 0, sizeof(double) * G.num_nodes, s));
    k_gather_cp<V><<<blocks_for(n, 256), 256, 0, s>>>(n, eb.cp_node, r, v.b);
    k_dense_gemv<V><<<blocks_for(n * 32, 256), 256, 0, s>>>(H.coarse_inv, n, v.b, v.x);
    k_scatter_cp<V><<<blocks_for(n, 256), 256, 0, s>>>(n, eb.cp_node, v.x, z);
    EB_CUDA(cudaGetLastError());
    S.nlaunch += 3;
    return 0;
  }
  const double inv_h2 = 1.0 / (G.h * G.h);
  const unsigned gb = tile_grid(eb);
  // list sweeps: one CP pair per thread (the partial-forming launch keeps the
  // fixed grid gb, whose CTA count is the number of partials)
  constexpr bool LIST = (DIM & DIM_LIST) != 0;
  const unsigned gl = LIST ? blocks_for(eb.num_pairs, TILE_NODES) : gb;
  const ChebCoef cc = cheb_coef(L0.rho, S.opts.cheb_degree);
  const TileView tv = eb.tv();
  using A = typename AccOf<V>::type;
  const GOp<A> o{(A)inv_h2, (A)S.shift, (A)(1.0 / (S.shift + 2.0 * G.dim * inv_h2))};
  const typename DiagOf<V>::type* diag = diag_of<V>(eb);
  S.nlaunch += 3 + 2 * cc.deg;
  VecSet<V>& g = LV::grid(H);
  // FP64 storage reads r directly; FP32 storage keeps a rounded copy in g.b
  V* bcopy = std::is_same<V, double>::value ? nullptr : g.b;
  const V* b = std::is_same<V, double>::value ? reinterpret_cast<const V*>(r) : g.b;
  V* x = g.x;
  V* x2 = g.x2;
  const bool rdf = dot && dot->df;
  if (first_done)
    S.nlaunch -= 1;  // amg_update_first did it
  else if (rdf)
    k_g_cheb_first<DIM, V, true><<<gl, TILE_NODES, 0, s>>>(tv, eb.code, diag, o, r, bcopy, x, g.d, (A)cc.theta);
  else
    k_g_cheb_first<DIM, V><<<gl, TILE_NODES, 0, s>>>(tv, eb.code, diag, o, r, bcopy, x, g.d, (A)cc.theta);
  // the tensor-copy step (batched 2D views, FP32 storage) or the sweep kernel
  auto step = [&](const V* xin, V* xout, int k) {
    if constexpr (std::is_same<V, float>::value && (DIM & (DIM_VB | DIM_LIST)) == 0 && dim_of(DIM) == 2) {
      if (ts_eligible(S, eb)) {
        ts_step(S, eb, o, b, xin, xout, g.d, (A)cc.c1[k], (A)cc.c2[k], s);
        return;
      }
    }
    k_g_cheb_step<DIM, V, V><<<gl, TILE_NODES, 0, s>>>(tv, eb.code, diag, o, b, xin, xout, g.d, (A)cc.c1[k],
                                                       (A)cc.c2[k]);
  };
  for (int k = 1; k < cc.deg; ++k) {
    S.prof_mark(s, true);
    step(x, x2, k);
    S.prof_mark(s, false);
    std::swap(x, x2);
  }
  k_g_resid<DIM, V><<<gl, TILE_NODES, 0, s>>>(tv, eb.code, diag, o, b, x, g.r);
  Level& C = H.L[1];
  VecSet<V>& cv = LV::vec(C);
  const CsrV<V> R0 = LV::R(L0), P0 = LV::P(L0);
  const int gR = group_width(L0.R.nnz, L0.R.n, S.csr_epl), gP = group_width(L0.P.nnz, L0.P.n, S.csr_epl);
  const MatrixFreeP& M = H.mf;
  using SC = typename std::conditional<std::is_same<V, double>::value, double, float>::type;
  const SC* sc = nullptr;
  if (M.on) sc = reinterpret_cast<const SC*>(std::is_same<V, double>::value ? (const void*)M.sc64 : (const void*)M.sc32);
  // restriction through the explicit R (its per-member stencil gathers made a
  // matrix-free restriction slower); prolongation matrix free
  EB_GROUP_LAUNCH(gR, k_restrict0, V, C.A.n, s, C.A.n, R0.rp, L0.R0node, R0.v, g.r, cv.b, coarse_first<V>(S, 1));
  vcycle_compact<V>(S, 1, s);
  if (S.opts.cycle == 2 && H.L.size() > 2) vcycle_compact<V>(S, 1, s, true);  // W-cycle
  if (M.on)
    k_prolong_mf<DIM, V, SC><<<gl, TILE_NODES, 0, s>>>(tv, eb.code, diag, o, (A)M.omega, M.agg_node, sc, cv.x, x);
  else
    EB_GROUP_LAUNCH(gP, k_prolong0, V, P0.n, s, P0.n, P0.rp, P0.ci, P0.v, eb.cp_node, cv.x, x);
  for (int k = 0; k < cc.deg; ++k) {
    // the launch that also forms the r'z partials is a different kernel: not
    // part of the smoother-step timing
    const bool mark = !(k == cc.deg - 1 && dot);
    if (mark) S.prof_mark(s, true);
    if (k == cc.deg - 1 && rdf && dot->part)  // z in FP32 for the DF outer iteration, with the r'z partials
      k_g_cheb_step<DIM, V, float, 2><<<gb, TILE_NODES, 0, s>>>(tv, eb.code, diag, o, b, x,
                                                                reinterpret_cast<float*>(z), g.d, (A)cc.c1[k],
                                                                (A)cc.c2[k], dot->r, dot->part);
    else if (k == cc.deg - 1 && rdf)  // z in FP32 on every node of the active tiles, 0 off the CPs
      k_g_cheb_step<(DIM & ~DIM_LIST), V, float><<<gb, TILE_NODES, 0, s>>>(
          tiles_only(tv), eb.code, diag, o, b, x, reinterpret_cast<float*>(z), g.d, (A)cc.c1[k], (A)cc.c2[k]);
    else if (k == cc.deg - 1 && dot)
      k_g_cheb_step<DIM, V, double, 1><<<gb, TILE_NODES, 0, s>>>(tv, eb.code, diag, o, b, x, z, g.d, (A)cc.c1[k],
                                                                 (A)cc.c2[k], dot->r, dot->part);
    else if (k == cc.deg - 1)  // z for a caller (amg_vcycle): every node of the active tiles, 0 off the CPs
      k_g_cheb_step<(DIM & ~DIM_LIST), V, double>
          <<<gb, TILE_NODES, 0, s>>>(tiles_only(tv), eb.code, diag, o, b, x, z, g.d, (A)cc.c1[k], (A)cc.c2[k]);
    else
      step(x, x2, k);
    if (mark) S.prof_mark(s, false);
    if (k != cc.deg - 1) std::swap(x, x2);
  }
  g.x = x;
  g.x2 = x2;
  EB_CUDA(cudaGetLastError());
  return (dot && dot->part) ? (int)gb : 0;
}

int amg_vcycle_grid(Solver& S, const double* r, double* z, cudaStream_t s, const VcycleDot* dot, bool first_done) {
  int ret = 0;
  dim_dispatch(*S.eb, [&](auto D) {
    constexpr int DL = D.value | DIM_LIST;
    const bool list = S.eb->pair_node != nullptr;
    if (S.opts.vcycle_prec == EB_F32)
      ret = list ? vcycle_grid<float, DL>(S, r, z, s, dot, first_done)
                 : vcycle_grid<float, D.value>(S, r, z, s, dot, first_done);
    else if (S.opts.vcycle_prec == EB_BF16)
      ret = list ? vcycle_grid<__nv_bfloat16, DL>(S, r, z, s, dot, first_done)
                 : vcycle_grid<__nv_bfloat16, D.value>(S, r, z, s, dot, first_done);
    else
      ret = list ? vcycle_grid<double, DL>(S, r, z, s, dot, first_done)
                 : vcycle_grid<double, D.value>(S, r, z, s, dot, first_done);
  });
  return ret;
}

template <class V, int DIM>
static void update_first(Solver& S, const PcgUpdate& u, cudaStream_t s) {
  using LV = LevelView<V>;
  using A = typename AccOf<V>::type;
  Hierarchy& H = *S.H;
  const EBHandle& eb = *S.eb;
  const Geometry& G = eb.g;
  const double inv_h2 = 1.0 / (G.h * G.h);
  const ChebCoef cc = cheb_coef(H.L[0].rho, S.opts.cheb_degree);
  const GOp<A> o{(A)inv_h2, (A)S.shift, (A)(1.0 / (S.shift + 2.0 * G.dim * inv_h2))};
  VecSet<V>& g = LV::grid(H);
  V* bcopy = std::is_same<V, double>::value ? nullptr : g.b;
  if constexpr (!std::is_same<V, double>::value) {
    if (u.df) {
      k_update_first_df<DIM, V><<<(unsigned)u.nblk, TILE_NODES, 0, s>>>(eb.pairs(), u, eb.code, diag_of<V>(eb), o,
                                                                        bcopy, g.x, g.d, (float)(1.0 / cc.theta));
      return;
    }
  }
  k_update_first<DIM, V><<<(unsigned)u.nblk, TILE_NODES, 0, s>>>(eb.pairs(), u, eb.code, diag_of<V>(eb), o, bcopy,
                                                                 g.x, g.d, (A)cc.theta);
}

int amg_levels(const Solver& S) { return S.H ? (int)S.H->L.size() : 0; }

int amg_update_first(Solver& S, const PcgUpdate& u, cudaStream_t s) {
  if (!S.H || S.H->L.size() == 1) return 0;  // a single level has no smoothing step
  const int dim = S.eb->g.dim;
  if (S.opts.vcycle_prec == EB_F32) {
    if (dim == 2) update_first<float, 2>(S, u, s);
    else update_first<float, 3>(S, u, s);
  } else if (S.opts.vcycle_prec == EB_BF16) {
    if (dim == 2) update_first<__nv_bfloat16, 2>(S, u, s);
    else update_first<__nv_bfloat16, 3>(S, u, s);
  } else {
    if (dim == 2) update_first<double, 2>(S, u, s);
    else update_first<double, 3>(S, u, s);
  }
  EB_CUDA(cudaGetLastError());
  return 1;
}

template <class V>
static void alloc_set(VecSet<V>& v, int64_t n, bool with_b, cudaStream_t s) {
  if (with_b) v.b = dalloc<V>(n, s);
  v.x = dalloc<V>(n, s);
  v.x2 = dalloc<V>(n, s);
  v.d = dalloc<V>(n, s);
  v.r = dalloc<V>(n, s);
}

template <class V>
static void free_set(VecSet<V>& v, cudaStream_t s) {
  dfree(v.b, s); dfree(v.x, s); dfree(v.x2, s); dfree(v.d, s); dfree(v.r, s);
}

static float* to_f32(const double* a, int64_t n, cudaStream_t s) {
  float* b = dalloc<float>(n, s, false);
  if (n > 0) k_to_f32<<<blocks_for(n, 256), 256, 0, s>>>(n, a, b);
  return b;
}

static __nv_bfloat16* to_bf16(const double* a, int64_t n, cudaStream_t s) {
  __nv_bfloat16* b = dalloc<__nv_bfloat16>(n, s, false);
  if (n > 0) k_to_bf16<<<blocks_for(n, 256), 256, 0, s>>>(n, a, b);
  return b;
}

void amg_alloc_vcycle(Solver& S, cudaStream_t s) {
  Hierarchy& H = *S.H;
  const int64_t nn = S.eb->g.num_nodes;
  const bool f32 = S.opts.vcycle_prec == EB_F32;
  const size_t first = H.L.size() == 1 ? 0 : 1;
  if (f32) {
    alloc_set(H.g32, nn, true, s);
    for (size_t l = first; l < H.L.size(); ++l) alloc_set(H.L[l].v32, H.L[l].A.n, true, s);
    for (size_t l = 0; l < H.L.size(); ++l) {
      Level& L = H.L[l];
      L.A32 = to_f32(L.A.v, L.A.nnz, s);
      if (L.dinv) L.dinv32 = to_f32(L.dinv, L.A.n, s);
      if (L.P.v) L.P32 = to_f32(L.P.v, L.P.nnz, s);
      if (L.R.v) L.R32 = to_f32(L.R.v, L.R.nnz, s);
    }
  } else if (S.opts.vcycle_prec == EB_BF16) {
    alloc_set(H.g16, nn, true, s);
    for (size_t l = first; l < H.L.size(); ++l) alloc_set(H.L[l].v16, H.L[l].A.n, true, s);
    for (size_t l = 0; l < H.L.size(); ++l) {
      Level& L = H.L[l];
      L.A16 = to_bf16(L.A.v, L.A.nnz, s);
      if (L.dinv) L.dinv16 = to_bf16(L.dinv, L.A.n, s);
      if (L.P.v) L.P16 = to_bf16(L.P.v, L.P.nnz, s);
      if (L.R.v) L.R16 = to_bf16(L.R.v, L.R.nnz, s);
    }
  } else {
    alloc_set(H.g64, nn, false, s);
    for (size_t l = first; l < H.L.size(); ++l) alloc_set(H.L[l].v64, H.L[l].A.n, true, s);
  }
  EB_CUDA(cudaGetLastError());
}

void amg_free_vcycle(Hierarchy& H, cudaStream_t s) {
  free_set(H.g64, s);
  free_set(H.g32, s);
  free_set(H.g16, s);
  for (Level& L : H.L) {
    free_set(L.v64, s);
    free_set(L.v32, s);
    free_set(L.v16, s);
    dfree(L.A32, s); dfree(L.P32, s); dfree(L.R32, s); dfree(L.dinv32, s);
    dfree(L.A16, s); dfree(L.P16, s); dfree(L.R16, s); dfree(L.dinv16, s);
  }
}

}  // namespace ebk

// ------------------------------------------------------- kernel timing alone
namespace ebk {

// Reads n 16-byte words (a buffer larger than L2), so that L2 then holds only
// clean lines of that buffer: the next kernel misses without write-backs, as
// after a cache flush.  The store never happens for a buffer of zeros
// (flag = 1); it only keeps the reads from being dropped.
__global__ void k_l2_clear(const uint4* __restrict__ p, int64_t n, int flag, unsigned* sink) {
  unsigned acc = 0u;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint4 v = __ldcg(p + i);
    acc |= v.x | v.y | v.z | v.w;
  }
  if (acc == 0u && flag == 0) *sink = acc;
}

// One Chebyshev smoothing step of level `level` (k = 1 coefficients, so that
// the step reads its previous direction), launched as in a V-cycle.
template <class V>
static void smoother_step(Solver& S, int level, cudaStream_t s) {
  using LV = LevelView<V>;
  using A = typename AccOf<V>::type;
  Hierarchy& H = *S.H;
  Level& L = H.L[level];
  const ChebCoef cc = cheb_coef(L.rho, S.opts.cheb_degree);
  const int k = cc.deg > 1 ? 1 : 0;
  if (level == 0) {
    const EBHandle& eb = *S.eb;
    const Geometry& G = eb.g;
    const double inv_h2 = 1.0 / (G.h * G.h);
    const GOp<A> o{(A)inv_h2, (A)S.shift, (A)(1.0 / (S.shift + 2.0 * G.dim * inv_h2))};
    VecSet<V>& g = LV::grid(H);
    const V* b = std::is_same<V, double>::value ? reinterpret_cast<const V*>(S.r) : g.b;
    dim_dispatch(eb, [&](auto D) {
      if (eb.pair_node)
        k_g_cheb_step<D.value | DIM_LIST, V, V><<<blocks_for(eb.num_pairs, TILE_NODES), TILE_NODES, 0, s>>>(
            eb.tv(), eb.code, diag_of<V>(eb), o, b, g.x, g.x2, g.d, (A)cc.c1[k], (A)cc.c2[k]);
      else
        k_g_cheb_step<D.value, V, V><<<tile_grid(eb), TILE_NODES, 0, s>>>(eb.tv(), eb.code, diag_of<V>(eb), o, b,
                                                                            g.x, g.x2, g.d, (A)cc.c1[k], (A)cc.c2[k]);
    });
  } else {
    VecSet<V>& v = LV::vec(L);
    const int gA = group_width(L.A.nnz, L.A.n, S.csr_epl);
    EB_GROUP_LAUNCH(gA, k_c_cheb_step, V, L.A.n, s, LV::A(L), LV::dinv(L), v.b, v.x, v.x2, v.d, (A)cc.c1[k],
                    (A)cc.c2[k]);
  }
}

// microseconds per launch of `launches` back-to-back launches captured in one
// graph (each preceded by an L2-clearing write when clear is given, whose own
// time, measured the same way, is subtracted)
static double time_alone(const std::function<void(cudaStream_t)>& launch, int launches, const uint4* clear,
                         int64_t nclear, cudaStream_t s) {
  cudaStream_t cap = nullptr;
  EB_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto graph_us = [&](bool with_kernel) {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    EB_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < launches; ++i) {
      if (clear) k_l2_clear<<<num_sms() * 4, 512, 0, cap>>>(clear, nclear, 1, nullptr);
      if (with_kernel) launch(cap);
    }
    EB_CUDA(cudaStreamEndCapture(cap, &g));
    const cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) throw Failure{EB_ERR_CUDA, std::string("amg_time_kernel: ") + cudaGetErrorString(ie)};
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      EB_CUDA(cudaEventRecord(e0, s));
      EB_CUDA(cudaGraphLaunch(ge, s));
      EB_CUDA(cudaEventRecord(e1, s));
      EB_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      EB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      best = std::min(best, ms);
    }
    cudaGraphExecDestroy(ge);
    return 1000.0 * best / launches;
  };
  double us = 0.0;
  try {
    EB_CUDA(cudaEventCreate(&e0));
    EB_CUDA(cudaEventCreate(&e1));
    us = graph_us(true);
    if (clear) us -= graph_us(false);
  } catch (...) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamDestroy(cap);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(cap);
  return us;
}

// plain streaming copy (16-byte loads and stores, grid-stride): the size-matched
// reference of eb_time_copy
__global__ void __launch_bounds__(256) k_stream_copy(const uint4* __restrict__ a, uint4* __restrict__ b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = __ldcs(a + i);
}

}  // namespace ebk

using namespace ebk;

extern "C" int eb_time_copy(int64_t bytes, int launches, int64_t clear_bytes, double* us_out, cudaStream_t stream) {
  if (!us_out || bytes < 32 || launches < 1 || launches > 10000 || clear_bytes < 0) {
    set_error("eb_time_copy: invalid argument");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    const int64_t n = bytes / 2 / (int64_t)sizeof(uint4);  // half read, half written
    uint4* a = dalloc<uint4>(n, stream);
    uint4* b = nullptr;
    const int64_t nclear = clear_bytes / (int64_t)sizeof(uint4);
    uint4* clear = nullptr;
    try {
      b = dalloc<uint4>(n, stream);
      clear = nclear > 0 ? dalloc<uint4>(nclear, stream) : nullptr;
      const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8);
      auto launch = [&](cudaStream_t s) { k_stream_copy<<<grid, 256, 0, s>>>(a, b, n); };
      EB_CUDA(cudaStreamSynchronize(stream));
      *us_out = time_alone(launch, launches, clear, nclear, stream);
    } catch (...) {
      dfree(a, stream);
      dfree(b, stream);
      dfree(clear, stream);
      throw;
    }
    dfree(a, stream);
    dfree(b, stream);
    dfree(clear, stream);
    EB_CUDA(cudaStreamSynchronize(stream));
  });
}

extern "C" int eb_time_apply(const eb_handle* eb, int prec, const void* x_dev, void* y_dev, int launches,
                             int64_t clear_bytes, double* us_out, cudaStream_t stream) {
  if (!eb || !x_dev || !y_dev || !us_out || launches < 1 || launches > 10000 || clear_bytes < 0 ||
      (prec != EB_F64 && prec != EB_F32 && prec != EB_BF16)) {
    set_error("eb_time_apply: invalid argument");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    const EBHandle& E = eb->h;
    const int64_t nclear = clear_bytes / (int64_t)sizeof(uint4);
    uint4* clear = nclear > 0 ? dalloc<uint4>(nclear, stream) : nullptr;
    double us = 0.0;
    try {
      auto launch = [&](cudaStream_t s) {
        if (prec == EB_F64) launch_apply<double>(E, (const double*)x_dev, (double*)y_dev, 0.0, s);
        else if (prec == EB_F32) launch_apply<float>(E, (const float*)x_dev, (float*)y_dev, 0.0, s);
        else launch_apply<__nv_bfloat16>(E, (const __nv_bfloat16*)x_dev, (__nv_bfloat16*)y_dev, 0.0, s);
      };
      EB_CUDA(cudaStreamSynchronize(stream));
      us = time_alone(launch, launches, clear, nclear, stream);
    } catch (...) {
      dfree(clear, stream);
      throw;
    }
    dfree(clear, stream);
    EB_CUDA(cudaStreamSynchronize(stream));
    *us_out = us;
  });
}

extern "C" int amg_time_kernel(const amg_handle* amg, int kernel, int level, int launches, int64_t clear_bytes,
                               double* us_out, cudaStream_t stream) {
  if (!amg || !us_out || launches < 1 || launches > 10000 || clear_bytes < 0) {
    set_error("amg_time_kernel: invalid argument");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    Solver& S = const_cast<Solver&>(amg->s);
    EB_REQUIRE(S.H != nullptr, EB_ERR_INVALID, "amg_time_kernel: handle has no hierarchy");
    EB_REQUIRE(kernel == EB_TK_SMOOTH_STEP, EB_ERR_INVALID, "amg_time_kernel: unknown kernel");
    EB_REQUIRE(level >= 0 && level + 1 < (int)S.H->L.size(), EB_ERR_INVALID,
               "amg_time_kernel: level must have a coarser level below it");
    EB_REQUIRE(S.r != nullptr, EB_ERR_INVALID, "amg_time_kernel: no work vectors");
    const int64_t nclear = clear_bytes / (int64_t)sizeof(uint4);
    uint4* clear = nclear > 0 ? dalloc<uint4>(nclear, stream) : nullptr;  // zero-filled
    double us = 0.0;
    try {
      auto launch = [&](cudaStream_t s) {
        if (S.opts.vcycle_prec == EB_F32) smoother_step<float>(S, level, s);
        else if (S.opts.vcycle_prec == EB_BF16) smoother_step<__nv_bfloat16>(S, level, s);
        else smoother_step<double>(S, level, s);
      };
      EB_CUDA(cudaStreamSynchronize(stream));
      us = time_alone(launch, launches, clear, nclear, stream);
    } catch (...) {
      dfree(clear, stream);
      throw;
    }
    dfree(clear, stream);
    EB_CUDA(cudaStreamSynchronize(stream));
    *us_out = us;
  });
}
