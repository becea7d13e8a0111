// Preconditioned conjugate gradients on the EB operator (Algorithm 1 step 4)
// and the theta-method heat step (Sec. 3.4).
//
// Vectors live in the full-grid layout and are touched on the active tiles
// only; the FP64 update kernels (x, r, p, q) run over the node pairs of the
// tiles that hold a CP (EBHandle::pairs): the other pairs' entries are never
// read at a CP, and GB300's narrow FP64 pipe makes the skipped pairs count.
// One iteration is the x/r update, the preconditioner and k_xpby_apply (the
// p update with the next operator apply).  Every reduction is two-pass and
// deterministic: each CTA of a fixed grid reduces its nodes in a fixed order
// to one partial; the partials are combined in a fixed order by the kernel
// that needs the result -- every CTA of the update kernels (x, r with alpha;
// p with beta) reduces them itself and CTA 0 records the scalars and, in the
// device-side loop, runs the convergence test -- or by one CTA (k_finalize).
// No scalar crosses to the host except at the end of the loop.
#include "df.cuh"
#include "eb_solver.cuh"
#include "stencil.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <type_traits>

namespace ebk {

struct OpParams {
  double inv_h2, sigma, dinv_int;
  double sigma_h2;  // sigma h^2: the shift of the unit stencil h^2 (sigma I + A)
};

// (sigma I + A) x for the pair at node
template <int DIM>
__device__ __forceinline__ void op_pair(const TileView& tv, const double* x, int32_t node, uint32_t c0, uint32_t c1,
                                        const double* diag, const OpParams& o, Two<double>& xc, Two<double>& ax) {
  Two<double> core;
  stencil_tv<DIM, LdRO>(tv, x, node, c0, c1, diag, xc, core);
  ax.x = core.x * o.inv_h2 + o.sigma * xc.x;
  ax.y = core.y * o.inv_h2 + o.sigma * xc.y;
}

// h^2 (sigma I + A) x for the pair at node: the unit stencil D_k x_k - sum of
// the CP-neighbour values, plus sigma h^2 x_k when SHIFT
template <int DIM, bool SHIFT>
__device__ __forceinline__ void op_pair_unit(const TileView& tv, const double* x, int32_t node, uint32_t c0,
                                             uint32_t c1, const double* diag, double sigma_h2, Two<double>& xc,
                                             Two<double>& ax) {
  stencil_tv<DIM, LdRO>(tv, x, node, c0, c1, diag, xc, ax);
  if (SHIFT) {
    ax.x += sigma_h2 * xc.x;
    ax.y += sigma_h2 * xc.y;
  }
}

// r = b - (sigma I + A) x  (b masked to the CPs); partials (b.b, r.r)
template <int DIM>
__global__ void __launch_bounds__(TILE_NODES) k_resid(TileView tv, const uint8_t* code, const double* diag, OpParams o,
                                                      const double* b, const double* x, double* r, double* part) {
  __shared__ double sm[32];
  double sbb = 0.0, srr = 0.0;
  EB_PAIR_LOOP(DIM, tv, node) {
    uint32_t c0, c1;
    ld_codes(code, node, c0, c1);
    Two<double> xc, ax;
    op_pair<DIM>(tv, x, node, c0, c1, diag, o, xc, ax);
    const Two<double> bv = LdRO::ld2(b + node);
    const double b0 = (c0 & CODE_CP) ? bv.x : 0.0, b1 = (c1 & CODE_CP) ? bv.y : 0.0;
    const double r0 = (c0 & CODE_CP) ? b0 - ax.x : 0.0, r1 = (c1 & CODE_CP) ? b1 - ax.y : 0.0;
    sbb += b0 * b0 + b1 * b1;
    srr += r0 * r0 + r1 * r1;
    st2(r + node, r0, r1);
  }
  const double a = block_sum(sbb, sm);
  const double q = block_sum(srr, sm);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = q;
  }
}

// alpha = rz / p'q from the partials of k_xpby_apply (every CTA; CTA 0 records
// pq, alpha and a breakdown); x += alpha h2 p; r -= alpha q; partial r.r.  q
// holds h^2 (sigma I + A) p (k_xpby_apply), so this alpha is the CG step
// length divided by h2 = h^2.  With rzo_part (flexible CG), also the partial
// of r.z for the new r and the z of the iteration ending (still in z): the
// r.zold term of the Polak-Ribiere beta.
template <int DIM>
__global__ void __launch_bounds__(TILE_NODES) k_update_xr(PairList pl, PcgScalars* sc, double* x, double* r,
                                                          const double* p, const double* q, const double* pq_part,
                                                          int nblk, double* part, double h2, const double* z,
                                                          double* rzo_part) {
  __shared__ double sm[32];
  __shared__ double s_alpha;
  if (cta_done(sc)) {
    if (threadIdx.x == 0) part[blockIdx.x] = 0.0;
    return;
  }
  const double alpha = pcg_alpha(sc, pq_part, nblk, sm, &s_alpha);
  const double ax = alpha * h2;
  double s = 0.0, so = 0.0;
  EB_LIST_LOOP(pl, node) {
    const Two<double> rv = ld2d(r + node), qv = LdRO::ld2(q + node), pv = LdRO::ld2(p + node), xv = ld2d(x + node);
    const double r0 = rv.x - alpha * qv.x, r1 = rv.y - alpha * qv.y;
    st2(x + node, xv.x + ax * pv.x, xv.y + ax * pv.y);
    st2(r + node, r0, r1);
    s += r0 * r0 + r1 * r1;
    if (rzo_part) {
      const Two<double> zv = LdRO::ld2(z + node);
      so += r0 * zv.x + r1 * zv.y;
    }
  }
  if (rzo_part) {
    const double t = block_sum(so, sm);
    if (threadIdx.x == 0) rzo_part[blockIdx.x] = t;
  }
  const double t = block_sum(s, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// z = D^-1 r (Jacobi); partial r.z
template <int DIM>
__global__ void __launch_bounds__(TILE_NODES) k_jacobi_dot(TileView tv, const uint8_t* code, const double* diag,
                                                           OpParams o, const double* r, double* z, double* part) {
  __shared__ double sm[32];
  double s = 0.0;
  EB_PAIR_LOOP(DIM, tv, node) {
    uint32_t c0, c1;
    ld_codes(code, node, c0, c1);
    const Two<double> rv = LdRO::ld2(r + node);
    const double z0 = (c0 & CODE_CP) ? inv_diag(c0, diag, node, o.inv_h2, o.sigma, o.dinv_int) * rv.x : 0.0;
    const double z1 = (c1 & CODE_CP) ? inv_diag(c1, diag, node + 1, o.inv_h2, o.sigma, o.dinv_int) * rv.y : 0.0;
    st2(z + node, z0, z1);
    s += rv.x * z0 + rv.y * z1;
  }
  const double t = block_sum(s, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

template <int DIM>
__global__ void __launch_bounds__(TILE_NODES) k_dot(TileView tv, const double* a, const double* b, double* part) {
  __shared__ double sm[32];
  double s = 0.0;
  EB_PAIR_LOOP(DIM, tv, node) {
    const Two<double> av = LdRO::ld2(a + node), bv = LdRO::ld2(b + node);
    s += av.x * bv.x + av.y * bv.y;
  }
  const double t = block_sum(s, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// The end of a PCG iteration in one pass over the CP pairs: beta = r.z / rz
// (Fletcher-Reeves), or (r.z - r.zold) / rz (Polak-Ribiere, flexible CG: the
// r.zold partials come from the x/r update), computed by every CTA (CTA 0
// records beta, the next rz and a breakdown), p = z + beta p, and the
// operator apply of the next iteration formed as
// q = B z + beta q with B = h^2 (sigma I + A) -- in exact arithmetic B (z +
// beta p), since q holds B p -- with the partials of p.q.  The stencil then
// reads z, which the preconditioner launch before has completed, instead of
// the p this launch writes, so the p update and the apply need no launch
// boundary between them.  nupd: partials per array of the x/r update (r'r,
// r'zold).  COND (device-side loop): CTA 0 also does the loop test and sets
// the loop condition h (a separate instance: profilers cannot replay graph
// kernel nodes that may set a condition).  B is the unit stencil (no 1/h^2
// multiply; the update kernels take the step as alpha h^2 for x), and SHIFT =
// false drops its sigma term for Poisson: two FP64 operations fewer per node
// on GB300's narrow FP64 pipe.  first: beta = 0, p = z, q = B z (the old p and
// q are not read).
template <int DIM, bool SHIFT, bool COND>
__global__ void __launch_bounds__(TILE_NODES) k_xpby_apply(TileView tv, PairList pl, PcgScalars* sc,
                                                           const uint8_t* code, const double* diag, OpParams o,
                                                           const double* z, double* p, double* q, int first,
                                                           const double* rz_part, int nrz, const double* rzo_part,
                                                           int nupd, double* pq_part, const double* rr_part,
                                                           cudaGraphConditionalHandle h) {
  __shared__ double sm[32];
  __shared__ double s_beta;
  if (cta_done(sc)) {
    if (COND && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
    return;
  }
  if (!first) {
    const double v = sum_parts(rz_part, nrz, 1, sm);
    __syncthreads();
    const double t = rzo_part ? sum_parts(rzo_part, nupd, 1, sm) : 0.0;
    if (threadIdx.x == 0) {
      const int k = sc->slot;  // not sc->iters: CTA 0 of this launch may advance it
      const bool ok = v > 0.0;
      const double beta = ok ? (v - t) / sc->rz[k] : 0.0;
      s_beta = beta;
      if (blockIdx.x == 0) {
        sc->beta = beta;
        sc->rz[k ^ 1] = v;
        if (!ok) {
          sc->flags |= isfinite(v) ? PCG_FLAG_BREAKDOWN : PCG_FLAG_NONFINITE;
          sc->done = 1;
        }
      }
    }
    __syncthreads();
  }
  const double beta = first ? 0.0 : s_beta;
  if (COND && blockIdx.x == 0) {
    // the device-side loop's test, after the beta breakdown check: r'r of
    // this iteration's update, then continue while not converged (or broken
    // down) and below the iteration limit.  CTAs that start after it and see
    // done skip the p, q update, which a finished loop does not use.
    const double v = sum_parts(rr_part, nupd, 1, sm);
    if (threadIdx.x == 0) {
      if (!sc->done) {
        sc->rr = v;
        sc->iters += 1;
        if (!isfinite(v)) {
          sc->flags |= PCG_FLAG_NONFINITE;
          sc->done = 1;
        } else if (v <= sc->tol2 * sc->bb) {
          sc->done = 1;
        }
      }
      cudaGraphSetConditional(h, (!sc->done && sc->iters < sc->maxit) ? 1u : 0u);
    }
  }
  double s = 0.0;
  EB_LIST_LOOP(pl, node) {
    uint32_t c0, c1;
    ld_codes(code, node, c0, c1);
    Two<double> zc, az;
    op_pair_unit<DIM, SHIFT>(tv, z, node, c0, c1, diag, o.sigma_h2, zc, az);
    double p0 = zc.x, p1 = zc.y, q0 = az.x, q1 = az.y;
    if (!first) {
      const Two<double> pv = ld2d(p + node), qv = ld2d(q + node);
      p0 = zc.x + beta * pv.x;
      p1 = zc.y + beta * pv.y;
      q0 = az.x + beta * qv.x;
      q1 = az.y + beta * qv.y;
    }
    q0 = (c0 & CODE_CP) ? q0 : 0.0;
    q1 = (c1 & CODE_CP) ? q1 : 0.0;
    st2(p + node, p0, p1);
    st2(q + node, q0, q1);
    s += p0 * q0 + p1 * q1;
  }
  const double t = block_sum(s, sm);
  if (threadIdx.x == 0) pq_part[blockIdx.x] = t;
}

// ------------------------------------------------- the DF outer iteration
// The same iteration with x, r, p, q as double-float vectors (double-float
// pairs in the buffers of doubles) and z in FP32 (the V-cycle's output, exact
// in DF).  The reduction partials are DF too (one per CTA in the 8 bytes of a
// slot), summed in DF by every CTA that needs them -- on the FP32 pipe, where
// the FP64 path's redundant per-CTA sums cost FP64 issue slots -- and rounded
// to FP64 once; alpha and beta are FP64 ratios, split into DF once per CTA.

// the DF copies of beta at the half points, per axis (variable coefficient)
struct DfBeta {
  const float2* b[3] = {nullptr, nullptr, nullptr};
};

// one pair's inputs of k_xpby_apply_df
struct XpIn {
  uint32_t c0, c1;
  float2 zc, dn, up, bk, fr;
  float left, right;
  DF po0, po1, qo0, qo1;
};

template <int DIM>
__device__ __forceinline__ void xp_load(XpIn& in, const TileView& tv, const uint8_t* code, const float* z,
                                        const double* p, const double* q, int first, int32_t node) {
  const int32_t nn = tv.nn, sy = tv.sy, sz = tv.sz;
  ld_codes(code, node, in.c0, in.c1);
  const float2 zero{0.0f, 0.0f};
  in.zc = __ldg(reinterpret_cast<const float2*>(z + node));
  in.left = node > 0 ? __ldg(z + node - 1) : 0.0f;
  in.right = node + 2 < nn ? __ldg(z + node + 2) : 0.0f;
  in.dn = node >= sy ? __ldg(reinterpret_cast<const float2*>(z + node - sy)) : zero;
  in.up = node + sy < nn ? __ldg(reinterpret_cast<const float2*>(z + node + sy)) : zero;
  in.bk = zero;
  in.fr = zero;
  if (dim_of(DIM) == 3) {
    in.bk = node >= sz ? __ldg(reinterpret_cast<const float2*>(z + node - sz)) : zero;
    in.fr = node + sz < nn ? __ldg(reinterpret_cast<const float2*>(z + node + sz)) : zero;
  }
  if (!first) {
    df_ld2_rw(p, node, in.po0, in.po1);
    df_ld2_rw(q, node, in.qo0, in.qo1);
  }
}

// B z at the pair, beta = 1: the neighbour sums by cascaded summation, then
// D_k z_k (an exact product: D_k = 2 dim at interior points, DF for cut ones)
// minus them
template <int D>
__device__ __forceinline__ void xp_unit(const XpIn& in, const float2* diag_df, int32_t node, DF& a0, DF& a1) {
  const uint32_t c0 = in.c0, c1 = in.c1;
  const float2 zc = in.zc;
  Sum2 s0 = sum2_start((c0 & 1) ? 0.0f : in.left), s1 = sum2_start((c1 & 1) ? 0.0f : zc.x);
  sum2_add(s0, (c0 & 2) ? 0.0f : zc.y);
  sum2_add(s1, (c1 & 2) ? 0.0f : in.right);
  sum2_add(s0, (c0 & 4) ? 0.0f : in.dn.x);
  sum2_add(s1, (c1 & 4) ? 0.0f : in.dn.y);
  sum2_add(s0, (c0 & 8) ? 0.0f : in.up.x);
  sum2_add(s1, (c1 & 8) ? 0.0f : in.up.y);
  if (D == 3) {
    sum2_add(s0, (c0 & 16) ? 0.0f : in.bk.x);
    sum2_add(s1, (c1 & 16) ? 0.0f : in.bk.y);
    sum2_add(s0, (c0 & 32) ? 0.0f : in.fr.x);
    sum2_add(s1, (c1 & 32) ? 0.0f : in.fr.y);
  }
  float d0h = (float)(2 * D), d0l = 0.0f, d1h = d0h, d1l = 0.0f;
  if (c0 & 0x7F) {
    const float2 t = __ldg(diag_df + node);
    d0h = t.x;
    d0l = t.y;
  }
  if (c1 & 0x7F) {
    const float2 t = __ldg(diag_df + node + 1);
    d1h = t.x;
    d1l = t.y;
  }
  float pr0, pe0, pr1, pe1;
  two_prod(d0h, zc.x, pr0, pe0);
  two_prod(d1h, zc.y, pr1, pe1);
  pe0 = __fmaf_rn(d0l, zc.x, pe0);
  pe1 = __fmaf_rn(d1l, zc.y, pe1);
  a0 = df_prod_minus_sum2(pr0, pe0, s0);
  a1 = df_prod_minus_sum2(pr1, pe1, s1);
}

// B z at the pair with a variable coefficient (eq. 3): D_k z_k minus the sum
// over the CP neighbours of beta_j z_j, beta_j at the half point between the
// node and the neighbour (beta_df: DF copies per axis), D_k read at every CP;
// the products in DF, summed by the two-step DF sum
template <int D>
__device__ __forceinline__ void xp_varbeta(const XpIn& in, const float2* diag_df, const float2* const* beta_df,
                                           int32_t node, int32_t sy, int32_t sz, DF& a0, DF& a1) {
  const uint32_t c0 = in.c0, c1 = in.c1;
  auto term = [&](uint32_t masked, int a, int32_t at, float v) {
    if (masked) return DF{0.0f, 0.0f};
    const float2 t = __ldg(beta_df[a] + at);
    return df_mul_f(DF{t.x, t.y}, v);
  };
  DF s0 = df_add_fast(term(c0 & 1, 0, node - 1, in.left), term(c0 & 2, 0, node, in.zc.y));
  DF s1 = df_add_fast(term(c1 & 1, 0, node, in.zc.x), term(c1 & 2, 0, node + 1, in.right));
  s0 = df_add_fast(s0, df_add_fast(term(c0 & 4, 1, node - sy, in.dn.x), term(c0 & 8, 1, node, in.up.x)));
  s1 = df_add_fast(s1, df_add_fast(term(c1 & 4, 1, node - sy + 1, in.dn.y), term(c1 & 8, 1, node + 1, in.up.y)));
  if (D == 3) {
    s0 = df_add_fast(s0, df_add_fast(term(c0 & 16, 2, node - sz, in.bk.x), term(c0 & 32, 2, node, in.fr.x)));
    s1 = df_add_fast(s1, df_add_fast(term(c1 & 16, 2, node - sz + 1, in.bk.y), term(c1 & 32, 2, node + 1, in.fr.y)));
  }
  const float2 e0 = (c0 & CODE_CP) ? __ldg(diag_df + node) : make_float2(0.0f, 0.0f);
  const float2 e1 = (c1 & CODE_CP) ? __ldg(diag_df + node + 1) : make_float2(0.0f, 0.0f);
  a0 = df_sub(df_mul_f(DF{e0.x, e0.y}, in.zc.x), s0);
  a1 = df_sub(df_mul_f(DF{e1.x, e1.y}, in.zc.y), s1);
}

// p, q of one pair from its inputs; the pair's p.q terms added to s.  DIM
// carrying DIM_VB: the variable-coefficient stencil
template <int DIM, bool SHIFT>
__device__ __forceinline__ void xp_compute(const XpIn& in, const float2* diag_df, DF sig_h2, DF beta, int first,
                                           double* p, double* q, int32_t node, DF& s, const float2* const* beta_df,
                                           int32_t sy, int32_t sz) {
  const uint32_t c0 = in.c0, c1 = in.c1;
  const float2 zc = in.zc;
  DF a0, a1;
  if constexpr ((DIM & DIM_VB) != 0) xp_varbeta<dim_of(DIM)>(in, diag_df, beta_df, node, sy, sz, a0, a1);
  else xp_unit<dim_of(DIM)>(in, diag_df, node, a0, a1);
  if (SHIFT) {
    a0 = df_add(a0, df_mul_f(sig_h2, zc.x));
    a1 = df_add(a1, df_mul_f(sig_h2, zc.y));
  }
  DF p0 = df_make(zc.x), p1 = df_make(zc.y), q0 = a0, q1 = a1;
  if (!first) {
    p0 = df_add_f(df_mul(beta, in.po0), zc.x);
    p1 = df_add_f(df_mul(beta, in.po1), zc.y);
    q0 = df_add_fast(df_mul(beta, in.qo0), a0);
    q1 = df_add_fast(df_mul(beta, in.qo1), a1);
  }
  if (!(c0 & CODE_CP)) q0 = DF{0.0f, 0.0f};
  if (!(c1 & CODE_CP)) q1 = DF{0.0f, 0.0f};
  df_st2(p, node, p0, p1);
  df_st2(q, node, q0, q1);
  df_acc_prod(s, p0, q0);
  df_acc_prod(s, p1, q1);
}

// The end of an iteration (k_xpby_apply in DF): p = z + beta p, q = B z + beta
// q, the p.q partials.  B z is the unit stencil D_k z_k - sum of the
// CP-neighbour values on the FP32 z: the neighbours by cascaded summation
// (TwoSum errors collected), D_k z_k an exact product (interior points) or a
// DF one (cut points), plus sigma h^2 z_k when SHIFT; with a variable
// coefficient (DIM_VB) the beta-weighted form of xp_varbeta.  The loads of a
// thread's first pair are issued before
// the partial sums that give beta (the pass is bound by its load latency; a
// double-buffered loop that also issued each pair's loads before the previous
// pair's arithmetic was no faster).
template <int DIM, bool SHIFT, bool COND>
__global__ void __launch_bounds__(TILE_NODES) k_xpby_apply_df(TileView tv, PairList pl, PcgScalars* sc,
                                                              const uint8_t* code, const float2* diag_df, DF sig_h2,
                                                              const float* z, double* p, double* q, int first,
                                                              const double* rz_part, int nrz, const double* rzo_part,
                                                              int nupd, double* pq_part, const double* rr_part,
                                                              cudaGraphConditionalHandle h, DfBeta bdf) {
  __shared__ DF dsm[32];
  __shared__ DF s_beta;
  if (cta_done(sc)) {
    if (COND && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
    return;
  }
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  XpIn cur;
  int32_t node = li < pl.n ? __ldg(pl.node + li) : 0;
  if (li < pl.n) xp_load<DIM>(cur, tv, code, z, p, q, first, node);
  if (threadIdx.x == 0) s_beta = DF{0.0f, 0.0f};
  if (!first) {
    const double v = df_sum_parts(rz_part, nrz, dsm);
    __syncthreads();
    const double t = rzo_part ? df_sum_parts(rzo_part, nupd, dsm) : 0.0;
    if (threadIdx.x == 0) {
      const int k = sc->slot;
      const bool ok = v > 0.0;
      const double beta = ok ? (v - t) / sc->rz[k] : 0.0;
      s_beta = df_from_double(beta);
      if (blockIdx.x == 0) {
        sc->beta = beta;
        sc->rz[k ^ 1] = v;
        if (!ok) {
          sc->flags |= isfinite(v) ? PCG_FLAG_BREAKDOWN : PCG_FLAG_NONFINITE;
          sc->done = 1;
        }
      }
    }
  }
  __syncthreads();
  const DF beta = s_beta;
  if (COND && blockIdx.x == 0) {
    const double v = df_sum_parts(rr_part, nupd, dsm);
    if (threadIdx.x == 0) {
      if (!sc->done) {
        sc->rr = v;
        sc->iters += 1;
        if (!isfinite(v)) {
          sc->flags |= PCG_FLAG_NONFINITE;
          sc->done = 1;
        } else if (v <= sc->tol2 * sc->bb) {
          sc->done = 1;
        }
      }
      cudaGraphSetConditional(h, (!sc->done && sc->iters < sc->maxit) ? 1u : 0u);
    }
  }
  DF s{0.0f, 0.0f};
  while (li < pl.n) {
    const int64_t ln = li + step;
    const int32_t nnode = ln < pl.n ? __ldg(pl.node + ln) : 0;
    xp_compute<DIM, SHIFT>(cur, diag_df, sig_h2, beta, first, p, q, node, s, bdf.b, tv.sy, tv.sz);
    if (ln < pl.n) xp_load<DIM>(cur, tv, code, z, p, q, first, nnode);
    li = ln;
    node = nnode;
  }
  const DF t = df_block_sum_df(s, dsm);
  if (threadIdx.x == 0) df_part_store(pq_part, blockIdx.x, t);
}

// Into DF: xd = scale x and, in place, r = scale r (FP64 -> DF), over the CP
// pairs; scale is a power of two (exact), chosen so that the scaled right-hand
// side has a unit root mean square, well inside FP32's exponent range.
__global__ void __launch_bounds__(TILE_NODES) k_df_in(PairList pl, const double* x, double* xd, double* r,
                                                      double scale) {
  EB_LIST_LOOP(pl, node) {
    const Two<double> xv = ld2d(x + node), rv = ld2d(r + node);
    df_st2(xd, node, df_from_double(xv.x * scale), df_from_double(xv.y * scale));
    df_st2(r, node, df_from_double(rv.x * scale), df_from_double(rv.y * scale));
  }
}

// Out of DF: x = xd / scale over the CP pairs
__global__ void __launch_bounds__(TILE_NODES) k_df_out(PairList pl, const double* xd, double* x, double inv_scale) {
  EB_LIST_LOOP(pl, node) {
    DF a, b;
    df_ld2_rw(xd, node, a, b);
    st2(x + node, df_to_double(a) * inv_scale, df_to_double(b) * inv_scale);
  }
}

// the DF copy of one axis of beta (every node: the stencil reads it at the
// neighbours' half points)
__global__ void k_df_full(int64_t n, const double* __restrict__ v, float2* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const DF d = df_from_double(v[i]);
    out[i] = make_float2(d.hi, d.lo);
  }
}

// the DF copy of the cut CPs' diagonals D_k (the interior value 2 dim is
// formed in the kernel; with a variable coefficient every CP's D_k)
__global__ void __launch_bounds__(TILE_NODES) k_df_diag(PairList pl, const uint8_t* code, const double* diag,
                                                        float2* out) {
  EB_LIST_LOOP(pl, node) {
    uint32_t c0, c1;
    ld_codes(code, node, c0, c1);
    if (c0 & 0x7F) {
      const DF v = df_from_double(diag[node]);
      out[node] = make_float2(v.hi, v.lo);
    }
    if (c1 & 0x7F) {
      const DF v = df_from_double(diag[node + 1]);
      out[node + 1] = make_float2(v.hi, v.lo);
    }
  }
}

// Right-hand side and guess of one implicit theta-scheme wave step (Sec. 3.5,
// theta > 0): (sigma I + A) u^{n+1} = sigma (2 u^n - u^{n-1}) - c A u^n -
// A u^{n-1}, sigma = 1 / (theta dt^2), c = (1 - 2 theta) / theta (the scheme
// divided by theta dt^2); guess = 2 u^n - u^{n-1} (0 off the CPs).
template <int DIM>
__global__ void __launch_bounds__(TILE_NODES) k_wave_theta_rhs(TileView tv, const uint8_t* code, const double* diag,
                                                               double inv_h2, double sigma, double c,
                                                               const double* un, const double* um, double* rhs,
                                                               double* guess) {
  EB_PAIR_LOOP(DIM, tv, node) {
    uint32_t c0, c1;
    ld_codes(code, node, c0, c1);
    Two<double> uc, ucore, mc, mcore;
    stencil_tv<DIM, LdRO>(tv, un, node, c0, c1, diag, uc, ucore);
    stencil_tv<DIM, LdRO>(tv, um, node, c0, c1, diag, mc, mcore);
    const double g0 = 2.0 * uc.x - mc.x, g1 = 2.0 * uc.y - mc.y;
    const double r0 = sigma * g0 - c * (ucore.x * inv_h2) - mcore.x * inv_h2;
    const double r1 = sigma * g1 - c * (ucore.y * inv_h2) - mcore.y * inv_h2;
    st2(rhs + node, (c0 & CODE_CP) ? r0 : 0.0, (c1 & CODE_CP) ? r1 : 0.0);
    st2(guess + node, (c0 & CODE_CP) ? g0 : 0.0, (c1 & CODE_CP) ? g1 : 0.0);
  }
}

// (a, b) <- (b, a) over the active tiles
template <int DIM>
__global__ void __launch_bounds__(TILE_NODES) k_swap_tiles(TileView tv, double* a, double* b) {
  EB_PAIR_LOOP(DIM, tv, node) {
    const Two<double> va = ld2d(a + node), vb = ld2d(b + node);
    st2(a + node, vb.x, vb.y);
    st2(b + node, va.x, va.y);
  }
}

template <int DIM>
__global__ void __launch_bounds__(TILE_NODES) k_copy_tiles(TileView tv, const double* a, double* b) {
  EB_PAIR_LOOP(DIM, tv, node) {
    const Two<double> v = LdRO::ld2(a + node);
    st2(b + node, v.x, v.y);
  }
}

// rhs of the theta-method: (u/dt - (1-theta) A u + theta b1 + (1-theta) b0) / theta
template <int DIM>
__global__ void __launch_bounds__(TILE_NODES) k_heat_rhs(TileView tv, const uint8_t* code, const double* diag,
                                                         double inv_h2, double dt, double theta, const double* u,
                                                         const double* b1, const double* b0, double* out) {
  EB_PAIR_LOOP(DIM, tv, node) {
    uint32_t c0, c1;
    ld_codes(code, node, c0, c1);
    Two<double> uc, core;
    stencil_tv<DIM, LdRO>(tv, u, node, c0, c1, diag, uc, core);
    const Two<double> b1v = LdRO::ld2(b1 + node), b0v = LdRO::ld2(b0 + node);
    double v0 = uc.x / dt + theta * b1v.x, v1 = uc.y / dt + theta * b1v.y;
    if (theta < 1.0) {
      v0 += (1.0 - theta) * (b0v.x - core.x * inv_h2);
      v1 += (1.0 - theta) * (b0v.y - core.y * inv_h2);
    }
    st2(out + node, (c0 & CODE_CP) ? v0 / theta : 0.0, (c1 & CODE_CP) ? v1 / theta : 0.0);
  }
}

template <int DIM>
__global__ void __launch_bounds__(TILE_NODES) k_mask_copy(TileView tv, const uint8_t* code, const double* in,
                                                          double* out) {
  EB_PAIR_LOOP(DIM, tv, node) {
    uint32_t c0, c1;
    ld_codes(code, node, c0, c1);
    const Two<double> v = ld2d(in + node);
    st2(out + node, (c0 & CODE_CP) ? v.x : 0.0, (c1 & CODE_CP) ? v.y : 0.0);
  }
}

// Combine partials in a fixed order and advance the scalar recurrences.
// df: the partials are DF (the DF outer iteration; never FIN_INIT), each
// thread's share summed in DF and rounded once
__global__ void k_finalize(const double* part, int nblk, int op, PcgScalars* sc, int df) {
  __shared__ double sm[2][1024];
  double a = 0.0, b = 0.0;
  const bool pairs = op == FIN_INIT;
  const int stride = pairs ? 2 : 1;
  if (df) {
    DF t{0.0f, 0.0f};
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) t = df_add(t, df_part_load(part, i));
    a = df_to_double(t);
  } else {
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
      a += part[stride * i];
      if (pairs) b += part[2 * i + 1];
    }
  }
  sm[0][threadIdx.x] = a;
  sm[1][threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sm[0][threadIdx.x] += sm[0][threadIdx.x + o];
      sm[1][threadIdx.x] += sm[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double v = sm[0][0];
  switch (op) {
    case FIN_INIT:
      sc->bb = v;
      sc->rr = sm[1][0];
      if (!isfinite(v) || !isfinite(sm[1][0])) sc->flags |= PCG_FLAG_NONFINITE;
      sc->done = (sm[1][0] <= sc->tol2 * v) ? 1 : 0;
      break;
    case FIN_RZ0:
      sc->rz[sc->iters & 1] = v;
      if (!isfinite(v)) sc->flags |= PCG_FLAG_NONFINITE;
      break;
    case FIN_RR:
      if (sc->done) break;
      sc->rr = v;
      sc->iters += 1;
      if (!isfinite(v)) {
        sc->flags |= PCG_FLAG_NONFINITE;
        sc->done = 1;
      } else if (v <= sc->tol2 * sc->bb) {
        sc->done = 1;
      }
      break;
  }
}

// ---------------------------------------------------------------- host side
#define EB_DIM_LAUNCH(dim, kernel, grid, ...)                                 \
  do {                                                                       \
    ++nlaunch;                                                               \
    if ((dim) == 2)                                                          \
      kernel<2><<<(grid), TILE_NODES, 0, s>>>(__VA_ARGS__);                  \
    else                                                                     \
      kernel<3><<<(grid), TILE_NODES, 0, s>>>(__VA_ARGS__);                  \
  } while (0)

// EB_DIM_LAUNCH for the kernels that apply the stencil: the grid's dimension
// with DIM_VB for a variable beta (dim_dispatch)
#define EB_DIMV_LAUNCH(ebh, kernel, grid, ...)                                        \
  do {                                                                                \
    ++nlaunch;                                                                        \
    dim_dispatch((ebh), [&](auto D_) { kernel<D_.value><<<(grid), TILE_NODES, 0, s>>>(__VA_ARGS__); }); \
  } while (0)

static OpParams op_params(const Solver& S) {
  const Geometry& G = S.eb->g;
  OpParams o;
  o.inv_h2 = 1.0 / (G.h * G.h);
  o.sigma = S.shift;
  o.dinv_int = 1.0 / (S.shift + 2.0 * G.dim * o.inv_h2);
  o.sigma_h2 = S.shift * G.h * G.h;
  return o;
}

void Solver::alloc_work(cudaStream_t s) {
  const int64_t nn = eb->g.num_nodes;
  r = dalloc<double>(nn, s);
  z = dalloc<double>(nn, s);
  p = dalloc<double>(nn, s);
  q = dalloc<double>(nn, s);
  tmp = dalloc<double>(nn, s);
  nblk = (int)std::min<int64_t>(std::max<int64_t>(eb->num_tiles, 1), (int64_t)num_sms() * 4);
  // p'q and r'r regions of 2 nblk, r'z of 2 max(nblk, 8 SMs) (the V-cycle's
  // grid sweeps use at most 8 CTAs per SM), then r'zold of nblk
  rz_cap = 2 * std::max<int64_t>(nblk, (int64_t)num_sms() * 8);
  part = dalloc<double>(5 * (int64_t)nblk + rz_cap, s);
  sc = dalloc<PcgScalars>(1, s);
  EB_CUDA(cudaMallocHost((void**)&sc_host, sizeof(PcgScalars)));
}

void Solver::free_work() {
  cudaStream_t s = home;
  graph_release();
  loop_release();
  if (cap_stream) cudaStreamDestroy(cap_stream);
  cap_stream = nullptr;
  dfree(r, s); dfree(z, s); dfree(p, s); dfree(q, s); dfree(tmp, s); dfree(part, s); dfree(sc, s); dfree(wx, s);
  dfree(diag_df, s); dfree(xdf, s); dfree(dev_err, s);
  for (auto& bd : beta_df) dfree(bd, s);
  if (sc_host) cudaFreeHost(sc_host);
  sc_host = nullptr;
}

void Solver::finalize(int op, const double* src, cudaStream_t s, int count) {
  ++nlaunch;
  k_finalize<<<1, 1024, 0, s>>>(src, count < 0 ? nblk : count, op, sc, (df_on && op != FIN_INIT) ? 1 : 0);
}

void Solver::precondition(int kind, const double* rin, double* zout, cudaStream_t s, bool first_done) {
  const int dim = eb->g.dim;
  const TileView tv = eb->tv();
  rz_n = nblk;
  if (kind == EB_PC_AMG_NN) {
    amg_vcycle_grid(*this, rin, zout, s);
    nn_stage_apply(nn, *eb, shift, nn_mode, rin, zout, nlaunch, this, s);
    EB_DIM_LAUNCH(dim, k_dot, nblk, tv, rin, zout, part_rz());
  } else if (kind == EB_PC_AMG && H) {
    // the V-cycle's last smoothing launch forms the r'z partials itself
    VcycleDot dot;
    dot.r = rin;
    dot.part = part_rz();
    dot.df = df_on;
    const int fused = amg_vcycle_grid(*this, rin, zout, s, &dot, first_done);
    if (fused) {
      rz_n = fused;
      return;
    }  // single-level hierarchy: no smoothing launch formed them
    EB_DIM_LAUNCH(dim, k_dot, nblk, tv, rin, zout, part_rz());
  } else if (kind == EB_PC_NONE) {
    EB_DIM_LAUNCH(dim, k_copy_tiles, nblk, tv, rin, zout);
    EB_DIM_LAUNCH(dim, k_dot, nblk, tv, rin, zout, part_rz());
  } else {
    EB_DIM_LAUNCH(dim, k_jacobi_dot, nblk, tv, eb->code, eb->diag, op_params(*this), rin, zout, part_rz());
  }
}

// the outer precision of the option-less solves: outer_default where the DF
// iteration applies (AMG with a reduced-precision V-cycle of two or more
// levels), else FP64
int Solver::default_outer() const {
  return (outer_default == EB_DF64 && H && flexible() && amg_levels(*this) > 1) ? EB_DF64 : EB_F64;
}

int Solver::pcg(const double* b, double* x, double rtol, int maxit, const pcg_opts& o, pcg_stats* stats,
                cudaStream_t s) {
  const int dim = eb->g.dim;
  const TileView tv = eb->tv();
  const OpParams op = op_params(*this);
  const int kind = o.precond;
  EB_REQUIRE(kind == EB_PC_AMG || kind == EB_PC_JACOBI || kind == EB_PC_NONE || kind == EB_PC_AMG_NN,
             EB_ERR_INVALID, "bad preconditioner");
  EB_REQUIRE(kind != EB_PC_AMG_NN || nn != nullptr, EB_ERR_INVALID,
             "the learned stage is selected by pcg_solve_nn");
  EB_REQUIRE((kind != EB_PC_AMG && kind != EB_PC_AMG_NN) || H != nullptr, EB_ERR_INVALID,
             "AMG preconditioner requested without a hierarchy");
  EB_REQUIRE(rtol > 0.0 && maxit >= 0, EB_ERR_INVALID, "rtol must be > 0 and maxit >= 0");
  EB_REQUIRE(b != x, EB_ERR_INVALID, "pcg: b and x must be different buffers");
  EB_REQUIRE(eb->pair_node != nullptr || eb->num_cp == 0, EB_ERR_INVALID, "pcg: the handle has no CP pair list");
  const int check = std::max(1, o.check_every);
  EB_REQUIRE(o.outer_prec == EB_F64 || o.outer_prec == EB_DF64, EB_ERR_INVALID,
             "pcg: outer_prec must be EB_F64 or EB_DF64");
  df_on = o.outer_prec == EB_DF64;
  if (df_on) {
    EB_REQUIRE(kind == EB_PC_AMG && flexible() && amg_levels(*this) > 1, EB_ERR_NOT_IMPLEMENTED,
               "pcg: the DF outer iteration needs the AMG preconditioner with an FP32 or BF16 V-cycle of at least "
               "two levels");
    // the DF copies of D_k and beta, rebuilt when the handle's geometry, tiles
    // or beta changed (tile_gen)
    if (!diag_df || df_gen != eb->tile_gen) {
      if (!diag_df) diag_df = dalloc<float2>(eb->g.num_nodes, s);
      ++nlaunch;
      k_df_diag<<<nblk, TILE_NODES, 0, s>>>(eb->pairs(), eb->code, eb->diag, diag_df);
      for (int a = 0; a < 3; ++a) {
        if (eb->has_beta() && a < eb->g.dim) {
          if (!beta_df[a]) beta_df[a] = dalloc<float2>(eb->g.num_nodes, s);
          ++nlaunch;
          k_df_full<<<(unsigned)(num_sms() * 8), 256, 0, s>>>(eb->g.num_nodes, eb->beta64[a], beta_df[a]);
        } else {
          dfree(beta_df[a], s);
        }
      }
      df_gen = eb->tile_gen;
    }
    if (!xdf) xdf = dalloc<double>(eb->g.num_nodes, s);
  }
  // the vector the iteration updates: x itself, or its DF image
  double* xi = df_on ? xdf : x;
  prof_begin(o.profile, s);
  nlaunch = 0;
  auto t0 = std::chrono::steady_clock::now();
  PcgScalars init{};
  init.tol2 = rtol * rtol;
  int total_iters = 0;
  const int pcg_maxit = maxit;
  bool converged = false;
  int flags = 0;
  double rel = 0.0;
  for (int restart = 0; restart < 4 && !converged; ++restart) {
    init.maxit = pcg_maxit - total_iters;
    EB_CUDA(cudaMemcpyAsync(sc, &init, sizeof(init), cudaMemcpyHostToDevice, s));
    // x is masked to the CPs (its non-CP entries are ignored on input)
    EB_DIM_LAUNCH(dim, k_mask_copy, nblk, tv, eb->code, x, x);
    EB_DIMV_LAUNCH(*eb, k_resid, nblk, tv, eb->code, eb->diag, op, b, x, r, part_pq());
    finalize(FIN_INIT, part_pq(), s);
    EB_CUDA(cudaMemcpyAsync(sc_host, sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
    EB_CUDA(cudaStreamSynchronize(s));
    if (sc_host->flags & PCG_FLAG_NONFINITE) {
      flags |= sc_host->flags;
      break;
    }
    if (sc_host->bb == 0.0) {  // b = 0: x = 0 is the solution
      EB_DIM_LAUNCH(dim, k_mask_copy, nblk, tv, eb->code, b, x);
      converged = true;
      rel = 0.0;
      break;
    }
    if (sc_host->done) {
      converged = true;
      rel = std::sqrt(sc_host->rr / sc_host->bb);
      break;
    }
    if (total_iters >= maxit) break;
    double scale = 1.0;
    if (df_on) {
      // scale by a power of two so that the scaled b has a unit root mean square
      const double ms = sc_host->bb / (double)std::max<int64_t>(eb->num_cp, 1);
      scale = std::ldexp(1.0, -(int)std::lround(0.5 * std::log2(ms)));
      ++nlaunch;
      k_df_in<<<nblk, TILE_NODES, 0, s>>>(eb->pairs(), x, xi, r, scale);
      sc_host->bb *= scale * scale;
      sc_host->rr *= scale * scale;
      EB_CUDA(cudaMemcpyAsync(sc, sc_host, sizeof(PcgScalars), cudaMemcpyHostToDevice, s));
    }
    precondition(kind, r, z, s);
    const bool flex = flex_for(kind);
    finalize(FIN_RZ0, part_rz(), s, rz_n);
    xpby_apply(op, flex, 1, s);
    int it = 0;
    bool stop = false;
    if (o.use_graph == 1 && !prof_on) {  // the whole loop on the device
      loop_prepare(kind, b, xi, s);
      EB_CUDA(cudaGraphLaunch(lexec, s));
      EB_CUDA(cudaMemcpyAsync(sc_host, sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
      EB_CUDA(cudaStreamSynchronize(s));
      nlaunch += l_launches * sc_host->iters;
      stop = true;
    }
    while (!stop) {
      const int nb = std::min(check, maxit - (total_iters + it));
      bool graphed = false;
      if (o.use_graph && nb == check) {
        graph_prepare(kind, b, xi, check, prof_on ? prof_what : 0, s);
        EB_CUDA(cudaGraphLaunch(gexec, s));
        nlaunch += g_launches;
        graphed = true;
        it += nb;
      } else {
        for (int j = 0; j < nb; ++j, ++it) iteration(kind, b, xi, s);
      }
      EB_CUDA(cudaGetLastError());
      EB_CUDA(cudaMemcpyAsync(sc_host, sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
      EB_CUDA(cudaStreamSynchronize(s));
      if (prof_on) {
        if (graphed) prof_collect(0, g_pairs);
        prof_collect(g_pairs, prof_n - g_pairs);
        prof_n = g_pairs;
      }
      if (sc_host->done || total_iters + it >= maxit) stop = true;
    }
    total_iters += sc_host->iters;
    flags |= sc_host->flags;
    if (df_on) {
      ++nlaunch;
      k_df_out<<<nblk, TILE_NODES, 0, s>>>(eb->pairs(), xi, x, 1.0 / scale);
    }
    if (flags & (PCG_FLAG_NONFINITE | PCG_FLAG_BREAKDOWN)) break;
    // true residual at exit (FP64)
    EB_DIMV_LAUNCH(*eb, k_resid, nblk, tv, eb->code, eb->diag, op, b, x, r, part_pq());
    finalize(FIN_INIT, part_pq(), s);
    EB_CUDA(cudaMemcpyAsync(sc_host, sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
    EB_CUDA(cudaStreamSynchronize(s));
    rel = sc_host->bb > 0 ? std::sqrt(sc_host->rr / sc_host->bb) : 0.0;
    if (sc_host->done) converged = true;
    if (total_iters >= maxit) break;
  }
  auto t1 = std::chrono::steady_clock::now();
  if (stats) {
    stats->iterations = total_iters;
    stats->rel_residual = rel;
    stats->true_rel_residual = rel;
    stats->solve_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    stats->converged = converged ? 1 : 0;
    stats->launches = nlaunch;
    prof_end(stats, s);
  }
  if (flags & PCG_FLAG_NONFINITE) {
    set_error("pcg: non-finite value in the right-hand side or a reduction");
    return EB_ERR_NONFINITE;
  }
  if (flags & PCG_FLAG_BREAKDOWN) {
    set_error("pcg: breakdown (p^T A p <= 0 or r^T z <= 0)");
    return EB_ERR_BREAKDOWN;
  }
  if (!converged) {
    set_error("pcg: maximum number of iterations reached");
    return EB_ERR_NO_CONVERGENCE;
  }
  return EB_OK;
}

int Solver::heat(double dt, double theta, const double* b1, const double* b0, double* u, double rtol, int maxit,
                 pcg_stats* stats, cudaStream_t s) {
  EB_REQUIRE(dt > 0.0 && theta > 0.0 && theta <= 1.0, EB_ERR_INVALID, "heat: need dt > 0 and 0 < theta <= 1");
  EB_REQUIRE(theta == 1.0 || b0 != nullptr, EB_ERR_INVALID, "heat: b0 required when theta < 1");
  const double want = 1.0 / (theta * dt);
  EB_REQUIRE(std::fabs(want - shift) <= 1e-12 * want, EB_ERR_INVALID,
             "heat: the hierarchy shift must equal 1/(theta dt)");
  const Geometry& G = eb->g;
  EB_DIMV_LAUNCH(*eb, k_heat_rhs, nblk, eb->tv(), eb->code, eb->diag, 1.0 / (G.h * G.h), dt, theta, u, b1,
                b0 ? b0 : b1, tmp);
  EB_CUDA(cudaGetLastError());
  // the loop on the device (tmp and u keep their addresses); the solver's
  // default outer precision (amg_set_outer_prec) where it applies
  pcg_opts o{H ? EB_PC_AMG : EB_PC_JACOBI, 1, 1, 0, default_outer()};
  return pcg(tmp, u, rtol, maxit, o, stats, s);
}

// nsteps implicit theta-scheme wave steps (Sec. 3.5): per step the right-hand
// side and the guess 2 u^n - u^{n-1} in one pass, AMG-PCG (device loop) into
// the solver's own x vector (fixed, so the captured loop is reused), and the
// result copied over u^{n-1}, whose buffer then plays u^n.
int Solver::wave_theta(double dt, double theta, double* ua, double* ub, int nsteps, double rtol, int maxit,
                       pcg_stats* stats, cudaStream_t s) {
  EB_REQUIRE(dt > 0.0 && theta > 0.0 && nsteps >= 0, EB_ERR_INVALID, "wave_theta_step: need dt > 0, theta > 0");
  const double sigma = 1.0 / (theta * dt * dt);
  EB_REQUIRE(std::fabs(sigma - shift) <= 1e-12 * sigma, EB_ERR_INVALID,
             "wave_theta_step: the hierarchy shift must equal 1/(theta dt^2)");
  const Geometry& G = eb->g;
  if (!wx) wx = dalloc<double>(G.num_nodes, s);
  const double c = (1.0 - 2.0 * theta) / theta;
  const double inv_h2 = 1.0 / (G.h * G.h);
  const TileView tv = eb->tv();
  pcg_opts o{H ? EB_PC_AMG : EB_PC_JACOBI, 1, 1, 0, default_outer()};
  pcg_stats total{};
  total.converged = 1;
  int rc = EB_OK;
  for (int k = 0; k < nsteps && rc == EB_OK; ++k) {
    double* prev = (k & 1) ? ub : ua;
    const double* cur = (k & 1) ? ua : ub;
    EB_DIMV_LAUNCH(*eb, k_wave_theta_rhs, nblk, tv, eb->code, eb->diag, inv_h2, sigma, c, cur, prev, tmp, wx);
    EB_CUDA(cudaGetLastError());
    pcg_stats st{};
    rc = pcg(tmp, wx, rtol, maxit, o, &st, s);
    EB_DIM_LAUNCH(G.dim, k_copy_tiles, nblk, tv, wx, prev);
    total.iterations += st.iterations;
    total.rel_residual = std::max(total.rel_residual, st.rel_residual);
    total.true_rel_residual = std::max(total.true_rel_residual, st.true_rel_residual);
    total.solve_ms += st.solve_ms;
    total.launches += st.launches + 2;
    total.converged = total.converged && st.converged;
  }
  if (rc == EB_OK && (nsteps & 1)) EB_DIM_LAUNCH(G.dim, k_swap_tiles, nblk, tv, ua, ub);
  EB_CUDA(cudaGetLastError());
  EB_CUDA(cudaStreamSynchronize(s));
  if (stats) *stats = total;
  return rc;
}

// One PCG iteration (device-side scalars; no host synchronisation).
// the k_xpby_apply instance for the dimension, the shift and the loop test
template <bool SHIFT, bool COND>
static void launch_xpby_apply(const EBHandle& eb, unsigned g, cudaStream_t s, const TileView& tv, const PairList& pl,
                              PcgScalars* sc, const uint8_t* code, const double* diag, const OpParams& op,
                              const double* z, double* p, double* q, int first, const double* rz, int nrz,
                              const double* rzo, int nupd, double* pq, const double* rr,
                              cudaGraphConditionalHandle h) {
  dim_dispatch(eb, [&](auto D) {
    k_xpby_apply<D.value, SHIFT, COND><<<g, TILE_NODES, 0, s>>>(tv, pl, sc, code, diag, op, z, p, q, first, rz, nrz,
                                                                rzo, nupd, pq, rr, h);
  });
}

void Solver::xpby_apply(const OpParams& op, bool flex, int first, cudaStream_t s,
                        const cudaGraphConditionalHandle* cond) {
  const TileView tv = eb->tv();
  const PairList pl = eb->pairs();
  const unsigned g = (unsigned)nblk_iter();
  const int dim = eb->g.dim;
  const double* rzo = flex ? part_rzo() : nullptr;
  const cudaGraphConditionalHandle h = cond ? *cond : cudaGraphConditionalHandle{};
  ++nlaunch;
  auto go = [&](auto shift, auto with_cond) {
    constexpr bool SH = decltype(shift)::value, CO = decltype(with_cond)::value;
    if (df_on) {
      const DF sig = df_from_double(op.sigma_h2);
      const float* zf = reinterpret_cast<const float*>(z);
      DfBeta bdf;
      for (int a = 0; a < 3; ++a) bdf.b[a] = beta_df[a];
      dim_dispatch(*eb, [&](auto D) {
        k_xpby_apply_df<D.value, SH, CO><<<g, TILE_NODES, 0, s>>>(tv, pl, sc, eb->code, diag_df, sig, zf, p, q, first,
                                                                  part_rz(), rz_n, rzo, (int)g, part_pq(), part_rr(),
                                                                  h, bdf);
      });
      return;
    }
    launch_xpby_apply<SH, CO>(*eb, g, s, tv, pl, sc, eb->code, eb->diag, op, z, p, q, first, part_rz(), rz_n, rzo,
                              nblk, part_pq(), part_rr(), h);
  };
  using T = std::true_type;
  using F = std::false_type;
  if (op.sigma_h2 != 0.0) {
    if (cond) go(T{}, T{});
    else go(T{}, F{});
  } else {
    if (cond) go(F{}, T{});
    else go(F{}, F{});
  }
}

void Solver::iteration(int kind, const double* b, double* x, cudaStream_t s,
                       const cudaGraphConditionalHandle* cond) {
  (void)b;
  const int dim = eb->g.dim;
  const OpParams op = op_params(*this);
  const bool flex = flex_for(kind);
  // q = h^2 (sigma I + A) p and the p.q partials come from the previous
  // k_xpby_apply; with an AMG V-cycle next, the x/r update also does its first
  // level-0 step
  prof_mark(s, true, PROF_UPDATE);  // exactly one launch until the matching mark: fused or not
  bool fused = false;
  if (kind == EB_PC_AMG && H) {
    PcgUpdate u;
    u.sc = sc;
    u.x = x;
    u.r = r;
    u.p = p;
    u.q = q;
    u.pq_part = part_pq();
    u.nblk = nblk_iter();
    u.rr_part = part_rr();
    u.h2 = eb->g.h * eb->g.h;
    u.z = z;
    u.rzo_part = flex ? part_rzo() : nullptr;
    u.df = df_on;
    fused = amg_update_first(*this, u, s) != 0;
    if (fused) ++nlaunch;
  }
  EB_REQUIRE(fused || !df_on, EB_ERR_INVALID, "pcg: the DF outer iteration needs the fused x/r update");
  if (!fused)
    EB_DIM_LAUNCH(dim, k_update_xr, nblk, eb->pairs(), sc, x, r, p, q, part_pq(), nblk, part_rr(), eb->g.h * eb->g.h, z,
                  flex ? part_rzo() : nullptr);
  prof_mark(s, false, PROF_UPDATE);
  precondition(kind, r, z, s, fused);
  // r'r and the convergence test end the iteration: in the device-side loop
  // the p, q launch does them and sets the loop condition
  prof_mark(s, true, PROF_XPBY);
  xpby_apply(op, flex, 0, s, cond);
  prof_mark(s, false, PROF_XPBY);
  if (!cond) finalize(FIN_RR, part_rr(), s, nblk_iter());
}

// Captures `iters` iterations into a CUDA graph (once per argument set).  The
// capture runs on a private stream forked from s, so s may be the legacy
// default stream.
void Solver::graph_prepare(int kind, const double* b, double* x, int iters, int profile, cudaStream_t s) {
  if (gexec && g_b == b && g_x == x && g_iters == iters && g_kind == kind && g_prof == profile && g_nn == nn &&
      g_nn_mode == nn_mode && g_tile_gen == eb->tile_gen && g_df == (int)df_on)
    return;
  if (prof_on) {  // settle event pairs recorded so far before the capture reuses them
    EB_CUDA(cudaStreamSynchronize(s));
    prof_collect(g_pairs, prof_n - g_pairs);
  }
  graph_release();
  if (!cap_stream) EB_CUDA(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
  cudaEvent_t fork;
  EB_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  EB_CUDA(cudaEventRecord(fork, s));
  EB_CUDA(cudaStreamWaitEvent(cap_stream, fork, 0));
  const int64_t n0 = nlaunch;
  prof_n = 0;
  EB_CUDA(cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal));
  for (int j = 0; j < iters; ++j) iteration(kind, b, x, cap_stream);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(cap_stream, &graph);
  cudaEventDestroy(fork);
  EB_CUDA(e);
  e = cudaGraphInstantiate(&gexec, graph, 0);
  cudaGraphDestroy(graph);
  EB_CUDA(e);
  g_launches = nlaunch - n0;
  nlaunch = n0;
  g_pairs = prof_n;
  g_b = b;
  g_x = x;
  g_iters = iters;
  g_kind = kind;
  g_prof = profile;
  g_nn = nn;
  g_nn_mode = nn_mode;
  g_tile_gen = eb->tile_gen;
  g_df = (int)df_on;
}

void Solver::graph_release() {
  if (gexec) cudaGraphExecDestroy(gexec);
  gexec = nullptr;
  g_pairs = 0;
  g_b = nullptr;
  g_x = nullptr;
}

cudaGraphExec_t build_while_graph(cudaStream_t cap,
                                  const std::function<void(cudaStream_t, cudaGraphConditionalHandle)>& body) {
  cudaGraph_t graph = nullptr;
  EB_CUDA(cudaGraphCreate(&graph, 0));
  cudaGraphExec_t exec = nullptr;
  try {
    cudaGraphConditionalHandle h;
    EB_CUDA(cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    EB_CUDA(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &p));
    cudaGraph_t bg = p.conditional.phGraph_out[0];
    EB_CUDA(cudaStreamBeginCaptureToGraph(cap, bg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    try {
      body(cap, h);
    } catch (...) {
      cudaGraph_t dummy = nullptr;
      cudaStreamEndCapture(cap, &dummy);
      throw;
    }
    EB_CUDA(cudaStreamEndCapture(cap, &bg));
    EB_CUDA(cudaGraphInstantiate(&exec, graph, 0));
  } catch (...) {
    cudaGraphDestroy(graph);
    throw;
  }
  cudaGraphDestroy(graph);
  return exec;
}

// Captures the device-side loop { while (!done && iters < maxit) iteration }
// (once per argument set).
void Solver::loop_prepare(int kind, const double* b, double* x, cudaStream_t s) {
  if (lexec && l_b == b && l_x == x && l_kind == kind && l_nn == nn && l_nn_mode == nn_mode &&
      l_tile_gen == eb->tile_gen && l_df == (int)df_on)
    return;
  loop_release();
  (void)s;  // capturing runs nothing; the graph is launched on s
  if (!cap_stream) EB_CUDA(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
  const int64_t n0 = nlaunch;
  lexec = build_while_graph(cap_stream,
                            [&](cudaStream_t cs, cudaGraphConditionalHandle h) { iteration(kind, b, x, cs, &h); });
  l_launches = nlaunch - n0;
  nlaunch = n0;
  l_b = b;
  l_x = x;
  l_kind = kind;
  l_nn = nn;
  l_nn_mode = nn_mode;
  l_tile_gen = eb->tile_gen;
  l_df = (int)df_on;
}

void Solver::loop_release() {
  if (lexec) cudaGraphExecDestroy(lexec);
  lexec = nullptr;
  l_b = nullptr;
  l_x = nullptr;
}

static bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(s, &st) == cudaSuccess && st == cudaStreamCaptureStatusActive;
}

// ---------------------------------------------------------- kernel timing
// Optional CUDA-event timing of the level-0 smoother launches (the kernel
// that dominates an AMG-PCG iteration), on the stream they are launched on.
// Inside a captured iteration the event records are graph nodes, so the
// pairs time the kernels back to back, without host-enqueue gaps.
void Solver::prof_begin(int mode, cudaStream_t) {
  prof_on = mode != 0;
  prof_what = (mode >= PROF_CONV && mode <= PROF_UPDATE) ? mode : PROF_SMOOTHER;
  prof_n = g_pairs;
  prof_acc_ms = 0.0;
  prof_acc_n = 0;
}

void Solver::prof_collect(int first, int count) {
  for (int i = first; i < first + count; ++i) {
    float ms = 0.0f;
    EB_CUDA(cudaEventElapsedTime(&ms, prof_ev[i].first, prof_ev[i].second));
    prof_acc_ms += ms;
    ++prof_acc_n;
  }
}

void Solver::prof_mark(cudaStream_t s, bool start, int what) {
  if (!prof_on || what != prof_what) return;
  if (start) {
    if (prof_n >= (int)prof_ev.size()) {
      cudaEvent_t a, b;
      EB_CUDA(cudaEventCreate(&a));
      EB_CUDA(cudaEventCreate(&b));
      prof_ev.push_back({a, b});
    }
    // external records stay observable (and timeable) when captured in a graph
    EB_CUDA(cudaEventRecordWithFlags(prof_ev[prof_n].first, s, capturing(s) ? cudaEventRecordExternal : 0));
  } else {
    EB_CUDA(cudaEventRecordWithFlags(prof_ev[prof_n].second, s, capturing(s) ? cudaEventRecordExternal : 0));
    ++prof_n;
  }
}

void Solver::prof_end(pcg_stats* st, cudaStream_t s) {
  st->prof_kernel_ms = 0.0;
  st->prof_launches = 0;
  if (!prof_on) return;
  EB_CUDA(cudaStreamSynchronize(s));
  prof_collect(g_pairs, prof_n - g_pairs);
  prof_n = g_pairs;
  st->prof_kernel_ms = prof_acc_ms;
  st->prof_launches = prof_acc_n;
  prof_on = false;
}

void Solver::prof_release() {
  for (auto& e : prof_ev) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  prof_ev.clear();
}

}  // namespace ebk
