// Device construction of the line-by-line EB operator (Algorithm 1 steps 1-3)
// and the matrix-free stencil apply / right-hand side.
//
// Level-set arithmetic is written with explicit round-to-nearest intrinsics
// (__dmul_rn, __dadd_rn, ...) so that no multiply-add is contracted: the
// quadric level set and its closed-form grid-line roots are then the same
// IEEE operations, in the same order, as the FP64 definition they follow.
#include "eb_internal.cuh"

#include <cmath>
#include <cstring>
#include <vector>

namespace ebk {

struct LSDev {
  int kind;
  int dim;
  double c[3], s[3], q[9];
  double r0;
  int nk;
  int k[EB_STAR_MAX_TERMS];
  double a[EB_STAR_MAX_TERMS], p[EB_STAR_MAX_TERMS];
  const double* psi;  // EB_LS_SAMPLED: psi at the nodes
  double m[4];        // 2D quadric: x = c + M y on the boundary, M = (Q2^T)^-1 (row-major 2 x 2)
};

__device__ __forceinline__ double node_coord(double lo, int64_t i, double h) {
  return __dadd_rn(lo, __dmul_rn((double)i, h));
}

// psi = sum_a (y_a/s_a)^2 - 1 with y = Q^T (x - c)  (fixed operation order)
__device__ double psi_quadric(const LSDev& L, const double* x) {
  double t0 = __dsub_rn(x[0], L.c[0]);
  double t1 = __dsub_rn(x[1], L.c[1]);
  double t2 = L.dim == 3 ? __dsub_rn(x[2], L.c[2]) : 0.0;
  double acc = 0.0;
  for (int a = 0; a < L.dim; ++a) {
    double y = __dadd_rn(__dmul_rn(L.q[0 * 3 + a], t0), __dmul_rn(L.q[1 * 3 + a], t1));
    if (L.dim == 3) y = __dadd_rn(y, __dmul_rn(L.q[2 * 3 + a], t2));
    double w = __ddiv_rn(y, L.s[a]);
    acc = (a == 0) ? __dmul_rn(w, w) : __dadd_rn(acc, __dmul_rn(w, w));
  }
  return __dsub_rn(acc, 1.0);
}

// psi = |x - c| - (r0 + sum_k a_k sin(k phi + p_k))
__device__ double psi_star(const LSDev& L, double x, double y) {
  double dx = __dsub_rn(x, L.c[0]);
  double dy = __dsub_rn(y, L.c[1]);
  double rho = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
  double phi = atan2(dy, dx);
  double r = L.r0;
  for (int j = 0; j < L.nk; ++j)
    r = __dadd_rn(r, __dmul_rn(L.a[j], sin(__dadd_rn(__dmul_rn((double)L.k[j], phi), L.p[j]))));
  return __dsub_rn(rho, r);
}

__device__ double psi_at(const LSDev& L, const double* x) {
  return L.kind == EB_LS_QUADRIC ? psi_quadric(L, x) : psi_star(L, x[0], x[1]);
}

// Positive root t of psi(p + sign t e_axis) = 0 for a quadric, p inside:
// alpha t^2 + beta t + gamma with the cancellation-free root formulas.
__device__ double quadric_root(const LSDev& L, const double* p, int axis, double sign) {
  double t0 = __dsub_rn(p[0], L.c[0]);
  double t1 = __dsub_rn(p[1], L.c[1]);
  double t2 = L.dim == 3 ? __dsub_rn(p[2], L.c[2]) : 0.0;
  double alpha = 0.0, dot = 0.0, gamma = 0.0;
  for (int a = 0; a < L.dim; ++a) {
    double y = __dadd_rn(__dmul_rn(L.q[0 * 3 + a], t0), __dmul_rn(L.q[1 * 3 + a], t1));
    if (L.dim == 3) y = __dadd_rn(y, __dmul_rn(L.q[2 * 3 + a], t2));
    double w = __ddiv_rn(y, L.s[a]);
    double u = __ddiv_rn(L.q[axis * 3 + a], L.s[a]);
    if (a == 0) {
      alpha = __dmul_rn(u, u);
      dot = __dmul_rn(w, u);
      gamma = __dmul_rn(w, w);
    } else {
      alpha = __dadd_rn(alpha, __dmul_rn(u, u));
      dot = __dadd_rn(dot, __dmul_rn(w, u));
      gamma = __dadd_rn(gamma, __dmul_rn(w, w));
    }
  }
  gamma = __dsub_rn(gamma, 1.0);
  double beta = __dmul_rn(2.0, __dmul_rn(sign, dot));
  double disc = __dsub_rn(__dmul_rn(beta, beta), __dmul_rn(__dmul_rn(4.0, alpha), gamma));
  double sq = __dsqrt_rn(disc);
  if (beta >= 0.0) return __ddiv_rn(__dmul_rn(-2.0, gamma), __dadd_rn(beta, sq));
  return __ddiv_rn(__dsub_rn(sq, beta), __dmul_rn(2.0, alpha));
}

// Illinois iteration on g(t) = psi(p + sign t e_axis) over [ta, tb],
// g(ta) < 0 <= g(tb); stops at g == 0 or when the iterate moves <= 1e-15 h.
__device__ double star_root(const LSDev& L, const double* p, int axis, double sign, double ta, double tb,
                            double h) {
  double q[2] = {p[0], p[1]};
  auto g = [&](double t) {
    double qq[2] = {q[0], q[1]};
    qq[axis] = __dadd_rn(p[axis], __dmul_rn(sign, t));
    return psi_star(L, qq[0], qq[1]);
  };
  double fa = g(ta), fb = g(tb);
  double t = tb;
  if (fb == 0.0) return t;
  int side = 0;
  double told = ta;
  for (int it = 0; it < 100; ++it) {
    double tn = __ddiv_rn(__dsub_rn(__dmul_rn(ta, fb), __dmul_rn(tb, fa)), __dsub_rn(fb, fa));
    double ft = g(tn);
    t = tn;
    if (ft == 0.0) break;
    if (ft < 0.0) {
      if (side == -1) fb = __dmul_rn(0.5, fb);
      ta = tn;
      fa = ft;
      side = -1;
    } else {
      if (side == 1) fa = __dmul_rn(0.5, fa);
      tb = tn;
      fb = ft;
      side = 1;
    }
    if (fabs(__dsub_rn(tn, told)) <= __dmul_rn(1e-15, h)) break;
    told = tn;
  }
  return t;
}

__device__ __forceinline__ void unflatten(const Geometry& G, int64_t node, int64_t* i) {
  i[0] = node % G.n0;
  int64_t r = node / G.n0;
  i[1] = r % G.n1;
  i[2] = r / G.n1;
}

__device__ __forceinline__ int64_t stride_of(const Geometry& G, int axis) {
  return axis == 0 ? 1 : (axis == 1 ? (int64_t)G.n0 : (int64_t)G.n0 * G.n1);
}

__device__ __forceinline__ bool on_border(const Geometry& G, const int64_t* i) {
  bool b = i[0] == 0 || i[0] == G.n0 - 1 || i[1] == 0 || i[1] == G.n1 - 1;
  if (G.dim == 3) b = b || i[2] == 0 || i[2] == G.n2 - 1;
  return b;
}

__device__ __forceinline__ void atomic_min_pos(double* addr, double v) {
  atomicMin(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}
// minimum of signed doubles through an order-preserving 64-bit key (init ~0)
__device__ __forceinline__ void atomic_min_signed(unsigned long long* key, double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  atomicMin(key, (u >> 63) ? ~u : (u | 0x8000000000000000ull));
}
static double decode_signed_key(unsigned long long k) {
  const unsigned long long u = (k & 0x8000000000000000ull) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  double v;
  std::memcpy(&v, &u, sizeof(v));
  return v;
}
__device__ __forceinline__ void atomic_max_pos(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

struct BuildStats {
  int border_inside;
  int pad;
  unsigned long long num_bp;
  unsigned long long num_far;
  double min_abs_psi;
  double max_delta_over_h;
  double min_margin;   // smallest sum of c_s over the BP directions of a CP
};

// pass 1: psi at every node; border check; |psi| margin
__global__ void k_psi(Geometry G, LSDev L, double* psi, BuildStats* st) {
  int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool live = node < G.num_nodes;
  if (!live) node = G.num_nodes - 1;   // keep the warp whole for the shuffle reduction
  int64_t i[3];
  unflatten(G, node, i);
  double v;
  if (L.kind == EB_LS_SAMPLED) {
    v = L.psi[node];
  } else {
    double x[3];
    for (int a = 0; a < 3; ++a) x[a] = a < G.dim ? node_coord(G.lo[a], i[a], G.h) : 0.0;
    v = psi_at(L, x);
  }
  if (live) psi[node] = v;
  if (v < 0.0 && on_border(G, i)) atomicExch(&st->border_inside, 1);
  double av = fabs(v);
  if (!(av >= 0.0)) av = 0.0;  // NaN -> 0 margin
  for (int o = 16; o > 0; o >>= 1) av = fmin(av, __shfl_xor_sync(0xffffffffu, av, o));
  if ((threadIdx.x & 31) == 0) atomic_min_pos(&st->min_abs_psi, av);
}

// pass 2: inside / BP / CP (Sec. 2 definitions)
__global__ void k_class(Geometry G, const double* psi, uint8_t* code, int32_t* is_cp, BuildStats* st) {
  int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= G.num_nodes) return;
  int64_t i[3];
  unflatten(G, node, i);
  uint8_t c = CODE_OUT;
  int cp = 0;
  if (psi[node] < 0.0 && !on_border(G, i)) {
    int cnt = 0;
    for (int a = 0; a < G.dim; ++a) {
      int64_t s = stride_of(G, a);
      cnt += (psi[node - s] < 0.0) + (psi[node + s] < 0.0);
    }
    if (cnt == 2 * G.dim) {
      c = CODE_CP;
      cp = 1;
    } else {
      c = CODE_BP;
    }
  }
  code[node] = c;
  unsigned bal = __ballot_sync(__activemask(), c == CODE_BP);
  if (bal && (threadIdx.x & 31) == (unsigned)(__ffs(bal) - 1)) atomicAdd(&st->num_bp, (unsigned long long)__popc(bal));
  is_cp[node] = cp;
}

// pass 3: CP numbering, BP-neighbour direction masks, cuts per CP
__global__ void k_cp_mask(Geometry G, uint8_t* code, const int32_t* cp_off, int32_t* cp_of_node,
                          int32_t* cp_node, int32_t* ncut, int64_t num_nodes) {
  int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= num_nodes) return;
  uint8_t c = code[node];
  if (!(c & CODE_CP)) {
    cp_of_node[node] = -1;
    return;
  }
  int32_t k = cp_off[node];
  cp_of_node[node] = k;
  cp_node[k] = (int32_t)node;
  uint8_t m = 0;
  for (int a = 0; a < G.dim; ++a) {
    int64_t s = stride_of(G, a);
    if (code[node - s] == CODE_BP) m |= (uint8_t)(1u << (2 * a));
    if (code[node + s] == CODE_BP) m |= (uint8_t)(1u << (2 * a + 1));
  }
  code[node] = (uint8_t)(CODE_CP | m);
  ncut[k] = __popc((unsigned)m);
}

// pass 4: per CP, its cuts (walk + root) and the diagonal D_k = sum_s c_s
__global__ void k_cut(Geometry G, LSDev L, const double* psi, const uint8_t* code, const int32_t* cp_node,
                      const int32_t* cut_off, int64_t num_cp, double* diag, int32_t* cut_cp, int32_t* cut_dir,
                      double* cut_delta, double* cut_c, double* cut_xg, int32_t* cut_far, BuildStats* st) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= num_cp) return;
  int64_t node = cp_node[k];
  uint8_t m = code[node] & 0x3F;
  double D = 0.0, margin = 0.0;
  int j = cut_off[k];
  int64_t i[3];
  unflatten(G, node, i);
  const double h = G.h;
  for (int s = 0; s < 2 * G.dim; ++s) {
    double cs = 1.0;
    if (m & (1u << s)) {
      int axis = s >> 1;
      int sg = (s & 1) ? 1 : -1;
      int64_t st_ax = stride_of(G, axis) * sg;
      int64_t bp = node + st_ax;
      int64_t cur = bp + st_ax;
      int64_t mm = 1;
      while (psi[cur] < 0.0) {
        ++mm;
        cur += st_ax;
      }
      double p[3];
      for (int a = 0; a < 3; ++a) {
        int64_t ia = i[a] + (a == axis ? sg : 0);
        p[a] = a < G.dim ? node_coord(G.lo[a], ia, h) : 0.0;
      }
      double delta;
      if (L.kind == EB_LS_QUADRIC) {
        delta = quadric_root(L, p, axis, (double)sg);
      } else if (L.kind == EB_LS_SAMPLED) {
        // linear ratio between the last inside node and the first outside one
        // (Sec. 3.3): delta = (mm - 1) h + psi_in / (psi_in - psi_out) h
        const double pin = psi[cur - st_ax], pout = psi[cur];
        delta = __dadd_rn(__dmul_rn((double)(mm - 1), h), __dmul_rn(__ddiv_rn(pin, __dsub_rn(pin, pout)), h));
      } else {
        double ta = __dmul_rn((double)(mm - 1), h);
        double tb = __dmul_rn((double)mm, h);
        delta = star_root(L, p, axis, (double)sg, ta, tb, h);
      }
      cs = __ddiv_rn(h, __dadd_rn(h, delta));
      cut_cp[j] = (int32_t)k;
      cut_dir[j] = s;
      cut_delta[j] = delta;
      cut_far[j] = mm > 1;  // the node past the BP is inside
      cut_c[j] = cs;
      for (int a = 0; a < G.dim; ++a)
        cut_xg[(int64_t)j * G.dim + a] = (a == axis) ? __dadd_rn(p[a], __dmul_rn((double)sg, delta)) : p[a];
      if (delta > h) atomicAdd(&st->num_far, 1ull);
      atomic_max_pos(&st->max_delta_over_h, fabs(delta / h));
      margin = __dadd_rn(margin, cs);
      ++j;
    }
    D = (s == 0) ? cs : __dadd_rn(D, cs);
  }
  diag[node] = D;
  if (m) atomic_min_pos(&st->min_margin, margin);
}

__global__ void k_tile_flags(Geometry G, const uint8_t* code, int32_t* tflag) {
  int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= G.num_nodes) return;
  if (!(code[node] & CODE_CP)) return;
  int64_t i[3];
  unflatten(G, node, i);
  int64_t t = i[0] / G.tx + (int64_t)G.ntx * (i[1] / G.ty + (int64_t)G.nty * (i[2] / G.tz));
  tflag[t] = 1;
}

__global__ void k_compact(const int32_t* flag, const int32_t* off, int64_t n, int32_t* out) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n && flag[t]) out[off[t]] = (int32_t)t;
}

__global__ void k_diag32(int64_t n, const double* d, float* f) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) f[i] = (float)d[i];
}

// corner node and extents of each listed tile
__global__ void k_tile_geom(Geometry G, const int32_t* tiles, int64_t nt, int32_t* base, int32_t* lim) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nt) return;
  int64_t t = tiles[k];
  int64_t bx = t % G.ntx, r = t / G.ntx, by = r % G.nty, bz = r / G.nty;
  int64_t x0 = bx * G.tx, y0 = by * G.ty, z0 = bz * G.tz;
  base[k] = (int32_t)(x0 + (int64_t)G.n0 * (y0 + (int64_t)G.n1 * z0));
  const int64_t rx = G.n0 - x0, ry = G.n1 - y0, rz = G.n2 - z0;
  const int lx = (int)(rx < G.tx ? rx : G.tx), ly = (int)(ry < G.ty ? ry : G.ty), lz = (int)(rz < G.tz ? rz : G.tz);
  lim[k] = lx | (ly << 8) | (lz << 16);
}

// Node pairs of listed tile blockIdx.x (128 threads, pair layout) that hold a
// CP: their count (fill == false) or their first nodes written from off[tile]
// on in pair order (fill == true).
__global__ void __launch_bounds__(128) k_cp_pairs(TileView tv, const uint8_t* __restrict__ code, bool fill,
                                                  int32_t* cnt, const int32_t* off, int32_t* list) {
  __shared__ int wc[4];
  const int64_t tt = blockIdx.x;
  int32_t node = 0;
  bool ok = tile_pair<3>(tv, tt, threadIdx.x, node);
  if (ok) {
    const uint32_t v = __ldg(reinterpret_cast<const unsigned short*>(code + node));
    ok = ((v | (v >> 8)) & CODE_CP) != 0;
  }
  const unsigned m = __ballot_sync(0xffffffffu, ok);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) wc[w] = __popc(m);
  __syncthreads();
  if (!fill) {
    if (threadIdx.x == 0) cnt[tt] = wc[0] + wc[1] + wc[2] + wc[3];
    return;
  }
  int before = 0;
  for (int k = 0; k < w; ++k) before += wc[k];
  if (ok) list[off[tt] + before + __popc(m & ((1u << lane) - 1u))] = node;
}

// ------------------------------------------------------- RBF closure (2D)
// Sec. 2.2: u_BP = w_ij u_ij + w_1 u_G1 + w_2 u_G2 from the cubic polyharmonic
// RBF interpolant with linear augmentation (eqs. 7-9) through the CP and two
// boundary points chosen by Algorithm 2.  The boundary is the parameterised
// curve of the descriptor: quadric x = c + M (s0 cos t, s1 sin t), star x =
// c + r(t) (cos t, sin t).
struct Pt {
  double x, y;
};

__device__ void rbf_curve(const LSDev& L, double t, Pt& g, Pt& g1, Pt& g2) {
  if (L.kind == EB_LS_QUADRIC) {
    const double ct = cos(t), st = sin(t);
    const double y0 = L.s[0] * ct, y1 = L.s[1] * st, d0 = -L.s[0] * st, d1 = L.s[1] * ct;
    g = {L.c[0] + L.m[0] * y0 + L.m[1] * y1, L.c[1] + L.m[2] * y0 + L.m[3] * y1};
    g1 = {L.m[0] * d0 + L.m[1] * d1, L.m[2] * d0 + L.m[3] * d1};
    g2 = {-(L.m[0] * y0 + L.m[1] * y1), -(L.m[2] * y0 + L.m[3] * y1)};
    return;
  }
  double r = L.r0, r1 = 0.0, r2 = 0.0;
  for (int j = 0; j < L.nk; ++j) {
    const double a = L.a[j], k = (double)L.k[j];
    const double sv = sin(k * t + L.p[j]), cv = cos(k * t + L.p[j]);
    r += a * sv;
    r1 += a * k * cv;
    r2 -= a * k * k * sv;
  }
  const double ct = cos(t), st = sin(t);
  g = {L.c[0] + r * ct, L.c[1] + r * st};
  g1 = {r1 * ct - r * st, r1 * st + r * ct};
  g2 = {r2 * ct - 2.0 * r1 * st - r * ct, r2 * st + 2.0 * r1 * ct - r * st};
}

// nearest point of Gamma to p: the nearest of RBF_GUESS uniform parameter
// samples, then Newton on (Gamma(t) - p) . Gamma'(t) = 0, steps limited to one
// sample spacing
constexpr int RBF_GUESS = 256;
// The uniform samples are split over the 32 lanes of a warp (lane l takes
// samples l, l + 32, ...); the nearest sample is the smallest distance with
// the smallest index among equal ones -- the first minimum of the sequential
// scan -- and every lane then runs the same Newton iteration from it.
__device__ Pt rbf_closest(const LSDev& L, Pt p, int lane) {
  const double two_pi = 6.283185307179586;
  const double dmax = two_pi / RBF_GUESS;
  double best = 1e300;
  int kb = 0;
  Pt g, g1, g2;
  for (int k = lane; k < RBF_GUESS; k += 32) {
    const double tk = two_pi * k / RBF_GUESS;
    rbf_curve(L, tk, g, g1, g2);
    const double d = (g.x - p.x) * (g.x - p.x) + (g.y - p.y) * (g.y - p.y);
    if (d < best) {
      best = d;
      kb = k;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int ok = __shfl_xor_sync(0xffffffffu, kb, o);
    if (ob < best || (ob == best && ok < kb)) {
      best = ob;
      kb = ok;
    }
  }
  double t = two_pi * kb / RBF_GUESS;
  for (int it = 0; it < 60; ++it) {
    rbf_curve(L, t, g, g1, g2);
    const double f = (g.x - p.x) * g1.x + (g.y - p.y) * g1.y;
    const double df = g1.x * g1.x + g1.y * g1.y + (g.x - p.x) * g2.x + (g.y - p.y) * g2.y;
    double step = df > 0.0 ? -f / df : (f > 0.0 ? -dmax : dmax);
    step = fmin(fmax(step, -dmax), dmax);
    t += step;
    if (fabs(step) <= 1e-15) break;
  }
  rbf_curve(L, t, g, g1, g2);
  return g;
}

__device__ double rbf_psi(const LSDev& L, double x, double y) {
  const double xx[3] = {x, y, 0.0};
  return psi_at(L, xx);
}

// first crossing of Gamma on the ray p + s d (p inside): march in steps of
// h/4, then the Illinois iteration on the bracket; -1 if none within the limit
constexpr int RBF_MARCH_LIMIT = 1 << 20;
__device__ double rbf_ray(const LSDev& L, Pt p, Pt d, double h) {
  const double step = 0.25 * h;
  double a = 0.0, fa = rbf_psi(L, p.x, p.y), b = step, fb = rbf_psi(L, p.x + b * d.x, p.y + b * d.y);
  int n = 0;
  while (fb < 0.0) {
    a = b;
    fa = fb;
    b += step;
    fb = rbf_psi(L, p.x + b * d.x, p.y + b * d.y);
    if (++n > RBF_MARCH_LIMIT) return -1.0;
  }
  if (fb == 0.0) return b;
  int side = 0;
  double told = a, t = b;
  for (int it = 0; it < 100; ++it) {
    t = (a * fb - b * fa) / (fb - fa);
    const double ft = rbf_psi(L, p.x + t * d.x, p.y + t * d.y);
    if (ft == 0.0) break;
    if (ft < 0.0) {
      if (side == -1) fb *= 0.5;
      a = t;
      fa = ft;
      side = -1;
    } else {
      if (side == 1) fa *= 0.5;
      b = t;
      fb = ft;
      side = 1;
    }
    if (fabs(t - told) <= 1e-15 * h) break;
    told = t;
  }
  return t;
}

// weights of eqs. 7-9 in coordinates relative to x_BP scaled by 1/h: the 6 x 6
// saddle system by Gaussian elimination with partial pivoting; false if it is
// singular
__device__ bool rbf_weights(const Pt* q, double* w) {
  double B[6][7];
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 7; ++b) B[a][b] = 0.0;
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) {
      const double r = hypot(q[a].x - q[b].x, q[a].y - q[b].y);
      B[a][b] = r * r * r;
    }
    B[3][a] = B[a][3] = 1.0;
    B[4][a] = B[a][4] = q[a].x;
    B[5][a] = B[a][5] = q[a].y;
    const double r = hypot(q[a].x, q[a].y);
    B[a][6] = r * r * r;
  }
  B[3][6] = 1.0;
  for (int c = 0; c < 6; ++c) {
    int piv = c;
    for (int r = c + 1; r < 6; ++r)
      if (fabs(B[r][c]) > fabs(B[piv][c])) piv = r;
    if (!(fabs(B[piv][c]) > 0.0)) return false;
    if (piv != c)
      for (int b = 0; b < 7; ++b) {
        const double t = B[c][b];
        B[c][b] = B[piv][b];
        B[piv][b] = t;
      }
    for (int r = c + 1; r < 6; ++r) {
      const double f = B[r][c] / B[c][c];
      for (int b = c; b < 7; ++b) B[r][b] -= f * B[c][b];
    }
  }
  double x[6];
  for (int r = 5; r >= 0; --r) {
    double acc = B[r][6];
    for (int b = r + 1; b < 6; ++b) acc -= B[r][b] * x[b];
    x[r] = acc / B[r][r];
  }
  w[0] = x[0];
  w[1] = x[1];
  w[2] = x[2];
  return isfinite(x[0]) && isfinite(x[1]) && isfinite(x[2]);
}

// One warp per RBF cut r (cut j = rbf_cut[r]): Algorithm 2 and the weights
// (the nearest-point searches split over the lanes, the rest on lane 0);
// the cut's diagonal contribution becomes 1 - w_ij, its crossing G1 (distance
// |x_BP - G1|), its first right-hand-side weight w_1; the second point G2 and
// weight w_2 are stored per RBF cut.  bad = 1 if a system was singular or a
// rotated line did not meet Gamma.
__global__ void k_rbf(Geometry G, LSDev L, double eps, const int32_t* cp_node, const int32_t* rbf_cut, int64_t nrbf,
                      const int32_t* cut_cp, const int32_t* cut_dir, double* cut_c, double* cut_w1, double* cut_delta,
                      double* cut_xg, double* rbf_xg2, double* rbf_w, int32_t* rbf_rot, int* bad) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= nrbf) return;  // whole warps: blockDim.x is a multiple of 32
  const int j = rbf_cut[r];
  const int64_t node = cp_node[cut_cp[j]];
  const int s = cut_dir[j];
  const int axis = s >> 1, sg = (s & 1) ? 1 : -1;
  int64_t ij[2] = {node % G.n0, node / G.n0};
  const Pt xij{node_coord(G.lo[0], ij[0], G.h), node_coord(G.lo[1], ij[1], G.h)};
  ij[axis] += sg;
  const Pt xbp{node_coord(G.lo[0], ij[0], G.h), node_coord(G.lo[1], ij[1], G.h)};
  const double h = G.h;
  const Pt g1 = rbf_closest(L, xbp, lane);
  Pt g2 = rbf_closest(L, xij, lane);
  if (lane != 0) return;
  int rot = 0;
  if (!(hypot(g1.x - g2.x, g1.y - g2.y) > eps * h)) {
    const Pt v{g1.x - xbp.x, g1.y - xbp.y};
    const double nv = hypot(v.x, v.y);
    const double c = cos(0.7853981633974483), sn = sin(0.7853981633974483);
    const Pt d{(c * v.x - sn * v.y) / nv, (sn * v.x + c * v.y) / nv};
    const double t = rbf_ray(L, xbp, d, h);
    if (t < 0.0) atomicExch(bad, 1);
    g2 = {xbp.x + t * d.x, xbp.y + t * d.y};
    rot = 1;
  }
  const Pt q[3] = {{(xij.x - xbp.x) / h, (xij.y - xbp.y) / h}, {(g1.x - xbp.x) / h, (g1.y - xbp.y) / h},
                   {(g2.x - xbp.x) / h, (g2.y - xbp.y) / h}};
  double w[3];
  if (!rbf_weights(q, w)) {
    atomicExch(bad, 1);
    w[0] = 0.0;
    w[1] = 1.0;
    w[2] = 0.0;
  }
  cut_c[j] = 1.0 - w[0];
  cut_w1[j] = w[1];
  cut_delta[j] = hypot(g1.x - xbp.x, g1.y - xbp.y);
  cut_xg[2 * (int64_t)j] = g1.x;
  cut_xg[2 * (int64_t)j + 1] = g1.y;
  rbf_xg2[2 * r] = g2.x;
  rbf_xg2[2 * r + 1] = g2.y;
  rbf_w[3 * r] = w[0];
  rbf_w[3 * r + 1] = w[1];
  rbf_w[3 * r + 2] = w[2];
  rbf_rot[r] = rot;
}

// RBF cuts of the closure mode (mixed: the far ones; rbf: all)
__global__ void k_rbf_flag(int64_t nc, const int32_t* cut_far, int all, int32_t* flag) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nc) flag[j] = all ? 1 : (cut_far[j] != 0);
}

__global__ void k_rbf_list(int64_t nc, const int32_t* flag, const int32_t* off, int32_t* rbf_cut, int32_t* cut_rbf) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nc) return;
  cut_rbf[j] = flag[j] ? off[j] : -1;
  if (flag[j]) rbf_cut[off[j]] = (int32_t)j;
}

__global__ void k_copy_f64(int64_t n, const double* a, double* b) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
}

// D_k = sum_s c_s (1 towards a CP) in direction order, after the RBF cuts
// changed their c_s; the dominance margin of the cut rows (signed: an RBF
// weight w_ij > 1 makes it negative)
__global__ void k_diag_from_cuts(Geometry G, const int32_t* cp_node, const uint8_t* code, const int32_t* cut_off,
                                 const double* cut_c, int64_t num_cp, double* diag, unsigned long long* margin_min) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= num_cp) return;
  const int64_t node = cp_node[k];
  const uint8_t m = code[node] & 0x3F;
  int j = cut_off[k];
  double D = 0.0, margin = 0.0;
  for (int sdir = 0; sdir < 2 * G.dim; ++sdir) {
    double cs = 1.0;
    if (m & (1u << sdir)) {
      cs = cut_c[j++];
      margin = __dadd_rn(margin, cs);
    }
    D = sdir == 0 ? cs : __dadd_rn(D, cs);
  }
  diag[node] = D;
  if (m) atomic_min_signed(margin_min, margin);
}

static LSDev to_dev(const eb_levelset& ls, int dim) {
  LSDev L{};
  L.kind = ls.kind;
  L.dim = dim;
  for (int a = 0; a < 3; ++a) {
    L.c[a] = ls.center[a];
    L.s[a] = ls.semi[a];
  }
  for (int a = 0; a < 9; ++a) L.q[a] = ls.rot[a];
  L.r0 = ls.r0;
  L.nk = ls.nk;
  for (int j = 0; j < ls.nk && j < EB_STAR_MAX_TERMS; ++j) {
    L.k[j] = ls.k[j];
    L.a[j] = ls.a[j];
    L.p[j] = ls.p[j];
  }
  L.psi = ls.psi;
  if (dim == 2 && ls.kind == EB_LS_QUADRIC) {
    // y = Q2^T (x - c): x = c + M y with M the inverse of Q2^T
    const double a = ls.rot[0], b = ls.rot[3], c = ls.rot[1], d = ls.rot[4];  // Q2^T = [[a, b], [c, d]]
    const double det = a * d - b * c;
    L.m[0] = d / det;
    L.m[1] = -b / det;
    L.m[2] = -c / det;
    L.m[3] = a / det;
  }
  return L;
}

void build_handle(EBHandle& eb, const eb_grid& grid, const eb_levelset& ls, cudaStream_t s,
                  const eb_build_opts* opts) {
  const int closure = opts ? opts->closure : EB_CLOSURE_LINE;
  const double rbf_eps = opts ? opts->rbf_eps : 0.025;
  EB_REQUIRE(closure == EB_CLOSURE_LINE || closure == EB_CLOSURE_MIXED || closure == EB_CLOSURE_RBF, EB_ERR_INVALID,
             "eb_build: closure must be EB_CLOSURE_LINE, EB_CLOSURE_MIXED or EB_CLOSURE_RBF");
  EB_REQUIRE(closure == EB_CLOSURE_LINE || (grid.dim == 2 && (ls.kind == EB_LS_QUADRIC || ls.kind == EB_LS_STAR2D)),
             EB_ERR_NOT_IMPLEMENTED, "eb_build: the RBF closure needs a 2D quadric or star level set");
  EB_REQUIRE(closure == EB_CLOSURE_LINE || (rbf_eps > 0.0 && std::isfinite(rbf_eps)), EB_ERR_INVALID,
             "eb_build: rbf_eps must be positive");
  EB_REQUIRE(grid.dim == 2 || grid.dim == 3, EB_ERR_INVALID, "grid.dim must be 2 or 3");
  EB_REQUIRE(grid.n[0] >= 3 && grid.n[1] >= 3 && (grid.dim == 2 ? grid.n[2] == 1 : grid.n[2] >= 3),
             EB_ERR_INVALID, "grid needs >= 3 nodes per used axis (and n[2] == 1 in 2D)");
  EB_REQUIRE(grid.n[0] % 2 == 0, EB_ERR_INVALID, "n[0] must be even");
  EB_REQUIRE(grid.h > 0.0 && std::isfinite(grid.h), EB_ERR_INVALID, "h must be positive");
  EB_REQUIRE(ls.kind == EB_LS_QUADRIC || (ls.kind == EB_LS_STAR2D && grid.dim == 2) || ls.kind == EB_LS_SAMPLED,
             EB_ERR_INVALID, "unknown level-set kind (STAR2D is 2D only)");
  EB_REQUIRE(ls.kind != EB_LS_SAMPLED || ls.psi != nullptr, EB_ERR_INVALID, "sampled level set: psi is NULL");
  EB_REQUIRE(ls.kind != EB_LS_STAR2D || (ls.nk >= 0 && ls.nk <= EB_STAR_MAX_TERMS), EB_ERR_INVALID,
             "star: nk out of range");
  if (ls.kind == EB_LS_QUADRIC)
    for (int a = 0; a < grid.dim; ++a) EB_REQUIRE(ls.semi[a] > 0.0, EB_ERR_INVALID, "quadric semi-axes must be > 0");
  int64_t nn = (int64_t)grid.n[0] * grid.n[1] * grid.n[2];
  EB_REQUIRE(nn < ((int64_t)1 << 31) - 1, EB_ERR_INVALID, "grid larger than 2^31 nodes");

  Geometry& G = eb.g;
  G.dim = grid.dim;
  G.n0 = grid.n[0];
  G.n1 = grid.n[1];
  G.n2 = grid.n[2];
  G.num_nodes = nn;
  for (int a = 0; a < 3; ++a) G.lo[a] = grid.lo[a];
  G.h = grid.h;
  eb.ls = ls;
  eb.ls.psi = nullptr;  // the sampled values are read during the build only
  eb.home = s;
  LSDev L = to_dev(ls, grid.dim);

  BuildStats* st = dalloc<BuildStats>(1, s);
  BuildStats init{};
  init.min_abs_psi = 1e300;
  init.max_delta_over_h = 0.0;
  init.min_margin = 1e300;
  EB_CUDA(cudaMemcpyAsync(st, &init, sizeof(init), cudaMemcpyHostToDevice, s));

  double* psi = dalloc<double>(nn, s, false);
  int32_t* is_cp = dalloc<int32_t>(nn, s, false);
  int32_t* cp_off = dalloc<int32_t>(nn + 1, s, false);
  eb.code = dalloc<uint8_t>(nn, s);
  eb.diag = dalloc<double>(nn, s);
  eb.cp_of_node = dalloc<int32_t>(nn, s, false);

  const int T = 256;
  k_psi<<<blocks_for(nn, T), T, 0, s>>>(G, L, psi, st);
  k_class<<<blocks_for(nn, T), T, 0, s>>>(G, psi, eb.code, is_cp, st);
  EB_CUDA(cudaGetLastError());
  exclusive_scan_i32(is_cp, cp_off, nn, s);
  BuildStats hst{};
  int32_t ncp = 0;
  EB_CUDA(cudaMemcpyAsync(&ncp, cp_off + nn, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  EB_CUDA(cudaMemcpyAsync(&hst, st, sizeof(hst), cudaMemcpyDeviceToHost, s));
  EB_CUDA(cudaStreamSynchronize(s));
  if (hst.border_inside || ncp == 0) {
    dfree(psi, s); dfree(is_cp, s); dfree(cp_off, s); dfree(st, s);
    EB_CUDA(cudaStreamSynchronize(s));
    throw Failure{EB_ERR_GEOMETRY, hst.border_inside ? "the geometry touches the outermost ring of grid nodes"
                                                     : "no computational point"};
  }
  eb.num_cp = ncp;
  eb.num_bp = (int64_t)hst.num_bp;
  eb.cp_node = dalloc<int32_t>(ncp, s, false);
  int32_t* ncut = dalloc<int32_t>(ncp + 1, s);
  eb.cut_off = dalloc<int32_t>(ncp + 1, s, false);
  k_cp_mask<<<blocks_for(nn, T), T, 0, s>>>(G, eb.code, cp_off, eb.cp_of_node, eb.cp_node, ncut, nn);
  EB_CUDA(cudaGetLastError());
  exclusive_scan_i32(ncut, eb.cut_off, ncp, s);
  int32_t nc = 0;
  EB_CUDA(cudaMemcpyAsync(&nc, eb.cut_off + ncp, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  EB_CUDA(cudaStreamSynchronize(s));
  eb.num_cut = nc;
  eb.cut_cp = dalloc<int32_t>(nc, s, false);
  eb.cut_dir = dalloc<int32_t>(nc, s, false);
  eb.cut_delta = dalloc<double>(nc, s, false);
  eb.cut_c = dalloc<double>(nc, s, false);
  eb.cut_xg = dalloc<double>((int64_t)nc * G.dim, s, false);
  int32_t* cut_far = dalloc<int32_t>(nc, s, false);
  k_cut<<<blocks_for(ncp, 128), 128, 0, s>>>(G, L, psi, eb.code, eb.cp_node, eb.cut_off, ncp, eb.diag, eb.cut_cp,
                                             eb.cut_dir, eb.cut_delta, eb.cut_c, eb.cut_xg, cut_far, st);
  EB_CUDA(cudaGetLastError());
  eb.closure = closure;
  double rbf_margin = 0.0;
  if (closure != EB_CLOSURE_LINE && nc > 0) {
    // Sec. 2.3: the RBF interpolation of Sec. 2.2 where the node past the BP
    // is inside (mixed) or at every cut (RBF-based)
    int32_t* flag = dalloc<int32_t>(nc + 1, s);
    int32_t* off = dalloc<int32_t>(nc + 1, s, false);
    int* bad = dalloc<int>(1, s);
    unsigned long long* mkey = dalloc<unsigned long long>(1, s, false);
    try {
      k_rbf_flag<<<blocks_for(nc, T), T, 0, s>>>(nc, cut_far, closure == EB_CLOSURE_RBF ? 1 : 0, flag);
      exclusive_scan_i32(flag, off, nc, s);
      int32_t nr = 0;
      EB_CUDA(cudaMemcpyAsync(&nr, off + nc, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      EB_CUDA(cudaStreamSynchronize(s));
      eb.num_rbf = nr;
      eb.rbf_cut = dalloc<int32_t>(nr, s, false);
      eb.cut_rbf = dalloc<int32_t>(nc, s, false);
      eb.rbf_xg2 = dalloc<double>(2 * (int64_t)nr, s, false);
      eb.rbf_w = dalloc<double>(3 * (int64_t)nr, s, false);
      eb.rbf_rot = dalloc<int32_t>(nr, s, false);
      eb.cut_w1 = dalloc<double>(nc, s, false);
      k_rbf_list<<<blocks_for(nc, T), T, 0, s>>>(nc, flag, off, eb.rbf_cut, eb.cut_rbf);
      k_copy_f64<<<blocks_for(nc, T), T, 0, s>>>(nc, eb.cut_c, eb.cut_w1);  // w_1 = c_s on line-by-line cuts
      if (nr > 0)
        k_rbf<<<blocks_for(32 * (int64_t)nr, 128), 128, 0, s>>>(G, L, rbf_eps, eb.cp_node, eb.rbf_cut, nr, eb.cut_cp,
                                                                eb.cut_dir, eb.cut_c, eb.cut_w1, eb.cut_delta,
                                                                eb.cut_xg, eb.rbf_xg2, eb.rbf_w, eb.rbf_rot, bad);
      const unsigned long long init = ~0ull;
      EB_CUDA(cudaMemcpyAsync(mkey, &init, sizeof(init), cudaMemcpyHostToDevice, s));
      k_diag_from_cuts<<<blocks_for(ncp, 128), 128, 0, s>>>(G, eb.cp_node, eb.code, eb.cut_off, eb.cut_c, ncp,
                                                            eb.diag, mkey);
      EB_CUDA(cudaGetLastError());
      int hb = 0;
      unsigned long long hk = 0;
      EB_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
      EB_CUDA(cudaMemcpyAsync(&hk, mkey, sizeof(hk), cudaMemcpyDeviceToHost, s));
      EB_CUDA(cudaStreamSynchronize(s));
      EB_REQUIRE(hb == 0, EB_ERR_GEOMETRY, "eb_build: an RBF closure found no usable boundary points");
      rbf_margin = decode_signed_key(hk);
      std::vector<int32_t> rot(nr);
      if (nr > 0) EB_CUDA(cudaMemcpy(rot.data(), eb.rbf_rot, sizeof(int32_t) * nr, cudaMemcpyDeviceToHost));
      eb.num_rbf_rot = 0;
      for (int32_t v : rot) eb.num_rbf_rot += v;
    } catch (...) {
      dfree(flag, s); dfree(off, s); dfree(bad, s); dfree(mkey, s); dfree(cut_far, s);
      throw;
    }
    dfree(flag, s); dfree(off, s); dfree(bad, s); dfree(mkey, s);
  }
  dfree(cut_far, s);

  if (grid.dim == 2)
    build_tiles(eb, TileShape<2>::X, TileShape<2>::Y, TileShape<2>::Z, s);
  else
    build_tiles(eb, TileShape<3>::X, TileShape<3>::Y, TileShape<3>::Z, s);
  EB_CUDA(cudaMemcpyAsync(&hst, st, sizeof(hst), cudaMemcpyDeviceToHost, s));
  EB_CUDA(cudaStreamSynchronize(s));
  eb.diag32 = dalloc<float>(nn, s, false);
  k_diag32<<<blocks_for(nn, T), T, 0, s>>>(nn, eb.diag, eb.diag32);
  EB_CUDA(cudaGetLastError());
  eb.num_far = (int64_t)hst.num_far;
  eb.max_delta_over_h = hst.max_delta_over_h;
  eb.min_abs_psi = hst.min_abs_psi;
  eb.min_margin = eb.num_cut > 0 ? (closure != EB_CLOSURE_LINE ? rbf_margin : hst.min_margin) : 0.0;
  dfree(psi, s); dfree(is_cp, s); dfree(cp_off, s); dfree(ncut, s); dfree(st, s);
  EB_CUDA(cudaStreamSynchronize(s));
}

bool tile_shape_ok(int dim, int tx, int ty, int tz) {
  auto pow2 = [](int v) { return v >= 1 && (v & (v - 1)) == 0; };
  if (!pow2(tx) || !pow2(ty) || !pow2(tz)) return false;
  if (tx * ty * tz != TILE_NODES || tx < 2 || tx > 128 || ty > 128 || tz > 128) return false;
  return dim == 3 || tz == 1;
}

void build_tiles(EBHandle& eb, int tx, int ty, int tz, cudaStream_t s) {
  EB_REQUIRE(tile_shape_ok(eb.g.dim, tx, ty, tz), EB_ERR_INVALID,
             "tile shape: powers of two with product 256, 2 <= x <= 128, y, z <= 128, z = 1 in 2D");
  Geometry& G = eb.g;
  G.tx = tx;
  G.ty = ty;
  G.tz = tz;
  G.ntx = (G.n0 + G.tx - 1) / G.tx;
  G.nty = (G.n1 + G.ty - 1) / G.ty;
  G.ntz = (G.n2 + G.tz - 1) / G.tz;
  dfree(eb.tiles, s);
  dfree(eb.tile_base, s);
  dfree(eb.tile_lim, s);
  eb.num_tiles = 0;
  const int T = 256;
  const int64_t nn = G.num_nodes;
  const int64_t ntiles_all = (int64_t)G.ntx * G.nty * G.ntz;
  int32_t* tflag = dalloc<int32_t>(ntiles_all, s);
  int32_t* toff = nullptr;
  try {
    toff = dalloc<int32_t>(ntiles_all + 1, s, false);
    k_tile_flags<<<blocks_for(nn, T), T, 0, s>>>(G, eb.code, tflag);
    exclusive_scan_i32(tflag, toff, ntiles_all, s);
    int32_t nt = 0;
    EB_CUDA(cudaMemcpyAsync(&nt, toff + ntiles_all, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    EB_CUDA(cudaStreamSynchronize(s));
    eb.tiles = dalloc<int32_t>(nt, s, false);
    k_compact<<<blocks_for(ntiles_all, T), T, 0, s>>>(tflag, toff, ntiles_all, eb.tiles);
    eb.tile_base = dalloc<int32_t>(nt, s, false);
    eb.tile_lim = dalloc<int32_t>(nt, s, false);
    k_tile_geom<<<blocks_for(nt, T), T, 0, s>>>(G, eb.tiles, nt, eb.tile_base, eb.tile_lim);
    EB_CUDA(cudaGetLastError());
    eb.num_tiles = nt;
  } catch (...) {
    dfree(tflag, s);
    dfree(toff, s);
    throw;
  }
  dfree(tflag, s);
  dfree(toff, s);
  build_cp_pairs(eb, s);
  ++eb.tile_gen;
}

// the CP pair list of the current tile view (EBHandle::pairs)
void build_cp_pairs(EBHandle& eb, cudaStream_t s) {
  dfree(eb.pair_node, s);
  eb.num_pairs = 0;
  const int64_t nt = eb.num_tiles;
  // views with per-tile shifts (batches) keep sweeping tiles: EB_SWEEP's list
  // mode has no tile index to read a shift with
  if (nt == 0 || eb.tile_shift64 || eb.tile_shift32) return;
  int32_t* cnt = dalloc<int32_t>(nt, s, false);
  int32_t* off = nullptr;
  try {
    off = dalloc<int32_t>(nt + 1, s, false);
    const TileView tv = eb.tv();
    k_cp_pairs<<<(unsigned)nt, 128, 0, s>>>(tv, eb.code, false, cnt, nullptr, nullptr);
    exclusive_scan_i32(cnt, off, nt, s);
    int32_t np = 0;
    EB_CUDA(cudaMemcpyAsync(&np, off + nt, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    EB_CUDA(cudaStreamSynchronize(s));
    if (np > 0) {
      eb.pair_node = dalloc<int32_t>(np, s, false);
      k_cp_pairs<<<(unsigned)nt, 128, 0, s>>>(tv, eb.code, true, nullptr, off, eb.pair_node);
      EB_CUDA(cudaGetLastError());
    }
    eb.num_pairs = np;
  } catch (...) {
    dfree(cnt, s);
    dfree(off, s);
    throw;
  }
  dfree(cnt, s);
  dfree(off, s);
}

void destroy_handle(EBHandle& eb) {
  cudaStream_t s = eb.home;
  eb.lf_graph.release();
  dfree(eb.code, s); dfree(eb.diag, s); dfree(eb.diag32, s); dfree(eb.cp_of_node, s); dfree(eb.cp_node, s);
  dfree(eb.tiles, s); dfree(eb.tile_base, s); dfree(eb.tile_lim, s); dfree(eb.pair_node, s); dfree(eb.cut_cp, s); dfree(eb.cut_dir, s); dfree(eb.cut_delta, s);
  dfree(eb.cut_c, s); dfree(eb.cut_xg, s); dfree(eb.cut_off, s); dfree(eb.cut_bc, s);
  dfree(eb.rbf_cut, s); dfree(eb.cut_rbf, s); dfree(eb.rbf_xg2, s); dfree(eb.rbf_w, s); dfree(eb.rbf_rot, s);
  dfree(eb.cut_w1, s); dfree(eb.cut_bw1, s); dfree(eb.rbf_bw2, s);
  for (int a = 0; a < 3; ++a) {
    dfree(eb.beta64[a], s);
    dfree(eb.beta32[a], s);
  }
  cudaStreamSynchronize(s);
}

// ------------------------------------------------------------------- RHS
// b_k = -f_k + sum over the cuts of k of (c_s u_Gamma) / h^2, summed in cut
// order; 0 at the non-CP nodes of the active tiles.
// RBF cuts (cut_rbf[j] = r >= 0) add their second value ug[num_cut + r] with
// weight w2[r * w2_stride] after all first values of the CP (the order of the
// assembled definition).
template <int DIM>
__global__ void __launch_bounds__(TILE_NODES) k_rhs(TileView tv, const uint8_t* code, const int32_t* cp_of_node,
                                                    const int32_t* cut_off, const double* cut_c, const double* f,
                                                    const double* ug, double* b, double h2, const int32_t* cut_rbf,
                                                    const double* w2, int w2_stride, int64_t num_cut) {
  EB_TILE_LOOP(DIM, tv, node) {
    const uint8_t c = code[node];
    double v = 0.0;
    if (c & CODE_CP) {
      double acc = 0.0;
      if (c & 0x3F) {
        const int32_t k = cp_of_node[node];
        for (int j = cut_off[k]; j < cut_off[k + 1]; ++j) acc = __dadd_rn(acc, __ddiv_rn(__dmul_rn(cut_c[j], ug[j]), h2));
        if (cut_rbf)
          for (int j = cut_off[k]; j < cut_off[k + 1]; ++j) {
            const int32_t r = cut_rbf[j];
            if (r >= 0)
              acc = __dadd_rn(acc, __ddiv_rn(__dmul_rn(w2[(int64_t)r * w2_stride], ug[num_cut + r]), h2));
          }
      }
      v = __dadd_rn(-f[node], acc);
    }
    b[node] = v;
  }
}

void launch_rhs(const EBHandle& eb, const double* f, const double* ug, double* b, cudaStream_t s) {
  const Geometry& G = eb.g;
  const double h2 = G.h * G.h;
  const unsigned blocks = tile_grid(eb);
  // weight of each cut's first value: c_s (line-by-line) or w_1 (RBF), times beta with a variable beta
  const double* w = eb.cut_bw1 ? eb.cut_bw1 : (eb.cut_bc && !eb.cut_w1) ? eb.cut_bc : eb.cut_w1 ? eb.cut_w1 : eb.cut_c;
  const bool rbf = eb.num_rbf > 0;
  const double* w2 = !rbf ? nullptr : eb.rbf_bw2 ? eb.rbf_bw2 : eb.rbf_w + 2;
  const int w2s = eb.rbf_bw2 ? 1 : 3;
  const int32_t* crbf = rbf ? eb.cut_rbf : nullptr;
  if (G.dim == 2)
    k_rhs<2><<<blocks, TILE_NODES, 0, s>>>(eb.tv(), eb.code, eb.cp_of_node, eb.cut_off, w, f, ug, b, h2, crbf, w2, w2s,
                                           eb.num_cut);
  else
    k_rhs<3><<<blocks, TILE_NODES, 0, s>>>(eb.tv(), eb.code, eb.cp_of_node, eb.cut_off, w, f, ug, b, h2, crbf, w2, w2s,
                                           eb.num_cut);
  EB_CUDA(cudaGetLastError());
}

// ------------------------------------------------------------ variable beta
// bad = 1 if a beta some CP uses (the half points between it and its 2 dim
// neighbours) is not positive and finite
__global__ void k_beta_check(Geometry G, const double* bx, const double* by, const double* bz, const int32_t* cp_node,
                             int64_t num_cp, int* bad) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= num_cp) return;
  const int64_t node = cp_node[k];
  const double* b[3] = {bx, by, bz};
  for (int sdir = 0; sdir < 2 * G.dim; ++sdir) {
    const int a = sdir >> 1;
    const double beta = b[a][(sdir & 1) ? node : node - stride_of(G, a)];
    if (!(beta > 0.0) || !isfinite(beta)) *bad = 1;
  }
}

// D_k = sum_s beta_s c_s (c_s = 1 towards a CP, h/(h+delta) towards a BP),
// summed in direction order with every product rounded (the same operations
// as the assembled definition); cut_bc[j] = beta_s c_s of each cut (the
// right-hand-side weights of Sec. 2.1 with beta); CODE_DIAG set on every CP;
// the dominance margin of the cut rows.
__global__ void k_beta_diag(Geometry G, const double* bx, const double* by, const double* bz, const int32_t* cp_node,
                            const int32_t* cut_off, const double* cut_c, int64_t num_cp, uint8_t* code, double* diag,
                            double* cut_bc, unsigned long long* margin_min) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= num_cp) return;
  const int64_t node = cp_node[k];
  const uint8_t c = code[node];
  const uint8_t m = c & 0x3F;
  const double* b[3] = {bx, by, bz};
  int j = cut_off[k];
  double D = 0.0, margin = 0.0;
  for (int sdir = 0; sdir < 2 * G.dim; ++sdir) {
    const int a = sdir >> 1;
    const int64_t st = stride_of(G, a);
    const double beta = b[a][(sdir & 1) ? node : node - st];
    double w = beta;
    if (m & (1u << sdir)) {
      w = __dmul_rn(beta, cut_c[j]);
      cut_bc[j] = w;
      margin = __dadd_rn(margin, w);
      ++j;
    } else {
      w = __dmul_rn(beta, 1.0);
    }
    D = sdir == 0 ? w : __dadd_rn(D, w);
  }
  diag[node] = D;
  code[node] = (uint8_t)(c | CODE_DIAG);
  if (m) atomic_min_signed(margin_min, margin);
}

// beta of each cut's half point times its first right-hand-side weight, and
// times the second weight of RBF cuts
__global__ void k_beta_rbf(Geometry G, const double* bx, const double* by, const int32_t* cp_node,
                           const int32_t* cut_cp, const int32_t* cut_dir, const double* cut_w1, const int32_t* cut_rbf,
                           const double* rbf_w, int64_t nc, double* cut_bw1, double* rbf_bw2) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nc) return;
  const int64_t node = cp_node[cut_cp[j]];
  const int sdir = cut_dir[j], a = sdir >> 1;
  const double* b = a == 0 ? bx : by;
  const double beta = b[(sdir & 1) ? node : node - stride_of(G, a)];
  cut_bw1[j] = __dmul_rn(beta, cut_w1[j]);
  const int32_t r = cut_rbf[j];
  if (r >= 0) rbf_bw2[r] = __dmul_rn(beta, rbf_w[3 * (int64_t)r + 2]);
}

void set_beta(EBHandle& eb, const double* const* beta, cudaStream_t s) {
  const Geometry& G = eb.g;
  EB_REQUIRE(!eb.has_beta(), EB_ERR_INVALID, "eb_set_beta: beta is already set on this grid");
  EB_REQUIRE(eb.tile_shift64 == nullptr, EB_ERR_NOT_IMPLEMENTED, "eb_set_beta: not available on batched grids");
  for (int a = 0; a < G.dim; ++a) EB_REQUIRE(beta[a] != nullptr, EB_ERR_INVALID, "eb_set_beta: NULL beta array");
  const int64_t nn = G.num_nodes;
  const int T = 256;
  unsigned long long* bmin = dalloc<unsigned long long>(1, s, false);
  int* bad = dalloc<int>(1, s);
  try {
    // validate before anything of the handle changes
    k_beta_check<<<blocks_for(eb.num_cp, 128), 128, 0, s>>>(G, beta[0], beta[1], G.dim == 3 ? beta[2] : nullptr,
                                                             eb.cp_node, eb.num_cp, bad);
    EB_CUDA(cudaGetLastError());
    int hb = 0;
    EB_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    EB_CUDA(cudaStreamSynchronize(s));
    if (hb) throw Failure{EB_ERR_INVALID, "eb_set_beta: beta must be positive and finite at every half point a CP uses"};
    const unsigned long long init = ~0ull;
    EB_CUDA(cudaMemcpyAsync(bmin, &init, sizeof(init), cudaMemcpyHostToDevice, s));
    for (int a = 0; a < G.dim; ++a) {
      eb.beta64[a] = dalloc<double>(nn, s, false);
      EB_CUDA(cudaMemcpyAsync(eb.beta64[a], beta[a], sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
      eb.beta32[a] = dalloc<float>(nn, s, false);
      k_diag32<<<blocks_for(nn, T), T, 0, s>>>(nn, eb.beta64[a], eb.beta32[a]);
    }
    eb.cut_bc = dalloc<double>(eb.num_cut, s, false);
    k_beta_diag<<<blocks_for(eb.num_cp, 128), 128, 0, s>>>(G, eb.beta64[0], eb.beta64[1],
                                                            G.dim == 3 ? eb.beta64[2] : nullptr, eb.cp_node,
                                                            eb.cut_off, eb.cut_c, eb.num_cp, eb.code, eb.diag,
                                                            eb.cut_bc, bmin);
    k_diag32<<<blocks_for(nn, T), T, 0, s>>>(nn, eb.diag, eb.diag32);
    if (eb.num_rbf > 0) {
      eb.cut_bw1 = dalloc<double>(eb.num_cut, s, false);
      eb.rbf_bw2 = dalloc<double>(eb.num_rbf, s, false);
      k_beta_rbf<<<blocks_for(eb.num_cut, 128), 128, 0, s>>>(G, eb.beta64[0], eb.beta64[1], eb.cp_node, eb.cut_cp,
                                                              eb.cut_dir, eb.cut_w1, eb.cut_rbf, eb.rbf_w, eb.num_cut,
                                                              eb.cut_bw1, eb.rbf_bw2);
    }
    EB_CUDA(cudaGetLastError());
    unsigned long long hk = 0;
    EB_CUDA(cudaMemcpyAsync(&hk, bmin, sizeof(hk), cudaMemcpyDeviceToHost, s));
    EB_CUDA(cudaStreamSynchronize(s));
    eb.min_margin = eb.num_cut > 0 ? decode_signed_key(hk) : 0.0;
  } catch (...) {
    dfree(bmin, s);
    dfree(bad, s);
    for (int a = 0; a < 3; ++a) {  // leave the handle without beta
      dfree(eb.beta64[a], s);
      dfree(eb.beta32[a], s);
    }
    dfree(eb.cut_bc, s);
    throw;
  }
  dfree(bmin, s);
  dfree(bad, s);
  eb.lf_graph.release();
  ++eb.tile_gen;  // captured graphs hold the view without beta
  EB_CUDA(cudaStreamSynchronize(s));
}

}  // namespace ebk
