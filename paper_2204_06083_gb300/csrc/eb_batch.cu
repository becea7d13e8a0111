// Batched grids: many geometries of uneven size advanced by one set of
// launches (implicit heat steps, Sec. 3.4, for a batch of domains).
//
// Batch layout.  Geometry g's full grid (n0_g x n1_g nodes, x fastest) sits
// at node offset off_g of one concatenated array whose rows all have the same
// stride S = max_g n0_g; node (i, j) of g is off_g + j S + i.  Every vector of
// the batch API uses this layout.  One list of active tiles, with the geometry
// of each tile, covers all grids, so the single-grid stencil kernels run
// unchanged on the batch (a grid's stencil never leaves its own rows because
// its outer ring of nodes is outside the domain).
//
// Scaling.  Geometry g's equations are multiplied by h_g^2: the operator of
// the batch is blockdiag(sigma'_g I + A~_g) with A~ the unit-spacing stencil
// (D_k x_k - sum of CP neighbours) and sigma'_g = h_g^2 / (theta dt_g), so all
// tiles share h = 1 and only the shift differs per tile.  Relative residuals
// are unchanged by this scaling.
//
// Solver.  One smoothed-aggregation hierarchy on the block-diagonal level-0
// matrix (aggregation never crosses blocks, so it is a hierarchy per
// geometry), and PCG with separate recurrences per geometry: kernels write
// one partial per tile, one CTA per geometry combines the partials of its
// tiles in a fixed order and advances that geometry's scalars; a converged
// geometry's tiles are skipped by the update kernels.  The iteration is
// captured in a CUDA graph.
#include "amg_internal.cuh"
#include "df.cuh"
#include "stencil.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>

namespace ebk {

constexpr int BT = PAIR_THREADS;  // one tile per CTA of 128 threads

struct GeoConst {
  double h2, dt, theta;
};

struct Batch {
  std::vector<eb_handle*> geo;
  std::vector<int64_t> node_off, cut_off, cp_off, tile_off;
  int64_t stride = 0;
  EBHandle view;                 // batch-layout view: code, diag, diag32, cp_node, cp_of_node, tiles
  int32_t* tile_geo = nullptr;   // [ntiles] geometry of each tile
  int32_t* geo_tile0 = nullptr;  // [ngeo + 1] first tile of each geometry
  int32_t* cut_off_cp = nullptr; // [num_cp + 1] global cut offset of each global CP
  double* cut_c = nullptr;       // [num_cut] c_s of every cut, geometry by geometry
  GeoConst* gconst = nullptr;    // [ngeo]
  std::vector<GeoConst> hconst;
  Solver* S = nullptr;
  PcgScalars* sc = nullptr;      // [ngeo]
  PcgScalars* sc_host = nullptr;
  double* part = nullptr;        // [2 ntiles]
  cudaStream_t home = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const double* g_b = nullptr;
  double* g_x = nullptr;
  int64_t g_launches = 0, nlaunch = 0;
  // event timing of the level-0 smoother launches inside the captured iteration
  bool profile = false;
  int g_prof = -1, g_pairs = 0;
  // the DF outer iteration (batch_set_outer_prec): requested precision, whether
  // the current solve runs it, per-geometry powers of two into DF, the DF copy
  // of the cut CPs' diagonals; g_df / l_df key the captured graphs
  int outer = EB_F64;
  bool l0_tma = true;  // batch_set_level0_tma, passed to the solver at setup
  bool df = false;
  double* gscale = nullptr;
  double* xdf = nullptr;  // the DF image of x (the solver's tmp holds the right-hand side)
  float2* diag_df = nullptr;
  int g_df = -1, l_df = -1;
  // the whole loop on the device (conditional WHILE node) when not profiling
  cudaGraphExec_t lexec = nullptr;
  const double* l_b = nullptr;
  double* l_x = nullptr;
  int64_t l_launches = 0;
  int ngeo() const { return (int)geo.size(); }
};

// ------------------------------------------------------------------ build
__global__ void k_map_cp(int64_t n, const int32_t* cp_node, int32_t n0, int64_t S, int64_t off, int32_t* out) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int32_t node = cp_node[k];
  out[k] = (int32_t)(off + (int64_t)(node / n0) * S + node % n0);
}

__global__ void k_rebase_tiles(int64_t n, const int32_t* base, int32_t n0, int64_t S, int64_t off, int32_t* out) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int32_t b = base[k];
  out[k] = (int32_t)(off + (int64_t)(b / n0) * S + b % n0);
}

__global__ void k_offset_cp(int64_t n, int32_t* v, int32_t add) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n && v[k] >= 0) v[k] += add;
}

__global__ void k_add_i32(int64_t n, const int32_t* in, int32_t add, int32_t* out) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = in[k] + add;
}

__global__ void k_fill_i32(int64_t n, int32_t v, int32_t* out) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = v;
}

__global__ void k_tile_shift(int64_t nt, const int32_t* tile_geo, const GeoConst* gc, double2* t64, float2* t32) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const GeoConst c = gc[tile_geo[t]];
  const double sig = c.h2 / (c.theta * c.dt);
  const double di = 1.0 / (sig + 4.0);
  t64[t] = make_double2(sig, di);
  t32[t] = make_float2((float)sig, (float)di);
}

static void batch_tiles(Batch& B, cudaStream_t s);

static void build_batch(Batch& B, const eb_grid* grids, const eb_levelset* lss, int count, cudaStream_t s) {
  EB_REQUIRE(count >= 1, EB_ERR_INVALID, "batch_build: need at least one geometry");
  B.home = s;
  int64_t S = 0, rows = 0;
  for (int g = 0; g < count; ++g) {
    EB_REQUIRE(grids[g].dim == 2, EB_ERR_INVALID, "batch_build: batches of 2D grids only");
    S = std::max<int64_t>(S, grids[g].n[0]);
  }
  S += S & 1;
  B.stride = S;
  B.node_off.assign(count + 1, 0);
  B.cut_off.assign(count + 1, 0);
  B.cp_off.assign(count + 1, 0);
  for (int g = 0; g < count; ++g) {
    eb_handle* e = new eb_handle();
    B.geo.push_back(e);
    build_handle(e->h, grids[g], lss[g], s);
    B.node_off[g + 1] = B.node_off[g] + S * (int64_t)grids[g].n[1];
    B.cut_off[g + 1] = B.cut_off[g] + e->h.num_cut;
    B.cp_off[g + 1] = B.cp_off[g] + e->h.num_cp;
    rows += grids[g].n[1];
  }
  const int64_t nn = B.node_off[count], ncp = B.cp_off[count], ncut = B.cut_off[count];
  EB_REQUIRE(nn < ((int64_t)1 << 31) - 1, EB_ERR_INVALID, "batch_build: batch above 2^31 nodes");
  EBHandle& V = B.view;
  V.home = s;
  Geometry& G = V.g;
  G.dim = 2;
  G.n0 = (int)S;
  G.n1 = (int)rows;
  G.n2 = 1;
  G.num_nodes = nn;
  G.lo[0] = G.lo[1] = G.lo[2] = 0.0;
  G.h = 1.0;
  V.num_cp = ncp;
  V.num_cut = ncut;
  V.code = dalloc<uint8_t>(nn, s);
  V.diag = dalloc<double>(nn, s);
  V.diag32 = dalloc<float>(nn, s);
  V.cp_of_node = dalloc<int32_t>(nn, s, false);
  k_fill_i32<<<blocks_for(nn, 256), 256, 0, s>>>(nn, -1, V.cp_of_node);
  V.cp_node = dalloc<int32_t>(ncp, s, false);
  B.cut_off_cp = dalloc<int32_t>(ncp + 1, s, false);
  B.cut_c = dalloc<double>(ncut, s, false);
  for (int g = 0; g < count; ++g) {
    const EBHandle& h = B.geo[g]->h;
    const int64_t n0 = h.g.n0, n1 = h.g.n1, off = B.node_off[g];
    EB_CUDA(cudaMemcpy2DAsync(V.code + off, S, h.code, n0, n0, n1, cudaMemcpyDeviceToDevice, s));
    EB_CUDA(cudaMemcpy2DAsync(V.diag + off, S * 8, h.diag, n0 * 8, n0 * 8, n1, cudaMemcpyDeviceToDevice, s));
    EB_CUDA(cudaMemcpy2DAsync(V.diag32 + off, S * 4, h.diag32, n0 * 4, n0 * 4, n1, cudaMemcpyDeviceToDevice, s));
    EB_CUDA(cudaMemcpy2DAsync(V.cp_of_node + off, S * 4, h.cp_of_node, n0 * 4, n0 * 4, n1,
                              cudaMemcpyDeviceToDevice, s));
    k_offset_cp<<<blocks_for(S * n1, 256), 256, 0, s>>>(S * n1, V.cp_of_node + off, (int32_t)B.cp_off[g]);
    k_map_cp<<<blocks_for(h.num_cp, 256), 256, 0, s>>>(h.num_cp, h.cp_node, h.g.n0, S, off, V.cp_node + B.cp_off[g]);
    k_add_i32<<<blocks_for(h.num_cp, 256), 256, 0, s>>>(h.num_cp, h.cut_off, (int32_t)B.cut_off[g],
                                                          B.cut_off_cp + B.cp_off[g]);
    if (h.num_cut)
      EB_CUDA(cudaMemcpyAsync(B.cut_c + B.cut_off[g], h.cut_c, 8 * h.num_cut, cudaMemcpyDeviceToDevice, s));
  }
  const int32_t ncut32 = (int32_t)ncut;
  EB_CUDA(cudaMemcpyAsync(B.cut_off_cp + ncp, &ncut32, 4, cudaMemcpyHostToDevice, s));
  B.gconst = dalloc<GeoConst>(count, s);
  B.hconst.resize(count);
  for (int g = 0; g < count; ++g) B.hconst[g] = GeoConst{grids[g].h * grids[g].h, 1.0, 1.0};
  EB_CUDA(cudaMemcpyAsync(B.gconst, B.hconst.data(), sizeof(GeoConst) * count, cudaMemcpyHostToDevice, s));
  B.sc = dalloc<PcgScalars>(count, s);
  EB_CUDA(cudaMallocHost((void**)&B.sc_host, sizeof(PcgScalars) * count));
  EB_CUDA(cudaStreamSynchronize(s));  // the host values above are read by the async copies
  batch_tiles(B, s);
  EB_CUDA(cudaGetLastError());
}

// (Re)builds the batch view's tile list from the geometries' tile lists (all
// geometries share one tile shape), with the per-tile geometry ids, shifts and
// reduction partials that depend on it.  Drops the captured iteration.
static void batch_tiles(Batch& B, cudaStream_t s) {
  EBHandle& V = B.view;
  const int count = B.ngeo();
  const Geometry& g0 = B.geo[0]->h.g;
  for (int g = 1; g < count; ++g)
    EB_REQUIRE(B.geo[g]->h.g.tx == g0.tx && B.geo[g]->h.g.ty == g0.ty, EB_ERR_INVALID,
               "batch: the geometries have different tile shapes");
  B.tile_off.assign(count + 1, 0);
  for (int g = 0; g < count; ++g) B.tile_off[g + 1] = B.tile_off[g] + B.geo[g]->h.num_tiles;
  const int64_t nt = B.tile_off[count];
  if (B.gexec) cudaGraphExecDestroy(B.gexec);
  B.gexec = nullptr;
  if (B.lexec) cudaGraphExecDestroy(B.lexec);
  B.lexec = nullptr;
  B.l_b = nullptr;
  B.l_x = nullptr;
  dfree(V.tile_base, s); dfree(V.tile_lim, s); dfree(V.tile_shift64, s); dfree(V.tile_shift32, s);
  dfree(B.tile_geo, s); dfree(B.geo_tile0, s); dfree(B.part, s);
  V.num_tiles = 0;
  Geometry& G = V.g;
  G.tx = g0.tx;
  G.ty = g0.ty;
  G.tz = 1;
  G.ntx = (int)((G.n0 + G.tx - 1) / G.tx);
  G.nty = (int)((G.n1 + G.ty - 1) / G.ty);
  G.ntz = 1;
  V.tile_base = dalloc<int32_t>(nt, s, false);
  V.tile_lim = dalloc<int32_t>(nt, s, false);
  V.tile_shift64 = dalloc<double2>(nt, s);
  V.tile_shift32 = dalloc<float2>(nt, s);
  B.tile_geo = dalloc<int32_t>(nt, s, false);
  B.part = dalloc<double>(2 * std::max<int64_t>(nt, 1), s);
  B.geo_tile0 = dalloc<int32_t>(count + 1, s, false);
  for (int g = 0; g < count; ++g) {
    const EBHandle& h = B.geo[g]->h;
    k_rebase_tiles<<<blocks_for(h.num_tiles, 256), 256, 0, s>>>(h.num_tiles, h.tile_base, h.g.n0, B.stride,
                                                                B.node_off[g], V.tile_base + B.tile_off[g]);
    EB_CUDA(cudaMemcpyAsync(V.tile_lim + B.tile_off[g], h.tile_lim, 4 * h.num_tiles, cudaMemcpyDeviceToDevice, s));
    k_fill_i32<<<blocks_for(h.num_tiles, 256), 256, 0, s>>>(h.num_tiles, g, B.tile_geo + B.tile_off[g]);
  }
  std::vector<int32_t> gt0(count + 1);
  for (int g = 0; g <= count; ++g) gt0[g] = (int32_t)B.tile_off[g];
  EB_CUDA(cudaMemcpyAsync(B.geo_tile0, gt0.data(), 4 * (count + 1), cudaMemcpyHostToDevice, s));
  V.num_tiles = nt;
  k_tile_shift<<<blocks_for(nt, 256), 256, 0, s>>>(nt, B.tile_geo, B.gconst, V.tile_shift64, V.tile_shift32);
  EB_CUDA(cudaGetLastError());
  ++V.tile_gen;
  EB_CUDA(cudaStreamSynchronize(s));  // gt0 is read by the copy above
}

static void destroy_batch(Batch& B) {
  cudaStream_t s = B.home;
  if (B.gexec) cudaGraphExecDestroy(B.gexec);
  if (B.lexec) cudaGraphExecDestroy(B.lexec);
  if (B.cap_stream) cudaStreamDestroy(B.cap_stream);
  if (B.S) {
    amg_free(*B.S);
    B.S->free_work();
    B.S->prof_release();
    delete B.S;
    B.S = nullptr;
  }
  EBHandle& V = B.view;
  dfree(V.code, s); dfree(V.diag, s); dfree(V.diag32, s); dfree(V.cp_of_node, s); dfree(V.cp_node, s);
  dfree(V.tile_base, s); dfree(V.tile_lim, s); dfree(V.tile_shift64, s); dfree(V.tile_shift32, s);
  dfree(B.tile_geo, s); dfree(B.geo_tile0, s); dfree(B.cut_off_cp, s); dfree(B.cut_c, s); dfree(B.gconst, s);
  dfree(B.sc, s); dfree(B.part, s); dfree(B.gscale, s); dfree(B.diag_df, s); dfree(B.xdf, s);
  if (B.sc_host) cudaFreeHost(B.sc_host);
  B.sc_host = nullptr;
  for (eb_handle* e : B.geo) {
    destroy_handle(e->h);
    delete e;
  }
  B.geo.clear();
  cudaStreamSynchronize(s);
}

// ------------------------------------------------------------------- RHS
// b = -f + sum over the cuts of (c_s u_Gamma) / h_g^2, batch layout
__global__ void __launch_bounds__(BT) k_b_rhs(TileView tv, const int32_t* tile_geo, const GeoConst* gc,
                                              const uint8_t* code, const int32_t* cp_of_node, const int32_t* cut_off,
                                              const double* cut_c, const double* f, const double* ug, double* b) {
  for (int64_t tt = blockIdx.x; tt < tv.ntiles; tt += gridDim.x) {
    int32_t node;
    if (!tile_pair<2>(tv, tt, threadIdx.x, node)) continue;
    const double h2 = gc[tile_geo[tt]].h2;
    for (int q = 0; q < 2; ++q) {
      const int32_t nd = node + q;
      const uint8_t c = code[nd];
      double v = 0.0;
      if (c & CODE_CP) {
        double acc = 0.0;
        if (c & 0x3F) {
          const int32_t k = cp_of_node[nd];
          for (int j = cut_off[k]; j < cut_off[k + 1]; ++j) acc += cut_c[j] * ug[j] / h2;
        }
        v = -f[nd] + acc;
      }
      b[nd] = v;
    }
  }
}

// ------------------------------------------------------------ batched PCG
__device__ __forceinline__ double tile_sum(double v, double* sm) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sm[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < BT / 32; ++i) s += sm[i];
  return s;
}

// unit-spacing operator with the tile's shift: (sigma' + D) x - sum of CP neighbours
__device__ __forceinline__ void b_op(const TileView& tv, int64_t tt, const double* x, int32_t node, uint32_t c0,
                                     uint32_t c1, const double* diag, Two<double>& xc, Two<double>& ax) {
  Two<double> core;
  stencil_pair<2, LdRO>(x, node, tv.nn, c0, c1, diag, tv.sy, tv.sz, xc, core);
  const double sig = __ldg(tv.tshift64 + tt).x;
  ax.x = core.x + sig * xc.x;
  ax.y = core.y + sig * xc.y;
}

// r = b - B x; per-tile partials (b.b, r.r)
__global__ void __launch_bounds__(BT) k_b_resid(TileView tv, const uint8_t* code, const double* diag, const double* b,
                                                const double* x, double* r, double* part) {
  __shared__ double sm[BT / 32];
  for (int64_t tt = blockIdx.x; tt < tv.ntiles; tt += gridDim.x) {
    int32_t node;
    double sbb = 0.0, srr = 0.0;
    if (tile_pair<2>(tv, tt, threadIdx.x, node)) {
      uint32_t c0, c1;
      ld_codes(code, node, c0, c1);
      Two<double> xc, ax;
      b_op(tv, tt, x, node, c0, c1, diag, xc, ax);
      const Two<double> bv = LdRO::ld2(b + node);
      const double b0 = (c0 & CODE_CP) ? bv.x : 0.0, b1 = (c1 & CODE_CP) ? bv.y : 0.0;
      const double r0 = (c0 & CODE_CP) ? b0 - ax.x : 0.0, r1 = (c1 & CODE_CP) ? b1 - ax.y : 0.0;
      sbb = b0 * b0 + b1 * b1;
      srr = r0 * r0 + r1 * r1;
      st2(r + node, r0, r1);
    }
    const double a = tile_sum(sbb, sm);
    const double q = tile_sum(srr, sm);
    if (threadIdx.x == 0) {
      part[2 * tt] = a;
      part[2 * tt + 1] = q;
    }
  }
}

// The end of a batched PCG iteration in one pass (tiles of converged
// geometries skipped): p = z + beta p and q = B z + beta q -- in exact
// arithmetic B (z + beta p), since q holds B p -- with the per-tile p.q
// partials, beta the geometry's (k_b_finalize FIN_BETA / FIN_BETAF).  The
// stencil reads z, which the preconditioner launch before completed, so the p
// update and the apply of the next iteration share one launch.  first: beta =
// 0, p = z, q = B z (the old p and q are not read).
__global__ void __launch_bounds__(BT) k_b_xpby_apply(TileView tv, const int32_t* tile_geo, const PcgScalars* sc,
                                                     const uint8_t* code, const double* diag, const double* z,
                                                     double* p, double* q, int first, double* part) {
  __shared__ double sm[BT / 32];
  for (int64_t tt = blockIdx.x; tt < tv.ntiles; tt += gridDim.x) {
    const PcgScalars& S = sc[tile_geo[tt]];
    if (S.done) continue;
    const double beta = first ? 0.0 : S.beta;
    int32_t node;
    double s = 0.0;
    if (tile_pair<2>(tv, tt, threadIdx.x, node)) {
      uint32_t c0, c1;
      ld_codes(code, node, c0, c1);
      Two<double> zc, az;
      b_op(tv, tt, z, node, c0, c1, diag, zc, az);
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
      s = p0 * q0 + p1 * q1;
    }
    const double t = tile_sum(s, sm);
    if (threadIdx.x == 0) part[tt] = t;
  }
}

// x += alpha p, r -= alpha q; per-tile partials r.r and, with z (flexible
// CG), r.z for the new r and the z still in place (the r.zold term of the
// Polak-Ribiere beta), as pairs; without z, single r.r partials
__global__ void __launch_bounds__(BT) k_b_update_xr(TileView tv, const int32_t* tile_geo, const PcgScalars* sc,
                                                    double* x, double* r, const double* p, const double* q,
                                                    const double* z, double* part) {
  __shared__ double sm[BT / 32];
  for (int64_t tt = blockIdx.x; tt < tv.ntiles; tt += gridDim.x) {
    const PcgScalars& S = sc[tile_geo[tt]];
    if (S.done) continue;
    const double alpha = S.alpha;
    int32_t node;
    double s = 0.0, so = 0.0;
    if (tile_pair<2>(tv, tt, threadIdx.x, node)) {
      const Two<double> rv = ld2d(r + node), qv = LdRO::ld2(q + node), pv = LdRO::ld2(p + node), xv = ld2d(x + node);
      const double r0 = rv.x - alpha * qv.x, r1 = rv.y - alpha * qv.y;
      st2(x + node, xv.x + alpha * pv.x, xv.y + alpha * pv.y);
      st2(r + node, r0, r1);
      s = r0 * r0 + r1 * r1;
      if (z) {
        const Two<double> zv = LdRO::ld2(z + node);
        so = r0 * zv.x + r1 * zv.y;
      }
    }
    const double t = tile_sum(s, sm);
    if (z) {
      const double u = tile_sum(so, sm);
      if (threadIdx.x == 0) {
        part[2 * tt] = t;
        part[2 * tt + 1] = u;
      }
    } else if (threadIdx.x == 0) {
      part[tt] = t;
    }
  }
}

// per-tile partials r.z (pairs (r.z, 0), the layout k_b_finalize reads for
// FIN_RZ0 / FIN_BETA)
__global__ void __launch_bounds__(BT) k_b_dot(TileView tv, const int32_t* tile_geo, const PcgScalars* sc,
                                              const double* r, const double* z, double* part) {
  __shared__ double sm[BT / 32];
  for (int64_t tt = blockIdx.x; tt < tv.ntiles; tt += gridDim.x) {
    if (sc[tile_geo[tt]].done) continue;
    int32_t node;
    double a = 0.0;
    if (tile_pair<2>(tv, tt, threadIdx.x, node)) {
      const Two<double> rv = LdRO::ld2(r + node), zv = LdRO::ld2(z + node);
      a = rv.x * zv.x + rv.y * zv.y;
    }
    const double u = tile_sum(a, sm);
    if (threadIdx.x == 0) {
      part[2 * tt] = u;
      part[2 * tt + 1] = 0.0;
    }
  }
}

__global__ void __launch_bounds__(BT) k_b_mask(TileView tv, const uint8_t* code, const double* in, double* out) {
  for (int64_t tt = blockIdx.x; tt < tv.ntiles; tt += gridDim.x) {
    int32_t node;
    if (!tile_pair<2>(tv, tt, threadIdx.x, node)) continue;
    uint32_t c0, c1;
    ld_codes(code, node, c0, c1);
    const Two<double> v = ld2d(in + node);
    st2(out + node, (c0 & CODE_CP) ? v.x : 0.0, (c1 & CODE_CP) ? v.y : 0.0);
  }
}

// scaled theta-method right-hand side:
// (h^2/theta) (u/dt + theta b1 + (1-theta) b0) - ((1-theta)/theta) A~ u
__global__ void __launch_bounds__(BT) k_b_heat_rhs(TileView tv, const int32_t* tile_geo, const GeoConst* gc,
                                                   const uint8_t* code, const double* diag, const double* u,
                                                   const double* b1, const double* b0, double* out) {
  for (int64_t tt = blockIdx.x; tt < tv.ntiles; tt += gridDim.x) {
    int32_t node;
    if (!tile_pair<2>(tv, tt, threadIdx.x, node)) continue;
    const GeoConst c = gc[tile_geo[tt]];
    uint32_t c0, c1;
    ld_codes(code, node, c0, c1);
    Two<double> uc, core;
    stencil_pair<2, LdRO>(u, node, tv.nn, c0, c1, diag, tv.sy, tv.sz, uc, core);
    const Two<double> v1 = LdRO::ld2(b1 + node);
    const double s = c.h2 / c.theta;
    double r0 = s * (uc.x / c.dt + c.theta * v1.x), r1 = s * (uc.y / c.dt + c.theta * v1.y);
    if (c.theta < 1.0) {
      const Two<double> v0 = LdRO::ld2(b0 + node);
      const double w = (1.0 - c.theta) / c.theta;
      r0 += s * (1.0 - c.theta) * v0.x - w * core.x;
      r1 += s * (1.0 - c.theta) * v0.y - w * core.y;
    }
    st2(out + node, (c0 & CODE_CP) ? r0 : 0.0, (c1 & CODE_CP) ? r1 : 0.0);
  }
}

// --------------------------------------------- the DF outer iteration (batch)
// The batched iteration with x, r, p, q as double-float vectors (DF pairs in
// the buffers of doubles), z the FP32 V-cycle output and DF per-tile partials
// (in the slots of the doubles), as the single-grid DF iteration: every vector
// operation on the FP32 pipe with error-free transformations.  A tile's
// scalars (alpha or beta, the shift sigma') are split into DF once per tile.

// x += alpha p, r -= alpha q in DF; per-tile DF partials r.r and, with z
// (flexible CG), r.zold as pairs, else r.r alone (k_b_update_xr's layout)
__global__ void __launch_bounds__(BT) k_b_update_xr_df(TileView tv, const int32_t* tile_geo, const PcgScalars* sc,
                                                       double* x, double* r, const double* p, const double* q,
                                                       const float* z, double* part) {
  __shared__ DF dsm[BT / 32];
  __shared__ DF s_a;
  for (int64_t tt = blockIdx.x; tt < tv.ntiles; tt += gridDim.x) {
    const PcgScalars& S = sc[tile_geo[tt]];
    if (S.done) continue;
    __syncthreads();  // s_a of the previous tile is read
    if (threadIdx.x == 0) s_a = df_from_double(S.alpha);
    __syncthreads();
    const DF a = s_a;
    int32_t node;
    DF srr{0.0f, 0.0f}, srzo{0.0f, 0.0f};
    if (tile_pair<2>(tv, tt, threadIdx.x, node)) {
      DF r0, r1, q0, q1, p0, p1, xa, xb;
      df_ld2_rw(r, node, r0, r1);
      df_ld2(q, node, q0, q1);
      df_ld2(p, node, p0, p1);
      df_ld2_rw(x, node, xa, xb);
      r0 = df_sub(r0, df_mul(a, q0));
      r1 = df_sub(r1, df_mul(a, q1));
      df_st2(x, node, df_add_fast(xa, df_mul(a, p0)), df_add_fast(xb, df_mul(a, p1)));
      df_st2(r, node, r0, r1);
      df_acc_prod(srr, r0, r0);
      df_acc_prod(srr, r1, r1);
      if (z) {
        const float2 zv = __ldg(reinterpret_cast<const float2*>(z + node));
        df_acc_prod_f(srzo, r0, zv.x);
        df_acc_prod_f(srzo, r1, zv.y);
      }
    }
    const DF t = df_block_sum_df(srr, dsm);
    if (z) {
      const DF u = df_block_sum_df(srzo, dsm);
      if (threadIdx.x == 0) {
        df_part_store(part, 2 * tt, t);
        df_part_store(part, 2 * tt + 1, u);
      }
    } else if (threadIdx.x == 0) {
      df_part_store(part, tt, t);
    }
  }
}

// per-tile DF partials r.z (pairs (r.z, 0)) for r in DF and the FP32 z
__global__ void __launch_bounds__(BT) k_b_dot_df(TileView tv, const int32_t* tile_geo, const PcgScalars* sc,
                                                 const double* r, const float* z, double* part) {
  __shared__ DF dsm[BT / 32];
  for (int64_t tt = blockIdx.x; tt < tv.ntiles; tt += gridDim.x) {
    if (sc[tile_geo[tt]].done) continue;
    int32_t node;
    DF a{0.0f, 0.0f};
    if (tile_pair<2>(tv, tt, threadIdx.x, node)) {
      DF r0, r1;
      df_ld2(r, node, r0, r1);
      const float2 zv = __ldg(reinterpret_cast<const float2*>(z + node));
      df_acc_prod_f(a, r0, zv.x);
      df_acc_prod_f(a, r1, zv.y);
    }
    const DF u = df_block_sum_df(a, dsm);
    if (threadIdx.x == 0) {
      df_part_store(part, 2 * tt, u);
      df_part_store(part, 2 * tt + 1, DF{0.0f, 0.0f});
    }
  }
}

// p = z + beta p, q = B z + beta q in DF with the per-tile DF partials p.q;
// B z = (sigma' + D_k) z_k - sum of the CP-neighbour values on the FP32 z (the
// neighbours by cascaded summation, D_k z_k exact or DF, sigma' z_k in DF)
__global__ void __launch_bounds__(BT) k_b_xpby_apply_df(TileView tv, const int32_t* tile_geo, const PcgScalars* sc,
                                                        const uint8_t* code, const float2* diag_df, const float* z,
                                                        double* p, double* q, int first, double* part) {
  __shared__ DF dsm[BT / 32];
  __shared__ DF s_c[2];
  for (int64_t tt = blockIdx.x; tt < tv.ntiles; tt += gridDim.x) {
    const PcgScalars& S = sc[tile_geo[tt]];
    if (S.done) continue;
    __syncthreads();  // s_c of the previous tile is read
    if (threadIdx.x == 0) {
      s_c[0] = df_from_double(first ? 0.0 : S.beta);
      s_c[1] = df_from_double(__ldg(tv.tshift64 + tt).x);
    }
    __syncthreads();
    const DF beta = s_c[0], sig = s_c[1];
    int32_t node;
    DF s{0.0f, 0.0f};
    if (tile_pair<2>(tv, tt, threadIdx.x, node)) {
      uint32_t c0, c1;
      ld_codes(code, node, c0, c1);
      const int32_t nn = tv.nn, sy = tv.sy;
      const float2 zero{0.0f, 0.0f};
      const float2 zc = __ldg(reinterpret_cast<const float2*>(z + node));
      const float left = node > 0 ? __ldg(z + node - 1) : 0.0f;
      const float right = node + 2 < nn ? __ldg(z + node + 2) : 0.0f;
      const float2 dn = node >= sy ? __ldg(reinterpret_cast<const float2*>(z + node - sy)) : zero;
      const float2 up = node + sy < nn ? __ldg(reinterpret_cast<const float2*>(z + node + sy)) : zero;
      Sum2 s0 = sum2_start((c0 & 1) ? 0.0f : left), s1 = sum2_start((c1 & 1) ? 0.0f : zc.x);
      sum2_add(s0, (c0 & 2) ? 0.0f : zc.y);
      sum2_add(s1, (c1 & 2) ? 0.0f : right);
      sum2_add(s0, (c0 & 4) ? 0.0f : dn.x);
      sum2_add(s1, (c1 & 4) ? 0.0f : dn.y);
      sum2_add(s0, (c0 & 8) ? 0.0f : up.x);
      sum2_add(s1, (c1 & 8) ? 0.0f : up.y);
      float d0h = 4.0f, d0l = 0.0f, d1h = 4.0f, d1l = 0.0f;
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
      const DF a0 = df_add(df_prod_minus_sum2(pr0, pe0, s0), df_mul_f(sig, zc.x));
      const DF a1 = df_add(df_prod_minus_sum2(pr1, pe1, s1), df_mul_f(sig, zc.y));
      DF p0 = df_make(zc.x), p1 = df_make(zc.y), q0 = a0, q1 = a1;
      if (!first) {
        DF po0, po1, qo0, qo1;
        df_ld2_rw(p, node, po0, po1);
        df_ld2_rw(q, node, qo0, qo1);
        p0 = df_add_f(df_mul(beta, po0), zc.x);
        p1 = df_add_f(df_mul(beta, po1), zc.y);
        q0 = df_add_fast(df_mul(beta, qo0), a0);
        q1 = df_add_fast(df_mul(beta, qo1), a1);
      }
      if (!(c0 & CODE_CP)) q0 = DF{0.0f, 0.0f};
      if (!(c1 & CODE_CP)) q1 = DF{0.0f, 0.0f};
      df_st2(p, node, p0, p1);
      df_st2(q, node, q0, q1);
      df_acc_prod(s, p0, q0);
      df_acc_prod(s, p1, q1);
    }
    const DF t = df_block_sum_df(s, dsm);
    if (threadIdx.x == 0) df_part_store(part, tt, t);
  }
}

// Into DF over the active tiles: xd = scale_g x and, in place, r = scale_g r,
// scale_g the power of two of the tile's geometry; and back: x = xd / scale_g
__global__ void __launch_bounds__(BT) k_b_df_in(TileView tv, const int32_t* tile_geo, const double* scale,
                                                const double* x, double* xd, double* r) {
  for (int64_t tt = blockIdx.x; tt < tv.ntiles; tt += gridDim.x) {
    int32_t node;
    if (!tile_pair<2>(tv, tt, threadIdx.x, node)) continue;
    const double sc = scale[tile_geo[tt]];
    const Two<double> xv = ld2d(x + node), rv = ld2d(r + node);
    df_st2(xd, node, df_from_double(xv.x * sc), df_from_double(xv.y * sc));
    df_st2(r, node, df_from_double(rv.x * sc), df_from_double(rv.y * sc));
  }
}

__global__ void __launch_bounds__(BT) k_b_df_out(TileView tv, const int32_t* tile_geo, const double* scale,
                                                 const double* xd, double* x) {
  for (int64_t tt = blockIdx.x; tt < tv.ntiles; tt += gridDim.x) {
    int32_t node;
    if (!tile_pair<2>(tv, tt, threadIdx.x, node)) continue;
    const double inv = 1.0 / scale[tile_geo[tt]];
    DF a, b;
    df_ld2_rw(xd, node, a, b);
    st2(x + node, df_to_double(a) * inv, df_to_double(b) * inv);
  }
}

// the DF copy of the cut CPs' diagonals of the batch view
__global__ void __launch_bounds__(BT) k_b_df_diag(TileView tv, const uint8_t* code, const double* diag,
                                                  float2* out) {
  for (int64_t tt = blockIdx.x; tt < tv.ntiles; tt += gridDim.x) {
    int32_t node;
    if (!tile_pair<2>(tv, tt, threadIdx.x, node)) continue;
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

// one CTA per geometry: combine the geometry's tile partials in a fixed order
// df: the partials are DF (the DF iteration; never FIN_INIT), each thread's
// share summed in DF and rounded once.
__global__ void k_b_finalize(const double* part, const int32_t* geo_tile0, int op, PcgScalars* sc, int df) {
  __shared__ double sm[2][256];
  const int g = blockIdx.x;
  const int t0 = geo_tile0[g], t1 = geo_tile0[g + 1];
  // k_b_resid, k_b_dot and the flexible x/r update (FIN_RRF) write pairs of
  // partials, the others single ones
  const bool pairs = op != FIN_ALPHA && op != FIN_RR;
  PcgScalars& S = sc[g];
  // a geometry already done (converged at FIN_INIT, e.g. on a restart) has no
  // fresh partials: the kernels skip its tiles
  if (op != FIN_INIT && S.done) return;
  double a = 0.0, b = 0.0;
  if (df) {
    DF da{0.0f, 0.0f}, db{0.0f, 0.0f};
    for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
      da = df_add(da, df_part_load(part, pairs ? 2 * (int64_t)t : t));
      if (pairs) db = df_add(db, df_part_load(part, 2 * (int64_t)t + 1));
    }
    a = df_to_double(da);
    b = df_to_double(db);
  } else {
    for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
      a += pairs ? part[2 * t] : part[t];
      if (pairs) b += part[2 * t + 1];
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
  const double v = sm[0][0], w = sm[1][0];
  switch (op) {
    case FIN_INIT:
      S.bb = v;
      S.rr = w;
      if (!isfinite(v) || !isfinite(w)) S.flags |= PCG_FLAG_NONFINITE;
      S.done = (w <= S.tol2 * v || !isfinite(v) || !isfinite(w)) ? 1 : 0;
      break;
    case FIN_RZ0:
    case FIN_RZ0F:
      S.rz[0] = v;
      if (!isfinite(v)) {
        S.flags |= PCG_FLAG_NONFINITE;
        S.done = 1;
      }
      break;
    case FIN_ALPHA:
      S.pq = v;
      if (!(v > 0.0)) {
        S.flags |= isfinite(v) ? PCG_FLAG_BREAKDOWN : PCG_FLAG_NONFINITE;
        S.done = 1;
        S.alpha = 0.0;
      } else {
        S.alpha = S.rz[0] / v;
      }
      break;
    case FIN_RR:
    case FIN_RRF:
      if (op == FIN_RRF) S.rzo = w;
      S.rr = v;
      S.iters += 1;
      if (!isfinite(v)) {
        S.flags |= PCG_FLAG_NONFINITE;
        S.done = 1;
      } else if (v <= S.tol2 * S.bb) {
        S.done = 1;
      }
      break;
    case FIN_BETA:
    case FIN_BETAF:
      if (!(v > 0.0)) {
        S.flags |= isfinite(v) ? PCG_FLAG_BREAKDOWN : PCG_FLAG_NONFINITE;
        S.done = 1;
        break;
      }
      S.beta = (op == FIN_BETAF ? v - S.rzo : v) / S.rz[0];
      S.rz[0] = v;
      break;
  }
}

// ------------------------------------------------------------ host side
static unsigned bgrid(const Batch& B) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(B.view.num_tiles, (int64_t)num_sms() * 16));
}

static void b_finalize(Batch& B, int op, cudaStream_t s) {
  ++B.nlaunch;
  k_b_finalize<<<B.ngeo(), 256, 0, s>>>(B.part, B.geo_tile0, op, B.sc, (B.df && op != FIN_INIT) ? 1 : 0);
}

// z = M^-1 r for all geometries at once (block-diagonal V-cycle), then the
// per-tile dot partials for beta
static void b_precondition(Batch& B, const double* r, double* z, cudaStream_t s) {
  Solver& S = *B.S;
  const int64_t n0 = S.nlaunch;
  if (B.df) {  // r in DF, z in FP32
    VcycleDot in;
    in.r = r;
    in.df = true;
    amg_vcycle_grid(S, r, z, s, &in);
  } else {
    amg_vcycle_grid(S, r, z, s);
  }
  B.nlaunch += S.nlaunch - n0;
  ++B.nlaunch;
  if (B.df)
    k_b_dot_df<<<bgrid(B), BT, 0, s>>>(B.view.tv(), B.tile_geo, B.sc, r, reinterpret_cast<const float*>(z), B.part);
  else
    k_b_dot<<<bgrid(B), BT, 0, s>>>(B.view.tv(), B.tile_geo, B.sc, r, z, B.part);
}

static void b_xpby_apply(Batch& B, int first, cudaStream_t s) {
  Solver& S = *B.S;
  ++B.nlaunch;
  if (B.df)
    k_b_xpby_apply_df<<<bgrid(B), BT, 0, s>>>(B.view.tv(), B.tile_geo, B.sc, B.view.code, B.diag_df,
                                              reinterpret_cast<const float*>(S.z), S.p, S.q, first, B.part);
  else
    k_b_xpby_apply<<<bgrid(B), BT, 0, s>>>(B.view.tv(), B.tile_geo, B.sc, B.view.code, B.view.diag, S.z, S.p, S.q,
                                           first, B.part);
}

// One batched iteration: alpha from the p.q partials of the previous
// k_b_xpby_apply, the x/r update (with r.zold when flexible), r.r and the
// convergence test, the V-cycle and r.z, beta, then p and the next q.
static void b_iteration(Batch& B, double* x, bool flex, cudaStream_t s) {
  Solver& S = *B.S;
  const TileView tv = B.view.tv();
  const unsigned gb = bgrid(B);
  ++B.nlaunch;
  b_finalize(B, FIN_ALPHA, s);
  if (B.df)
    k_b_update_xr_df<<<gb, BT, 0, s>>>(tv, B.tile_geo, B.sc, x, S.r, S.p, S.q,
                                       flex ? reinterpret_cast<const float*>(S.z) : nullptr, B.part);
  else
    k_b_update_xr<<<gb, BT, 0, s>>>(tv, B.tile_geo, B.sc, x, S.r, S.p, S.q, flex ? S.z : nullptr, B.part);
  b_finalize(B, flex ? FIN_RRF : FIN_RR, s);
  b_precondition(B, S.r, S.z, s);
  b_finalize(B, flex ? FIN_BETAF : FIN_BETA, s);
  b_xpby_apply(B, 0, s);
}

static void b_graph_prepare(Batch& B, const double* b, double* x, bool flex, cudaStream_t s) {
  if (B.gexec && B.g_b == b && B.g_x == x && B.g_prof == (int)B.profile && B.g_df == (int)B.df) return;
  Solver& S = *B.S;
  if (B.gexec) cudaGraphExecDestroy(B.gexec);
  B.gexec = nullptr;
  if (!B.cap_stream) EB_CUDA(cudaStreamCreateWithFlags(&B.cap_stream, cudaStreamNonBlocking));
  cudaEvent_t fork;
  EB_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  EB_CUDA(cudaEventRecord(fork, s));
  EB_CUDA(cudaStreamWaitEvent(B.cap_stream, fork, 0));
  const int64_t n0 = B.nlaunch;
  // the graph records event pairs 0 .. g_pairs-1 around its level-0 smoother launches
  S.prof_on = B.profile;
  S.prof_n = 0;
  EB_CUDA(cudaStreamBeginCapture(B.cap_stream, cudaStreamCaptureModeThreadLocal));
  b_iteration(B, x, flex, B.cap_stream);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(B.cap_stream, &graph);
  S.prof_on = false;
  B.g_pairs = S.prof_n;
  B.g_prof = (int)B.profile;
  cudaEventDestroy(fork);
  EB_CUDA(e);
  e = cudaGraphInstantiate(&B.gexec, graph, 0);
  cudaGraphDestroy(graph);
  EB_CUDA(e);
  B.g_launches = B.nlaunch - n0;
  B.nlaunch = n0;
  B.g_b = b;
  B.g_x = x;
  B.g_df = (int)B.df;
}

// continue while some geometry is neither converged nor at its iteration limit
__global__ void k_b_loop_cond(cudaGraphConditionalHandle h, const PcgScalars* sc, int ng) {
  int active = 0;
  for (int g = threadIdx.x; g < ng; g += blockDim.x) active |= (!sc[g].done && sc[g].iters < sc[g].maxit) ? 1 : 0;
  active = __syncthreads_or(active);
  if (threadIdx.x == 0) cudaGraphSetConditional(h, active ? 1u : 0u);
}

static void b_loop_release(Batch& B) {
  if (B.lexec) cudaGraphExecDestroy(B.lexec);
  B.lexec = nullptr;
  B.l_b = nullptr;
  B.l_x = nullptr;
}

static void b_loop_prepare(Batch& B, const double* b, double* x, bool flex) {
  if (B.lexec && B.l_b == b && B.l_x == x && B.l_df == (int)B.df) return;
  b_loop_release(B);
  if (!B.cap_stream) EB_CUDA(cudaStreamCreateWithFlags(&B.cap_stream, cudaStreamNonBlocking));
  const int64_t n0 = B.nlaunch;
  B.lexec = build_while_graph(B.cap_stream, [&](cudaStream_t cs, cudaGraphConditionalHandle h) {
    b_iteration(B, x, flex, cs);
    k_b_loop_cond<<<1, 256, 0, cs>>>(h, B.sc, B.ngeo());
    ++B.nlaunch;
  });
  B.l_launches = B.nlaunch - n0;
  B.nlaunch = n0;
  B.l_b = b;
  B.l_x = x;
  B.l_df = (int)B.df;
}

static int batch_pcg(Batch& B, const double* b, double* x, double rtol, int maxit, pcg_stats* stats, cudaStream_t s) {
  Solver& S = *B.S;
  const int ng = B.ngeo();
  const TileView tv = B.view.tv();
  const unsigned gb = bgrid(B);
  const bool flex = S.opts.vcycle_prec != EB_F64;
  EB_REQUIRE(rtol > 0.0 && maxit >= 0, EB_ERR_INVALID, "batch: rtol must be > 0 and maxit >= 0");
  B.df = B.outer == EB_DF64;
  if (B.df) {
    EB_REQUIRE(flex && amg_levels(S) > 1, EB_ERR_NOT_IMPLEMENTED,
               "batch: the DF outer iteration needs an FP32 or BF16 V-cycle of at least two levels");
    if (!B.gscale) B.gscale = dalloc<double>(ng, s);
    if (!B.xdf) B.xdf = dalloc<double>(B.view.g.num_nodes, s);
    if (!B.diag_df) {
      B.diag_df = dalloc<float2>(B.view.g.num_nodes, s);
      ++B.nlaunch;
      k_b_df_diag<<<gb, BT, 0, s>>>(tv, B.view.code, B.view.diag, B.diag_df);
    }
  }
  // the vector the iteration updates: x itself, or its DF image
  double* xi = B.df ? B.xdf : x;
  EB_REQUIRE(xi != b, EB_ERR_INVALID, "batch: x and b share a buffer");
  std::vector<double> gsc(ng, 1.0);
  auto t0 = std::chrono::steady_clock::now();
  std::vector<PcgScalars> init(ng);
  for (auto& p : init) {
    p = PcgScalars{};
    p.tol2 = rtol * rtol;
  }
  std::vector<int> iters(ng, 0), flags(ng, 0), conv(ng, 0);
  std::vector<double> rel(ng, 0.0);
  B.nlaunch = 0;
  S.prof_on = false;
  S.prof_what = PROF_SMOOTHER;
  S.prof_acc_ms = 0.0;
  S.prof_acc_n = 0;
  for (int restart = 0; restart < 4; ++restart) {
    const int done_its = *std::max_element(iters.begin(), iters.end());
    for (auto& p : init) p.maxit = maxit - done_its;
    EB_CUDA(cudaMemcpyAsync(B.sc, init.data(), sizeof(PcgScalars) * ng, cudaMemcpyHostToDevice, s));
    B.nlaunch += 2;
    k_b_mask<<<gb, BT, 0, s>>>(tv, B.view.code, x, x);
    k_b_resid<<<gb, BT, 0, s>>>(tv, B.view.code, B.view.diag, b, x, S.r, B.part);
    b_finalize(B, FIN_INIT, s);
    int its = *std::max_element(iters.begin(), iters.end());
    if (its < maxit && B.df) {
      // per geometry a power of two that gives its b a unit root mean square
      EB_CUDA(cudaMemcpyAsync(B.sc_host, B.sc, sizeof(PcgScalars) * ng, cudaMemcpyDeviceToHost, s));
      EB_CUDA(cudaStreamSynchronize(s));
      for (int g = 0; g < ng; ++g) {
        const double ncp = (double)std::max<int64_t>(B.cp_off[g + 1] - B.cp_off[g], 1);
        const double ms = B.sc_host[g].bb / ncp;
        gsc[g] = (ms > 0.0 && std::isfinite(ms)) ? std::ldexp(1.0, -(int)std::lround(0.5 * std::log2(ms))) : 1.0;
        B.sc_host[g].bb *= gsc[g] * gsc[g];
        B.sc_host[g].rr *= gsc[g] * gsc[g];
      }
      EB_CUDA(cudaMemcpyAsync(B.sc, B.sc_host, sizeof(PcgScalars) * ng, cudaMemcpyHostToDevice, s));
      EB_CUDA(cudaMemcpyAsync(B.gscale, gsc.data(), sizeof(double) * ng, cudaMemcpyHostToDevice, s));
      ++B.nlaunch;
      k_b_df_in<<<gb, BT, 0, s>>>(tv, B.tile_geo, B.gscale, x, xi, S.r);
    }
    if (its < maxit) {
      b_precondition(B, S.r, S.z, s);
      b_finalize(B, FIN_RZ0, s);
      b_xpby_apply(B, 1, s);
      int it = 0;
      if (!B.profile) {  // the whole loop on the device
        b_loop_prepare(B, b, xi, flex);
        EB_CUDA(cudaGraphLaunch(B.lexec, s));
        EB_CUDA(cudaMemcpyAsync(B.sc_host, B.sc, sizeof(PcgScalars) * ng, cudaMemcpyDeviceToHost, s));
        EB_CUDA(cudaStreamSynchronize(s));
        int most = 0;
        for (int g = 0; g < ng; ++g) most = std::max(most, B.sc_host[g].iters);
        B.nlaunch += B.l_launches * most;
        it = maxit;  // skip the host loop below
      }
      while (true) {
        if (its + it >= maxit) break;
        b_graph_prepare(B, b, xi, flex, s);
        EB_CUDA(cudaGraphLaunch(B.gexec, s));
        B.nlaunch += B.g_launches;
        ++it;
        EB_CUDA(cudaMemcpyAsync(B.sc_host, B.sc, sizeof(PcgScalars) * ng, cudaMemcpyDeviceToHost, s));
        EB_CUDA(cudaStreamSynchronize(s));
        if (B.profile) S.prof_collect(0, B.g_pairs);
        bool all = true;
        for (int g = 0; g < ng; ++g) all = all && B.sc_host[g].done;
        if (all) break;
      }
    }
    EB_CUDA(cudaMemcpyAsync(B.sc_host, B.sc, sizeof(PcgScalars) * ng, cudaMemcpyDeviceToHost, s));
    EB_CUDA(cudaStreamSynchronize(s));
    bool hard = false;
    for (int g = 0; g < ng; ++g) {
      iters[g] += B.sc_host[g].iters;
      flags[g] |= B.sc_host[g].flags;
      hard = hard || (flags[g] & (PCG_FLAG_NONFINITE | PCG_FLAG_BREAKDOWN));
    }
    if (B.df && its < maxit) {
      ++B.nlaunch;
      k_b_df_out<<<gb, BT, 0, s>>>(tv, B.tile_geo, B.gscale, xi, x);
    }
    // true residuals at exit (FP64)
    B.nlaunch += 1;
    k_b_resid<<<gb, BT, 0, s>>>(tv, B.view.code, B.view.diag, b, x, S.r, B.part);
    b_finalize(B, FIN_INIT, s);
    EB_CUDA(cudaMemcpyAsync(B.sc_host, B.sc, sizeof(PcgScalars) * ng, cudaMemcpyDeviceToHost, s));
    EB_CUDA(cudaStreamSynchronize(s));
    bool all = true;
    for (int g = 0; g < ng; ++g) {
      const PcgScalars& p = B.sc_host[g];
      rel[g] = p.bb > 0 ? std::sqrt(p.rr / p.bb) : 0.0;
      conv[g] = p.bb == 0.0 || p.rr <= p.tol2 * p.bb;
      all = all && conv[g];
    }
    if (all || hard || *std::max_element(iters.begin(), iters.end()) >= maxit) break;
  }
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  int worst = EB_OK;
  if (S.dev_err) {  // a bounded wait of a tensor-copy smoothing step gave up
    int e = 0;
    EB_CUDA(cudaMemcpyAsync(&e, S.dev_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    EB_CUDA(cudaStreamSynchronize(s));
    if (e) {
      EB_CUDA(cudaMemsetAsync(S.dev_err, 0, sizeof(int), s));
      set_error("batch_heat_step: a tensor-copy wait of the level-0 smoother gave up");
      return EB_ERR_TIMEOUT;
    }
  }
  for (int g = 0; g < ng; ++g) {
    if (stats) {
      stats[g] = pcg_stats{};
      stats[g].iterations = iters[g];
      stats[g].rel_residual = rel[g];
      stats[g].true_rel_residual = rel[g];
      stats[g].solve_ms = ms;
      stats[g].converged = conv[g];
      stats[g].launches = B.nlaunch;
      stats[g].prof_kernel_ms = S.prof_acc_ms;
      stats[g].prof_launches = S.prof_acc_n;
    }
    if (flags[g] & PCG_FLAG_NONFINITE) worst = EB_ERR_NONFINITE;
    else if ((flags[g] & PCG_FLAG_BREAKDOWN) && worst == EB_OK) worst = EB_ERR_BREAKDOWN;
    else if (!conv[g] && worst == EB_OK) worst = EB_ERR_NO_CONVERGENCE;
  }
  if (worst != EB_OK) set_error("batch_heat_step: a geometry did not converge (see its statistics)");
  return worst;
}

}  // namespace ebk

struct batch_handle {
  ebk::Batch b;
};

using namespace ebk;

extern "C" {

int batch_build(const eb_grid* grids, const eb_levelset* lss, int count, batch_handle** out, cudaStream_t stream) {
  if (!grids || !lss || !out || count < 1) {
    set_error("batch_build: invalid argument");
    return EB_ERR_INVALID;
  }
  *out = nullptr;
  batch_handle* h = new (std::nothrow) batch_handle();
  if (!h) {
    set_error("batch_build: host allocation failed");
    return EB_ERR_OOM;
  }
  int st = guarded([&] { build_batch(h->b, grids, lss, count, stream); });
  if (st != EB_OK) {
    destroy_batch(h->b);
    delete h;
    return st;
  }
  *out = h;
  return EB_OK;
}

void batch_destroy(batch_handle* b) {
  if (!b) return;
  destroy_batch(b->b);
  delete b;
}

int batch_info(const batch_handle* b, batch_info_t* out) {
  if (!b || !out) {
    set_error("batch_info: NULL argument");
    return EB_ERR_INVALID;
  }
  const Batch& B = b->b;
  out->count = B.ngeo();
  out->stride = B.stride;
  out->num_nodes = B.view.g.num_nodes;
  out->num_cp = B.view.num_cp;
  out->num_cut = B.view.num_cut;
  out->num_tiles = B.view.num_tiles;
  return EB_OK;
}

int batch_offsets(const batch_handle* b, int64_t* node_off, int64_t* cut_off, int64_t* cp_off) {
  if (!b) {
    set_error("batch_offsets: NULL handle");
    return EB_ERR_INVALID;
  }
  const Batch& B = b->b;
  for (int g = 0; g <= B.ngeo(); ++g) {
    if (node_off) node_off[g] = B.node_off[g];
    if (cut_off) cut_off[g] = B.cut_off[g];
    if (cp_off) cp_off[g] = B.cp_off[g];
  }
  return EB_OK;
}

const eb_handle* batch_geometry(const batch_handle* b, int g) {
  if (!b || g < 0 || g >= b->b.ngeo()) {
    set_error("batch_geometry: index out of range");
    return nullptr;
  }
  return b->b.geo[g];
}

int batch_rhs(const batch_handle* b, const double* f_all, const double* ug_all, double* b_all, cudaStream_t stream) {
  if (!b || !f_all || !b_all || (!ug_all && b->b.view.num_cut > 0)) {
    set_error("batch_rhs: NULL argument");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    const Batch& B = b->b;
    k_b_rhs<<<bgrid(B), BT, 0, stream>>>(B.view.tv(), B.tile_geo, B.gconst, B.view.code, B.view.cp_of_node,
                                         B.cut_off_cp, B.cut_c, f_all, ug_all, b_all);
    EB_CUDA(cudaGetLastError());
  });
}

// out[g] = sum over geometry g's nodes of w u (one CTA per geometry, a fixed
// summation order: deterministic)
__global__ void __launch_bounds__(256) k_b_wsum(const int64_t* node_off, const int32_t* n0, const int32_t* n1,
                                                int64_t stride, const double* w, const double* u, double* out) {
  __shared__ double sm[32];
  const int g = blockIdx.x;
  const int64_t base = node_off[g];
  const int64_t nx = n0[g], cnt = nx * n1[g];
  double acc = 0.0;
  for (int64_t k = threadIdx.x; k < cnt; k += blockDim.x) {
    const int64_t node = base + (k / nx) * stride + (k % nx);
    acc += w[node] * u[node];
  }
  const double t = block_sum(acc, sm);
  if (threadIdx.x == 0) out[g] = t;
}

int batch_weighted_sum(const batch_handle* b, const double* w_all, const double* u_all, double* out_dev,
                       cudaStream_t stream) {
  if (!b || !w_all || !u_all || !out_dev) {
    set_error("batch_weighted_sum: NULL argument");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    const Batch& B = b->b;
    const int ng = B.ngeo();
    std::vector<int32_t> nx(ng), ny(ng);
    for (int g = 0; g < ng; ++g) {
      nx[g] = B.geo[g]->h.g.n0;
      ny[g] = B.geo[g]->h.g.n1;
    }
    int64_t* off = dalloc<int64_t>(ng, stream, false);
    int32_t* d0 = dalloc<int32_t>(ng, stream, false);
    int32_t* d1 = dalloc<int32_t>(ng, stream, false);
    EB_CUDA(cudaMemcpyAsync(off, B.node_off.data(), sizeof(int64_t) * ng, cudaMemcpyHostToDevice, stream));
    EB_CUDA(cudaMemcpyAsync(d0, nx.data(), sizeof(int32_t) * ng, cudaMemcpyHostToDevice, stream));
    EB_CUDA(cudaMemcpyAsync(d1, ny.data(), sizeof(int32_t) * ng, cudaMemcpyHostToDevice, stream));
    k_b_wsum<<<ng, 256, 0, stream>>>(off, d0, d1, B.stride, w_all, u_all, out_dev);
    const cudaError_t e = cudaGetLastError();
    EB_CUDA(cudaStreamSynchronize(stream));
    dfree(off, stream);
    dfree(d0, stream);
    dfree(d1, stream);
    EB_CUDA(e);
  });
}

int batch_heat_setup(batch_handle* b, const double* dt, double theta, const amg_opts* opts, cudaStream_t stream) {
  if (!b || !dt || !(theta > 0.0 && theta <= 1.0)) {
    set_error("batch_heat_setup: invalid argument");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    Batch& B = b->b;
    const int ng = B.ngeo();
    B.hconst.resize(ng);
    for (int g = 0; g < ng; ++g) {
      EB_REQUIRE(dt[g] > 0.0 && (std::isfinite(dt[g]) || (std::isinf(dt[g]) && theta == 1.0)), EB_ERR_INVALID,
                 "batch_heat_setup: dt must be > 0 (+infinity only with theta = 1)");
      const double h = B.geo[g]->h.g.h;
      B.hconst[g] = GeoConst{h * h, dt[g], theta};
    }
    EB_CUDA(cudaMemcpyAsync(B.gconst, B.hconst.data(), sizeof(GeoConst) * ng, cudaMemcpyHostToDevice, stream));
    k_tile_shift<<<blocks_for(B.view.num_tiles, 256), 256, 0, stream>>>(B.view.num_tiles, B.tile_geo, B.gconst,
                                                                        B.view.tile_shift64, B.view.tile_shift32);
    if (B.S) {
      amg_free(*B.S);
      B.S->free_work();
      B.S->prof_release();
      delete B.S;
      B.S = nullptr;
    }
    if (B.gexec) cudaGraphExecDestroy(B.gexec);
    B.gexec = nullptr;
    b_loop_release(B);
    amg_opts o{25, 1024, 0.02, 2, EB_F64, EB_AMG_SA, 1};
    if (opts) o = *opts;
    EB_REQUIRE(o.max_levels >= 1 && o.max_levels <= 32, EB_ERR_INVALID, "batch_heat_setup: max_levels in [1, 32]");
    EB_REQUIRE(o.vcycle_prec == EB_F64 || o.vcycle_prec == EB_F32 || o.vcycle_prec == EB_BF16, EB_ERR_INVALID,
               "batch_heat_setup: vcycle_prec must be EB_F64, EB_F32 or EB_BF16");
    EB_REQUIRE((o.coarsening == EB_AMG_SA || o.coarsening == EB_AMG_RS) && (o.cycle == 1 || o.cycle == 2),
               EB_ERR_INVALID, "batch_heat_setup: coarsening EB_AMG_SA / EB_AMG_RS, cycle 1 or 2");
    B.S = new Solver();
    Solver& S = *B.S;
    S.eb = &B.view;
    S.l0_tma = B.l0_tma;
    S.home = stream;
    S.shift = 0.0;  // per-tile shifts of the view take over
    S.opts = o;
    S.alloc_work(stream);
    // block-diagonal level-0 matrix of the scaled operators, geometry by geometry
    std::vector<DCsr> parts(ng);
    int64_t nnz = 0;
    for (int g = 0; g < ng; ++g) {
      EBHandle unit = B.geo[g]->h;  // shallow copy with unit spacing: off-diagonals -1, diagonal D + sigma'
      unit.g.h = 1.0;
      parts[g] = level0_csr(unit, B.hconst[g].h2 / (theta * dt[g]), stream);
      nnz += parts[g].nnz;
    }
    DCsr A0;
    A0.n = A0.m = B.view.num_cp;
    A0.nnz = nnz;
    A0.rp = dalloc<int32_t>(A0.n + 1, stream, false);
    A0.ci = dalloc<int32_t>(nnz, stream, false);
    A0.v = dalloc<double>(nnz, stream, false);
    int64_t e0 = 0;
    for (int g = 0; g < ng; ++g) {
      DCsr& P = parts[g];
      k_add_i32<<<blocks_for(P.n, 256), 256, 0, stream>>>(P.n, P.rp, (int32_t)e0, A0.rp + B.cp_off[g]);
      k_add_i32<<<blocks_for(P.nnz, 256), 256, 0, stream>>>(P.nnz, P.ci, (int32_t)B.cp_off[g], A0.ci + e0);
      EB_CUDA(cudaMemcpyAsync(A0.v + e0, P.v, 8 * P.nnz, cudaMemcpyDeviceToDevice, stream));
      e0 += P.nnz;
    }
    const int32_t nnz32 = (int32_t)nnz;
    EB_CUDA(cudaMemcpyAsync(A0.rp + A0.n, &nnz32, 4, cudaMemcpyHostToDevice, stream));
    EB_CUDA(cudaStreamSynchronize(stream));
    for (DCsr& P : parts) csr_free(P, stream);
    auto t0 = std::chrono::steady_clock::now();
    amg_build_from(S, A0, stream);
    EB_CUDA(cudaStreamSynchronize(stream));
    S.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  });
}

int batch_autotune(batch_handle* b, int reps, eb_tune_t* out, cudaStream_t stream) {
  if (!b) {
    set_error("batch_autotune: NULL handle");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    Batch& B = b->b;
    EB_REQUIRE(B.S != nullptr, EB_ERR_INVALID, "batch_autotune: call batch_heat_setup first");
    const int64_t nn = B.view.g.num_nodes;
    double* r = dalloc<double>(nn, stream);
    double* z = nullptr;
    try {
      z = dalloc<double>(nn, stream);
      auto retile = [&](const TileDims& t) {
        for (eb_handle* e : B.geo) build_tiles(e->h, t.x, t.y, t.z, stream);
        batch_tiles(B, stream);
      };
      run_tuner(2, retile, [&] { amg_vcycle_grid(*B.S, r, z, stream); }, reps, out, stream);
    } catch (...) {
      dfree(r, stream);
      dfree(z, stream);
      throw;
    }
    dfree(r, stream);
    dfree(z, stream);
    EB_CUDA(cudaStreamSynchronize(stream));
  });
}

int batch_set_profile(batch_handle* b, int on) {
  if (!b) {
    set_error("batch_set_profile: NULL handle");
    return EB_ERR_INVALID;
  }
  b->b.profile = on != 0;
  return EB_OK;
}

int batch_set_level0_tma(batch_handle* b, int on) {
  if (!b) {
    set_error("batch_set_level0_tma: NULL handle");
    return EB_ERR_INVALID;
  }
  b->b.l0_tma = on != 0;
  if (b->b.S) b->b.S->l0_tma = b->b.l0_tma;
  return EB_OK;
}

int batch_set_outer_prec(batch_handle* b, int prec) {
  if (!b || (prec != EB_F64 && prec != EB_DF64)) {
    set_error("batch_set_outer_prec: NULL handle or precision other than EB_F64 / EB_DF64");
    return EB_ERR_INVALID;
  }
  b->b.outer = prec;
  return EB_OK;
}

int batch_heat_step(batch_handle* b, const double* b1_all, const double* b0_all, double* u_all, double rtol,
                    int maxit, pcg_stats* stats, cudaStream_t stream) {
  if (!b || !b1_all || !u_all) {
    set_error("batch_heat_step: NULL argument");
    return EB_ERR_INVALID;
  }
  int rc = EB_OK;
  int st = guarded([&] {
    Batch& B = b->b;
    EB_REQUIRE(B.S != nullptr, EB_ERR_INVALID, "batch_heat_step: call batch_heat_setup first");
    const double theta = B.hconst[0].theta;
    EB_REQUIRE(theta == 1.0 || b0_all != nullptr, EB_ERR_INVALID, "batch_heat_step: b0 required when theta < 1");
    Solver& S = *B.S;
    k_b_heat_rhs<<<bgrid(B), BT, 0, stream>>>(B.view.tv(), B.tile_geo, B.gconst, B.view.code, B.view.diag, u_all,
                                              b1_all, b0_all ? b0_all : b1_all, S.tmp);
    EB_CUDA(cudaGetLastError());
    rc = batch_pcg(B, S.tmp, u_all, rtol, maxit, stats, stream);
  });
  return st != EB_OK ? st : rc;
}

}  // extern "C"
