// Preconditioned MINRES on the EB operator: (sigma I + A) x = b for any real
// sigma, in particular the indefinite Helmholtz operator omega^2 u + Lap u of
// Sec. 3.3.2 (sigma = -omega^2, A = -L), which the paper solves by MINRES.
//
// The Lanczos process runs in the inner product of an SPD preconditioner M
// (the hierarchy's V-cycle, a Jacobi sweep, or none) and the tridiagonal
// system is reduced by Givens rotations (Paige & Saunders 1975, in the
// three-term form of Elman, Silvester & Wathen, ch. 6).  One iteration:
//   k_mr_apply   zs = z / gamma_j, Az = (sigma I + A) zs, partials of zs'Az
//   k_mr_lanczos delta = zs'Az; v_{j+1} = Az - (delta/gamma_j) v_j
//                - (gamma_j/gamma_{j-1}) v_{j-1} (v_{j-1} <- v_j in place)
//   z = M v_{j+1} with the partials of v'z (the V-cycle's last smoothing
//                launch forms them)
//   k_mr_update  gamma_{j+1} = sqrt(v'z), the rotation, w_{j+1} = (zs -
//                a3 w_{j-1} - a2 w_j) / a1 (in place), x += c eta w_{j+1},
//                eta = -s eta; CTA 0 records the scalars, tests |eta| <= rtol
//                gamma_1 and sets the loop condition.
// Every reduction is deterministic: each CTA reduces its pairs to one partial
// and every consumer sums the partials in the same order.  The loop runs on
// the device (a conditional WHILE node around one captured iteration).
#include "eb_solver.cuh"
#include "stencil.cuh"

#include <chrono>
#include <cmath>

namespace ebk {

// The rotation state of the current iteration lives in st[iters & 1]: the
// update launch reads st[slot] (slot = iters & 1, recorded by the launch
// before it) and CTA 0 writes the next state to st[slot ^ 1] and advances
// iters, so no CTA of a launch sees a state another CTA of it is rewriting.
struct MrRot {
  double gamma, gamma_prev, c_prev, c, s_prev, s, eta;
  int done;
};
struct MrScalars {
  MrRot st[2];
  double gamma1, delta, tol, bb;
  int iters, slot, maxit, flags;
};
enum { MR_FLAG_NONFINITE = 1, MR_FLAG_BREAKDOWN = 2 };

struct MrOp {
  double inv_h2, sigma;
};

// v = b - (sigma I + A) x over the CP pairs (x masked to the CPs first by the
// caller's contract: its non-CP entries are never read at a CP); v_prev = w =
// w_prev = 0; partials of b'b
template <int DIM>
__global__ void __launch_bounds__(TILE_NODES) k_mr_init(TileView tv, PairList pl, const uint8_t* code,
                                                        const double* diag, MrOp o, const double* b, const double* x,
                                                        double* v, double* v_prev, double* w, double* w_prev,
                                                        double* part) {
  __shared__ double sm[32];
  double sbb = 0.0;
  EB_LIST_LOOP(pl, node) {
    uint32_t c0, c1;
    ld_codes(code, node, c0, c1);
    Two<double> xc, core;
    stencil_tv<DIM, LdRO>(tv, x, node, c0, c1, diag, xc, core);
    const Two<double> bv = LdRO::ld2(b + node);
    const double b0 = (c0 & CODE_CP) ? bv.x : 0.0, b1 = (c1 & CODE_CP) ? bv.y : 0.0;
    const double r0 = (c0 & CODE_CP) ? b0 - (core.x * o.inv_h2 + o.sigma * xc.x) : 0.0;
    const double r1 = (c1 & CODE_CP) ? b1 - (core.y * o.inv_h2 + o.sigma * xc.y) : 0.0;
    st2(v + node, r0, r1);
    st2(v_prev + node, 0.0, 0.0);
    st2(w + node, 0.0, 0.0);
    st2(w_prev + node, 0.0, 0.0);
    sbb += b0 * b0 + b1 * b1;
  }
  const double t = block_sum(sbb, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// gamma_1 = sqrt(v'z) from the preconditioner's partials; the rotation state
// and eta = gamma_1 (one CTA)
__global__ void k_mr_start(MrScalars* sc, const double* bb_part, int nbb, const double* vz_part, int nvz, double rtol,
                           int maxit) {
  __shared__ double sm[32];
  const double bb = sum_parts(bb_part, nbb, 1, sm);
  __syncthreads();
  const double vz = sum_parts(vz_part, nvz, 1, sm);
  if (threadIdx.x == 0) {
    MrScalars m{};
    MrRot& r = m.st[0];
    m.bb = bb;
    m.tol = rtol;
    m.maxit = maxit;
    r.gamma_prev = 1.0;
    r.c_prev = r.c = 1.0;
    r.s_prev = r.s = 0.0;
    if (!(vz >= 0.0) || !isfinite(vz)) {
      m.flags = isfinite(vz) ? MR_FLAG_BREAKDOWN : MR_FLAG_NONFINITE;
      r.done = 1;
    } else {
      r.gamma = sqrt(vz);
      m.gamma1 = r.gamma;
      r.eta = r.gamma;
      r.done = (r.gamma == 0.0 || maxit <= 0) ? 1 : 0;
    }
    m.st[1] = r;
    *sc = m;
  }
}

// the rotation state st[idx] as thread 0 of the CTA reads it, for all threads
// (idx = -1: the current state st[iters & 1])
__device__ __forceinline__ MrRot mr_view(const MrScalars* sc, int idx) {
  __shared__ MrRot v;
  if (threadIdx.x == 0) {
    const volatile MrScalars* p = sc;
    const int k = idx < 0 ? (p->iters & 1) : idx;
    v.gamma = p->st[k].gamma;
    v.gamma_prev = p->st[k].gamma_prev;
    v.c_prev = p->st[k].c_prev;
    v.c = p->st[k].c;
    v.s_prev = p->st[k].s_prev;
    v.s = p->st[k].s;
    v.eta = p->st[k].eta;
    v.done = p->st[k].done;
  }
  __syncthreads();
  return v;
}

template <int DIM>
__global__ void __launch_bounds__(TILE_NODES) k_mr_apply(TileView tv, PairList pl, const uint8_t* code,
                                                         const double* diag, MrOp o, const MrScalars* sc,
                                                         const double* z, double* zs, double* az, double* part) {
  __shared__ double sm[32];
  const MrRot m = mr_view(sc, -1);
  if (m.done) {
    if (threadIdx.x == 0) part[blockIdx.x] = 0.0;
    return;
  }
  const double ig = 1.0 / m.gamma;
  double sd = 0.0;
  EB_LIST_LOOP(pl, node) {
    uint32_t c0, c1;
    ld_codes(code, node, c0, c1);
    Two<double> zc, core;
    stencil_tv<DIM, LdRO>(tv, z, node, c0, c1, diag, zc, core);
    const double s0 = (c0 & CODE_CP) ? zc.x * ig : 0.0, s1 = (c1 & CODE_CP) ? zc.y * ig : 0.0;
    const double a0 = (c0 & CODE_CP) ? (core.x * o.inv_h2 + o.sigma * zc.x) * ig : 0.0;
    const double a1 = (c1 & CODE_CP) ? (core.y * o.inv_h2 + o.sigma * zc.y) * ig : 0.0;
    st2(zs + node, s0, s1);
    st2(az + node, a0, a1);
    sd += s0 * a0 + s1 * a1;
  }
  const double t = block_sum(sd, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void __launch_bounds__(TILE_NODES) k_mr_lanczos(PairList pl, MrScalars* sc, const double* d_part, int nd,
                                                           const double* az, double* v, double* v_prev) {
  __shared__ double sm[32];
  __shared__ double s_delta;
  const MrRot m = mr_view(sc, -1);
  if (m.done) return;
  const double delta = sum_parts(d_part, nd, 1, sm);
  if (threadIdx.x == 0) {
    s_delta = delta;
    if (blockIdx.x == 0) {
      sc->delta = delta;
      sc->slot = sc->iters & 1;
    }
  }
  __syncthreads();
  const double a = s_delta / m.gamma, b = m.gamma / m.gamma_prev;
  EB_LIST_LOOP(pl, node) {
    const Two<double> av = LdRO::ld2(az + node), vv = ld2d(v + node), vp = ld2d(v_prev + node);
    st2(v_prev + node, vv.x, vv.y);
    st2(v + node, av.x - a * vv.x - b * vp.x, av.y - a * vv.y - b * vp.y);
  }
}

// the rotation of the new column (every CTA, same order), then the w and x
// updates; CTA 0 records the scalars, runs the test and sets the condition
template <bool COND>
__global__ void __launch_bounds__(TILE_NODES) k_mr_update(PairList pl, MrScalars* sc, const double* vz_part, int nvz,
                                                          const double* zs, double* w, double* w_prev, double* x,
                                                          cudaGraphConditionalHandle h) {
  __shared__ double sm[32];
  __shared__ double s_k[4];  // a2, a3, 1 / a1, c_{j+1} eta
  __shared__ int s_slot;
  if (threadIdx.x == 0) s_slot = *(volatile const int*)&sc->slot;  // written by the launch before
  __syncthreads();
  const int slot = s_slot;
  const MrRot m = mr_view(sc, slot);
  if (m.done) {
    if (COND && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
    return;
  }
  const double vz = sum_parts(vz_part, nvz, 1, sm);
  if (threadIdx.x == 0) {
    const double delta = sc->delta;  // written by the launch before
    const bool ok = vz >= 0.0 && isfinite(vz);
    const double gn = ok ? sqrt(vz) : 0.0;
    const double a0 = m.c * delta - m.c_prev * m.s * m.gamma;
    const double a1 = sqrt(a0 * a0 + gn * gn);
    const double a2 = m.s * delta + m.c_prev * m.c * m.gamma;
    const double a3 = m.s_prev * m.gamma;
    const bool fine = ok && a1 > 0.0 && isfinite(a1);
    const double cn = fine ? a0 / a1 : 0.0, sn = fine ? gn / a1 : 0.0;
    s_k[0] = a2;
    s_k[1] = a3;
    s_k[2] = fine ? 1.0 / a1 : 0.0;
    s_k[3] = cn * m.eta;
    if (blockIdx.x == 0) {
      MrRot& nx = sc->st[slot ^ 1];
      nx.gamma_prev = m.gamma;
      nx.gamma = gn;
      nx.c_prev = m.c;
      nx.c = cn;
      nx.s_prev = m.s;
      nx.s = sn;
      nx.eta = -sn * m.eta;
      nx.done = 0;
      if (!fine) {
        sc->flags |= isfinite(vz) && isfinite(a1) ? MR_FLAG_BREAKDOWN : MR_FLAG_NONFINITE;
        nx.done = 1;
      } else if (fabs(nx.eta) <= sc->tol * sc->gamma1 || gn == 0.0) {
        nx.done = 1;
      }
      sc->iters += 1;
      if (COND) cudaGraphSetConditional(h, (!nx.done && sc->iters < sc->maxit) ? 1u : 0u);
    }
  }
  __syncthreads();
  const double a2 = s_k[0], a3 = s_k[1], ia1 = s_k[2], ce = s_k[3];
  EB_LIST_LOOP(pl, node) {
    const Two<double> zv = LdRO::ld2(zs + node), wv = ld2d(w + node), wp = ld2d(w_prev + node),
                      xv = ld2d(x + node);
    const double n0 = (zv.x - a3 * wp.x - a2 * wv.x) * ia1, n1 = (zv.y - a3 * wp.y - a2 * wv.y) * ia1;
    st2(w_prev + node, wv.x, wv.y);
    st2(w + node, n0, n1);
    st2(x + node, xv.x + ce * n0, xv.y + ce * n1);
  }
}

// partials of a'b over the CP pairs
__global__ void __launch_bounds__(TILE_NODES) k_mr_dot(PairList pl, const double* a, const double* b, double* part) {
  __shared__ double sm[32];
  double s = 0.0;
  EB_LIST_LOOP(pl, node) {
    const Two<double> av = LdRO::ld2(a + node), bv = LdRO::ld2(b + node);
    s += av.x * bv.x + av.y * bv.y;
  }
  const double t = block_sum(s, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// z = D^-1 v (Jacobi with the diagonal of sigma_m I + A, sigma_m the
// hierarchy's shift) or z = v (none)
__global__ void __launch_bounds__(TILE_NODES) k_mr_diag(PairList pl, const uint8_t* code, const double* diag,
                                                        double inv_h2, double sigma_m, double dim2, bool jacobi,
                                                        const double* v, double* z) {
  EB_LIST_LOOP(pl, node) {
    uint32_t c0, c1;
    ld_codes(code, node, c0, c1);
    const Two<double> vv = LdRO::ld2(v + node);
    double d0 = 1.0, d1 = 1.0;
    if (jacobi) {
      d0 = 1.0 / (sigma_m + ((c0 & 0x7F) ? diag[node] : dim2) * inv_h2);
      d1 = 1.0 / (sigma_m + ((c1 & 0x7F) ? diag[node + 1] : dim2) * inv_h2);
    }
    st2(z + node, (c0 & CODE_CP) ? d0 * vv.x : 0.0, (c1 & CODE_CP) ? d1 * vv.y : 0.0);
  }
}

// ||b - (sigma I + A) x||^2 partials (true residual at exit)
template <int DIM>
__global__ void __launch_bounds__(TILE_NODES) k_mr_resid(TileView tv, PairList pl, const uint8_t* code,
                                                         const double* diag, MrOp o, const double* b, const double* x,
                                                         double* part) {
  __shared__ double sm[32];
  double srr = 0.0;
  EB_LIST_LOOP(pl, node) {
    uint32_t c0, c1;
    ld_codes(code, node, c0, c1);
    Two<double> xc, core;
    stencil_tv<DIM, LdRO>(tv, x, node, c0, c1, diag, xc, core);
    const Two<double> bv = LdRO::ld2(b + node);
    const double r0 = (c0 & CODE_CP) ? bv.x - (core.x * o.inv_h2 + o.sigma * xc.x) : 0.0;
    const double r1 = (c1 & CODE_CP) ? bv.y - (core.y * o.inv_h2 + o.sigma * xc.y) : 0.0;
    srr += r0 * r0 + r1 * r1;
  }
  const double t = block_sum(srr, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_mr_sum(const double* part, int n, double* out) {
  __shared__ double sm[32];
  const double v = sum_parts(part, n, 1, sm);
  if (threadIdx.x == 0) *out = v;
}

// 0 at the non-CP nodes of the active tiles (the output contract)
template <int DIM>
__global__ void __launch_bounds__(TILE_NODES) k_mr_mask(TileView tv, const uint8_t* code, double* x) {
  EB_PAIR_LOOP(DIM, tv, node) {
    uint32_t c0, c1;
    ld_codes(code, node, c0, c1);
    const Two<double> v = ld2d(x + node);
    st2(x + node, (c0 & CODE_CP) ? v.x : 0.0, (c1 & CODE_CP) ? v.y : 0.0);
  }
}

struct MinresState {
  MrScalars* sc = nullptr;
  MrScalars* host = nullptr;
  double *v = nullptr, *v_prev = nullptr, *zs = nullptr, *az = nullptr, *w = nullptr, *w_prev = nullptr;
  double* part = nullptr;  // [3 * nblk + rz_cap]: apply, b'b / residual, v'z
  double* scal = nullptr;
};

int minres(Solver& S, double sigma, int precond, const double* b, double* x, double rtol, int maxit,
           pcg_stats* stats, cudaStream_t s) {
  const EBHandle& eb = *S.eb;
  const Geometry& G = eb.g;
  EB_REQUIRE(precond == EB_PC_AMG || precond == EB_PC_JACOBI || precond == EB_PC_NONE, EB_ERR_INVALID,
             "minres_solve: precond must be EB_PC_AMG, EB_PC_JACOBI or EB_PC_NONE");
  EB_REQUIRE(precond != EB_PC_AMG || S.H != nullptr, EB_ERR_INVALID, "minres_solve: the handle has no hierarchy");
  EB_REQUIRE(rtol > 0.0 && maxit >= 0 && b != x, EB_ERR_INVALID, "minres_solve: rtol > 0, maxit >= 0, b != x");
  EB_REQUIRE(std::isfinite(sigma), EB_ERR_INVALID, "minres_solve: sigma must be finite");
  const int64_t nn = G.num_nodes;
  const int nblk = S.nblk;
  const TileView tv = eb.tv();
  const PairList pl = eb.pairs();
  const MrOp op{1.0 / (G.h * G.h), sigma};
  MinresState M;
  auto release = [&] {
    dfree(M.sc, s); dfree(M.v, s); dfree(M.v_prev, s); dfree(M.zs, s); dfree(M.az, s); dfree(M.w, s);
    dfree(M.w_prev, s); dfree(M.part, s); dfree(M.scal, s);
    if (M.host) cudaFreeHost(M.host);
    M.host = nullptr;
  };
  int rc = EB_OK;
  auto t0 = std::chrono::steady_clock::now();
  cudaGraphExec_t exec = nullptr;
  try {
    M.sc = dalloc<MrScalars>(1, s);
    M.v = dalloc<double>(nn, s);
    M.v_prev = dalloc<double>(nn, s);
    M.zs = dalloc<double>(nn, s);
    M.az = dalloc<double>(nn, s);
    M.w = dalloc<double>(nn, s);
    M.w_prev = dalloc<double>(nn, s);
    M.part = dalloc<double>(3 * (int64_t)nblk + S.rz_cap, s);
    M.scal = dalloc<double>(2, s);
    EB_CUDA(cudaMallocHost((void**)&M.host, sizeof(MrScalars)));
    double* p_apply = M.part;
    double* p_bb = M.part + nblk;
    double* p_vz = M.part + 2 * (int64_t)nblk;
    double* z = S.z;  // the preconditioned vector (unscaled z_j)
    int64_t nl = 0;
    // z = M v with the v'z partials; returns their count
    auto precondition = [&](cudaStream_t st) -> int {
      if (precond == EB_PC_AMG) {
        VcycleDot dot;
        dot.r = M.v;
        dot.part = p_vz;
        const int fused = amg_vcycle_grid(S, M.v, z, st, &dot);
        if (fused) return fused;
      } else {
        k_mr_diag<<<nblk, TILE_NODES, 0, st>>>(pl, eb.code, eb.diag, op.inv_h2, S.shift, 2.0 * G.dim,
                                               precond == EB_PC_JACOBI, M.v, z);
        ++nl;
      }
      k_mr_dot<<<nblk, TILE_NODES, 0, st>>>(pl, M.v, z, p_vz);
      ++nl;
      return nblk;
    };
    dim_dispatch(eb, [&](auto D) {
      k_mr_mask<D.value><<<nblk, TILE_NODES, 0, s>>>(tv, eb.code, x);
      k_mr_init<D.value><<<nblk, TILE_NODES, 0, s>>>(tv, pl, eb.code, eb.diag, op, b, x, M.v, M.v_prev, M.w,
                                                      M.w_prev, p_bb);
    });
    const int nvz0 = precondition(s);
    k_mr_start<<<1, 1024, 0, s>>>(M.sc, p_bb, nblk, p_vz, nvz0, rtol, maxit);
    EB_CUDA(cudaGetLastError());
    // the iteration as the body of a device-side WHILE loop
    if (!S.cap_stream) EB_CUDA(cudaStreamCreateWithFlags(&S.cap_stream, cudaStreamNonBlocking));
    int64_t per_iter = 0;
    exec = build_while_graph(S.cap_stream, [&](cudaStream_t cs, cudaGraphConditionalHandle h) {
      const int64_t n0 = nl;
      dim_dispatch(eb, [&](auto D) {
        k_mr_apply<D.value><<<nblk, TILE_NODES, 0, cs>>>(tv, pl, eb.code, eb.diag, op, M.sc, z, M.zs, M.az, p_apply);
      });
      k_mr_lanczos<<<nblk, TILE_NODES, 0, cs>>>(pl, M.sc, p_apply, nblk, M.az, M.v, M.v_prev);
      const int nvz = precondition(cs);
      k_mr_update<true><<<nblk, TILE_NODES, 0, cs>>>(pl, M.sc, p_vz, nvz, M.zs, M.w, M.w_prev, x, h);
      per_iter = nl - n0 + 3;
    });
    EB_CUDA(cudaMemcpyAsync(M.host, M.sc, sizeof(MrScalars), cudaMemcpyDeviceToHost, s));
    EB_CUDA(cudaStreamSynchronize(s));
    if (!M.host->st[0].done) EB_CUDA(cudaGraphLaunch(exec, s));
    // true residual at exit
    dim_dispatch(eb, [&](auto D) {
      k_mr_resid<D.value><<<nblk, TILE_NODES, 0, s>>>(tv, pl, eb.code, eb.diag, op, b, x, p_bb);
    });
    k_mr_sum<<<1, 1024, 0, s>>>(p_bb, nblk, M.scal);
    double rr = 0.0;
    EB_CUDA(cudaMemcpyAsync(&rr, M.scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    EB_CUDA(cudaMemcpyAsync(M.host, M.sc, sizeof(MrScalars), cudaMemcpyDeviceToHost, s));
    EB_CUDA(cudaStreamSynchronize(s));
    const MrScalars& m = *M.host;
    const MrRot& cur = m.st[m.iters & 1];
    auto t1 = std::chrono::steady_clock::now();
    const double tr = m.bb > 0.0 ? std::sqrt(rr / m.bb) : 0.0;
    if (stats) {
      stats->iterations = m.iters;
      stats->rel_residual = m.gamma1 > 0.0 ? std::fabs(cur.eta) / m.gamma1 : 0.0;
      stats->true_rel_residual = tr;
      stats->solve_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
      stats->converged = (cur.done && !m.flags) ? 1 : 0;
      stats->prof_kernel_ms = 0.0;
      stats->prof_launches = 0;
      stats->launches = 3 + nvz0 + per_iter * m.iters;
    }
    if (m.flags & MR_FLAG_NONFINITE) {
      set_error("minres_solve: non-finite value in the iteration");
      rc = EB_ERR_NONFINITE;
    } else if (m.flags & MR_FLAG_BREAKDOWN) {
      set_error("minres_solve: breakdown (preconditioner not positive definite)");
      rc = EB_ERR_BREAKDOWN;
    } else if (!cur.done) {
      set_error("minres_solve: maxit reached");
      rc = EB_ERR_NO_CONVERGENCE;
    }
  } catch (...) {
    if (exec) cudaGraphExecDestroy(exec);
    release();
    throw;
  }
  if (exec) cudaGraphExecDestroy(exec);
  release();
  EB_CUDA(cudaStreamSynchronize(s));
  return rc;
}

}  // namespace ebk

using namespace ebk;

extern "C" int minres_solve(const amg_handle* amg, double sigma, int precond, const double* b_dev, double* x_dev,
                            double rtol, int maxit, pcg_stats* stats, cudaStream_t stream) {
  if (!amg || !b_dev || !x_dev) {
    set_error("minres_solve: NULL argument");
    return EB_ERR_INVALID;
  }
  int rc = EB_OK;
  int st = guarded([&] {
    Solver& S = const_cast<Solver&>(amg->s);
    EB_REQUIRE(S.eb->pair_node != nullptr, EB_ERR_INVALID, "minres_solve: the grid has no CP pair list");
    rc = minres(S, sigma, precond, b_dev, x_dev, rtol, maxit, stats, stream);
  });
  return st != EB_OK ? st : rc;
}
