// Preconditioned conjugate gradients on the EB operator (Algorithm 1 step 4)
// and the theta-method heat step (Sec. 3.4).
//
// Vectors live in the full-grid layout and are touched on the active tiles
// only.  Every reduction is two-pass and deterministic: each CTA of a fixed
// grid reduces its nodes in a fixed order to one partial, and a single CTA
// combines the partials in a fixed tree and updates the scalar recurrences
// (alpha, beta, ...) in device memory, so no scalar crosses to the host except
// the convergence flag, read every check_every iterations.
#include "eb_solver.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>

namespace ebk {

constexpr int VT = 256;

__device__ __forceinline__ double block_sum(double v, double* sm) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sm[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sm[i];
  return s;
}

struct TileIt {
  const Geometry G;
  __device__ __forceinline__ bool node(int64_t t, int l, int64_t& out) const {
    int64_t bx = t % G.ntx, r = t / G.ntx, by = r % G.nty, bz = r / G.nty;
    int lx = l % G.tx, ly = (l / G.tx) % G.ty, lz = l / (G.tx * G.ty);
    int64_t ix = bx * G.tx + lx, iy = by * G.ty + ly, iz = bz * G.tz + lz;
    out = ix + (int64_t)G.n0 * (iy + (int64_t)G.n1 * iz);
    return ix < G.n0 && iy < G.n1 && iz < G.n2;
  }
};

#define FOR_TILE_NODES(G, tiles, ntiles, node)                                  \
  const int tsz_ = (G).tx * (G).ty * (G).tz;                                    \
  TileIt it_{G};                                                                \
  for (int64_t tt_ = blockIdx.x; tt_ < (ntiles); tt_ += gridDim.x)              \
    for (int l_ = threadIdx.x; l_ < tsz_; l_ += blockDim.x)                     \
      if (int64_t node = 0; it_.node((tiles)[tt_], l_, node))

__device__ __forceinline__ double cp_stencil(const Geometry& G, const double* x, int64_t node, uint8_t c,
                                             const double* diag, double inv_h2, double sigma) {
  const int64_t sy = G.n0, sz = (int64_t)G.n0 * G.n1;
  const double xc = x[node];
  const uint8_t m = c & 0x3F;
  double sum = 0.0;
  if (!(m & 1)) sum += x[node - 1];
  if (!(m & 2)) sum += x[node + 1];
  if (!(m & 4)) sum += x[node - sy];
  if (!(m & 8)) sum += x[node + sy];
  if (G.dim == 3) {
    if (!(m & 16)) sum += x[node - sz];
    if (!(m & 32)) sum += x[node + sz];
  }
  const double D = m ? diag[node] : (double)(2 * G.dim);
  return (D * xc - sum) * inv_h2 + sigma * xc;
}

// dinv = 1 / (sigma + D/h^2) at the CPs
__global__ void k_dinv(Geometry G, const int32_t* tiles, int64_t ntiles, const uint8_t* code, const double* diag,
                       double sigma, double inv_h2, double* dinv) {
  FOR_TILE_NODES(G, tiles, ntiles, node) {
    uint8_t c = code[node];
    double v = 0.0;
    if (c & CODE_CP) {
      double D = (c & 0x3F) ? diag[node] : (double)(2 * G.dim);
      v = 1.0 / (sigma + D * inv_h2);
    }
    dinv[node] = v;
  }
}

// r = b - (sigma I + A) x  (b masked to the CPs); partials (b.b, r.r)
__global__ void k_resid(Geometry G, const int32_t* tiles, int64_t ntiles, const uint8_t* code, const double* diag,
                        double sigma, double inv_h2, const double* b, const double* x, double* r, double* part) {
  __shared__ double sm[32];
  double sbb = 0.0, srr = 0.0;
  FOR_TILE_NODES(G, tiles, ntiles, node) {
    uint8_t c = code[node];
    double rv = 0.0;
    if (c & CODE_CP) {
      double bv = b[node];
      rv = bv - cp_stencil(G, x, node, c, diag, inv_h2, sigma);
      sbb += bv * bv;
      srr += rv * rv;
    }
    r[node] = rv;
  }
  double a = block_sum(sbb, sm);
  double bsum = block_sum(srr, sm);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = bsum;
  }
}

// q = (sigma I + A) p; partial p.q
__global__ void k_apply_dot(Geometry G, const int32_t* tiles, int64_t ntiles, const uint8_t* code, const double* diag,
                            double sigma, double inv_h2, const double* p, double* q, double* part) {
  __shared__ double sm[32];
  double s = 0.0;
  FOR_TILE_NODES(G, tiles, ntiles, node) {
    uint8_t c = code[node];
    double qv = 0.0;
    if (c & CODE_CP) {
      qv = cp_stencil(G, p, node, c, diag, inv_h2, sigma);
      s += p[node] * qv;
    }
    q[node] = qv;
  }
  double t = block_sum(s, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// x += alpha p; r -= alpha q; partial r.r
__global__ void k_update_xr(Geometry G, const int32_t* tiles, int64_t ntiles, const PcgScalars* sc, double* x,
                            double* r, const double* p, const double* q, double* part) {
  __shared__ double sm[32];
  if (sc->done) {
    if (threadIdx.x == 0) part[blockIdx.x] = 0.0;
    return;
  }
  const double alpha = sc->alpha;
  double s = 0.0;
  FOR_TILE_NODES(G, tiles, ntiles, node) {
    double rv = r[node] - alpha * q[node];
    x[node] += alpha * p[node];
    r[node] = rv;
    s += rv * rv;
  }
  double t = block_sum(s, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// z = dinv r; partial r.z
__global__ void k_jacobi_dot(Geometry G, const int32_t* tiles, int64_t ntiles, const double* dinv, const double* r,
                             double* z, double* part) {
  __shared__ double sm[32];
  double s = 0.0;
  FOR_TILE_NODES(G, tiles, ntiles, node) {
    double rv = r[node];
    double zv = dinv[node] * rv;
    z[node] = zv;
    s += rv * zv;
  }
  double t = block_sum(s, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_dot(Geometry G, const int32_t* tiles, int64_t ntiles, const double* a, const double* b, double* part) {
  __shared__ double sm[32];
  double s = 0.0;
  FOR_TILE_NODES(G, tiles, ntiles, node) { s += a[node] * b[node]; }
  double t = block_sum(s, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// p = z + beta p   (beta = 0 on the first iteration of a cycle)
__global__ void k_xpby(Geometry G, const int32_t* tiles, int64_t ntiles, const PcgScalars* sc, const double* z,
                       double* p, int first) {
  if (sc->done) return;
  const double beta = first ? 0.0 : sc->beta;
  FOR_TILE_NODES(G, tiles, ntiles, node) { p[node] = first ? z[node] : z[node] + beta * p[node]; }
}

// rhs for the theta-method: (u/dt - (1-theta) A u + theta b1 + (1-theta) b0) / theta
__global__ void k_heat_rhs(Geometry G, const int32_t* tiles, int64_t ntiles, const uint8_t* code, const double* diag,
                           double inv_h2, double dt, double theta, const double* u, const double* b1,
                           const double* b0, double* out) {
  FOR_TILE_NODES(G, tiles, ntiles, node) {
    uint8_t c = code[node];
    double v = 0.0;
    if (c & CODE_CP) {
      double uv = u[node];
      v = uv / dt + theta * b1[node];
      if (theta < 1.0) v += (1.0 - theta) * (b0[node] - cp_stencil(G, u, node, c, diag, inv_h2, 0.0));
      v /= theta;
    }
    out[node] = v;
  }
}

__global__ void k_mask_copy(Geometry G, const int32_t* tiles, int64_t ntiles, const uint8_t* code, const double* in,
                            double* out) {
  FOR_TILE_NODES(G, tiles, ntiles, node) { out[node] = (code[node] & CODE_CP) ? in[node] : 0.0; }
}

// Combine partials in a fixed order and advance the scalar recurrences.
__global__ void k_finalize(const double* part, int nblk, int op, PcgScalars* sc) {
  __shared__ double sm[2][1024];
  double a = 0.0, b = 0.0;
  const int stride = (op == FIN_INIT) ? 2 : 1;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
    a += part[stride * i];
    if (op == FIN_INIT) b += part[2 * i + 1];
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
      sc->rz = v;
      if (!isfinite(v)) sc->flags |= PCG_FLAG_NONFINITE;
      break;
    case FIN_ALPHA:
      if (sc->done) break;
      sc->pq = v;
      if (!(v > 0.0)) {
        sc->flags |= isfinite(v) ? PCG_FLAG_BREAKDOWN : PCG_FLAG_NONFINITE;
        sc->done = 1;
        sc->alpha = 0.0;
      } else {
        sc->alpha = sc->rz / v;
      }
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
    case FIN_BETA:
      if (sc->done) break;
      if (!(v > 0.0)) {
        sc->flags |= isfinite(v) ? PCG_FLAG_BREAKDOWN : PCG_FLAG_NONFINITE;
        sc->done = 1;
        break;
      }
      sc->beta = v / sc->rz;
      sc->rz = v;
      break;
  }
}

// ---------------------------------------------------------------- host side
void Solver::alloc_work(cudaStream_t s) {
  const int64_t nn = eb->g.num_nodes;
  r = dalloc<double>(nn, s);
  z = dalloc<double>(nn, s);
  p = dalloc<double>(nn, s);
  q = dalloc<double>(nn, s);
  tmp = dalloc<double>(nn, s);
  dinv = dalloc<double>(nn, s);
  nblk = (int)std::min<int64_t>(std::max<int64_t>(eb->num_tiles, 1), (int64_t)num_sms() * 4);
  nblk = std::min(nblk, 1024 * 8);
  part = dalloc<double>(2 * (int64_t)nblk, s);
  sc = dalloc<PcgScalars>(1, s);
  EB_CUDA(cudaMallocHost((void**)&sc_host, sizeof(PcgScalars)));
  const Geometry& G = eb->g;
  k_dinv<<<nblk, VT, 0, s>>>(G, eb->tiles, eb->num_tiles, eb->code, eb->diag, shift, 1.0 / (G.h * G.h), dinv);
  EB_CUDA(cudaGetLastError());
}

void Solver::free_work() {
  cudaStream_t s = eb->home;
  dfree(r, s); dfree(z, s); dfree(p, s); dfree(q, s); dfree(tmp, s); dfree(dinv, s); dfree(part, s); dfree(sc, s);
  if (sc_host) cudaFreeHost(sc_host);
  sc_host = nullptr;
}

void Solver::finalize(int op, cudaStream_t s) {
  k_finalize<<<1, 1024, 0, s>>>(part, nblk, op, sc);
}

void Solver::precondition(int kind, const double* rin, double* zout, cudaStream_t s) {
  const Geometry& G = eb->g;
  if (kind == EB_PC_AMG && H) {
    amg_vcycle_grid(*this, rin, zout, s);
    k_dot<<<nblk, VT, 0, s>>>(G, eb->tiles, eb->num_tiles, rin, zout, part);
  } else if (kind == EB_PC_NONE) {
    EB_CUDA(cudaMemcpyAsync(zout, rin, sizeof(double) * G.num_nodes, cudaMemcpyDeviceToDevice, s));
    k_dot<<<nblk, VT, 0, s>>>(G, eb->tiles, eb->num_tiles, rin, zout, part);
  } else {
    k_jacobi_dot<<<nblk, VT, 0, s>>>(G, eb->tiles, eb->num_tiles, dinv, rin, zout, part);
  }
}

int Solver::pcg(const double* b, double* x, double rtol, int maxit, const pcg_opts& o, pcg_stats* stats,
                cudaStream_t s) {
  const Geometry& G = eb->g;
  const double inv_h2 = 1.0 / (G.h * G.h);
  const int kind = o.precond;
  EB_REQUIRE(kind == EB_PC_AMG || kind == EB_PC_JACOBI || kind == EB_PC_NONE, EB_ERR_INVALID, "bad preconditioner");
  EB_REQUIRE(kind != EB_PC_AMG || H != nullptr, EB_ERR_INVALID, "AMG preconditioner requested without a hierarchy");
  EB_REQUIRE(rtol > 0.0 && maxit >= 0, EB_ERR_INVALID, "rtol must be > 0 and maxit >= 0");
  const int check = std::max(1, o.check_every);
  auto t0 = std::chrono::steady_clock::now();
  PcgScalars init{};
  init.tol2 = rtol * rtol;
  int total_iters = 0;
  bool converged = false;
  int flags = 0;
  double rel = 0.0;
  for (int restart = 0; restart < 4 && !converged; ++restart) {
    EB_CUDA(cudaMemcpyAsync(sc, &init, sizeof(init), cudaMemcpyHostToDevice, s));
    // x is masked to the CPs (its non-CP entries are ignored on input)
    k_mask_copy<<<nblk, VT, 0, s>>>(G, eb->tiles, eb->num_tiles, eb->code, x, x);
    k_resid<<<nblk, VT, 0, s>>>(G, eb->tiles, eb->num_tiles, eb->code, eb->diag, shift, inv_h2, b, x, r, part);
    finalize(FIN_INIT, s);
    EB_CUDA(cudaMemcpyAsync(sc_host, sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
    EB_CUDA(cudaStreamSynchronize(s));
    if (sc_host->flags & PCG_FLAG_NONFINITE) {
      flags |= sc_host->flags;
      break;
    }
    if (sc_host->bb == 0.0) {  // b = 0: x = 0 is the solution
      EB_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * G.num_nodes, s));
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
    precondition(kind, r, z, s);
    finalize(FIN_RZ0, s);
    k_xpby<<<nblk, VT, 0, s>>>(G, eb->tiles, eb->num_tiles, sc, z, p, 1);
    int it = 0;
    bool stop = false;
    while (!stop) {
      for (int j = 0; j < check && total_iters + it < maxit; ++j, ++it) {
        k_apply_dot<<<nblk, VT, 0, s>>>(G, eb->tiles, eb->num_tiles, eb->code, eb->diag, shift, inv_h2, p, q, part);
        finalize(FIN_ALPHA, s);
        k_update_xr<<<nblk, VT, 0, s>>>(G, eb->tiles, eb->num_tiles, sc, x, r, p, q, part);
        finalize(FIN_RR, s);
        precondition(kind, r, z, s);
        finalize(FIN_BETA, s);
        k_xpby<<<nblk, VT, 0, s>>>(G, eb->tiles, eb->num_tiles, sc, z, p, 0);
      }
      EB_CUDA(cudaGetLastError());
      EB_CUDA(cudaMemcpyAsync(sc_host, sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
      EB_CUDA(cudaStreamSynchronize(s));
      if (sc_host->done || total_iters + it >= maxit) stop = true;
    }
    total_iters += sc_host->iters;
    flags |= sc_host->flags;
    if (flags & (PCG_FLAG_NONFINITE | PCG_FLAG_BREAKDOWN)) break;
    // true residual at exit
    k_resid<<<nblk, VT, 0, s>>>(G, eb->tiles, eb->num_tiles, eb->code, eb->diag, shift, inv_h2, b, x, r, part);
    finalize(FIN_INIT, s);
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
  k_heat_rhs<<<nblk, VT, 0, s>>>(G, eb->tiles, eb->num_tiles, eb->code, eb->diag, 1.0 / (G.h * G.h), dt, theta, u,
                                 b1, b0 ? b0 : b1, tmp);
  EB_CUDA(cudaGetLastError());
  pcg_opts o{EB_PC_AMG, 1, 0};
  if (!H) o.precond = EB_PC_JACOBI;
  return pcg(tmp, u, rtol, maxit, o, stats, s);
}

}  // namespace ebk
