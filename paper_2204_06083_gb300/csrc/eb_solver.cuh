// Internal solver state: PCG scalars, work vectors and the AMG hierarchy.
#pragma once

#include <utility>
#include <vector>

#include "eb_internal.cuh"

namespace ebk {

// Flexible CG (Polak-Ribiere beta): the x/r update also forms r.z_previous
// (the r'zold term) from the z still in place.  FIN_RRF: the batch's (r.r,
// r.z_previous) pairs, recorded per geometry; FIN_BETAF then takes r.z_previous
// from there; FIN_RZ0F is FIN_RZ0.  The single-grid PCG combines FIN_ALPHA and
// FIN_BETA inside its update kernels; the batch finalizes every op in its
// per-geometry kernel.
enum { FIN_INIT = 0, FIN_RZ0 = 1, FIN_ALPHA = 2, FIN_RR = 3, FIN_BETA = 4, FIN_RZ0F = 5, FIN_BETAF = 6, FIN_RRF = 7 };
enum { PCG_FLAG_NONFINITE = 1, PCG_FLAG_BREAKDOWN = 2 };
// what pcg_opts.profile times: the level-0 smoother launches, the learned stage's 32 -> 32
// convolutions, the level-1 (first coarse, CSR) smoother launches, the PCG's p update +
// apply launches (k_xpby_apply) or its x/r update launches (fused with the first level-0
// smoothing step when an AMG V-cycle follows)
enum { PROF_SMOOTHER = 1, PROF_CONV = 2, PROF_LEVEL1 = 3, PROF_XPBY = 4, PROF_UPDATE = 5 };

// rz[iters & 1] holds r'z of the current iteration; the kernel that computes
// the next one writes the other slot, so that no CTA reads a value another CTA
// of the same kernel is rewriting (the batch keeps using rz[0])
struct PcgScalars {
  double bb, rr, rz[2], pq, alpha, beta, tol2;
  int iters, flags, done;
  int maxit;  // iteration limit of the device-side loop (counted like iters)
  // iters & 1 as the x/r update of the iteration saw it: the r'z slot of the
  // p update, whose launch may also advance iters (device-side loop)
  int slot;
  double rzo;  // batched flexible PCG: r'zold of the iteration (FIN_RRF)
};

struct Hierarchy;  // AMG levels (amg.cu)
struct OpParams;   // operator constants of the PCG kernels (eb_solve.cu)

struct Solver {
  EBHandle* eb = nullptr;
  // stream the solver's memory belongs to (set at setup); destroying a solver
  // never reads *eb, which may already be gone
  cudaStream_t home = 0;
  double shift = 0.0;
  amg_opts opts{};
  Hierarchy* H = nullptr;
  double setup_ms = 0.0;
  int csr_epl = 2;  // CSR kernels of the V-cycle: target entries per lane of a row group (amg_tune_csr)
  // full-grid work vectors (touched on the active tiles only)
  double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *tmp = nullptr;
  double* wx = nullptr;  // the implicit wave step's solution vector (allocated on first use)
  bool flexible() const { return H != nullptr && (opts.vcycle_prec == EB_F32 || opts.vcycle_prec == EB_BF16); }
  // the flexible (Polak-Ribiere) beta: reduced-precision V-cycle or learned stage
  bool flex_for(int kind) const { return kind == EB_PC_AMG_NN || (kind == EB_PC_AMG && flexible()); }
  nn_handle* nn = nullptr;  // learned stage of EB_PC_AMG_NN (set for one solve)
  int nn_mode = 0;          // eb_nn_mode of that stage
  // reduction partials: [p'q | r'r] regions of 2 nblk each, then the r'z region
  // of 2 max(nblk, 8 SMs): r'z comes from the PCG's own dot kernel (nblk
  // partials) or from the V-cycle's last smoothing launch (one per CTA of it),
  // then the r'zold region of nblk
  double* part = nullptr;
  double* part_pq() const { return part; }
  double* part_rr() const { return part + 2 * (int64_t)nblk; }
  double* part_rz() const { return part + 4 * (int64_t)nblk; }
  // r'zold partials of the flexible beta (nblk, from the x/r update)
  double* part_rzo() const { return part + 4 * (int64_t)nblk + rz_cap; }
  // CTAs (= partials) of the iteration's x/r update and p update + apply
  int nblk_iter() const { return nblk; }
  int64_t rz_cap = 0;
  int nblk = 1;
  int rz_n = 1;  // r'z partials written by the last precondition()
  PcgScalars* sc = nullptr;
  PcgScalars* sc_host = nullptr;
  int64_t nlaunch = 0;  // kernel launches issued (reported per solve)
  // event timing of the level-0 smoother launches
  bool prof_on = false;
  int prof_what = PROF_SMOOTHER;
  int prof_n = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev;
  double prof_acc_ms = 0.0;
  int prof_acc_n = 0;
  // captured PCG iteration (CUDA graph), keyed by its arguments
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const double* g_b = nullptr;
  double* g_x = nullptr;
  const nn_handle* g_nn = nullptr;
  int g_tile_gen = -1;
  int g_nn_mode = -1;
  int g_iters = 0, g_kind = -1, g_prof = -1, g_pairs = 0;
  int64_t g_launches = 0;
  // the whole iteration loop on the device: a conditional WHILE node whose
  // body is one iteration (no host round trip per iteration)
  cudaGraphExec_t lexec = nullptr;
  const double* l_b = nullptr;
  double* l_x = nullptr;
  int l_kind = -1, l_nn_mode = -1, l_tile_gen = -1;
  const nn_handle* l_nn = nullptr;
  int64_t l_launches = 0;  // kernel launches per loop iteration
  // the DF outer iteration (pcg_opts.outer_prec = EB_DF64) for the current
  // solve: x, r, p, q hold double-float pairs (x in xdf), z FP32; diag_df is
  // the DF copy of the cut CPs' D_k (built on first use)
  bool df_on = false;
  float2* diag_df = nullptr;
  float2* beta_df[3] = {nullptr, nullptr, nullptr};  // DF copies of beta per axis (variable coefficient)
  int df_gen = -1;  // the handle's tile_gen the DF copies were built for
  // outer precision of the solves without their own options: heat_step,
  // wave_theta_step, pcg_solve with NULL opts (amg_set_outer_prec)
  int outer_default = EB_F64;
  int default_outer() const;
  // level-0 smoothing steps of batched 2D views through tensor copies (on by
  // default; batch_set_level0_tma), and the device flag their bounded waits set
  bool l0_tma = true;
  int* dev_err = nullptr;
  double* xdf = nullptr;  // the DF image of x (tmp may hold the right-hand side)
  int g_df = -1, l_df = -1;

  void alloc_work(cudaStream_t s);
  void free_work();
  void finalize(int op, const double* src, cudaStream_t s, int count = -1);  // count < 0: nblk partials
  // first_done: amg_update_first did the V-cycle's first level-0 step for r
  void precondition(int kind, const double* r, double* z, cudaStream_t s, bool first_done = false);
  int pcg(const double* b, double* x, double rtol, int maxit, const pcg_opts& o, pcg_stats* stats, cudaStream_t s);
  int heat(double dt, double theta, const double* b1, const double* b0, double* u, double rtol, int maxit,
           pcg_stats* stats, cudaStream_t s);
  int wave_theta(double dt, double theta, double* ua, double* ub, int nsteps, double rtol, int maxit,
                 pcg_stats* stats, cudaStream_t s);
  void prof_begin(int mode, cudaStream_t s);
  void prof_mark(cudaStream_t s, bool start, int what = PROF_SMOOTHER);
  void prof_collect(int first, int count);
  void prof_end(pcg_stats* st, cudaStream_t s);
  void prof_release();
  // cond: inside the device-side loop, the handle its last launch sets
  void iteration(int kind, const double* b, double* x, cudaStream_t s,
                 const cudaGraphConditionalHandle* cond = nullptr);
  // p = z + beta p and q = h^2 (sigma I + A) z + beta q with the p.q partials
  // (eb_solve.cu); flex: the Polak-Ribiere beta (r'zold partials in part_rzo)
  void xpby_apply(const OpParams& op, bool flex, int first, cudaStream_t s,
                  const cudaGraphConditionalHandle* cond = nullptr);
  void graph_prepare(int kind, const double* b, double* x, int iters, int profile, cudaStream_t s);
  void graph_release();
  void loop_prepare(int kind, const double* b, double* x, cudaStream_t s);
  void loop_release();
};

// Instantiates { while (condition) body } as one executable graph: body(st,
// h) enqueues one pass on the capture stream st and must end with a kernel
// that sets the condition handle h (cudaGraphSetConditional); the condition
// starts at 1.  cap is a non-blocking stream used only for the capture.
cudaGraphExec_t build_while_graph(cudaStream_t cap,
                                  const std::function<void(cudaStream_t, cudaGraphConditionalHandle)>& body);

// AMG (amg.cu)
void amg_build(Solver& S, cudaStream_t s);
void amg_free(Solver& S);
// Sum of v over the CTA (warp shuffles, then the warps in order); thread 0
// holds the result.  Every reduction partial of the PCG is formed this way.
__device__ __forceinline__ double block_sum(double v, double* sm) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sm[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sm[i];
  return s;
}

// sc->done as thread 0 of the CTA reads it, the same for all its threads (CTA
// 0 of the launch may set it meanwhile, so threads reading it themselves could
// disagree and part of the CTA skip the barriers the rest waits at); all
// threads call it.
__device__ __forceinline__ bool cta_done(const PcgScalars* sc) {
  __shared__ int s_done;
  if (threadIdx.x == 0) s_done = *(volatile const int*)&sc->done;
  __syncthreads();
  return s_done != 0;
}

// sum of n partials (stride apart) in a fixed order, the same in every CTA;
// thread 0 holds the result
__device__ __forceinline__ double sum_parts(const double* part, int n, int stride, double* sm) {
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += part[stride * i];
  return block_sum(a, sm);
}

// alpha = rz / p'q from the nblk partials of k_xpby_apply (q scaled by h^2:
// the CG step length over h^2), formed by every CTA in
// the same order; CTA 0 records p'q, alpha and a breakdown (p'q <= 0 or not
// finite).  All threads of the CTA call it; returns alpha to every thread.
// thread 0's part of pcg_alpha, given the summed p'q: returns alpha (CTA 0
// records p'q, alpha and a breakdown)
__device__ __forceinline__ double pcg_alpha_from(PcgScalars* sc, double pq) {
  const bool ok = pq > 0.0;  // false for NaN too
  const double alpha = ok ? sc->rz[sc->iters & 1] / pq : 0.0;
  if (blockIdx.x == 0) {
    sc->pq = pq;
    sc->alpha = alpha;
    sc->slot = sc->iters & 1;
    if (!ok) {
      sc->flags |= isfinite(pq) ? PCG_FLAG_BREAKDOWN : PCG_FLAG_NONFINITE;
      sc->done = 1;
    }
  }
  return alpha;
}

__device__ __forceinline__ double pcg_alpha(PcgScalars* sc, const double* pq_part, int nblk, double* sm,
                                            double* s_alpha) {
  const double pq = sum_parts(pq_part, nblk, 1, sm);
  if (threadIdx.x == 0) *s_alpha = pcg_alpha_from(sc, pq);
  __syncthreads();
  return *s_alpha;
}

// The PCG update x += alpha p, r -= alpha q (with the r'r partials of
// k_update_xr) fused with the first level-0 smoothing step of the V-cycle that
// follows (which then starts at its second step); 0 if the hierarchy has no
// such step (a single level), else the launch was issued.
struct PcgUpdate {
  PcgScalars* sc = nullptr;
  double *x = nullptr, *r = nullptr;
  const double *p = nullptr, *q = nullptr, *pq_part = nullptr;
  int nblk = 0;
  double* rr_part = nullptr;
  double h2 = 1.0;  // q holds h2 (sigma I + A) p: x takes the step alpha h2
  // flexible CG: partials of (new r).z with the z still in z (r'zold)
  const double* z = nullptr;
  double* rzo_part = nullptr;
  // the DF outer iteration: x, r, p, q hold double-float pairs, z FP32
  bool df = false;
};
int amg_update_first(Solver& S, const PcgUpdate& u, cudaStream_t s);

// z = V r.  With dot, the last level-0 smoothing launch also writes per-CTA
// partials of r.z to dot->part; returns their count, or 0 if no launch wrote
// them (single-level hierarchy), in which case the caller computes the dot
// itself.
struct VcycleDot {
  const double* r = nullptr;
  double* part = nullptr;
  // the DF outer iteration: r holds double-float pairs, z is written in FP32
  // (part null: no partials, z on every node of the active tiles)
  bool df = false;
};
// first_done: amg_update_first already did the first level-0 step for this r.
int amg_vcycle_grid(Solver& S, const double* r, double* z, cudaStream_t s, const VcycleDot* dot = nullptr,
                    bool first_done = false);
void amg_fill_info(const Solver& S, amg_info_t* out);
int amg_levels(const Solver& S);  // levels of the hierarchy (0 without one)
void amg_copy_level(const Solver& S, int level, int which, int32_t* rowptr, int32_t* col, double* val, cudaStream_t s);

// learned stage (cnn.cu): buffers for grids of eb's size (before any capture),
// then z <- z + omega h^2 rms(s) N(s / rms(s), m), s = r - (shift I + A) z
void nn_stage_prepare(nn_handle* nn, const EBHandle& eb, cudaStream_t s);
void nn_stage_apply(nn_handle* nn, const EBHandle& eb, double shift, int mode, const double* r, double* z,
                    int64_t& nlaunch, Solver* prof, cudaStream_t s);

}  // namespace ebk

// the opaque AMG / solver handle of the C ABI
struct amg_handle {
  ebk::Solver s;
};
