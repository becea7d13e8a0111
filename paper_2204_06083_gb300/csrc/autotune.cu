// Tile-shape autotuner.  The active-tile kernels cut the grid into blocks of
// 256 nodes whose extents are powers of two; the shape only changes how the
// work is split into CTAs and how far apart in memory the rows of one tile
// lie, never a result.  The tuner rebuilds the tile list for each candidate
// shape, times the operation it is asked about with CUDA events on the
// caller's stream, and keeps the fastest shape.
#include "eb_solver.cuh"

#include <algorithm>
#include <vector>

namespace ebk {

std::vector<TileDims> tile_candidates(int dim) {
  if (dim == 2) return {{32, 8, 1}, {64, 4, 1}, {16, 16, 1}, {128, 2, 1}, {8, 32, 1}};
  return {{16, 4, 4}, {32, 4, 2}, {8, 8, 4}, {16, 8, 2}, {32, 2, 4}, {64, 2, 2},
          {8, 4, 8}, {16, 2, 8}, {32, 8, 1}, {64, 4, 1}};
}

double time_us(const std::function<void()>& op, int reps, cudaStream_t s) {
  for (int i = 0; i < 3; ++i) op();
  cudaEvent_t a, b;
  EB_CUDA(cudaEventCreate(&a));
  cudaError_t e = cudaEventCreate(&b);
  if (e != cudaSuccess) {
    cudaEventDestroy(a);
    EB_CUDA(e);
  }
  float ms = 0.0f;
  try {
    EB_CUDA(cudaEventRecord(a, s));
    for (int i = 0; i < reps; ++i) op();
    EB_CUDA(cudaEventRecord(b, s));
    EB_CUDA(cudaEventSynchronize(b));
    EB_CUDA(cudaEventElapsedTime(&ms, a, b));
  } catch (...) {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    throw;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return 1000.0 * ms / reps;
}

void run_tuner(int dim, const std::function<void(const TileDims&)>& retile, const std::function<void()>& op,
               int reps, eb_tune_t* out, cudaStream_t s) {
  EB_REQUIRE(reps >= 1 && reps <= 100000, EB_ERR_INVALID, "autotune: reps in [1, 100000]");
  const std::vector<TileDims> cand = tile_candidates(dim);
  eb_tune_t r{};
  r.count = (int)cand.size();
  int best = 0;
  for (int i = 0; i < r.count; ++i) {
    retile(cand[i]);
    r.tile[i][0] = cand[i].x;
    r.tile[i][1] = cand[i].y;
    r.tile[i][2] = cand[i].z;
    r.us[i] = time_us(op, reps, s);
    if (r.us[i] < r.us[best]) best = i;
  }
  if (best != r.count - 1) retile(cand[best]);
  r.best = best;
  if (out) *out = r;
}

}  // namespace ebk

using namespace ebk;

extern "C" {

int eb_retile(eb_handle* eb, const int tile[3], cudaStream_t stream) {
  if (!eb || !tile) {
    set_error("eb_retile: NULL argument");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    build_tiles(eb->h, tile[0], tile[1], tile[2], stream);
    EB_CUDA(cudaStreamSynchronize(stream));
  });
}

int eb_autotune(eb_handle* eb, int op_kind, int prec, int reps, eb_tune_t* out, cudaStream_t stream) {
  if (!eb) {
    set_error("eb_autotune: NULL handle");
    return EB_ERR_INVALID;
  }
  if (op_kind != EB_TUNE_APPLY && op_kind != EB_TUNE_LEAPFROG) {
    set_error("eb_autotune: op must be EB_TUNE_APPLY or EB_TUNE_LEAPFROG");
    return EB_ERR_INVALID;
  }
  if (prec != EB_F64 && prec != EB_F32 && (prec != EB_BF16 || op_kind == EB_TUNE_LEAPFROG)) {
    set_error("eb_autotune: prec must be EB_F64, EB_F32 or (apply only) EB_BF16");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    EBHandle& E = eb->h;
    const int64_t nn = E.g.num_nodes;
    const size_t es = prec == EB_F64 ? 8 : (prec == EB_F32 ? 4 : 2);
    uint8_t* x = dalloc<uint8_t>(nn * es, stream);
    uint8_t* y = nullptr;
    try {
      y = dalloc<uint8_t>(nn * es, stream);
      // leapfrog: 16 step launches per timed call (dt = 0: fields stay finite)
      auto leap = [&] {
        int rc = prec == EB_F64
                     ? launch_leapfrog<double>(E, reinterpret_cast<double*>(x), reinterpret_cast<double*>(y), 16, 0.0,
                                               stream, false)
                     : launch_leapfrog<float>(E, reinterpret_cast<float*>(x), reinterpret_cast<float*>(y), 16, 0.0,
                                              stream, false);
        EB_REQUIRE(rc == EB_OK, rc, "eb_autotune: leapfrog launch failed");
      };
      auto op = [&] {
        if (op_kind == EB_TUNE_LEAPFROG)
          leap();
        else if (prec == EB_F64)
          launch_apply<double>(E, reinterpret_cast<double*>(x), reinterpret_cast<double*>(y), 0.0, stream);
        else if (prec == EB_F32)
          launch_apply<float>(E, reinterpret_cast<float*>(x), reinterpret_cast<float*>(y), 0.0, stream);
        else
          launch_apply<__nv_bfloat16>(E, reinterpret_cast<__nv_bfloat16*>(x), reinterpret_cast<__nv_bfloat16*>(y),
                                      0.0, stream);
      };
      run_tuner(E.g.dim, [&](const TileDims& t) { build_tiles(E, t.x, t.y, t.z, stream); }, op, reps, out, stream);
    } catch (...) {
      dfree(x, stream);
      dfree(y, stream);
      throw;
    }
    dfree(x, stream);
    dfree(y, stream);
    EB_CUDA(cudaStreamSynchronize(stream));
  });
}

int amg_autotune(amg_handle* amg, int reps, eb_tune_t* out, cudaStream_t stream) {
  if (!amg) {
    set_error("amg_autotune: NULL handle");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    Solver& S = amg->s;
    EB_REQUIRE(S.H != nullptr, EB_ERR_INVALID, "amg_autotune: handle has no hierarchy");
    EBHandle& E = *S.eb;
    const int64_t nn = E.g.num_nodes;
    double* r = dalloc<double>(nn, stream);
    double* z = nullptr;
    try {
      z = dalloc<double>(nn, stream);
      run_tuner(E.g.dim, [&](const TileDims& t) { build_tiles(E, t.x, t.y, t.z, stream); },
                [&] { amg_vcycle_grid(S, r, z, stream); }, reps, out, stream);
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

int amg_tune_csr(amg_handle* amg, int reps, double* us_out, int* best_out, cudaStream_t stream) {
  if (!amg) {
    set_error("amg_tune_csr: NULL handle");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    Solver& S = amg->s;
    EB_REQUIRE(S.H != nullptr, EB_ERR_INVALID, "amg_tune_csr: handle has no hierarchy");
    EB_REQUIRE(reps >= 1 && reps <= 100000, EB_ERR_INVALID, "amg_tune_csr: reps in [1, 100000]");
    const int64_t nn = S.eb->g.num_nodes;
    double* r = dalloc<double>(nn, stream);
    double* z = nullptr;
    try {
      z = dalloc<double>(nn, stream);
      const int cand[4] = {1, 2, 4, 8};
      double us[4];
      int best = 0;
      for (int i = 0; i < 4; ++i) {
        S.csr_epl = cand[i];
        us[i] = time_us([&] { amg_vcycle_grid(S, r, z, stream); }, reps, stream);
        if (us[i] < us[best]) best = i;
      }
      S.csr_epl = cand[best];
      S.graph_release();  // captured iterations hold the old launch shapes
      S.loop_release();
      if (us_out)
        for (int i = 0; i < 4; ++i) us_out[i] = us[i];
      if (best_out) *best_out = cand[best];
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

}  // extern "C"

namespace ebk {
// FP64 arithmetic peak: every thread runs 8 independent chains of fused
// multiply-adds (no memory traffic in the loop), so the FP64 pipes, not
// latency, bound it.  The result is stored only if it were NaN (never), which
// keeps the chains alive without a store per thread.
constexpr int FP64_PEAK_ITERS = 2048;
constexpr int FP64_PEAK_CHAINS = 8;
__global__ void __launch_bounds__(256) k_fp64_fma_peak(double seed, double* sink) {
  double a[FP64_PEAK_CHAINS];
  const double m = 1.0 - 1e-9 * (threadIdx.x & 7);
  const double c = 1e-9 * seed;
#pragma unroll
  for (int k = 0; k < FP64_PEAK_CHAINS; ++k) a[k] = seed + k;
  for (int i = 0; i < FP64_PEAK_ITERS; ++i) {
#pragma unroll
    for (int k = 0; k < FP64_PEAK_CHAINS; ++k) a[k] = fma(a[k], m, c);
  }
  double t = 0.0;
#pragma unroll
  for (int k = 0; k < FP64_PEAK_CHAINS; ++k) t += a[k];
  if (t != t) sink[0] = t;
}
}  // namespace ebk

extern "C" {

int eb_fp64_peak(int reps, double* tflops_out, cudaStream_t stream) {
  if (!tflops_out || reps < 1 || reps > 10000) {
    set_error("eb_fp64_peak: NULL output or reps not in [1, 10000]");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    double* sink = dalloc<double>(1, stream);
    try {
      int per_sm = 0;
      EB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_fma_peak, 256, 0));
      const unsigned blocks = (unsigned)(std::max(per_sm, 1) * num_sms() * 4);
      const double us = time_us([&] { k_fp64_fma_peak<<<blocks, 256, 0, stream>>>(1.0, sink); }, reps, stream);
      EB_CUDA(cudaGetLastError());
      const double flop = 2.0 * FP64_PEAK_ITERS * FP64_PEAK_CHAINS * 256.0 * blocks;
      *tflops_out = flop / (us * 1e-6) / 1e12;
    } catch (...) {
      dfree(sink, stream);
      throw;
    }
    dfree(sink, stream);
    EB_CUDA(cudaStreamSynchronize(stream));
  });
}

int amg_set_csr_epl(amg_handle* amg, int epl) {
  if (!amg || (epl != 1 && epl != 2 && epl != 4 && epl != 8)) {
    set_error("amg_set_csr_epl: NULL handle or entries per lane not 1, 2, 4 or 8");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    Solver& S = amg->s;
    if (S.csr_epl == epl) return;
    S.csr_epl = epl;
    S.graph_release();  // captured iterations hold the old launch shapes
    S.loop_release();
  });
}

}  // extern "C"
