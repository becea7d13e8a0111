// extern "C" entry points of include/eb.h.  Each call validates its arguments,
// runs under a guard that turns internal failures into eb_status codes, and
// records a thread-local message for eb_last_error().
#include "eb_solver.cuh"

#include <chrono>
#include <cmath>

namespace ebk {
static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
const char* last_error() { return g_last_error.c_str(); }
const EBHandle& handle_of(const eb_handle* eb) { return eb->h; }
}  // namespace ebk

using namespace ebk;

extern "C" {

const char* eb_last_error(void) { return ebk::last_error(); }

int eb_build(const eb_grid* grid, const eb_levelset* ls, eb_handle** out, cudaStream_t stream) {
  return eb_build_ex(grid, ls, nullptr, out, stream);
}

int eb_build_ex(const eb_grid* grid, const eb_levelset* ls, const eb_build_opts* opts, eb_handle** out,
                cudaStream_t stream) {
  if (!grid || !ls || !out) {
    set_error("eb_build: NULL argument");
    return EB_ERR_INVALID;
  }
  *out = nullptr;
  eb_handle* e = new (std::nothrow) eb_handle();
  if (!e) {
    set_error("eb_build: host allocation failed");
    return EB_ERR_OOM;
  }
  int st = guarded([&] { build_handle(e->h, *grid, *ls, stream, opts); });
  if (st != EB_OK) {
    destroy_handle(e->h);
    delete e;
    return st;
  }
  *out = e;
  return EB_OK;
}

void eb_destroy(eb_handle* eb) {
  if (!eb) return;
  destroy_handle(eb->h);
  delete eb;
}

int eb_info(const eb_handle* eb, eb_info_t* out) {
  if (!eb || !out) {
    set_error("eb_info: NULL argument");
    return EB_ERR_INVALID;
  }
  const EBHandle& h = eb->h;
  out->num_nodes = h.g.num_nodes;
  out->num_cp = h.num_cp;
  out->num_bp = h.num_bp;
  out->num_cut = h.num_cut;
  out->num_far = h.num_far;
  out->num_tiles = h.num_tiles;
  out->tile[0] = h.g.tx;
  out->tile[1] = h.g.ty;
  out->tile[2] = h.g.tz;
  out->max_delta_over_h = h.max_delta_over_h;
  out->min_abs_psi = h.min_abs_psi;
  out->min_dominance_margin = h.min_margin;
  out->num_rbf = h.num_rbf;
  out->num_rbf_rotated = h.num_rbf_rot;
  return EB_OK;
}

int eb_rbf_cuts(const eb_handle* eb, int32_t* cut_index_dev, double* xg2_dev, double* weights_dev,
                int32_t* rotated_dev, cudaStream_t stream) {
  if (!eb) {
    set_error("eb_rbf_cuts: NULL handle");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    const EBHandle& h = eb->h;
    const size_t n = (size_t)h.num_rbf;
    if (n == 0) return;
    if (cut_index_dev) EB_CUDA(cudaMemcpyAsync(cut_index_dev, h.rbf_cut, 4 * n, cudaMemcpyDeviceToDevice, stream));
    if (xg2_dev) EB_CUDA(cudaMemcpyAsync(xg2_dev, h.rbf_xg2, 16 * n, cudaMemcpyDeviceToDevice, stream));
    if (weights_dev) EB_CUDA(cudaMemcpyAsync(weights_dev, h.rbf_w, 24 * n, cudaMemcpyDeviceToDevice, stream));
    if (rotated_dev) EB_CUDA(cudaMemcpyAsync(rotated_dev, h.rbf_rot, 4 * n, cudaMemcpyDeviceToDevice, stream));
  });
}

// the public code bytes: the internal CODE_DIAG flag of CPs cleared
__global__ void k_public_codes(int64_t n, const uint8_t* in, uint8_t* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const uint8_t c = in[i];
    out[i] = (c & CODE_CP) ? (uint8_t)(c & ~CODE_DIAG) : c;
  }
}

int eb_classes(const eb_handle* eb, uint8_t* code_dev, cudaStream_t stream) {
  if (!eb || !code_dev) {
    set_error("eb_classes: NULL argument");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    if (eb->h.has_beta()) {
      k_public_codes<<<blocks_for(eb->h.g.num_nodes, 256), 256, 0, stream>>>(eb->h.g.num_nodes, eb->h.code, code_dev);
      EB_CUDA(cudaGetLastError());
    } else {
      EB_CUDA(cudaMemcpyAsync(code_dev, eb->h.code, eb->h.g.num_nodes, cudaMemcpyDeviceToDevice, stream));
    }
  });
}

int eb_set_beta(eb_handle* eb, const double* beta_x_dev, const double* beta_y_dev, const double* beta_z_dev,
                cudaStream_t stream) {
  if (!eb) {
    set_error("eb_set_beta: NULL handle");
    return EB_ERR_INVALID;
  }
  const double* b[3] = {beta_x_dev, beta_y_dev, beta_z_dev};
  return guarded([&] { set_beta(eb->h, b, stream); });
}

__global__ void k_gather_diag(const int32_t* cp_node, const double* diag, int64_t n, double* out) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = diag[cp_node[k]];
}

int eb_cp_data(const eb_handle* eb, int32_t* cp_node_dev, double* diag_dev, cudaStream_t stream) {
  if (!eb) {
    set_error("eb_cp_data: NULL handle");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    const EBHandle& h = eb->h;
    if (cp_node_dev)
      EB_CUDA(cudaMemcpyAsync(cp_node_dev, h.cp_node, sizeof(int32_t) * h.num_cp, cudaMemcpyDeviceToDevice, stream));
    if (diag_dev) {
      k_gather_diag<<<blocks_for(h.num_cp, 256), 256, 0, stream>>>(h.cp_node, h.diag, h.num_cp, diag_dev);
      EB_CUDA(cudaGetLastError());
    }
  });
}

int eb_cuts(const eb_handle* eb, int32_t* cut_cp_dev, int32_t* cut_dir_dev, double* delta_dev, double* xg_dev,
            cudaStream_t stream) {
  if (!eb) {
    set_error("eb_cuts: NULL handle");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    const EBHandle& h = eb->h;
    const size_t n = (size_t)h.num_cut;
    if (n == 0) return;
    if (cut_cp_dev) EB_CUDA(cudaMemcpyAsync(cut_cp_dev, h.cut_cp, 4 * n, cudaMemcpyDeviceToDevice, stream));
    if (cut_dir_dev) EB_CUDA(cudaMemcpyAsync(cut_dir_dev, h.cut_dir, 4 * n, cudaMemcpyDeviceToDevice, stream));
    if (delta_dev) EB_CUDA(cudaMemcpyAsync(delta_dev, h.cut_delta, 8 * n, cudaMemcpyDeviceToDevice, stream));
    if (xg_dev)
      EB_CUDA(cudaMemcpyAsync(xg_dev, h.cut_xg, 8 * n * h.g.dim, cudaMemcpyDeviceToDevice, stream));
  });
}

int eb_rhs(const eb_handle* eb, const double* f_dev, const double* ugamma_dev, double* b_dev, cudaStream_t stream) {
  if (!eb || !f_dev || !b_dev || (!ugamma_dev && eb->h.num_cut + eb->h.num_rbf > 0)) {
    set_error("eb_rhs: NULL argument");
    return EB_ERR_INVALID;
  }
  return guarded([&] { launch_rhs(eb->h, f_dev, ugamma_dev, b_dev, stream); });
}

int eb_apply(const eb_handle* eb, int prec, const void* x_dev, void* y_dev, cudaStream_t stream) {
  if (!eb || !x_dev || !y_dev) {
    set_error("eb_apply: NULL argument");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    switch (prec) {
      case EB_F64:
        launch_apply<double>(eb->h, (const double*)x_dev, (double*)y_dev, 0.0, stream);
        break;
      case EB_F32:
        launch_apply<float>(eb->h, (const float*)x_dev, (float*)y_dev, 0.0, stream);
        break;
      case EB_BF16:
        launch_apply<__nv_bfloat16>(eb->h, (const __nv_bfloat16*)x_dev, (__nv_bfloat16*)y_dev, 0.0, stream);
        break;
      default:
        throw Failure{EB_ERR_INVALID, "eb_apply: unknown precision"};
    }
  });
}

int wave_step(const eb_handle* eb, int prec, double dt, void* u_prev_dev, void* u_cur_dev, int nsteps,
              cudaStream_t stream) {
  if (!eb || !u_prev_dev || !u_cur_dev || nsteps < 0 || !(dt > 0.0) || u_prev_dev == u_cur_dev) {
    set_error("wave_step: invalid argument");
    return EB_ERR_INVALID;
  }
  int rc = EB_OK;
  int st = guarded([&] {
    if (prec == EB_F64)
      rc = launch_leapfrog<double>(eb->h, (double*)u_prev_dev, (double*)u_cur_dev, nsteps, dt, stream, true);
    else if (prec == EB_F32)
      rc = launch_leapfrog<float>(eb->h, (float*)u_prev_dev, (float*)u_cur_dev, nsteps, dt, stream, true);
    else
      throw Failure{EB_ERR_INVALID, "wave_step: precision must be EB_F64 or EB_F32"};
  });
  return st != EB_OK ? st : rc;
}

// ------------------------------------------------------------------ solver
int amg_setup(const eb_handle* eb, double shift, const amg_opts* opts, amg_handle** out, cudaStream_t stream) {
  if (!eb || !out || !(shift >= 0.0) || !std::isfinite(shift)) {
    set_error("amg_setup: invalid argument");
    return EB_ERR_INVALID;
  }
  *out = nullptr;
  amg_handle* a = new (std::nothrow) amg_handle();
  if (!a) {
    set_error("amg_setup: host allocation failed");
    return EB_ERR_OOM;
  }
  Solver& S = a->s;
  S.eb = const_cast<EBHandle*>(&eb->h);
  S.home = stream;
  S.shift = shift;
  amg_opts o{25, 1024, 0.02, 2, EB_F64, EB_AMG_SA, 1};
  if (opts) o = *opts;
  S.opts = o;
  int st = guarded([&] {
    EB_REQUIRE(o.max_levels >= 0 && o.max_levels <= 32, EB_ERR_INVALID, "amg_setup: max_levels out of range");
    EB_REQUIRE(o.coarse_max >= 1 && o.coarse_max <= 4096, EB_ERR_INVALID, "amg_setup: coarse_max in [1, 4096]");
    EB_REQUIRE(o.cheb_degree >= 1 && o.cheb_degree <= 8, EB_ERR_INVALID, "amg_setup: cheb_degree in [1, 8]");
    EB_REQUIRE(o.vcycle_prec == EB_F64 || o.vcycle_prec == EB_F32 || o.vcycle_prec == EB_BF16, EB_ERR_INVALID,
               "amg_setup: vcycle_prec must be EB_F64, EB_F32 or EB_BF16");
    EB_REQUIRE(o.coarsening == EB_AMG_SA || o.coarsening == EB_AMG_RS, EB_ERR_INVALID,
               "amg_setup: coarsening must be EB_AMG_SA or EB_AMG_RS");
    EB_REQUIRE(o.cycle == 1 || o.cycle == 2, EB_ERR_INVALID, "amg_setup: cycle must be 1 (V) or 2 (W)");
    auto t0 = std::chrono::steady_clock::now();
    S.alloc_work(stream);
    if (o.max_levels > 0) amg_build(S, stream);
    EB_CUDA(cudaStreamSynchronize(stream));
    S.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  });
  if (st != EB_OK) {
    amg_free(S);
    S.free_work();
    delete a;
    return st;
  }
  *out = a;
  return EB_OK;
}

void amg_destroy(amg_handle* amg) {
  if (!amg) return;
  amg_free(amg->s);
  amg->s.free_work();
  amg->s.prof_release();
  cudaStreamSynchronize(amg->s.home);
  delete amg;
}

int amg_info(const amg_handle* amg, amg_info_t* out) {
  if (!amg || !out) {
    set_error("amg_info: NULL argument");
    return EB_ERR_INVALID;
  }
  *out = amg_info_t{};
  amg_fill_info(amg->s, out);
  out->setup_ms = amg->s.setup_ms;
  return EB_OK;
}

int amg_level_copy(const amg_handle* amg, int level, int which, int32_t* rowptr_dev, int32_t* col_dev,
                   double* val_dev, cudaStream_t stream) {
  if (!amg) {
    set_error("amg_level_copy: NULL handle");
    return EB_ERR_INVALID;
  }
  return guarded([&] { amg_copy_level(amg->s, level, which, rowptr_dev, col_dev, val_dev, stream); });
}

int amg_set_outer_prec(amg_handle* amg, int prec) {
  if (!amg || (prec != EB_F64 && prec != EB_DF64)) {
    set_error("amg_set_outer_prec: NULL handle or precision other than EB_F64 / EB_DF64");
    return EB_ERR_INVALID;
  }
  amg->s.outer_default = prec;
  return EB_OK;
}

int amg_vcycle(const amg_handle* amg, const double* r_dev, double* z_dev, cudaStream_t stream) {
  if (!amg || !r_dev || !z_dev) {
    set_error("amg_vcycle: NULL argument");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    EB_REQUIRE(amg->s.H != nullptr, EB_ERR_INVALID, "amg_vcycle: handle has no hierarchy (max_levels = 0)");
    amg_vcycle_grid(const_cast<Solver&>(amg->s), r_dev, z_dev, stream);
  });
}

int pcg_solve(const amg_handle* amg, const double* b_dev, double* x_dev, double rtol, int maxit, const pcg_opts* opts,
              pcg_stats* stats, cudaStream_t stream) {
  if (!amg || !b_dev || !x_dev) {
    set_error("pcg_solve: NULL argument");
    return EB_ERR_INVALID;
  }
  pcg_opts o{amg->s.H ? EB_PC_AMG : EB_PC_JACOBI, 1, 1, 0, amg->s.default_outer()};
  if (opts) o = *opts;
  int rc = EB_OK;
  int st = guarded([&] { rc = const_cast<Solver&>(amg->s).pcg(b_dev, x_dev, rtol, maxit, o, stats, stream); });
  return st != EB_OK ? st : rc;
}

int wave_theta_step(const amg_handle* amg, double dt, double theta, double* u_prev_dev, double* u_cur_dev,
                    int nsteps, double rtol, int maxit, pcg_stats* stats, cudaStream_t stream) {
  if (!amg || !u_prev_dev || !u_cur_dev || u_prev_dev == u_cur_dev) {
    set_error("wave_theta_step: NULL or aliased argument");
    return EB_ERR_INVALID;
  }
  int rc = EB_OK;
  int st = guarded([&] {
    rc = const_cast<Solver&>(amg->s).wave_theta(dt, theta, u_prev_dev, u_cur_dev, nsteps, rtol, maxit, stats, stream);
  });
  return st != EB_OK ? st : rc;
}

int heat_step(const amg_handle* amg, double dt, double theta, const double* b1_dev, const double* b0_dev,
              double* u_dev, double rtol, int maxit, pcg_stats* stats, cudaStream_t stream) {
  if (!amg || !b1_dev || !u_dev) {
    set_error("heat_step: NULL argument");
    return EB_ERR_INVALID;
  }
  int rc = EB_OK;
  int st = guarded([&] {
    rc = const_cast<Solver&>(amg->s).heat(dt, theta, b1_dev, b0_dev, u_dev, rtol, maxit, stats, stream);
  });
  return st != EB_OK ? st : rc;
}

}  // extern "C"
