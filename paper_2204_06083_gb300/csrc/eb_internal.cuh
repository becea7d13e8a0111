// Internal declarations of the EB library (sm_103a).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <cstdio>
#include <functional>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/eb.h"
#include "tiles.cuh"

namespace ebk {

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
const char* last_error();

struct Failure {
  int code;
  std::string msg;
};

#define EB_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      throw ::ebk::Failure{EB_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

#define EB_REQUIRE(cond, code, msg)                   \
  do {                                                \
    if (!(cond)) throw ::ebk::Failure{(code), (msg)}; \
  } while (0)

// Runs body, translating Failure / std exceptions into a status code.
template <class F>
int guarded(F&& body) {
  try {
    body();
    return EB_OK;
  } catch (const Failure& f) {
    set_error(f.msg);
    return f.code;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return EB_ERR_OOM;
  } catch (...) {
    set_error("unexpected internal error");
    return EB_ERR_INVALID;
  }
}

// Device allocation that reports EB_ERR_OOM.
template <class T>
T* dalloc(size_t count, cudaStream_t s, bool zero = true) {
  if (count == 0) count = 1;
  void* p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, count * sizeof(T), s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Failure{EB_ERR_OOM, std::string("device allocation of ") + std::to_string(count * sizeof(T)) +
                                  " bytes failed: " + cudaGetErrorString(e)};
  }
  if (zero) EB_CUDA(cudaMemsetAsync(p, 0, count * sizeof(T), s));
  return static_cast<T*>(p);
}

template <class T>
void dfree(T*& p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
  p = nullptr;
}

// ------------------------------------------------------------- node codes
constexpr uint8_t CODE_OUT = 0x00;
constexpr uint8_t CODE_BP = 0x40;
constexpr uint8_t CODE_CP = 0x80;   // | mask of BP-neighbour directions
// set on every CP once a variable beta is given: D_k is then read from the
// diagonal array at every CP (interior CPs no longer have D = 2 dim)
constexpr uint8_t CODE_DIAG = 0x40;

// --------------------------------------------------------------- geometry
struct Geometry {
  int dim;
  int n0, n1, n2;
  int64_t num_nodes;
  double lo[3];
  double h;
  int tx, ty, tz;          // tile extents (nodes)
  int ntx, nty, ntz;       // tiles per axis
};

// ------------------------------------------------------------------ handle
// CUDA graph of CHUNK consecutive leapfrog launches, cached per handle for
// the fields, precision, dt and tile list it was built with
struct LeapfrogGraph {
  static constexpr int CHUNK = 32;  // even: a chunk leaves the roles of the two fields unchanged
  cudaGraphExec_t exec = nullptr;
  const void* ua = nullptr;
  const void* ub = nullptr;
  int prec = -1, tile_gen = -1;
  double c2 = 0.0;
  void release();
};

struct EBHandle {
  Geometry g;
  eb_levelset ls;
  int64_t num_cp = 0, num_bp = 0, num_cut = 0, num_far = 0, num_tiles = 0;
  double max_delta_over_h = 0.0, min_abs_psi = 0.0, min_margin = 0.0;
  uint8_t* code = nullptr;       // [num_nodes]
  double* diag = nullptr;        // [num_nodes] D_k (h^2 units) at CPs, 0 elsewhere
  float* diag32 = nullptr;       // [num_nodes] FP32 copy for the FP32 / BF16 kernels
  int32_t* cp_of_node = nullptr; // [num_nodes]
  int32_t* cp_node = nullptr;    // [num_cp]
  int32_t* tiles = nullptr;      // [num_tiles] linear tile index, ascending
  int32_t* tile_base = nullptr;  // [num_tiles] corner node of each listed tile
  int32_t* tile_lim = nullptr;   // [num_tiles] extents x | y << 8 | z << 16
  double2* tile_shift64 = nullptr;  // batched view only: per-tile (sigma, 1 / (sigma + 2 dim))
  float2* tile_shift32 = nullptr;
  int tile_gen = 0;  // bumped whenever the tile list is rebuilt (captured graphs key on it)
  // node pairs of the tile view holding a CP (rebuilt with the tiles; single
  // grids only): the PCG's FP64 update kernels run over these
  int32_t* pair_node = nullptr;
  int64_t num_pairs = 0;
  PairList pairs() const { return PairList{pair_node, num_pairs}; }
  TileView tv() const {
    TileView v{tile_base, tile_lim, num_tiles, g.n0, g.n0 * g.n1, (int32_t)g.num_nodes, tile_shift64, tile_shift32};
    v.bx = ilog2(g.tx);
    v.by = ilog2(g.ty);
    v.pair_node = pair_node;
    v.npairs = num_pairs;
    for (int a = 0; a < 3; ++a) {
      v.beta64[a] = beta64[a];
      v.beta32[a] = beta32[a];
    }
    return v;
  }
  // variable beta (eq. 3): null for beta = 1
  double* beta64[3] = {nullptr, nullptr, nullptr};
  float* beta32[3] = {nullptr, nullptr, nullptr};
  double* cut_bc = nullptr;      // [num_cut] beta of the cut's half point times c_s (the diagonal's terms)
  // RBF closure (Sec. 2.2) of the mixed / RBF-based methods: null for the line-by-line closure
  int closure = EB_CLOSURE_LINE;
  int64_t num_rbf = 0, num_rbf_rot = 0;
  int32_t* rbf_cut = nullptr;    // [num_rbf] the cuts closed by RBF interpolation (ascending)
  int32_t* cut_rbf = nullptr;    // [num_cut] index in rbf_cut, -1 for line-by-line cuts
  double* rbf_xg2 = nullptr;     // [num_rbf x 2] second boundary point G2
  double* rbf_w = nullptr;       // [num_rbf x 3] weights (w_ij, w_1, w_2)
  int32_t* rbf_rot = nullptr;    // [num_rbf] G2 from Algorithm 2's rotated line
  double* cut_w1 = nullptr;      // [num_cut] right-hand-side weight of the first value (c_s on line cuts)
  double* cut_bw1 = nullptr;     // [num_cut] beta times cut_w1 (variable beta with RBF cuts)
  double* rbf_bw2 = nullptr;     // [num_rbf] beta times w_2
  bool has_beta() const { return beta64[0] != nullptr; }
  static int ilog2(int v) {
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
  }
  int32_t* cut_cp = nullptr;     // [num_cut]
  int32_t* cut_dir = nullptr;    // [num_cut]
  double* cut_delta = nullptr;   // [num_cut]
  double* cut_c = nullptr;       // [num_cut]
  double* cut_xg = nullptr;      // [num_cut * dim]
  int32_t* cut_off = nullptr;    // [num_cp + 1] first cut of CP k
  cudaStream_t home = 0;
  mutable LeapfrogGraph lf_graph;
};

}  // namespace ebk

// the opaque handle of the C ABI
struct eb_handle {
  ebk::EBHandle h;
};

namespace ebk {

// D_k array matching a kernel's element type: FP64 kernels read the FP64
// diagonal, FP32 / BF16 kernels its FP32 copy (no FP64 instruction in them)
template <class T>
struct DiagOf {
  using type = float;
};
template <>
struct DiagOf<double> {
  using type = double;
};
template <class T>
inline const typename DiagOf<T>::type* diag_of(const EBHandle& eb) {
  return eb.diag32;
}
template <>
inline const double* diag_of<double>(const EBHandle& eb) {
  return eb.diag;
}

// Calls f(std::integral_constant<int, D>{}) with the DIM template argument of
// the grid kernels for eb: its dimension, with DIM_VB added when the grid has
// a variable beta (the kernels then instantiate the weighted stencil).
template <class F>
inline void dim_dispatch(const EBHandle& eb, F&& f) {
  const bool vb = eb.has_beta();
  if (eb.g.dim == 2) {
    if (vb) f(std::integral_constant<int, 2 | DIM_VB>{});
    else f(std::integral_constant<int, 2>{});
  } else {
    if (vb) f(std::integral_constant<int, 3 | DIM_VB>{});
    else f(std::integral_constant<int, 3>{});
  }
}

// ----------------------------------------------------------- build / apply
void build_handle(EBHandle& eb, const eb_grid& grid, const eb_levelset& ls, cudaStream_t s,
                  const eb_build_opts* opts = nullptr);
void destroy_handle(EBHandle& eb);

// y = (sigma I + A) x at the CPs, 0 at the other node of a pair holding a CP
// (the CP pair list), every other node untouched.
template <class T>
void launch_apply(const EBHandle& eb, const T* x, T* y, double sigma, cudaStream_t s);

void launch_rhs(const EBHandle& eb, const double* f, const double* ug, double* b, cudaStream_t s);
// variable beta of eq. 3 (device arrays, one per axis, beta at node + h/2 e_a)
void set_beta(EBHandle& eb, const double* const* beta, cudaStream_t s);

// Scans: exclusive prefix sum of n int32 values into out (out[n] = total).
void exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s);
int64_t scan_total(const int32_t* out, int64_t n, cudaStream_t s);

// --------------------------------------------------------- launch helpers
inline int num_sms() {
  static int v = 0;
  if (!v) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (v <= 0) v = 1;
  }
  return v;
}

// CTAs for a grid-stride loop over the active tiles (8 resident per SM)
inline unsigned tile_grid(const EBHandle& eb, int per_sm = 8) {
  int64_t b = eb.num_tiles < (int64_t)num_sms() * per_sm ? eb.num_tiles : (int64_t)num_sms() * per_sm;
  return (unsigned)(b < 1 ? 1 : b);
}

inline unsigned blocks_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > (int64_t)1 << 30) b = (int64_t)1 << 30;
  return (unsigned)b;
}

}  // namespace ebk

namespace ebk {
// Rebuilds the list of active tiles of eb for tiles of tx x ty x tz nodes
// (powers of two, product 256, tx >= 2, tz = 1 in 2D); bumps eb.tile_gen.
void build_tiles(EBHandle& eb, int tx, int ty, int tz, cudaStream_t s);
void build_cp_pairs(EBHandle& eb, cudaStream_t s);
// whether (tx, ty, tz) is a valid tile shape for dim
bool tile_shape_ok(int dim, int tx, int ty, int tz);
// tile-shape autotuner (autotune.cu): candidate shapes, event timing of an
// operation on a stream, and the tuning loop (retile, time, keep the fastest)
struct TileDims {
  int x, y, z;
};
std::vector<TileDims> tile_candidates(int dim);
double time_us(const std::function<void()>& op, int reps, cudaStream_t s);
void run_tuner(int dim, const std::function<void(const TileDims&)>& retile, const std::function<void()>& op,
               int reps, eb_tune_t* out, cudaStream_t s);
template <class T>
int launch_leapfrog(const EBHandle& eb, T* ua, T* ub, int nsteps, double dt, cudaStream_t s, bool use_graph);
}
