// AMG hierarchy storage shared by the setup (amg.cu) and the V-cycle
// (amg_vcycle.cu).
#pragma once

#include <vector>

#include "eb_solver.cuh"

namespace ebk {

struct DCsr {
  int64_t n = 0, m = 0, nnz = 0;
  int32_t* rp = nullptr;
  int32_t* ci = nullptr;
  double* v = nullptr;
};

inline void csr_free(DCsr& A, cudaStream_t s) {
  dfree(A.rp, s);
  dfree(A.ci, s);
  dfree(A.v, s);
  A.n = A.m = A.nnz = 0;
}

// V-cycle vectors of one level in the storage type V
template <class V>
struct VecSet {
  V *b = nullptr, *x = nullptr, *x2 = nullptr, *d = nullptr, *r = nullptr;
};

struct Level {
  DCsr A, P, R;               // FP64 hierarchy (exact setup)
  int32_t* R0node = nullptr;  // level 0 only: R's columns as grid node indices
  int32_t* agg = nullptr;
  double* dinv = nullptr;     // compact levels
  double rho = 0.0;
  VecSet<double> v64;
  VecSet<float> v32;
  VecSet<__nv_bfloat16> v16;
  // FP32 / BF16 copies of the values for the reduced-precision V-cycles
  float *A32 = nullptr, *P32 = nullptr, *R32 = nullptr, *dinv32 = nullptr;
  __nv_bfloat16 *A16 = nullptr, *P16 = nullptr, *R16 = nullptr, *dinv16 = nullptr;
};

// Level-0 prolongation applied matrix free (single grids): with
// P = (I - omega D^-1 A) P_hat, x += P e is one stencil pass over the tiles on
// t = P_hat e, t_j = e[agg(j)] / sqrt(|agg(j)|).
struct MatrixFreeP {
  bool on = false;
  double omega = 0.0;             // 4 / (3 rho_0)
  int32_t* agg_node = nullptr;    // [num_nodes] aggregate of a CP node, -1 elsewhere
  double* sc64 = nullptr;         // [nc] P_hat value of aggregate c: 1 / sqrt(|c|)
  float* sc32 = nullptr;
  int64_t nc = 0;
};

struct Hierarchy {
  std::vector<Level> L;
  double* coarse_inv = nullptr;  // FP64 inverse of the coarsest matrix
  int64_t nc = 0;
  MatrixFreeP mf;
  VecSet<double> g64;            // level-0 grid vectors (full grid)
  VecSet<float> g32;
  VecSet<__nv_bfloat16> g16;
};

DCsr level0_csr(const EBHandle& eb, double sigma, cudaStream_t s);
void amg_build_from(Solver& S, DCsr A0, cudaStream_t s);
void amg_alloc_vcycle(Solver& S, cudaStream_t s);
void amg_free_vcycle(Hierarchy& H, cudaStream_t s);

}  // namespace ebk
