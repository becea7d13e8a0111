// Internal solver state: PCG scalars, work vectors and the AMG hierarchy.
#pragma once

#include "eb_internal.cuh"

namespace ebk {

enum { FIN_INIT = 0, FIN_RZ0 = 1, FIN_ALPHA = 2, FIN_RR = 3, FIN_BETA = 4 };
enum { PCG_FLAG_NONFINITE = 1, PCG_FLAG_BREAKDOWN = 2 };

struct PcgScalars {
  double bb, rr, rz, pq, alpha, beta, tol2;
  int iters, flags, done, pad;
};

struct Hierarchy;  // AMG levels (amg.cu)

struct Solver {
  EBHandle* eb = nullptr;
  double shift = 0.0;
  amg_opts opts{};
  Hierarchy* H = nullptr;
  double setup_ms = 0.0;
  // full-grid work vectors
  double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *tmp = nullptr, *dinv = nullptr;
  double* part = nullptr;
  int nblk = 1;
  PcgScalars* sc = nullptr;
  PcgScalars* sc_host = nullptr;

  void alloc_work(cudaStream_t s);
  void free_work();
  void finalize(int op, cudaStream_t s);
  void precondition(int kind, const double* r, double* z, cudaStream_t s);
  int pcg(const double* b, double* x, double rtol, int maxit, const pcg_opts& o, pcg_stats* stats, cudaStream_t s);
  int heat(double dt, double theta, const double* b1, const double* b0, double* u, double rtol, int maxit,
           pcg_stats* stats, cudaStream_t s);
};

// AMG (amg.cu)
void amg_build(Solver& S, cudaStream_t s);
void amg_free(Solver& S);
void amg_vcycle_grid(Solver& S, const double* r, double* z, cudaStream_t s);
void amg_fill_info(const Solver& S, amg_info_t* out);
void amg_copy_level(const Solver& S, int level, int which, int32_t* rowptr, int32_t* col, double* val, cudaStream_t s);

}  // namespace ebk
