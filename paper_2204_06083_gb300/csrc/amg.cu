// Smoothed-aggregation AMG on the device: setup and V-cycle.
//
// The paper preconditions CG with a library AMG (Sec. 3, first paragraph) and
// fixes none of its parameters; the hierarchy built here is deterministic so
// that it can be checked against an independent sequential implementation:
//   strength   |a_ij| >= theta sqrt(a_ii a_jj)
//   MIS-2      synchronous rounds; key (state << 62 | lowbias32(i) << 30 | i),
//              state 2 root / 1 undecided / 0 removed; closed-neighbourhood
//              maximum taken twice; a node whose distance-2 maximum is itself
//              becomes a root, one that sees a root becomes removed
//   aggregates roots numbered in index order; strong root neighbour first, then
//              the strongest strong neighbour assigned in that first pass
//              (ties to the lowest aggregate id)
//   P          (I - omega D^-1 A) P_hat, omega = 4 / (3 rho), rho the
//              Gershgorin bound of D^-1 A; P_hat the normalised constant
//              vector of each aggregate
//   A_c        P^T A P, sparsity = the symbolic product (cancellations kept)
//   coarsest   explicit inverse by a Gauss-Jordan sweep (A_c is SPD, no pivoting)
//   smoother   Chebyshev of degree k for D^-1 A on [rho/30, 1.1 rho], one
//              sweep before and after the coarse correction
//
// SpGEMM C = A B: one warp per row of C.  The output pattern of a row is a
// bitmap over the column range of its products (sorted order for free); the
// values are accumulated k by k in the order of A's row, the lanes handling the
// distinct columns of row k of B, so every entry of C is the sum of its
// products in ascending k -- the summation order of a sequential row-by-row
// product.
#include "eb_solver.cuh"
#include "stencil.cuh"

#include <algorithm>
#include <cmath>

#include "amg_internal.cuh"

namespace ebk {

// ------------------------------------------------------------ level 0 CSR
__global__ void k_l0_count(Geometry G, const int32_t* cp_node, const uint8_t* code, int64_t ncp, int32_t* cnt) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ncp) return;
  uint8_t m = code[cp_node[k]] & 0x3F;
  cnt[k] = 1 + 2 * G.dim - __popc((unsigned)m);
}

// beta pointers of a variable-coefficient grid (all null for beta = 1)
struct BetaArgs {
  const double* b[3];
};

__global__ void k_l0_fill(Geometry G, const int32_t* cp_node, const int32_t* cp_of_node, const uint8_t* code,
                          const double* diag, int64_t ncp, double sigma, const int32_t* rp, int32_t* ci, double* v,
                          BetaArgs beta) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ncp) return;
  const int64_t node = cp_node[k];
  const uint8_t c = code[node];
  const uint8_t m = c & 0x3F;
  const double h2 = __dmul_rn(G.h, G.h);
  const double off = __ddiv_rn(-1.0, h2);
  const int64_t st[3] = {1, (int64_t)G.n0, (int64_t)G.n0 * G.n1};
  int32_t e = rp[k];
  // neighbours in ascending node order: -z, -y, -x, self, +x, +y, +z; with a
  // variable beta the coupling is -beta(half point) / h^2 (eq. 3)
  for (int a = G.dim - 1; a >= 0; --a)
    if (!(m & (1u << (2 * a)))) {
      ci[e] = cp_of_node[node - st[a]];
      v[e++] = beta.b[0] ? __ddiv_rn(-beta.b[a][node - st[a]], h2) : off;
    }
  const double D = (c & 0x7F) ? diag[node] : (double)(2 * G.dim);
  ci[e] = (int32_t)k;
  v[e++] = sigma == 0.0 ? __ddiv_rn(D, h2) : __dadd_rn(__ddiv_rn(D, h2), sigma);
  for (int a = 0; a < G.dim; ++a)
    if (!(m & (1u << (2 * a + 1)))) {
      ci[e] = cp_of_node[node + st[a]];
      v[e++] = beta.b[0] ? __ddiv_rn(-beta.b[a][node], h2) : off;
    }
}

// -------------------------------------------------------- row information
__global__ void k_rowinfo(DCsr A, double* d, double* dinv, double* rho_max) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double ratio = 0.0;
  if (i < A.n) {
    double s = 0.0, di = 0.0;
    for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e) {
      double v = A.v[e];
      s = (e == A.rp[i]) ? fabs(v) : __dadd_rn(s, fabs(v));
      if (A.ci[e] == i) di = v;
    }
    d[i] = di;
    dinv[i] = __ddiv_rn(1.0, di);
    ratio = __ddiv_rn(s, di);
    if (!(ratio >= 0.0)) ratio = 1e300;
  }
  for (int o = 16; o > 0; o >>= 1) ratio = fmax(ratio, __shfl_xor_sync(0xffffffffu, ratio, o));
  if ((threadIdx.x & 31) == 0)
    atomicMax(reinterpret_cast<unsigned long long*>(rho_max), (unsigned long long)__double_as_longlong(ratio));
}

__global__ void k_strength(DCsr A, const double* d, double theta, uint8_t* strong) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const double di = d[i];
  for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e) {
    int32_t j = A.ci[e];
    strong[e] = (j != i) && (fabs(A.v[e]) >= __dmul_rn(theta, __dsqrt_rn(__dmul_rn(di, d[j]))));
  }
}

// ------------------------------------------------------------------ MIS-2
__device__ __forceinline__ uint32_t lowbias32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

__device__ __forceinline__ uint64_t mis_key(uint8_t state, int64_t i) {
  return ((uint64_t)state << 62) | ((uint64_t)lowbias32((uint32_t)i) << 30) | (uint64_t)i;
}

__global__ void k_mis_max1(DCsr A, const uint8_t* strong, const uint8_t* state, uint64_t* k1) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  uint64_t m = mis_key(state[i], i);
  for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e)
    if (strong[e]) {
      int32_t j = A.ci[e];
      uint64_t kj = mis_key(state[j], j);
      m = kj > m ? kj : m;
    }
  k1[i] = m;
}

__global__ void k_mis_max2(DCsr A, const uint8_t* strong, const uint64_t* k1, uint8_t* state, int* undecided) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int und = 0;
  if (i < A.n) {
    uint64_t m = k1[i];
    for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e)
      if (strong[e]) {
        uint64_t kj = k1[A.ci[e]];
        m = kj > m ? kj : m;
      }
    if (state[i] == 1) {
      if ((m & ((1ull << 30) - 1)) == (uint64_t)i)
        state[i] = 2;
      else if ((m >> 62) == 2)
        state[i] = 0;
      else
        und = 1;
    }
  }
  unsigned bal = __ballot_sync(0xffffffffu, und);
  if ((threadIdx.x & 31) == 0 && bal) atomicAdd(undecided, __popc(bal));
}

__global__ void k_is_root(int64_t n, const uint8_t* state, int32_t* flag) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = state[i] == 2;
}

__global__ void k_agg_pass1(DCsr A, const uint8_t* strong, const uint8_t* state, const int32_t* root_off,
                            int32_t* agg1) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  int32_t a = -1;
  if (state[i] == 2) {
    a = root_off[i];
  } else {
    for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e)
      if (strong[e] && state[A.ci[e]] == 2) {
        a = root_off[A.ci[e]];
        break;
      }
  }
  agg1[i] = a;
}

__global__ void k_agg_pass2(DCsr A, const uint8_t* strong, const int32_t* agg1, int32_t* agg, int* unassigned) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  int32_t a = agg1[i];
  if (a < 0) {
    // weights compared rounded to single precision, ties to the lowest id
    float bw = -1.0f;
    int32_t ba = -1;
    for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e) {
      if (!strong[e]) continue;
      int32_t c = agg1[A.ci[e]];
      if (c < 0) continue;
      float w = __double2float_rn(fabs(A.v[e]));
      if (w > bw || (w == bw && c < ba)) {
        bw = w;
        ba = c;
      }
    }
    a = ba;
    if (a < 0) atomicAdd(unassigned, 1);
  }
  agg[i] = a;
}

// ------------------------------------------------- classical (RS) coarsening
// Strength, PMIS splitting and direct interpolation of the classical method
// (the specification the sequential reference implementation states in its
// header): S_i = {j != i : -a_ij >= 0.25 max_k(-a_ik)}, compared in single
// precision; lambda_i = |S_i^T|; key (lambda << 32 | lowbias32(i)).
constexpr double RS_THETA = 0.25;

__global__ void k_rs_strength(DCsr A, uint8_t* strong) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  double m = -INFINITY;
  for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e)
    if (A.ci[e] != i) m = fmax(m, -A.v[e]);
  const float thr = __double2float_rn(__dmul_rn(RS_THETA, m));
  for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e)
    strong[e] = (A.ci[e] != i) && m > 0.0 && __double2float_rn(-A.v[e]) >= thr;
}

// strongT[e] for entry e = (i, j): whether i is in S_j (the strength flag of
// the transposed entry (j, i), found by binary search in row j; the pattern of
// every level is symmetric); lambda_i = sum over row i of strongT
__global__ void k_rs_transpose(DCsr A, const uint8_t* strong, uint8_t* strongT, int32_t* lambda) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  int32_t lam = 0;
  for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e) {
    const int32_t j = A.ci[e];
    uint8_t t = 0;
    if (j != i) {
      int32_t lo = A.rp[j], hi = A.rp[j + 1];
      while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (A.ci[mid] < i) lo = mid + 1;
        else hi = mid;
      }
      if (lo < A.rp[j + 1] && A.ci[lo] == i) t = strong[lo];
    }
    strongT[e] = t;
    lam += t;
  }
  lambda[i] = lam;
}

__device__ __forceinline__ uint64_t rs_key(int32_t lam, int64_t i) {
  return ((uint64_t)(uint32_t)lam << 32) | (uint64_t)lowbias32((uint32_t)i);
}

// state: -1 undecided, 1 C, 0 F; points no one depends on start as F
__global__ void k_rs_init(int64_t n, const int32_t* lambda, int8_t* state) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) state[i] = lambda[i] == 0 ? 0 : -1;
}

// a PMIS round, part 1: undecided i whose key exceeds those of all undecided
// strong neighbours (either direction) is marked for C (state unchanged)
__global__ void k_rs_select(DCsr A, const uint8_t* strong, const uint8_t* strongT, const int32_t* lambda,
                            const int8_t* state, uint8_t* newc) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  uint8_t c = 0;
  if (state[i] < 0) {
    const uint64_t ki = rs_key(lambda[i], i);
    c = 1;
    for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e) {
      const int32_t j = A.ci[e];
      if (j == i || !(strong[e] || strongT[e]) || state[j] >= 0) continue;
      if (rs_key(lambda[j], j) > ki) {
        c = 0;
        break;
      }
    }
  }
  newc[i] = c;
}

__global__ void k_rs_apply(int64_t n, const uint8_t* newc, int8_t* state) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && newc[i]) state[i] = 1;
}

// part 2: undecided points with a C point in their S become F; counts the
// points still undecided
__global__ void k_rs_fassign(DCsr A, const uint8_t* strong, int8_t* state, int* undecided) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int und = 0;
  if (i < A.n && state[i] < 0) {
    bool dep = false;
    for (int32_t e = A.rp[i]; e < A.rp[i + 1] && !dep; ++e) dep = strong[e] && state[A.ci[e]] == 1;
    if (dep) state[i] = 0;
    else und = 1;
  }
  unsigned bal = __ballot_sync(0xffffffffu, und);
  if ((threadIdx.x & 31) == 0 && bal) atomicAdd(undecided, __popc(bal));
}

__global__ void k_rs_cflag(int64_t n, const int8_t* state, int32_t* flag) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = state[i] == 1;
}

// entries of P's row i: 1 for a C point, its strong C neighbours for an F point
__global__ void k_rs_pcount(DCsr A, const uint8_t* strong, const int8_t* state, int32_t* cnt) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  int32_t c = 0;
  if (state[i] == 1) {
    c = 1;
  } else {
    for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e) c += strong[e] && state[A.ci[e]] == 1;
  }
  cnt[i] = c;
}

// direct interpolation (the sums in the row's column order, as the sequential
// definition); agg records the coarse index of C points, -1 for F points
__global__ void k_rs_pfill(DCsr A, const uint8_t* strong, const int8_t* state, const int32_t* cidx, DCsr P,
                           int32_t* agg) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  int32_t o = P.rp[i];
  if (state[i] == 1) {
    P.ci[o] = cidx[i];
    P.v[o] = 1.0;
    agg[i] = cidx[i];
    return;
  }
  agg[i] = -1;
  double aii = 0.0, sneg = 0.0, spos = 0.0, pneg = 0.0, ppos = 0.0;
  for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e) {
    const int32_t j = A.ci[e];
    const double v = A.v[e];
    if (j == i) {
      aii = v;
      continue;
    }
    if (v < 0.0) sneg = __dadd_rn(sneg, v);
    else spos = __dadd_rn(spos, v);
    if (strong[e] && state[j] == 1) {
      if (v < 0.0) pneg = __dadd_rn(pneg, v);
      else ppos = __dadd_rn(ppos, v);
    }
  }
  if (ppos == 0.0) aii = __dadd_rn(aii, spos);
  const double alpha = pneg != 0.0 ? __ddiv_rn(sneg, pneg) : 0.0;
  const double beta = ppos != 0.0 ? __ddiv_rn(spos, ppos) : 0.0;
  for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e) {
    const int32_t j = A.ci[e];
    if (j == i || !(strong[e] && state[j] == 1)) continue;
    const double v = A.v[e];
    P.ci[o] = cidx[j];
    P.v[o] = __ddiv_rn(__dmul_rn(-(v < 0.0 ? alpha : beta), v), aii);
    ++o;
  }
}

__global__ void k_agg_sizes(int64_t n, const int32_t* agg, int32_t* size) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(&size[agg[i]], 1);
}

__global__ void k_phat(int64_t n, const int32_t* agg, const int32_t* size, int32_t* rp, int32_t* ci, double* v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  rp[i] = (int32_t)i;
  if (i == n) return;
  ci[i] = agg[i];
  v[i] = __ddiv_rn(1.0, __dsqrt_rn((double)size[agg[i]]));
}

// P = P_hat - omega (dinv (A P_hat)) on the pattern of A P_hat
__global__ void k_smooth_p(DCsr T, const int32_t* agg, const double* phat, const double* dinv, double omega,
                           double* pv) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= T.n) return;
  for (int32_t e = T.rp[i]; e < T.rp[i + 1]; ++e) {
    double z = __dmul_rn(omega, __dmul_rn(dinv[i], T.v[e]));
    pv[e] = (T.ci[e] == agg[i]) ? __dsub_rn(phat[i], z) : -z;
  }
}

// ------------------------------------------------------------------ SpGEMM
constexpr int SPG_WARPS = 4;
constexpr int SPG_BITS = 1 << 16;            // bitmap capacity (column range per row)
constexpr int SPG_WORDS = SPG_BITS / 32;

struct SpgSmem {
  uint32_t bits[SPG_WORDS];
  int32_t pre[SPG_WORDS];
};

// column range of the products of row i; false when the row is empty
__device__ __forceinline__ bool spg_range(const DCsr& A, const DCsr& B, int64_t i, int lane, int32_t& cmin,
                                          int32_t& cmax) {
  int32_t lo = INT32_MAX, hi = -1;
  for (int32_t e = A.rp[i] + lane; e < A.rp[i + 1]; e += 32) {
    int32_t k = A.ci[e];
    int32_t b0 = B.rp[k], b1 = B.rp[k + 1];
    if (b1 > b0) {
      lo = min(lo, B.ci[b0]);
      hi = max(hi, B.ci[b1 - 1]);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  cmin = lo;
  cmax = hi;
  return hi >= lo;
}

__device__ void spg_mark(const DCsr& A, const DCsr& B, int64_t i, int lane, int32_t cmin, int nwords,
                         uint32_t* bits) {
  for (int w = lane; w < nwords; w += 32) bits[w] = 0u;
  __syncwarp();
  for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e) {
    int32_t k = A.ci[e];
    for (int32_t f = B.rp[k] + lane; f < B.rp[k + 1]; f += 32) {
      int32_t off = B.ci[f] - cmin;
      atomicOr(&bits[off >> 5], 1u << (off & 31));
    }
  }
  __syncwarp();
}

// warp-wide exclusive prefix of popcounts over the bitmap words; returns total
__device__ int32_t spg_prefix(int lane, int nwords, const uint32_t* bits, int32_t* pre) {
  int32_t carry = 0;
  for (int w0 = 0; w0 < nwords; w0 += 32) {
    int w = w0 + lane;
    int32_t c = w < nwords ? __popc(bits[w]) : 0;
    int32_t x = c;
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (w < nwords) pre[w] = carry + x - c;
    carry += __shfl_sync(0xffffffffu, x, 31);
  }
  __syncwarp();
  return carry;
}

// phase 0: count of the output row; rows whose column range exceeds the bitmap
// are flagged
__global__ void k_spg_count(DCsr A, DCsr B, int32_t* cnt, int* overflow) {
  extern __shared__ SpgSmem sm_spg[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  SpgSmem& S = sm_spg[warp];
  for (int64_t i = (int64_t)blockIdx.x * SPG_WARPS + warp; i < A.n; i += (int64_t)gridDim.x * SPG_WARPS) {
    int32_t cmin, cmax;
    if (!spg_range(A, B, i, lane, cmin, cmax)) {
      if (lane == 0) cnt[i] = 0;
      continue;
    }
    int64_t range = (int64_t)cmax - cmin + 1;
    if (range > SPG_BITS) {
      if (lane == 0) {
        cnt[i] = 0;
        atomicAdd(overflow, 1);
      }
      continue;
    }
    int nwords = (int)((range + 31) >> 5);
    spg_mark(A, B, i, lane, cmin, nwords, S.bits);
    int32_t tot = 0;
    for (int w = lane; w < nwords; w += 32) tot += __popc(S.bits[w]);
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (lane == 0) cnt[i] = tot;
    __syncwarp();
  }
}

// phase 1: sorted columns and values of the output rows
__global__ void k_spg_fill(DCsr A, DCsr B, DCsr C) {
  extern __shared__ SpgSmem sm_spg[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  SpgSmem& S = sm_spg[warp];
  for (int64_t i = (int64_t)blockIdx.x * SPG_WARPS + warp; i < A.n; i += (int64_t)gridDim.x * SPG_WARPS) {
    int32_t cmin, cmax;
    if (!spg_range(A, B, i, lane, cmin, cmax)) continue;
    int nwords = (int)((((int64_t)cmax - cmin + 1) + 31) >> 5);
    spg_mark(A, B, i, lane, cmin, nwords, S.bits);
    spg_prefix(lane, nwords, S.bits, S.pre);
    const int32_t base = C.rp[i];
    for (int w = lane; w < nwords; w += 32) {
      uint32_t word = S.bits[w];
      int32_t p = base + S.pre[w];
      while (word) {
        int b = __ffs(word) - 1;
        word &= word - 1;
        C.ci[p] = cmin + 32 * w + b;
        C.v[p] = 0.0;
        ++p;
      }
    }
    __syncwarp();
    // values: k in the order of A's row; lanes over the distinct columns of B_k
    for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e) {
      const int32_t k = A.ci[e];
      const double a = A.v[e];
      for (int32_t f = B.rp[k] + lane; f < B.rp[k + 1]; f += 32) {
        int32_t off = B.ci[f] - cmin;
        uint32_t word = S.bits[off >> 5];
        int32_t pos = base + S.pre[off >> 5] + __popc(word & ((1u << (off & 31)) - 1u));
        C.v[pos] = __dadd_rn(C.v[pos], __dmul_rn(a, B.v[f]));
      }
      __syncwarp();
    }
  }
}

static DCsr spgemm(const DCsr& A, const DCsr& B, cudaStream_t s) {
  EB_REQUIRE(A.m == B.n, EB_ERR_INVALID, "spgemm: inner dimensions differ");
  DCsr C;
  C.n = A.n;
  C.m = B.m;
  int32_t* cnt = dalloc<int32_t>(A.n + 1, s);
  int* ovf = dalloc<int>(1, s);
  const size_t smem = sizeof(SpgSmem) * SPG_WARPS;
  static bool attr = false;
  if (!attr) {
    EB_CUDA(cudaFuncSetAttribute(k_spg_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    EB_CUDA(cudaFuncSetAttribute(k_spg_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((A.n + SPG_WARPS - 1) / SPG_WARPS,
                                                                     (int64_t)num_sms() * 16));
  k_spg_count<<<blocks, 32 * SPG_WARPS, smem, s>>>(A, B, cnt, ovf);
  EB_CUDA(cudaGetLastError());
  int hovf = 0;
  EB_CUDA(cudaMemcpyAsync(&hovf, ovf, sizeof(int), cudaMemcpyDeviceToHost, s));
  C.rp = dalloc<int32_t>(A.n + 1, s, false);
  exclusive_scan_i32(cnt, C.rp, A.n, s);
  int32_t nnz = 0;
  EB_CUDA(cudaMemcpyAsync(&nnz, C.rp + A.n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  EB_CUDA(cudaStreamSynchronize(s));
  dfree(cnt, s);
  dfree(ovf, s);
  EB_REQUIRE(hovf == 0, EB_ERR_OOM, "spgemm: a product row spans more than 65536 columns");
  C.nnz = nnz;
  C.ci = dalloc<int32_t>(nnz, s, false);
  C.v = dalloc<double>(nnz, s, false);
  k_spg_fill<<<blocks, 32 * SPG_WARPS, smem, s>>>(A, B, C);
  EB_CUDA(cudaGetLastError());
  return C;
}

// -------------------------------------------------------------- transpose
__global__ void k_tr_count(DCsr A, int32_t* cnt) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < A.nnz) atomicAdd(&cnt[A.ci[e]], 1);
}

__global__ void k_tr_scatter(DCsr A, const int32_t* rp, int32_t* fill, int32_t* ci, double* v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e) {
    int32_t c = A.ci[e];
    int32_t p = rp[c] + atomicAdd(&fill[c], 1);
    ci[p] = (int32_t)i;
    v[p] = A.v[e];
  }
}

// Sorts every row of C by column: one warp per row, bitonic sort in shared
// memory for rows of up to SORT_CAP entries (column indices are distinct), a
// serial insertion sort by lane 0 beyond.
constexpr int SORT_WARPS = 2;  // 2 x 2048 x 12 B = 48 KB of static shared memory
constexpr int SORT_CAP = 2048;

__global__ void k_row_sort(DCsr C) {
  __shared__ int32_t skey[SORT_WARPS][SORT_CAP];
  __shared__ double sval[SORT_WARPS][SORT_CAP];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t* key = skey[warp];
  double* val = sval[warp];
  for (int64_t i = (int64_t)blockIdx.x * SORT_WARPS + warp; i < C.n; i += (int64_t)gridDim.x * SORT_WARPS) {
    const int32_t b = C.rp[i], e = C.rp[i + 1], m = e - b;
    if (m <= 1) continue;
    if (m > SORT_CAP) {
      if (lane == 0) {
        for (int32_t p = b + 1; p < e; ++p) {
          const int32_t kc = C.ci[p];
          const double kv = C.v[p];
          int32_t q = p - 1;
          while (q >= b && C.ci[q] > kc) {
            C.ci[q + 1] = C.ci[q];
            C.v[q + 1] = C.v[q];
            --q;
          }
          C.ci[q + 1] = kc;
          C.v[q + 1] = kv;
        }
      }
      __syncwarp();
      continue;
    }
    int M = 1;
    while (M < m) M <<= 1;
    for (int t = lane; t < M; t += 32) {
      key[t] = t < m ? C.ci[b + t] : INT32_MAX;
      val[t] = t < m ? C.v[b + t] : 0.0;
    }
    __syncwarp();
    for (int k = 2; k <= M; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int t = lane; t < M; t += 32) {
          const int u = t ^ j;
          if (u > t) {
            const bool up = (t & k) == 0;
            const int32_t kt = key[t], ku = key[u];
            if ((kt > ku) == up) {
              key[t] = ku;
              key[u] = kt;
              const double vt = val[t];
              val[t] = val[u];
              val[u] = vt;
            }
          }
        }
        __syncwarp();
      }
    for (int t = lane; t < m; t += 32) {
      C.ci[b + t] = key[t];
      C.v[b + t] = val[t];
    }
    __syncwarp();
  }
}

static DCsr transpose(const DCsr& A, cudaStream_t s) {
  DCsr T;
  T.n = A.m;
  T.m = A.n;
  T.nnz = A.nnz;
  int32_t* cnt = dalloc<int32_t>(A.m + 1, s);
  T.rp = dalloc<int32_t>(A.m + 1, s, false);
  T.ci = dalloc<int32_t>(A.nnz, s, false);
  T.v = dalloc<double>(A.nnz, s, false);
  k_tr_count<<<blocks_for(A.nnz, 256), 256, 0, s>>>(A, cnt);
  exclusive_scan_i32(cnt, T.rp, A.m, s);
  EB_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (A.m + 1), s));
  k_tr_scatter<<<blocks_for(A.n, 256), 256, 0, s>>>(A, T.rp, cnt, T.ci, T.v);
  k_row_sort<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((T.n + SORT_WARPS - 1) / SORT_WARPS, (int64_t)num_sms() * 16)), 32 * SORT_WARPS, 0, s>>>(T);
  EB_CUDA(cudaGetLastError());
  dfree(cnt, s);
  return T;
}

// ---------------------------------------------------- coarsest: inversion
// In-place Gauss-Jordan sweep of an SPD matrix (no pivoting), one cooperative
// launch; for pivot k: save row / column k, barrier, update, barrier.
struct CoopBarrier {
  unsigned int count, gen;
  int err, pad;
};

__device__ bool coop_sync(CoopBarrier* gb) {
  __syncthreads();
  __shared__ int failed;
  if (threadIdx.x == 0) {
    failed = 0;
    volatile int* perr = &gb->err;
    if (*perr) {
      failed = 1;
    } else {
      volatile unsigned int* pgen = &gb->gen;
      unsigned int g = *pgen;
      __threadfence();
      if (atomicAdd(&gb->count, 1u) + 1u == gridDim.x) {
        gb->count = 0;
        __threadfence();
        atomicAdd(&gb->gen, 1u);
      } else {
        long long spins = 0;
        while (*pgen == g) {
          if (*perr || ++spins > 20000000LL) {
            atomicExch(&gb->err, 1);
            failed = 1;
            break;
          }
          __nanosleep(32);
        }
      }
      __threadfence();
    }
  }
  __syncthreads();
  return failed == 0;
}

__global__ void k_gauss_jordan(double* M, int n, double* rowk, double* colk, CoopBarrier* gb) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const int64_t nn = (int64_t)n * n;
  for (int k = 0; k < n; ++k) {
    for (int64_t t = tid; t < n; t += nth) {
      rowk[t] = __ldcg(M + (int64_t)k * n + t);
      colk[t] = __ldcg(M + t * n + k);
    }
    if (!coop_sync(gb)) return;
    const double p = __ldcg(rowk + k);
    const double ip = 1.0 / p;
    for (int64_t t = tid; t < nn; t += nth) {
      const int64_t i = t / n, j = t % n;
      double v;
      if (i == k && j == k)
        v = ip;
      else if (i == k)
        v = __ldcg(rowk + j) * ip;
      else if (j == k)
        v = -__ldcg(colk + i) * ip;
      else
        v = __ldcg(M + t) - __ldcg(colk + i) * __ldcg(rowk + j) * ip;
      M[t] = v;
    }
    if (!coop_sync(gb)) return;
  }
}

__global__ void k_csr_to_dense(DCsr A, double* M) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e) M[i * A.n + A.ci[e]] = A.v[e];
}

static void coarse_inverse(Hierarchy& H, const DCsr& A, cudaStream_t s) {
  const int n = (int)A.n;
  H.nc = n;
  H.coarse_inv = dalloc<double>((int64_t)n * n, s);
  k_csr_to_dense<<<blocks_for(n, 128), 128, 0, s>>>(A, H.coarse_inv);
  double* rowk = dalloc<double>(n, s);
  double* colk = dalloc<double>(n, s);
  CoopBarrier* gb = dalloc<CoopBarrier>(1, s);
  int per_sm = 0;
  EB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gauss_jordan, 256, 0));
  EB_REQUIRE(per_sm > 0, EB_ERR_INVALID, "coarse inverse kernel cannot be resident");
  int64_t want = ((int64_t)n * n + 255) / 256;
  unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms() * std::min(per_sm, 2)));
  double* M = H.coarse_inv;
  int nn = n;
  void* args[] = {(void*)&M, (void*)&nn, (void*)&rowk, (void*)&colk, (void*)&gb};
  EB_CUDA(cudaLaunchCooperativeKernel((void*)k_gauss_jordan, dim3(blocks), dim3(256), args, 0, s));
  CoopBarrier hb{};
  EB_CUDA(cudaMemcpyAsync(&hb, gb, sizeof(hb), cudaMemcpyDeviceToHost, s));
  EB_CUDA(cudaStreamSynchronize(s));
  dfree(rowk, s);
  dfree(colk, s);
  dfree(gb, s);
  EB_REQUIRE(hb.err == 0, EB_ERR_TIMEOUT, "coarse inverse: grid barrier timed out");
}

// ------------------------------------------------------------------ setup
__global__ void k_map_cols(int64_t nnz, const int32_t* ci, const int32_t* map, int32_t* out) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nnz) out[e] = map[ci[e]];
}

// ---------------------------------------- matrix-free level-0 prolongation data
__global__ void k_agg_node(int64_t ncp, const int32_t* cp_node, const int32_t* agg, int32_t* agg_node) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < ncp) agg_node[cp_node[k]] = agg[k];
}

__global__ void k_agg_scale(int64_t nc, const int32_t* size, double* sc64, float* sc32) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const double v = __ddiv_rn(1.0, __dsqrt_rn((double)size[c]));  // the P_hat value of k_phat
  sc64[c] = v;
  sc32[c] = (float)v;
}

static void build_mf(MatrixFreeP& M, const EBHandle& eb, const Level& L0, int32_t nc, const int32_t* size,
                     cudaStream_t s) {
  const int64_t ncp = eb.num_cp, nn = eb.g.num_nodes;
  M.omega = 4.0 / (3.0 * L0.rho);
  M.nc = nc;
  M.agg_node = dalloc<int32_t>(nn, s, false);
  EB_CUDA(cudaMemsetAsync(M.agg_node, 0xFF, sizeof(int32_t) * nn, s));
  k_agg_node<<<blocks_for(ncp, 256), 256, 0, s>>>(ncp, eb.cp_node, L0.agg, M.agg_node);
  M.sc64 = dalloc<double>(nc, s, false);
  M.sc32 = dalloc<float>(nc, s, false);
  k_agg_scale<<<blocks_for(nc, 256), 256, 0, s>>>(nc, size, M.sc64, M.sc32);
  EB_CUDA(cudaGetLastError());
  M.on = true;
}

static void free_mf(MatrixFreeP& M, cudaStream_t s) {
  dfree(M.agg_node, s); dfree(M.sc64, s); dfree(M.sc32, s);
  M.on = false;
}

// level-0 matrix sigma I + A over the CPs of one grid, in CSR
DCsr level0_csr(const EBHandle& eb, double sigma, cudaStream_t s) {
  const Geometry& G = eb.g;
  const int64_t ncp = eb.num_cp;
  DCsr A0;
  A0.n = A0.m = ncp;
  int32_t* cnt = dalloc<int32_t>(ncp + 1, s);
  k_l0_count<<<blocks_for(ncp, 256), 256, 0, s>>>(G, eb.cp_node, eb.code, ncp, cnt);
  A0.rp = dalloc<int32_t>(ncp + 1, s, false);
  exclusive_scan_i32(cnt, A0.rp, ncp, s);
  int32_t nnz = 0;
  EB_CUDA(cudaMemcpyAsync(&nnz, A0.rp + ncp, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  EB_CUDA(cudaStreamSynchronize(s));
  A0.nnz = nnz;
  A0.ci = dalloc<int32_t>(nnz, s, false);
  A0.v = dalloc<double>(nnz, s, false);
  const BetaArgs beta{{eb.beta64[0], eb.beta64[1], eb.beta64[2]}};
  k_l0_fill<<<blocks_for(ncp, 256), 256, 0, s>>>(G, eb.cp_node, eb.cp_of_node, eb.code, eb.diag, ncp, sigma, A0.rp,
                                                  A0.ci, A0.v, beta);
  EB_CUDA(cudaGetLastError());
  dfree(cnt, s);
  return A0;
}

void amg_build(Solver& S, cudaStream_t s) { amg_build_from(S, level0_csr(*S.eb, S.shift, s), s); }

// Hierarchy from a given level-0 CSR whose row k is the CP at node
// S.eb->cp_node[k] of the (possibly batched) grid view.
void amg_build_from(Solver& S, DCsr A0, cudaStream_t s) {
  const EBHandle& eb = *S.eb;
  Hierarchy* H = new Hierarchy();
  S.H = H;
  DCsr A = A0;
  const int max_levels = std::max(1, S.opts.max_levels);
  for (int lev = 0;; ++lev) {
    H->L.emplace_back();
    Level& L = H->L.back();
    L.A = A;
    double* d = dalloc<double>(A.n, s, false);
    L.dinv = dalloc<double>(A.n, s, false);
    double* rho = dalloc<double>(1, s);
    k_rowinfo<<<blocks_for(A.n, 256), 256, 0, s>>>(A, d, L.dinv, rho);
    EB_CUDA(cudaMemcpyAsync(&L.rho, rho, sizeof(double), cudaMemcpyDeviceToHost, s));
    EB_CUDA(cudaStreamSynchronize(s));
    dfree(rho, s);
    EB_REQUIRE(std::isfinite(L.rho) && L.rho > 0.0 && L.rho < 1e299, EB_ERR_NONFINITE,
               "amg_setup: non-finite or non-positive diagonal");
    if (A.n <= S.opts.coarse_max || (int)H->L.size() >= max_levels) {
      dfree(d, s);
      break;
    }
    if (S.opts.coarsening == EB_AMG_RS) {
      // classical coarsening: strength, PMIS splitting, direct interpolation
      uint8_t* strong = dalloc<uint8_t>(A.nnz, s, false);
      uint8_t* strongT = dalloc<uint8_t>(A.nnz, s, false);
      int32_t* lam = dalloc<int32_t>(A.n, s, false);
      int8_t* state = dalloc<int8_t>(A.n, s, false);
      uint8_t* newc = dalloc<uint8_t>(A.n, s, false);
      int* und = dalloc<int>(1, s);
      const unsigned bn = blocks_for(A.n, 256);
      k_rs_strength<<<bn, 256, 0, s>>>(A, strong);
      k_rs_transpose<<<bn, 256, 0, s>>>(A, strong, strongT, lam);
      k_rs_init<<<bn, 256, 0, s>>>(A.n, lam, state);
      for (int round = 0;; ++round) {
        EB_REQUIRE(round < 1000, EB_ERR_INVALID, "amg_setup: PMIS did not terminate");
        EB_CUDA(cudaMemsetAsync(und, 0, sizeof(int), s));
        k_rs_select<<<bn, 256, 0, s>>>(A, strong, strongT, lam, state, newc);
        k_rs_apply<<<bn, 256, 0, s>>>(A.n, newc, state);
        k_rs_fassign<<<bn, 256, 0, s>>>(A, strong, state, und);
        int hund = 0;
        EB_CUDA(cudaMemcpyAsync(&hund, und, sizeof(int), cudaMemcpyDeviceToHost, s));
        EB_CUDA(cudaStreamSynchronize(s));
        if (hund == 0) break;
      }
      int32_t* cflag = dalloc<int32_t>(A.n + 1, s);
      int32_t* cidx = dalloc<int32_t>(A.n + 1, s, false);
      k_rs_cflag<<<bn, 256, 0, s>>>(A.n, state, cflag);
      exclusive_scan_i32(cflag, cidx, A.n, s);
      int32_t nc = 0;
      EB_CUDA(cudaMemcpyAsync(&nc, cidx + A.n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      EB_CUDA(cudaStreamSynchronize(s));
      auto release = [&] {
        dfree(strong, s); dfree(strongT, s); dfree(lam, s); dfree(state, s); dfree(newc, s); dfree(und, s);
        dfree(cflag, s); dfree(cidx, s); dfree(d, s);
      };
      if (nc >= A.n || nc == 0) {
        release();
        break;
      }
      int32_t* pc = dalloc<int32_t>(A.n + 1, s);
      DCsr P;
      P.n = A.n;
      P.m = nc;
      P.rp = dalloc<int32_t>(A.n + 1, s, false);
      k_rs_pcount<<<bn, 256, 0, s>>>(A, strong, state, pc);
      exclusive_scan_i32(pc, P.rp, A.n, s);
      int32_t pnnz = 0;
      EB_CUDA(cudaMemcpyAsync(&pnnz, P.rp + A.n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      EB_CUDA(cudaStreamSynchronize(s));
      P.nnz = pnnz;
      P.ci = dalloc<int32_t>(pnnz, s, false);
      P.v = dalloc<double>(pnnz, s, false);
      L.agg = dalloc<int32_t>(A.n, s, false);
      k_rs_pfill<<<bn, 256, 0, s>>>(A, strong, state, cidx, P, L.agg);
      EB_CUDA(cudaGetLastError());
      dfree(pc, s);
      release();
      L.P = P;
      L.R = transpose(L.P, s);
      if (lev == 0) {
        L.R0node = dalloc<int32_t>(L.R.nnz, s, false);
        k_map_cols<<<blocks_for(L.R.nnz, 256), 256, 0, s>>>(L.R.nnz, L.R.ci, eb.cp_node, L.R0node);
      }
      DCsr AP = spgemm(A, L.P, s);
      DCsr Ac = spgemm(L.R, AP, s);
      csr_free(AP, s);
      A = Ac;
      continue;
    }
    // strength + MIS-2
    uint8_t* strong = dalloc<uint8_t>(A.nnz, s, false);
    k_strength<<<blocks_for(A.n, 256), 256, 0, s>>>(A, d, S.opts.strength, strong);
    uint8_t* state = dalloc<uint8_t>(A.n, s, false);
    EB_CUDA(cudaMemsetAsync(state, 1, A.n, s));
    uint64_t* k1 = dalloc<uint64_t>(A.n, s, false);
    int* und = dalloc<int>(1, s);
    for (int round = 0; round < 1000; ++round) {
      EB_CUDA(cudaMemsetAsync(und, 0, sizeof(int), s));
      k_mis_max1<<<blocks_for(A.n, 256), 256, 0, s>>>(A, strong, state, k1);
      k_mis_max2<<<blocks_for(A.n, 256), 256, 0, s>>>(A, strong, k1, state, und);
      int hund = 0;
      EB_CUDA(cudaMemcpyAsync(&hund, und, sizeof(int), cudaMemcpyDeviceToHost, s));
      EB_CUDA(cudaStreamSynchronize(s));
      if (hund == 0) break;
      EB_REQUIRE(round < 999, EB_ERR_INVALID, "amg_setup: MIS-2 did not terminate");
    }
    int32_t* rflag = dalloc<int32_t>(A.n + 1, s);
    int32_t* roff = dalloc<int32_t>(A.n + 1, s, false);
    k_is_root<<<blocks_for(A.n, 256), 256, 0, s>>>(A.n, state, rflag);
    exclusive_scan_i32(rflag, roff, A.n, s);
    int32_t nc = 0;
    EB_CUDA(cudaMemcpyAsync(&nc, roff + A.n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    int32_t* agg1 = dalloc<int32_t>(A.n, s, false);
    L.agg = dalloc<int32_t>(A.n, s, false);
    int* unas = dalloc<int>(1, s);
    k_agg_pass1<<<blocks_for(A.n, 256), 256, 0, s>>>(A, strong, state, roff, agg1);
    k_agg_pass2<<<blocks_for(A.n, 256), 256, 0, s>>>(A, strong, agg1, L.agg, unas);
    int hun = 0;
    EB_CUDA(cudaMemcpyAsync(&hun, unas, sizeof(int), cudaMemcpyDeviceToHost, s));
    EB_CUDA(cudaStreamSynchronize(s));
    dfree(strong, s); dfree(state, s); dfree(k1, s); dfree(und, s); dfree(rflag, s); dfree(roff, s);
    dfree(agg1, s); dfree(unas, s); dfree(d, s);
    EB_REQUIRE(hun == 0, EB_ERR_INVALID, "amg_setup: aggregation left a node unassigned");
    if (nc >= A.n || nc == 0) break;
    // tentative and smoothed prolongators
    int32_t* size = dalloc<int32_t>(nc, s);
    k_agg_sizes<<<blocks_for(A.n, 256), 256, 0, s>>>(A.n, L.agg, size);
    DCsr Ph;
    Ph.n = A.n;
    Ph.m = nc;
    Ph.nnz = A.n;
    Ph.rp = dalloc<int32_t>(A.n + 1, s, false);
    Ph.ci = dalloc<int32_t>(A.n, s, false);
    Ph.v = dalloc<double>(A.n, s, false);
    k_phat<<<blocks_for(A.n + 1, 256), 256, 0, s>>>(A.n, L.agg, size, Ph.rp, Ph.ci, Ph.v);
    EB_CUDA(cudaGetLastError());
    DCsr T = spgemm(A, Ph, s);
    const double omega = 4.0 / (3.0 * L.rho);
    k_smooth_p<<<blocks_for(T.n, 256), 256, 0, s>>>(T, L.agg, Ph.v, L.dinv, omega, T.v);
    EB_CUDA(cudaGetLastError());
    L.P = T;
    csr_free(Ph, s);
    // a single grid (no per-tile shifts) applies the level-0 P and R matrix free
    if (lev == 0 && eb.tile_shift64 == nullptr && A.n == eb.num_cp) build_mf(H->mf, eb, L, nc, size, s);
    dfree(size, s);
    L.R = transpose(L.P, s);
    if (lev == 0) {
      L.R0node = dalloc<int32_t>(L.R.nnz, s, false);
      k_map_cols<<<blocks_for(L.R.nnz, 256), 256, 0, s>>>(L.R.nnz, L.R.ci, eb.cp_node, L.R0node);
    }
    DCsr AP = spgemm(A, L.P, s);
    DCsr Ac = spgemm(L.R, AP, s);
    csr_free(AP, s);
    A = Ac;
  }
  // coarsest level
  EB_REQUIRE(H->L.back().A.n <= 8192, EB_ERR_INVALID,
             "amg_setup: coarsest level above 8192 rows for the dense solve; raise max_levels");
  coarse_inverse(*H, H->L.back().A, s);
  amg_alloc_vcycle(S, s);
  EB_CUDA(cudaStreamSynchronize(s));
}

void amg_free(Solver& S) {
  if (!S.H) return;
  cudaStream_t s = S.home;
  Hierarchy* H = S.H;
  amg_free_vcycle(*H, s);
  free_mf(H->mf, s);
  for (Level& L : H->L) {
    csr_free(L.A, s);
    csr_free(L.P, s);
    csr_free(L.R, s);
    dfree(L.R0node, s); dfree(L.agg, s); dfree(L.dinv, s);
  }
  dfree(H->coarse_inv, s);
  cudaStreamSynchronize(s);
  delete H;
  S.H = nullptr;
}

void amg_fill_info(const Solver& S, amg_info_t* out) {
  if (!S.H) {
    out->num_levels = 0;
    return;
  }
  const Hierarchy& H = *S.H;
  out->num_levels = (int)H.L.size();
  double tot = 0.0;
  for (size_t l = 0; l < H.L.size() && l < 32; ++l) {
    out->rows[l] = H.L[l].A.n;
    out->nnz[l] = H.L[l].A.nnz;
    tot += (double)H.L[l].A.nnz;
  }
  out->operator_complexity = tot / (double)std::max<int64_t>(1, H.L[0].A.nnz);
}

void amg_copy_level(const Solver& S, int level, int which, int32_t* rowptr, int32_t* col, double* val,
                    cudaStream_t s) {
  EB_REQUIRE(S.H != nullptr, EB_ERR_INVALID, "amg_level_copy: no hierarchy");
  const Hierarchy& H = *S.H;
  EB_REQUIRE(level >= 0 && level < (int)H.L.size(), EB_ERR_INVALID, "amg_level_copy: level out of range");
  const Level& L = H.L[level];
  if (which == 2) {
    EB_REQUIRE(L.agg != nullptr && col != nullptr, EB_ERR_INVALID, "amg_level_copy: no aggregates on this level");
    EB_CUDA(cudaMemcpyAsync(col, L.agg, sizeof(int32_t) * L.A.n, cudaMemcpyDeviceToDevice, s));
    return;
  }
  EB_REQUIRE(which == 0 || which == 1, EB_ERR_INVALID, "amg_level_copy: which must be 0, 1 or 2");
  const DCsr& M = which == 0 ? L.A : L.P;
  EB_REQUIRE(M.rp != nullptr, EB_ERR_INVALID, "amg_level_copy: matrix not present on this level");
  if (rowptr) EB_CUDA(cudaMemcpyAsync(rowptr, M.rp, sizeof(int32_t) * (M.n + 1), cudaMemcpyDeviceToDevice, s));
  if (col) EB_CUDA(cudaMemcpyAsync(col, M.ci, sizeof(int32_t) * M.nnz, cudaMemcpyDeviceToDevice, s));
  if (val) EB_CUDA(cudaMemcpyAsync(val, M.v, sizeof(double) * M.nnz, cudaMemcpyDeviceToDevice, s));
}

}  // namespace ebk
