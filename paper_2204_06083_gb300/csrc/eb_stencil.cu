// Matrix-free EB stencil (eq. 3 with the line-by-line diagonal of Sec. 2.1),
// device prefix scan, and the leapfrog step kernel (theta-scheme of
// Sec. 3.5 at theta = 0).
//
// Layout: full grid, x fastest; work is distributed over the active tiles
// (tiles.cuh), the leapfrog steps over their node pairs that hold a CP.  The node code byte carries the CP flag and the mask of
// directions whose neighbour is a BP, so a CP never reads a non-CP value:
// interior CPs (code 0x80) use D = 2 dim, cut CPs read D_k (stencil.cuh).
#include "eb_internal.cuh"
#include "stencil.cuh"

#include <algorithm>

namespace ebk {

// ------------------------------------------------------------------- scan
// Three-phase exclusive scan of int32 values: per-block sums, a single-block
// scan of the block sums, and a per-block scan with the block offset added.
constexpr int SCAN_T = 256;
constexpr int SCAN_PER = 4;
constexpr int SCAN_TILE = SCAN_T * SCAN_PER;

__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t* sm, int32_t* total) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sm[w] = x;
  __syncthreads();
  if (w == 0) {
    int32_t s = lane < (int)(blockDim.x >> 5) ? sm[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    sm[lane] = s;
  }
  __syncthreads();
  int32_t base = w ? sm[w - 1] : 0;
  *total = sm[(blockDim.x >> 5) - 1];
  __syncthreads();
  return base + x - v;
}

__global__ void k_scan_sums(const int32_t* in, int64_t n, int32_t* bsum) {
  __shared__ int32_t sm[32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int32_t s = 0;
  for (int j = 0; j < SCAN_PER; ++j) {
    int64_t i = base + (int64_t)j * SCAN_T + threadIdx.x;
    if (i < n) s += in[i];
  }
  int32_t tot;
  block_excl_scan(s, sm, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_top(int32_t* bsum, int64_t nb) {
  __shared__ int32_t sm[32];
  int32_t carry = 0;
  for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
    int64_t i = b0 + threadIdx.x;
    int32_t v = i < nb ? bsum[i] : 0;
    int32_t tot;
    int32_t e = block_excl_scan(v, sm, &tot);
    if (i < nb) bsum[i] = carry + e;
    carry += tot;
  }
}

__global__ void k_scan_final(const int32_t* in, int64_t n, const int32_t* boff, int32_t* out) {
  __shared__ int32_t sm[32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int32_t v[SCAN_PER];
  int32_t s = 0;
  int64_t i0 = base + (int64_t)threadIdx.x * SCAN_PER;
  for (int j = 0; j < SCAN_PER; ++j) {
    int64_t i = i0 + j;
    v[j] = i < n ? in[i] : 0;
    s += v[j];
  }
  int32_t tot;
  int32_t e = block_excl_scan(s, sm, &tot) + boff[blockIdx.x];
  for (int j = 0; j < SCAN_PER; ++j) {
    int64_t i = i0 + j;
    if (i < n) out[i] = e;
    e += v[j];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) out[n] = e;
}

void exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s) {
  if (n <= 0) {
    EB_CUDA(cudaMemsetAsync(out, 0, sizeof(int32_t), s));
    return;
  }
  int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  int32_t* bsum = dalloc<int32_t>(nb, s, false);
  // k_scan_sums uses a strided layout per block, k_scan_final a blocked one;
  // both cover the same SCAN_TILE range per block, so the block sums agree.
  k_scan_sums<<<(unsigned)nb, SCAN_T, 0, s>>>(in, n, bsum);
  k_scan_top<<<1, 1024, 0, s>>>(bsum, nb);
  k_scan_final<<<(unsigned)nb, SCAN_T, 0, s>>>(in, n, bsum, out);
  EB_CUDA(cudaGetLastError());
  dfree(bsum, s);
}

// ---------------------------------------------------------------- stencil
// y = (sigma I + A) x at the CPs, 0 at the other node of a pair that holds a
// CP.  With the view's CP pair list (every single grid that has a CP) one
// thread takes one pair of the list, one pass over the grid of CTAs; without
// it (no CP) the pairs of the active tiles, grid-stride.
constexpr int APPLY_THREADS = 256;

template <class T, int DIM>
__global__ void __launch_bounds__(APPLY_THREADS) k_apply(TileView tv, const uint8_t* __restrict__ code,
                                                         const typename DiagOf<T>::type* __restrict__ diag,
                                                         const T* __restrict__ x, T* __restrict__ y,
                                                         typename AccOf<T>::type sigma,
                                                         typename AccOf<T>::type inv_h2) {
  using A = typename AccOf<T>::type;
  EB_SWEEP(DIM, tv, node) {
    uint32_t c0, c1;
    ld_codes(code, node, c0, c1);
    Two<A> xc, core;
    stencil_tv<DIM, LdRO>(tv, x, node, c0, c1, diag, xc, core);
    const A v0 = (c0 & CODE_CP) ? core.x * inv_h2 + sigma * xc.x : (A)0;
    const A v1 = (c1 & CODE_CP) ? core.y * inv_h2 + sigma * xc.y : (A)0;
    st2(y + node, v0, v1);
  }
}

template <class T>
void launch_apply(const EBHandle& eb, const T* x, T* y, double sigma, cudaStream_t s) {
  using A = typename AccOf<T>::type;
  const A inv_h2 = (A)(1.0 / (eb.g.h * eb.g.h));
  const TileView tv = eb.tv();
  dim_dispatch(eb, [&](auto D) {
    if (tv.pair_node)
      k_apply<T, D.value | DIM_LIST><<<blocks_for(tv.npairs, APPLY_THREADS), APPLY_THREADS, 0, s>>>(
          tv, eb.code, diag_of<T>(eb), x, y, (A)sigma, inv_h2);
    else
      k_apply<T, D.value><<<tile_grid(eb), APPLY_THREADS, 0, s>>>(tv, eb.code, diag_of<T>(eb), x, y, (A)sigma,
                                                                  inv_h2);
  });
  EB_CUDA(cudaGetLastError());
}

template void launch_apply<double>(const EBHandle&, const double*, double*, double, cudaStream_t);
template void launch_apply<float>(const EBHandle&, const float*, float*, double, cudaStream_t);
template void launch_apply<__nv_bfloat16>(const EBHandle&, const __nv_bfloat16*, __nv_bfloat16*, double, cudaStream_t);

// -------------------------------------------------------------- leapfrog
// One leapfrog step per launch: u_new = 2 u - u_old - dt^2 A u, u_new
// overwriting u_old in place.  A launch boundary is the cheapest grid-wide
// barrier on this part: a persistent cooperative kernel with a software grid
// barrier between its steps measured 9.6-14.8 us per step at 4096^2 against
// 8.3 us for one launch per step inside a CUDA graph.  512-thread CTAs sized
// to one resident wave, over the view's CP pair list (four tiles per pass over
// every tile pair for a view without one).
constexpr int LF_THREADS = 512;

template <class T, int DIM>
__global__ void __launch_bounds__(LF_THREADS) k_leapfrog(TileView tv, const uint8_t* __restrict__ code,
                                                         const typename DiagOf<T>::type* __restrict__ diag,
                                                         const T* __restrict__ cur, T* __restrict__ prev,
                                                         typename AccOf<T>::type c2) {
  using A = typename AccOf<T>::type;
  auto step = [&](int32_t node) {
    uint32_t c0, c1;
    ld_codes(code, node, c0, c1);
    Two<A> xc, core;
    stencil_tv<DIM, LdRO>(tv, cur, node, c0, c1, diag, xc, core);
    const Two<A> po = LdCG::ld2(prev + node);  // read, then overwritten, by this thread only
    const A n0 = (c0 & CODE_CP) ? (A)2 * xc.x - po.x - c2 * core.x : (A)0;
    const A n1 = (c1 & CODE_CP) ? (A)2 * xc.y - po.y - c2 * core.y : (A)0;
    st2(prev + node, n0, n1);
  };
  if (tv.pair_node) {  // the CP pairs (the others hold 0 in both fields: k_field_mask)
    for (int64_t li = (int64_t)blockIdx.x * LF_THREADS + threadIdx.x; li < tv.npairs;
         li += (int64_t)gridDim.x * LF_THREADS)
      step(__ldg(tv.pair_node + li));
    return;
  }
  constexpr int TPP = LF_THREADS / PAIR_THREADS;
  for (int64_t tt = (int64_t)TPP * blockIdx.x + (threadIdx.x >> 7); tt < tv.ntiles; tt += (int64_t)TPP * gridDim.x) {
    int32_t node;
    if (!tile_pair<DIM>(tv, tt, threadIdx.x & (PAIR_THREADS - 1), node)) continue;
    step(node);
  }
}

// 0 at the non-CP nodes of every pair of the active tiles, in both fields: the
// values a step over every tile pair writes there, so that stepping only the
// CP pairs leaves the same fields
template <class T, int DIM>
__global__ void __launch_bounds__(LF_THREADS) k_field_mask(TileView tv, const uint8_t* __restrict__ code, T* ua,
                                                           T* ub) {
  constexpr int TPP = LF_THREADS / PAIR_THREADS;
  for (int64_t tt = (int64_t)TPP * blockIdx.x + (threadIdx.x >> 7); tt < tv.ntiles; tt += (int64_t)TPP * gridDim.x) {
    int32_t node;
    if (!tile_pair<DIM>(tv, tt, threadIdx.x & (PAIR_THREADS - 1), node)) continue;
    uint32_t c0, c1;
    ld_codes(code, node, c0, c1);
    if ((c0 & c1 & CODE_CP) != 0) continue;  // both CPs: nothing to clear
    const bool k0 = (c0 & CODE_CP) != 0, k1 = (c1 & CODE_CP) != 0;
    const Two<T> a{ua[node], ua[node + 1]}, b{ub[node], ub[node + 1]};
    st2(ua + node, k0 ? a.x : (T)0, k1 ? a.y : (T)0);
    st2(ub + node, k0 ? b.x : (T)0, k1 ? b.y : (T)0);
  }
}

// (ua, ub) <- (ub, ua) over the active tiles: after an odd number of steps the
// newest field sits in ua
template <class T, int DIM>
__global__ void __launch_bounds__(LF_THREADS) k_field_swap(TileView tv, T* ua, T* ub) {
  using A = typename AccOf<T>::type;
  constexpr int TPP = LF_THREADS / PAIR_THREADS;
  for (int64_t tt = (int64_t)TPP * blockIdx.x + (threadIdx.x >> 7); tt < tv.ntiles; tt += (int64_t)TPP * gridDim.x) {
    int32_t node;
    if (!tile_pair<DIM>(tv, tt, threadIdx.x & (PAIR_THREADS - 1), node)) continue;
    const Two<A> a = LdCG::ld2(ua + node);
    const Two<A> b = LdCG::ld2(ub + node);
    st2(ua + node, b.x, b.y);
    st2(ub + node, a.x, a.y);
  }
}

template <class T>
static unsigned leapfrog_grid(const EBHandle& eb, const void* fn) {
  static int per_sm[2][2] = {{0, 0}, {0, 0}};  // [T is double][dim 3]
  int& ps = per_sm[sizeof(T) == 8][eb.g.dim == 3];
  if (!ps) {
    EB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, fn, LF_THREADS, 0));
    EB_REQUIRE(ps > 0, EB_ERR_INVALID, "leapfrog kernel cannot be resident");
  }
  constexpr int TPP = LF_THREADS / PAIR_THREADS;
  const int64_t need = (eb.num_tiles + TPP - 1) / TPP;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)ps * num_sms()));
}

void LeapfrogGraph::release() {
  if (exec) cudaGraphExecDestroy(exec);
  exec = nullptr;
}

// nsteps launches of k_leapfrog, alternating the roles of ua and ub, then the
// swap if nsteps is odd.  With use_graph, whole chunks of LeapfrogGraph::CHUNK
// steps run as one launch of a graph cached on the handle (rebuilt when the
// fields, the precision, dt or the tile list change); the rest are launched
// one by one, as are all steps without use_graph (no allocation then).
template <class T>
int launch_leapfrog(const EBHandle& eb, T* ua, T* ub, int nsteps, double dt, cudaStream_t s, bool use_graph) {
  if (nsteps <= 0) return EB_OK;
  const Geometry& G = eb.g;
  using A = typename AccOf<T>::type;
  const void* fn = nullptr;
  dim_dispatch(eb, [&](auto D) { fn = (const void*)k_leapfrog<T, D.value>; });
  const unsigned blocks = leapfrog_grid<T>(eb, fn);
  A c2 = (A)(dt * dt / (G.h * G.h));  // dt^2 / h^2, the only constant of the step
  TileView tv = eb.tv();
  const uint8_t* code = eb.code;
  const typename DiagOf<T>::type* diag = diag_of<T>(eb);
  auto step_args = [&](int k, const T*& cur, T*& prev) {
    cur = (k & 1) ? ua : ub;
    prev = (k & 1) ? ub : ua;
  };
  if (tv.pair_node) {  // the steps touch only the CP pairs
    if (G.dim == 2)
      k_field_mask<T, 2><<<blocks, LF_THREADS, 0, s>>>(tv, code, ua, ub);
    else
      k_field_mask<T, 3><<<blocks, LF_THREADS, 0, s>>>(tv, code, ua, ub);
  }
  int done = 0;
  if (use_graph && nsteps >= LeapfrogGraph::CHUNK) {
    LeapfrogGraph& lg = eb.lf_graph;
    const int prec = sizeof(T) == 8 ? EB_F64 : EB_F32;
    if (!lg.exec || lg.ua != ua || lg.ub != ub || lg.prec != prec || lg.c2 != (double)c2 || lg.tile_gen != eb.tile_gen) {
      lg.release();
      cudaGraph_t g = nullptr;
      EB_CUDA(cudaGraphCreate(&g, 0));
      cudaGraphNode_t last = nullptr;
      for (int k = 0; k < LeapfrogGraph::CHUNK; ++k) {
        const T* cur;
        T* prev;
        step_args(k, cur, prev);
        void* args[] = {(void*)&tv, (void*)&code, (void*)&diag, (void*)&cur, (void*)&prev, (void*)&c2};
        cudaKernelNodeParams p{};
        p.func = const_cast<void*>(fn);
        p.gridDim = dim3(blocks);
        p.blockDim = dim3(LF_THREADS);
        p.kernelParams = args;
        cudaGraphNode_t nd = nullptr;
        const cudaError_t e = cudaGraphAddKernelNode(&nd, g, last ? &last : nullptr, last ? 1 : 0, &p);
        if (e != cudaSuccess) {
          cudaGraphDestroy(g);
          throw Failure{EB_ERR_CUDA, std::string("wave_step: cudaGraphAddKernelNode failed: ") + cudaGetErrorString(e)};
        }
        last = nd;
      }
      const cudaError_t e = cudaGraphInstantiate(&lg.exec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        lg.exec = nullptr;
        throw Failure{EB_ERR_CUDA, std::string("wave_step: cudaGraphInstantiate failed: ") + cudaGetErrorString(e)};
      }
      lg.ua = ua;
      lg.ub = ub;
      lg.prec = prec;
      lg.c2 = (double)c2;
      lg.tile_gen = eb.tile_gen;
    }
    for (; done + LeapfrogGraph::CHUNK <= nsteps; done += LeapfrogGraph::CHUNK) EB_CUDA(cudaGraphLaunch(lg.exec, s));
  }
  for (int k = done; k < nsteps; ++k) {
    const T* cur;
    T* prev;
    step_args(k, cur, prev);  // CHUNK is even: step k has the parity of k
    dim_dispatch(eb, [&](auto D) { k_leapfrog<T, D.value><<<blocks, LF_THREADS, 0, s>>>(tv, code, diag, cur, prev, c2); });
  }
  if (nsteps & 1) {
    if (G.dim == 2)
      k_field_swap<T, 2><<<blocks, LF_THREADS, 0, s>>>(tv, ua, ub);
    else
      k_field_swap<T, 3><<<blocks, LF_THREADS, 0, s>>>(tv, ua, ub);
  }
  EB_CUDA(cudaGetLastError());
  return EB_OK;
}

template int launch_leapfrog<double>(const EBHandle&, double*, double*, int, double, cudaStream_t, bool);
template int launch_leapfrog<float>(const EBHandle&, float*, float*, int, double, cudaStream_t, bool);

}  // namespace ebk
