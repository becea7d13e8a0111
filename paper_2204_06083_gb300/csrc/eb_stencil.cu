// Matrix-free EB stencil (eq. 3 with the line-by-line diagonal of Sec. 2.1),
// device prefix scan, and the persistent leapfrog kernel (theta-scheme of
// Sec. 3.5 at theta = 0).
//
// Layout: full grid, x fastest.  Work is distributed over the list of active
// tiles (tiles holding at least one CP); a CTA of 256 threads covers one tile
// per iteration of a grid-stride loop.  The node code byte carries the CP flag
// and the mask of directions whose neighbour is a BP, so a CP never reads a
// non-CP value: interior CPs (code 0x80) use D = 2 dim, cut CPs read D_k.
#include "eb_internal.cuh"

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
template <class T>
struct Acc {
  using type = float;
};
template <>
struct Acc<double> {
  using type = double;
};

__device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
__device__ __forceinline__ double ld(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(p[0]); }
__device__ __forceinline__ void st(float* p, float v) { *p = v; }
__device__ __forceinline__ void st(double* p, double v) { *p = v; }
__device__ __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

// L2-coherent loads for data written by other CTAs during the same launch
__device__ __forceinline__ double ld_plain(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ld_plain(const float* p) { return __ldcg(p); }

struct TileCursor {
  int64_t node;
  bool valid;
};

__device__ __forceinline__ TileCursor tile_node(const Geometry& G, int64_t t, int l) {
  int64_t bx = t % G.ntx, r = t / G.ntx, by = r % G.nty, bz = r / G.nty;
  int lx = l % G.tx, ly = (l / G.tx) % G.ty, lz = l / (G.tx * G.ty);
  int64_t ix = bx * G.tx + lx, iy = by * G.ty + ly, iz = bz * G.tz + lz;
  TileCursor c;
  c.valid = ix < G.n0 && iy < G.n1 && iz < G.n2;
  c.node = ix + (int64_t)G.n0 * (iy + (int64_t)G.n1 * iz);
  return c;
}

// (sigma I + A) x at one CP, in the accumulation type of T
template <class T, int DIM>
__device__ __forceinline__ typename Acc<T>::type stencil_at(const T* x, int64_t node, uint8_t c, const double* diag,
                                                            int64_t sy, int64_t sz, typename Acc<T>::type inv_h2,
                                                            typename Acc<T>::type sigma) {
  using A = typename Acc<T>::type;
  const A xc = ld(x + node);
  const uint8_t m = c & 0x3F;
  A sum = 0;
  if (!(m & 1)) sum += ld(x + node - 1);
  if (!(m & 2)) sum += ld(x + node + 1);
  if (!(m & 4)) sum += ld(x + node - sy);
  if (!(m & 8)) sum += ld(x + node + sy);
  if (DIM == 3) {
    if (!(m & 16)) sum += ld(x + node - sz);
    if (!(m & 32)) sum += ld(x + node + sz);
  }
  const A D = m ? (A)__ldg(diag + node) : (A)(2 * DIM);
  return (D * xc - sum) * inv_h2 + sigma * xc;
}

template <class T, int DIM>
__global__ void __launch_bounds__(256) k_apply(Geometry G, const int32_t* __restrict__ tiles, int64_t ntiles,
                                               const uint8_t* __restrict__ code, const double* __restrict__ diag,
                                               const T* __restrict__ x, T* __restrict__ y, double sigma, double inv_h2) {
  using A = typename Acc<T>::type;
  const int tsz = G.tx * G.ty * G.tz;
  const int64_t sy = G.n0, sz = (int64_t)G.n0 * G.n1;
  for (int64_t tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
    const int64_t t = tiles[tt];
    for (int l = threadIdx.x; l < tsz; l += blockDim.x) {
      TileCursor cur = tile_node(G, t, l);
      if (!cur.valid) continue;
      const uint8_t c = code[cur.node];
      A v = 0;
      if (c & CODE_CP) v = stencil_at<T, DIM>(x, cur.node, c, diag, sy, sz, (A)inv_h2, (A)sigma);
      st(y + cur.node, v);
    }
  }
}

inline unsigned tile_blocks(const EBHandle& eb, int per_sm = 8) {
  int64_t b = std::min<int64_t>(eb.num_tiles, (int64_t)num_sms() * per_sm);
  return (unsigned)std::max<int64_t>(b, 1);
}

template <class T>
void launch_apply(const EBHandle& eb, const T* x, T* y, double sigma, cudaStream_t s) {
  const Geometry& G = eb.g;
  double inv_h2 = 1.0 / (G.h * G.h);
  if (G.dim == 2)
    k_apply<T, 2><<<tile_blocks(eb), 256, 0, s>>>(G, eb.tiles, eb.num_tiles, eb.code, eb.diag, x, y, sigma, inv_h2);
  else
    k_apply<T, 3><<<tile_blocks(eb), 256, 0, s>>>(G, eb.tiles, eb.num_tiles, eb.code, eb.diag, x, y, sigma, inv_h2);
  EB_CUDA(cudaGetLastError());
}

template void launch_apply<double>(const EBHandle&, const double*, double*, double, cudaStream_t);
template void launch_apply<float>(const EBHandle&, const float*, float*, double, cudaStream_t);
template void launch_apply<__nv_bfloat16>(const EBHandle&, const __nv_bfloat16*, __nv_bfloat16*, double, cudaStream_t);

// -------------------------------------------------------------- leapfrog
// Grid-wide barrier for a cooperative launch: sense-reversing counter with a
// bounded spin.  On timeout the block sets *err and every later barrier of
// the launch returns at once, so the kernel always terminates.
struct GridBarrier {
  unsigned int count;
  unsigned int gen;
  int err;
  int pad;
};

constexpr long long BARRIER_SPIN_LIMIT = 20000000;  // ~ seconds of polling

__device__ bool grid_sync(GridBarrier* gb) {
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
      unsigned int arrived = atomicAdd(&gb->count, 1u) + 1u;
      if (arrived == gridDim.x) {
        gb->count = 0;
        __threadfence();
        atomicAdd(&gb->gen, 1u);
      } else {
        long long spins = 0;
        while (*pgen == g) {
          if (*perr || ++spins > BARRIER_SPIN_LIMIT) {
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

template <class T, int DIM>
__global__ void __launch_bounds__(256) k_leapfrog(Geometry G, const int32_t* __restrict__ tiles, int64_t ntiles,
                                                  const uint8_t* __restrict__ code, const double* __restrict__ diag,
                                                  T* ua, T* ub, int nsteps, double dt2, double inv_h2, GridBarrier* gb) {
  using A = typename Acc<T>::type;
  const int tsz = G.tx * G.ty * G.tz;
  const int64_t sy = G.n0, sz = (int64_t)G.n0 * G.n1;
  // step s reads cur = (s even ? ub : ua) and overwrites prev = the other
  for (int s = 0; s < nsteps; ++s) {
    T* prev = (s & 1) ? ub : ua;
    const T* cur = (s & 1) ? ua : ub;
    for (int64_t tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
      const int64_t t = tiles[tt];
      for (int l = threadIdx.x; l < tsz; l += blockDim.x) {
        TileCursor c = tile_node(G, t, l);
        if (!c.valid) continue;
        const uint8_t cc = code[c.node];
        if (!(cc & CODE_CP)) continue;
        // plain loads: cur was written by other CTAs in the previous step
        const A xc = (A)ld_plain(cur + c.node);
        const uint8_t m = cc & 0x3F;
        A sum = 0;
        if (!(m & 1)) sum += (A)ld_plain(cur + c.node - 1);
        if (!(m & 2)) sum += (A)ld_plain(cur + c.node + 1);
        if (!(m & 4)) sum += (A)ld_plain(cur + c.node - sy);
        if (!(m & 8)) sum += (A)ld_plain(cur + c.node + sy);
        if (DIM == 3) {
          if (!(m & 16)) sum += (A)ld_plain(cur + c.node - sz);
          if (!(m & 32)) sum += (A)ld_plain(cur + c.node + sz);
        }
        const A D = m ? (A)__ldg(diag + c.node) : (A)(2 * DIM);
        const A Au = (D * xc - sum) * (A)inv_h2;
        const A un = (A)2 * xc - (A)ld_plain(prev + c.node) - (A)dt2 * Au;
        st(prev + c.node, un);
      }
    }
    if (!grid_sync(gb)) return;
  }
  // odd step count: the newest field is in ua; swap so that (ua, ub) = (prev, cur)
  if (nsteps & 1) {
    for (int64_t tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
      const int64_t t = tiles[tt];
      for (int l = threadIdx.x; l < tsz; l += blockDim.x) {
        TileCursor c = tile_node(G, t, l);
        if (!c.valid) continue;
        T a = __ldcg(ua + c.node);
        ua[c.node] = __ldcg(ub + c.node);
        ub[c.node] = a;
      }
    }
  }
}

}  // namespace ebk

namespace ebk {

template <class T>
int launch_leapfrog(const EBHandle& eb, T* ua, T* ub, int nsteps, double dt, cudaStream_t s) {
  const Geometry& G = eb.g;
  if (nsteps <= 0) return EB_OK;
  GridBarrier* gb = dalloc<GridBarrier>(1, s);
  int dev = 0;
  EB_CUDA(cudaGetDevice(&dev));
  int per_sm = 0;
  void* fn = G.dim == 2 ? (void*)k_leapfrog<T, 2> : (void*)k_leapfrog<T, 3>;
  EB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0));
  EB_REQUIRE(per_sm > 0, EB_ERR_INVALID, "leapfrog kernel cannot be resident");
  int64_t nb = std::min<int64_t>(eb.num_tiles, (int64_t)per_sm * num_sms());
  unsigned blocks = (unsigned)std::max<int64_t>(nb, 1);
  double dt2 = dt * dt, inv_h2 = 1.0 / (G.h * G.h);
  int64_t ntiles = eb.num_tiles;
  const int32_t* tiles = eb.tiles;
  const uint8_t* code = eb.code;
  const double* diag = eb.diag;
  Geometry g = G;
  void* args[] = {(void*)&g, (void*)&tiles, (void*)&ntiles, (void*)&code, (void*)&diag, (void*)&ua, (void*)&ub,
                  (void*)&nsteps, (void*)&dt2, (void*)&inv_h2, (void*)&gb};
  EB_CUDA(cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(256), args, 0, s));
  GridBarrier hb{};
  EB_CUDA(cudaMemcpyAsync(&hb, gb, sizeof(hb), cudaMemcpyDeviceToHost, s));
  EB_CUDA(cudaStreamSynchronize(s));
  dfree(gb, s);
  if (hb.err) {
    set_error("leapfrog: grid barrier timed out");
    return EB_ERR_TIMEOUT;
  }
  return EB_OK;
}

template int launch_leapfrog<double>(const EBHandle&, double*, double*, int, double, cudaStream_t);
template int launch_leapfrog<float>(const EBHandle&, float*, float*, int, double, cudaStream_t);

}  // namespace ebk
