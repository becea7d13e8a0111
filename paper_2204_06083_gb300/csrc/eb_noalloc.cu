// wave_step_noalloc: the leapfrog steps of wave_step for callers that must
// not allocate any memory during the call.
//
// wave_step runs whole chunks of steps as a CUDA graph that it builds and
// caches on the handle the first time it sees a set of fields; building that
// graph allocates.  Some callers cannot allow any allocation inside the call:
// loops with a fixed memory budget that must not touch the allocator after
// start-up, processes whose device memory is held by another framework's pool,
// and time-critical loops for which the implicit device synchronisation of
// cudaMalloc / cudaFree is unacceptable.  This variant runs all nsteps in one
// persistent cooperative launch whose scratch -- the state of its grid-wide
// barrier between steps -- lives in a file-scope device array, so a call
// performs no cudaMalloc / cudaFree and calls no allocating library routine.
// The fields and the eb handle are the caller's, created beforehand.
//
// Scratch: one flag per cooperative CTA plus a release counter and an error
// word, at most EB_NOALLOC_MAX_CTAS CTAs (8 KB of flags); the grid is capped
// at that many CTAs.  Every GPU that
// loads the library holds this array until the process exits.  The first call
// on a device looks up the array's device address with that device current
// (cudaGetSymbolAddress, no allocation); make that first call before any
// stream capture.  All calls share the array and it keeps the last call's
// contents, so each call clears the part it uses before its launch; two calls
// whose kernels overlap on the GPU race on it and must not be issued.
#include "eb_internal.cuh"
#include "stencil.cuh"

#include <algorithm>
#include <cstddef>
#include <mutex>

#define EB_NOALLOC_MAX_CTAS 2048

namespace ebk {

struct NoAllocWaveScratch {
  unsigned int gen;                           // steps released by CTA 0
  int err;                                    // set when a bounded wait gave up
  unsigned int pad[62];                       // arrival flags start on their own 256-byte line
  unsigned int arrive[EB_NOALLOC_MAX_CTAS];   // steps finished by each CTA
};

static __device__ __align__(256) NoAllocWaveScratch g_wave_scratch;

constexpr long long NOALLOC_SPIN_LIMIT = 20000000;  // ~ a second of polling

// Barrier after step k (1-based): every CTA publishes k in its flag, CTA 0
// waits for all flags and then publishes k in gen, the others wait for gen.
// Every wait is bounded; on timeout err is set and all later barriers return.
__device__ bool noalloc_sync(NoAllocWaveScratch* sc, unsigned int k) {
  __shared__ int failed;
  if (threadIdx.x == 0) failed = 0;  // before the barrier: pollers below may set it
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicExch(&sc->arrive[blockIdx.x], k);
  }
  volatile int* perr = &sc->err;
  if (blockIdx.x == 0) {
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
      volatile unsigned int* pa = &sc->arrive[b];
      long long spins = 0;
      while (*pa < k) {
        if (*perr || ++spins > NOALLOC_SPIN_LIMIT) {
          atomicExch(&sc->err, 1);
          failed = 1;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();  // acquire: order this thread's observations before the release below
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicExch(&sc->gen, k);
    }
  } else if (threadIdx.x == 0) {
    volatile unsigned int* pg = &sc->gen;
    long long spins = 0;
    while (*pg < k) {
      if (*perr || ++spins > NOALLOC_SPIN_LIMIT) {
        atomicExch(&sc->err, 1);
        failed = 1;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0 && *perr) failed = 1;
  __syncthreads();
  return failed == 0;
}

// Same per-node arithmetic as the leapfrog kernel of wave_step (same results).
template <class T, int DIM>
__global__ void __launch_bounds__(TILE_NODES) k_leapfrog_noalloc(TileView tv, const uint8_t* __restrict__ code,
                                                                 const typename DiagOf<T>::type* __restrict__ diag,
                                                                 T* ua, T* ub, int nsteps, typename AccOf<T>::type c2,
                                                                 NoAllocWaveScratch* sc) {
  using A = typename AccOf<T>::type;
  for (int s = 0; s < nsteps; ++s) {
    T* prev = (s & 1) ? ub : ua;
    const T* cur = (s & 1) ? ua : ub;
    EB_PAIR_LOOP(DIM, tv, node) {
      uint32_t c0, c1;
      ld_codes(code, node, c0, c1);
      Two<A> xc, core;
      stencil_tv<DIM, LdCG>(tv, cur, node, c0, c1, diag, xc, core);
      const Two<A> po = LdCG::ld2(prev + node);
      const A n0 = (c0 & CODE_CP) ? (A)2 * xc.x - po.x - c2 * core.x : (A)0;
      const A n1 = (c1 & CODE_CP) ? (A)2 * xc.y - po.y - c2 * core.y : (A)0;
      st2(prev + node, n0, n1);
    }
    if (!noalloc_sync(sc, (unsigned int)s + 1u)) return;
  }
  // After an odd number of steps the newest field sits in ua: swap.  With a
  // single step ub was never written, so its non-CP entries still hold the
  // caller's input; both fields are masked here (0 off the CPs), as wave_step's
  // masking pass leaves them.
  if (nsteps & 1) {
    EB_PAIR_LOOP(DIM, tv, node) {
      uint32_t c0, c1;
      ld_codes(code, node, c0, c1);
      const bool k0 = (c0 & CODE_CP) != 0, k1 = (c1 & CODE_CP) != 0;
      const Two<A> a = LdCG::ld2(ua + node);
      const Two<A> b = LdCG::ld2(ub + node);
      st2(ua + node, k0 ? b.x : (A)0, k1 ? b.y : (A)0);
      st2(ub + node, k0 ? a.x : (A)0, k1 ? a.y : (A)0);
    }
  }
}

// Device address of the scratch array, looked up once per device with that
// device current (the lookup allocates nothing).
static NoAllocWaveScratch* scratch_for_current_device() {
  static std::mutex mu;
  static NoAllocWaveScratch* addr[64] = {};
  int dev = 0;
  EB_CUDA(cudaGetDevice(&dev));
  EB_REQUIRE(dev >= 0 && dev < 64, EB_ERR_INVALID, "wave_step_noalloc: device ordinal above 63");
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_wave_scratch);
    if (e != cudaSuccess)
      throw Failure{EB_ERR_CUDA, std::string("wave_step_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e)};
    addr[dev] = static_cast<NoAllocWaveScratch*>(p);
  }
  return addr[dev];
}

template <class T>
static int leapfrog_noalloc(const EBHandle& eb, T* ua, T* ub, int nsteps, double dt, cudaStream_t s) {
  NoAllocWaveScratch* sc = scratch_for_current_device();
  if (nsteps <= 0) return EB_OK;
  const Geometry& G = eb.g;
  void* fn = nullptr;
  dim_dispatch(eb, [&](auto D) { fn = (void*)k_leapfrog_noalloc<T, D.value>; });
  int per_sm = 0;
  EB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, TILE_NODES, 0));
  EB_REQUIRE(per_sm > 0, EB_ERR_INVALID, "wave_step_noalloc: kernel cannot be resident");
  // the step body is a grid-stride loop over the tile pairs, so a grid capped
  // at the scratch's flag count gives the same fields (the cap limits
  // parallelism on parts with more resident CTAs, never the result)
  const int64_t nb = std::max<int64_t>(
      1, std::min<int64_t>({eb.num_tiles, (int64_t)per_sm * num_sms(), (int64_t)EB_NOALLOC_MAX_CTAS}));
  // clear the counter, the error word and the flags this launch uses
  EB_CUDA(cudaMemsetAsync(sc, 0, offsetof(NoAllocWaveScratch, arrive) + sizeof(unsigned int) * (size_t)nb, s));
  typename AccOf<T>::type c2 = (typename AccOf<T>::type)(dt * dt / (G.h * G.h));
  TileView tv = eb.tv();
  const uint8_t* code = eb.code;
  const typename DiagOf<T>::type* diag = diag_of<T>(eb);
  void* args[] = {(void*)&tv, (void*)&code, (void*)&diag, (void*)&ua, (void*)&ub, (void*)&nsteps,
                  (void*)&c2, (void*)&sc};
  EB_CUDA(cudaLaunchCooperativeKernel(fn, dim3((unsigned)nb), dim3(TILE_NODES), args, 0, s));
  int err = 0;
  EB_CUDA(cudaMemcpyAsync(&err, &sc->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  EB_CUDA(cudaStreamSynchronize(s));
  if (err) {
    set_error("wave_step_noalloc: grid barrier timed out");
    return EB_ERR_TIMEOUT;
  }
  return EB_OK;
}

}  // namespace ebk

struct eb_handle;
namespace ebk {
const EBHandle& handle_of(const eb_handle* eb);
}

using namespace ebk;

extern "C" int wave_step_noalloc(const eb_handle* eb, int prec, double dt, void* u_prev_dev, void* u_cur_dev,
                                 int nsteps, cudaStream_t stream) {
  if (!eb || !u_prev_dev || !u_cur_dev || nsteps < 0 || !(dt > 0.0) || u_prev_dev == u_cur_dev) {
    set_error("wave_step_noalloc: invalid argument");
    return EB_ERR_INVALID;
  }
  int rc = EB_OK;
  int st = guarded([&] {
    const EBHandle& h = handle_of(eb);
    if (prec == EB_F64)
      rc = leapfrog_noalloc<double>(h, (double*)u_prev_dev, (double*)u_cur_dev, nsteps, dt, stream);
    else if (prec == EB_F32)
      rc = leapfrog_noalloc<float>(h, (float*)u_prev_dev, (float*)u_cur_dev, nsteps, dt, stream);
    else
      throw Failure{EB_ERR_INVALID, "wave_step_noalloc: precision must be EB_F64 or EB_F32"};
  });
  return st != EB_OK ? st : rc;
}
