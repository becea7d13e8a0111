// Learned correction stage of the preconditioner: a small convolutional
// network on the 2D Cartesian grid, its training on the device, the
// solver-generated training pairs, and the stage inside the flexible PCG.
// The paper has no learned component; this extends its AMG-PCG (Algorithm 1
// step 4).  Definitions (network, pairs, loss, stage) are those of include/eb.h.
//
// Storage: hidden activations BF16 NHWC (32 channels = 64 bytes per pixel);
// FP32 master parameters, BF16 copies of the 32 -> 32 weights; every sum in
// FP32.  The four 32 -> 32 layers (99.6 % of the FLOPs) are implicit GEMMs on
// the 5th-generation tensor cores (tcgen05.mma, accumulators in tensor memory),
// fed by tensor copies (TMA) in a warp-specialised pipeline: a job is 128
// pixels of one image row and all 32 output channels; its three input rows
// (130 pixels x 32 channels) and the 9 x 32 x 32 weights sit in shared memory;
// K = 9 taps x 32 channels.  Data gradients run through
// the same kernel with flipped, transposed weights and the ReLU mask of the
// layer input applied in its epilogue; weight gradients are GEMMs over pixels
// (mma.sync fragments) with per-CTA partials summed in a fixed order.  The
// 2 -> 32 and 32 -> 1 layers run on the CUDA cores.  Inference (nn_forward,
// the stage in the PCG) runs all six layers in one launch instead
// (k_net_fwd), with the hidden activations kept in shared memory and tensor
// memory and results identical to the layer-by-layer launches.
#include "eb_solver.cuh"
#include "tma.cuh"

#include <mma.h>

#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

namespace ebk {

using bf16 = __nv_bfloat16;
namespace wm = nvcuda::wmma;

constexpr int NC = 32;    // hidden channels
constexpr int NMID = 4;   // 32 -> 32 layers
constexpr int TPX = 128;  // pixels per CTA job (one row segment)
constexpr int LDA = 48;   // weight-gradient staging: pixel stride in bf16 (96 bytes: 32-byte aligned rows)

// flat parameter vector
constexpr int W1_N = NC * 9 * 2, B1_N = NC;
constexpr int WM_N = NC * 9 * NC, BM_N = NC;
constexpr int W6_N = 9 * NC, B6_N = 1;
constexpr int OFF_W1 = 0;
constexpr int OFF_WM = OFF_W1 + W1_N + B1_N;  // middle layer l at OFF_WM + l (WM_N + BM_N)
constexpr int OFF_W6 = OFF_WM + NMID * (WM_N + BM_N);
constexpr int NPARAM = OFF_W6 + W6_N + B6_N;
static_assert(NPARAM == 37889, "parameter layout");

__host__ __device__ constexpr int off_wm(int l) { return OFF_WM + l * (WM_N + BM_N); }

// A stack of images: H rows of W pixels, image boundaries every R rows.
struct Image {
  int W, H, R;
  __device__ int64_t npx() const { return (int64_t)W * H; }
};

// ------------------------------------------------------------ forward
// layer 1 (2 -> 32) + ReLU; in: (s_hat, m) per pixel.  A thread computes two
// x-adjacent pixels: the 3 x 4 input window is loaded once and every weight
// -- read from shared memory as float4s, two taps' two channels at a time --
// is applied to both pixels, one FMA per multiply-add.
__global__ void __launch_bounds__(128) k_l1_fwd(Image im, const float2* __restrict__ in, const float* __restrict__ P,
                                                bf16* __restrict__ y) {
  constexpr int WS = 20;  // a channel's 9 x 2 weights padded to five float4s
  __shared__ __align__(16) float w[NC * WS + NC];
  for (int i = threadIdx.x; i < NC * WS; i += blockDim.x) {
    const int co = i / WS, j = i % WS;
    w[i] = j < 18 ? P[OFF_W1 + co * 18 + j] : 0.0f;
  }
  for (int i = threadIdx.x; i < NC; i += blockDim.x) w[NC * WS + i] = P[OFF_W1 + W1_N + i];
  __syncthreads();
  const int half = (im.W + 1) >> 1;
  const int64_t pp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pp >= (int64_t)half * im.H) return;
  const int r = (int)(pp / half), x = 2 * (int)(pp - (int64_t)r * half);
  const int lo = (r / im.R) * im.R, hi = lo + im.R;
  float2 v[3][4];
#pragma unroll
  for (int dy = 0; dy < 3; ++dy) {
    const int rr = r + dy - 1;
#pragma unroll
    for (int dx = 0; dx < 4; ++dx) {
      const int xx = x + dx - 1;
      v[dy][dx] = (xx >= 0 && xx < im.W && rr >= lo && rr < hi) ? in[(int64_t)rr * im.W + xx] : make_float2(0.f, 0.f);
    }
  }
  uint32_t o0[NC / 2], o1[NC / 2];
#pragma unroll
  for (int co = 0; co < NC; co += 2) {
    float a[2][2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const float* wc = w + (co + k) * WS;
      float a0 = w[NC * WS + co + k], a1 = a0;
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const float4 t = *reinterpret_cast<const float4*>(wc + 4 * q);
        const int d0 = 2 * q, d1 = 2 * q + 1;
        a0 = fmaf(t.x, v[d0 / 3][d0 % 3].x, a0);
        a0 = fmaf(t.y, v[d0 / 3][d0 % 3].y, a0);
        a1 = fmaf(t.x, v[d0 / 3][d0 % 3 + 1].x, a1);
        a1 = fmaf(t.y, v[d0 / 3][d0 % 3 + 1].y, a1);
        if (d1 < 9) {
          a0 = fmaf(t.z, v[d1 / 3][d1 % 3].x, a0);
          a0 = fmaf(t.w, v[d1 / 3][d1 % 3].y, a0);
          a1 = fmaf(t.z, v[d1 / 3][d1 % 3 + 1].x, a1);
          a1 = fmaf(t.w, v[d1 / 3][d1 % 3 + 1].y, a1);
        }
      }
      a[k][0] = fmaxf(a0, 0.0f);
      a[k][1] = fmaxf(a1, 0.0f);
    }
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(a[0][0], a[1][0]);
    const __nv_bfloat162 h1 = __floats2bfloat162_rn(a[0][1], a[1][1]);
    o0[co / 2] = *reinterpret_cast<const uint32_t*>(&h0);
    o1[co / 2] = *reinterpret_cast<const uint32_t*>(&h1);
  }
  const int64_t p = (int64_t)r * im.W + x;
  int4* dst = reinterpret_cast<int4*>(y + p * NC);
#pragma unroll
  for (int q = 0; q < 4; ++q) dst[q] = make_int4(o0[4 * q], o0[4 * q + 1], o0[4 * q + 2], o0[4 * q + 3]);
  if (x + 1 < im.W) {
#pragma unroll
    for (int q = 0; q < 4; ++q) dst[4 + q] = make_int4(o1[4 * q], o1[4 * q + 1], o1[4 * q + 2], o1[4 * q + 3]);
  }
}

// Stages the rows r-1, r, r+1 (pixels x0-1 .. x0+TPX) of x into sIn [3][TPX+2][LDA],
// zero outside the image.
__device__ __forceinline__ void stage_rows(const Image& im, const bf16* __restrict__ x, int r, int x0, bf16* sIn) {
  const int lo = (r / im.R) * im.R, hi = lo + im.R;
  for (int i = threadIdx.x; i < 3 * (TPX + 2) * 4; i += blockDim.x) {
    const int q = i & 3, px = (i >> 2) % (TPX + 2), rr = (i >> 2) / (TPX + 2);
    const int gx = x0 - 1 + px, gr = r - 1 + rr;
    int4 v = make_int4(0, 0, 0, 0);
    if (gx >= 0 && gx < im.W && gr >= lo && gr < hi)
      v = *reinterpret_cast<const int4*>(x + ((int64_t)gr * im.W + gx) * NC + q * 8);
    *reinterpret_cast<int4*>(sIn + (rr * (TPX + 2) + px) * LDA + q * 8) = v;
  }
}

// ------------------------------------------- 32 -> 32 convolution (tcgen05)
// Implicit GEMM on the 5th-generation tensor cores (kernel k_conv32_tma below).
// The B operand, the weights, sits in shared memory in the no-swizzle K-major
// layout of "core matrices" (8 rows x 16 bytes stored contiguously):
// [tap][channel group g][n][8 k] (SBO = 128 B between 8-row blocks of n,
// LBO = 32 x 16 B between channel groups).  The A operand (activations) uses the
// 64-byte swizzled layout written by the tensor copies (tc_desc_sw64).
constexpr int TC_PIX = TPX + 2;                  // pixels of a job's rows with their two halo pixels
constexpr int TC_A = 3 * TC_PIX * NC * 2;        // a job's three rows: 24,960 bytes
constexpr int TC_WTAP = 4 * NC * 16;             // 2048 per tap
constexpr int TC_W = 9 * TC_WTAP;                // 18,432
constexpr uint32_t TC_SPIN = 1u << 22;           // bounded mbarrier polls (~0.1 s)

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, LBO, SBO (bytes), version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// shared-memory matrix descriptor of a K-major operand in the 64-byte swizzled
// layout: rows of 64 bytes (32 bf16 along K), the 16-byte chunks of a row
// permuted by the address bits 7-8 as the tensor copies write them, 8-row
// groups 512 bytes apart (SBO); LBO unused (the K extent of one MMA, 32 bytes,
// lies inside a row); swizzle mode 4 (64 bytes) in bits 61-63
__device__ __forceinline__ uint64_t tc_desc_sw64(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

// instruction descriptor of kind::f16: D f32, A and B bf16, both K-major, N, M
__device__ __forceinline__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ------------------------- 32 -> 32 convolution, TMA-fed warp-specialised pipeline
// y = conv(x; wk) + bias (if bias), then ReLU (if relu), then 0 where
// mask_ref <= 0 (if mask_ref: the ReLU derivative of a data gradient).
// wk: bf16 [9][32 (n)][32 (k)].  A job is 128 pixels of one image row and all
// 32 output channels: M = 128, N = 32, K = 9 taps x 32 channels = 18 MMAs of
// 128 x 32 x 16 (bf16 in, f32 in TMEM).  One thread issues, per job, one 4D
// tensor copy (cp.async.bulk.tensor) of the job's 3 rows x 130 pixels x 32
// channels into a ring of CP_STAGES buffers, in the 64-byte swizzled K-major
// layout (a pixel's 32 channels are one 64-byte row); the operand of tap
// (dy, dx) and channel half kh starts at row dy * 130 + dx, byte 32 kh.  One
// thread issues the 18 MMAs of each job into one of two TMEM accumulators;
// four warps drain the accumulators (tcgen05.ld: warp w reads TMEM lanes
// 32 w .. 32 w + 31, its 32 pixels) and run the epilogue while the next jobs
// load and multiply.  The tensor map views the activations as (32 channels,
// pixel, row in image, image), so the rows outside an image and the pixels
// outside a row are filled with zeros by the copy.
// Barriers: full[s] (copy -> MMA, transaction bytes), empty[s] (MMA commit ->
// copy), tfull[a] (MMA commit -> epilogue), tempty[a] (4 epilogue warps ->
// MMA).  Every wait is bounded; a wait that gives up raises a shared abort
// flag that ends every role's loop, sets *err, and the CTA waits (bounded) for
// its copies and MMAs in flight before freeing TMEM.
constexpr int CP_STAGES = 2;
constexpr int CP_STAGE = 25600;                        // TC_A rounded up to 1 KB (swizzle atoms stay aligned)
constexpr int CP_W = CP_STAGES * CP_STAGE;             // weights after the stages
constexpr int CP_BAR = CP_W + TC_W;                    // barriers after the weights
constexpr int CP_NBAR = 2 * CP_STAGES + 4;
constexpr int CP_SMEM = CP_BAR + 8 * CP_NBAR + 16;     // + TMEM slot and abort flag
constexpr int CP_THREADS = 192;                        // warps 0-3 epilogue, 4 copies, 5 MMAs
constexpr uint32_t CP_BOX_BYTES = 3 * TC_PIX * NC * 2;  // 24,960
static_assert(CP_BOX_BYTES == TC_A, "box = staged operand");

__device__ __forceinline__ bool cp_wait(uint32_t bar, uint32_t parity, volatile int* abort) {
  for (uint32_t it = 0; it < TC_SPIN; ++it) {
    uint32_t ok = 0;
    asm volatile(
        "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 63) == 63 && *abort) return false;
  }
  *abort = 1;
  return false;
}

__global__ void __launch_bounds__(CP_THREADS, 3) k_conv32_tma(const __grid_constant__ CUtensorMap xmap, Image im,
                                                               const bf16* __restrict__ wk,
                                                               const float* __restrict__ bias, bf16* __restrict__ y,
                                                               int relu, const bf16* __restrict__ mask_ref,
                                                               int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sW = smem_raw + CP_W;
  const uint32_t base = smem_addr(smem_raw);
  const uint32_t a0 = base, w0 = base + CP_W, bars = base + CP_BAR;
  auto full = [&](int st) { return bars + 8 * st; };
  auto empty = [&](int st) { return bars + 8 * (CP_STAGES + st); };
  auto tfull = [&](int a) { return bars + 8 * (2 * CP_STAGES + a); };
  auto tempty = [&](int a) { return bars + 8 * (2 * CP_STAGES + 2 + a); };
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem_raw + CP_BAR + 8 * CP_NBAR);
  volatile int* abort = reinterpret_cast<volatile int*>(smem_raw + CP_BAR + 8 * CP_NBAR + 8);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < 9 * NC * 4; i += CP_THREADS) {  // weights once per CTA
    const int g = i & 3, n = (i >> 2) % NC, d = (i >> 2) / NC;
    *reinterpret_cast<int4*>(sW + d * TC_WTAP + g * (NC * 16) + n * 16) =
        *reinterpret_cast<const int4*>(wk + (d * NC + n) * NC + g * 8);
  }
  if (tid == 0) {
    for (int b = 0; b < CP_NBAR; ++b) {
      const uint32_t cnt = (b >= 2 * CP_STAGES + 2) ? 4u : 1u;  // tempty: one arrive per epilogue warp
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bars + 8 * b), "r"(cnt));
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_addr(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;");  // weights (generic stores) are read by the tensor cores
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  const int segs = (im.W + TPX - 1) / TPX;
  const int64_t jobs = (int64_t)segs * im.H;
  const int64_t njob = jobs > (int64_t)blockIdx.x ? (jobs - 1 - blockIdx.x) / gridDim.x + 1 : 0;  // this CTA's jobs
  if (warp == 4) {
    // copies: stage s = k mod S, its u-th use waits for the MMAs of use u - 1
    if (lane == 0) {
      const uint64_t map = reinterpret_cast<uint64_t>(&xmap);
      asm volatile("prefetch.tensormap [%0];" ::"l"(map) : "memory");
      int64_t k = 0;
      for (; k < njob; ++k) {
        const int st = (int)(k % CP_STAGES);
        const uint32_t u = (uint32_t)(k / CP_STAGES);
        if (u > 0 && !cp_wait(empty(st), (u - 1) & 1u, abort)) break;
        const int64_t job = blockIdx.x + k * gridDim.x;
        const int r = (int)(job / segs), x0 = (int)(job % segs) * TPX;
        const int img = r / im.R, rin = r - img * im.R;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(full(st)), "r"(CP_BOX_BYTES)
                     : "memory");
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
            "%5}], [%6];" ::"r"(a0 + st * CP_STAGE),
            "l"(map), "r"(0), "r"(x0 - 1), "r"(rin - 1), "r"(img), "r"(full(st))
            : "memory");
      }
      // copies still in flight (an aborted run) land before the CTA ends
      for (int64_t q = k > CP_STAGES ? k - CP_STAGES : 0; q < k; ++q) {
        volatile int never = 0;
        cp_wait(full((int)(q % CP_STAGES)), (uint32_t)(q / CP_STAGES) & 1u, &never);
      }
    }
  } else if (warp == 5) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc_idesc(128, NC);
      int64_t k = 0;
      for (; k < njob; ++k) {
        const int st = (int)(k % CP_STAGES);
        const int a = (int)(k & 1);
        if (!cp_wait(full(st), (uint32_t)(k / CP_STAGES) & 1u, abort)) break;
        if (k >= 2 && !cp_wait(tempty(a), (uint32_t)((k >> 1) - 1) & 1u, abort)) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t sa = a0 + st * CP_STAGE;
#pragma unroll 1
        for (int q = 0; q < 18; ++q) {
          const int d = q >> 1, kh = q & 1, dy = d / 3, dx = d % 3;
          const uint64_t da = tc_desc_sw64(sa + (dy * TC_PIX + dx) * 64 + kh * 32);
          const uint64_t db = tc_desc(w0 + d * TC_WTAP + (2 * kh) * (NC * 16), NC * 16, 128);
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem + (uint32_t)(a * NC)),
              "l"(da), "l"(db), "r"(idesc), "r"((uint32_t)(q > 0)));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(empty(st))
                     : "memory");
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tfull(a))
                     : "memory");
      }
      if (k > 0) {  // the last MMAs complete before TMEM is freed
        volatile int never = 0;
        cp_wait(tfull((int)((k - 1) & 1)), (uint32_t)(((k - 1) >> 1) & 1), &never);
      }
    }
  } else {
    // epilogue: warp w drains TMEM lanes 32 w .. 32 w + 31 (pixels x0 + 32 w + lane)
    float bv[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) bv[c] = bias ? bias[c] : 0.0f;
    for (int64_t k = 0; k < njob; ++k) {
      const int a = (int)(k & 1);
      // the warp leaves together or not at all (tcgen05.ld is warp-collective)
      const bool okl = cp_wait(tfull(a), (uint32_t)(k >> 1) & 1u, abort);
      if (!__all_sync(0xffffffffu, okl)) {
        *abort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      uint32_t v[NC];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
          "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
            "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
            "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
          : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(a * NC)));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tempty(a)) : "memory");
      const int64_t job = blockIdx.x + k * gridDim.x;
      const int r = (int)(job / segs), x0 = (int)(job % segs) * TPX;
      const int gx = x0 + warp * 32 + lane;
      if (gx < im.W) {
        const int64_t p = (int64_t)r * im.W + gx;
        __align__(16) bf16 ov[NC];
        __align__(16) bf16 mr[NC];
        if (mask_ref) {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            reinterpret_cast<int4*>(mr)[q] = reinterpret_cast<const int4*>(mask_ref + p * NC)[q];
        }
#pragma unroll
        for (int co = 0; co < NC; ++co) {
          float f = __uint_as_float(v[co]) + bv[co];
          if (relu) f = fmaxf(f, 0.0f);
          if (mask_ref && !(__bfloat162float(mr[co]) > 0.0f)) f = 0.0f;
          ov[co] = __float2bfloat16_rn(f);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) reinterpret_cast<int4*>(y + p * NC)[q] = reinterpret_cast<const int4*>(ov)[q];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid == 0 && *abort) atomicExch(err, 1);
  if (warp == 5) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem));
  }
}

// layer 6 (32 -> 1); out = m * (conv + b6).  Each tap's 32-channel sum is
// formed on its own (one FMA chain from 0) and the nine are added to b6 in tap
// order: the order of k_net_fwd, whose results this kernel reproduces bit for
// bit.
__global__ void k_l6_fwd(Image im, const bf16* __restrict__ y5, const float* __restrict__ P,
                         const float2* __restrict__ in, float* __restrict__ out) {
  __shared__ float w[W6_N + B6_N];
  for (int i = threadIdx.x; i < W6_N + B6_N; i += blockDim.x) w[i] = P[OFF_W6 + i];
  __syncthreads();
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= im.npx()) return;
  const int x = (int)(p % im.W), r = (int)(p / im.W);
  const int lo = (r / im.R) * im.R, hi = lo + im.R;
  float a = w[W6_N];
  for (int d = 0; d < 9; ++d) {
    const int xx = x + d % 3 - 1, rr = r + d / 3 - 1;
    if (xx < 0 || xx >= im.W || rr < lo || rr >= hi) continue;
    const int4* src = reinterpret_cast<const int4*>(y5 + ((int64_t)rr * im.W + xx) * NC);
    float t = 0.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int4 v = src[q];
      const bf16* e = reinterpret_cast<const bf16*>(&v);
#pragma unroll
      for (int c = 0; c < 8; ++c) t = __fmaf_rn(w[d * NC + q * 8 + c], __bfloat162float(e[c]), t);
    }
    a = __fadd_rn(a, t);
  }
  out[p] = in[p].y * a;
}

// --------------------------------------------- fused forward: all six layers
// One launch computes N(in) with every hidden activation kept on chip.  A CTA
// owns a strip of FZ_OUT = 116 output columns and a run of rows of one image
// and walks down it one step at a time; step tau computes layer 1 at row tau,
// layer l (2..5) at row tau - 2 (l - 1) and layer 6 at row tau - 10, so the
// rows a step reads were all finished in earlier steps and the layers of one
// step are independent.  Every layer computes 128 columns (the tensor cores'
// M), the strip's 116 plus 6 on each side: layer l is exact on 128 - 2 (l - 1)
// of them, which leaves layer 6 exact on the strip.
//   * layer 1 (2 -> 32, CUDA cores, warps 4-7): one pixel per thread, eight
//     output channels' FMA chains side by side, each in k_l1_fwd's order;
//     bf16 result into ring 0.  The input window is loaded a step ahead.
//   * layers 2-5 (tcgen05, lane 0 of warp 8 + l - 2): the MMAs are input-row
//     stationary.  At step tau layer l takes its newest input row, rho + 1
//     (rho = the output row it finishes), from ring l - 2 (64-byte swizzled
//     K-major rows of 64 bytes, one per pixel, as k_conv32_tma's tensor
//     copies lay them out) and multiplies it, shifted by dx = 0, 1, 2 pixels
//     and split in two channel halves, by the weights of the three tap rows
//     at once: N = 96 = (dy, n), contributions to output rows rho + 2 - dy.
//     Each output row accumulates in one of four 32-column TMEM slots per
//     layer, placed so that rows rho + 2, rho + 1, rho lie at increasing
//     columns; runs of adjacent slots take one MMA per (dx, kh), so a layer
//     issues 6 MMAs per step (12 when the three slots wrap), a third of the
//     18 of the output-stationary form.  The slot of row rho receives its taps
//     in (dy, dx, kh) order, the order of k_conv32_tma's 18 MMAs, from zero.
//   * epilogues of layers 2-4 (warps 0-3, one TMEM lane = one pixel per
//     thread): read the finished slot of row rho and zero it for row rho + 4,
//     bias, ReLU, bf16, 0 outside the image (the next layer's zero padding),
//     into ring l - 1 (the swizzle applied by hand).
//   * layers 5-6 (warps 12-15): layer 5's epilogue forms the nine tap
//     partials of layer 6 (a float per tap and pixel, ring T) from its
//     bf16-rounded values, nine FMA chains side by side; layer 6 adds them up:
//     out = m (b6 + sum).
// Activation rings hold 2 rows (row rho in slot rho & 1): a step reads row
// rho + 1 of a ring and writes row rho + 2.  T holds 4.  Every layer's
// arithmetic is that of the layer-by-layer path (k_l1_fwd, k_conv32_tma,
// k_l6_fwd), so the two give identical outputs.
// Barriers (mbarriers, two of each kind per layer, by step parity): rdy[j][b]
// (ring j row of step k written: 4 warp arrivals -> MMA of layer j + 2 at
// step k + 1), mdone[j][b] (commit of layer j + 2's MMAs at step k ->
// epilogue; mdone[0] also frees ring 0's older row for layer 1), tempty[j][b]
// (slot read and zeroed: 4 warp arrivals -> MMA at step k + 2, or k + 1 at a
// unit's first step, after the last step of the unit before has cleared every
// slot).  With two barriers per kind no waiter can fall two phases behind.
// The epilogue of layer l at step k overwrites the row of ring l - 1 that
// layer l + 1's MMAs read at step k - 1: for l = 2, 3 the epilogue warps
// waited for those (mdone of layer l + 1, step k - 1) earlier in their own
// program order, for l = 4 they wait for layer 5's explicitly.  Every wait is
// bounded; one that gives up raises a shared abort flag, after which every
// role runs its remaining steps without waiting or computing (so the named
// barriers still match), the CTA waits (bounded) for its MMAs in flight,
// frees TMEM and sets *err.
constexpr int FZ_OUT = TPX - 12;                       // 116
constexpr int FZ_ROW = TC_PIX * NC * 2;                // 8320 bytes: one activation row, 130 pixel slots
constexpr int FZ_RING = 2;                             // rows per activation ring
constexpr int FZ_RINGB = FZ_RING * FZ_ROW;             // 16,640
constexpr int FZ_W = 4 * FZ_RINGB;                     // weights of layers 2-5: 66,560
constexpr int FZ_WDX = 4 * 96 * 16;                    // B bytes of one horizontal tap: 6144
constexpr int FZ_TRING = 4;                            // rows of the tap-partial ring
constexpr int FZ_TROW = 9 * TC_PIX;                    // floats of a T row: 9 taps x 130 slots
constexpr int FZ_T = FZ_W + NMID * TC_W;               // 140,288
constexpr int FZ_W1 = FZ_T + FZ_TRING * FZ_TROW * 4;   // 159,008: layer-1 weights [d][ci][co], then b1
constexpr int FZ_W6 = FZ_W1 + (NC * 20 + NC) * 4;      // 161,696: W6 as [c][12 taps], then b6
constexpr int FZ_BM = FZ_W6 + 1552;                    // 163,248: biases of layers 2-5
constexpr int FZ_BAR = FZ_BM + NMID * NC * 4;          // 163,760
constexpr int FZ_NBAR = 24;
constexpr int FZ_SMEM = FZ_BAR + 8 * FZ_NBAR + 16;     // 163,968
constexpr int FZ_THREADS = 512;  // warps 0-3 epilogues 2-4, 4-7 layer 1, 8-11 MMAs, 12-15 layers 5-6
static_assert(FZ_SMEM <= 232448, "fused forward: shared memory");
static_assert(FZ_W % 1024 == 0 && FZ_T % 16 == 0 && FZ_BAR % 8 == 0, "fused forward: alignment");

struct FzArgs {
  Image im;
  const float2* in;
  float* out;
  const float* P;
  const bf16* wf;  // [4][9][32 n][32 k] bf16
  int strips, segs, seg_rows;
  int64_t units;
  int* err;
};

// 64 bytes (32 bf16 = 16 words) into the pixel row at shared address row (a
// multiple of 64) in the 64-byte swizzled layout: 16-byte chunk c of the row
// lands at chunk c ^ (address bits 7-8)
__device__ __forceinline__ void fz_st_row(uint32_t row, const uint32_t (&w)[NC / 2]) {
  const uint32_t sw = (row >> 7) & 3u;
#pragma unroll
  for (int c = 0; c < 4; ++c)
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(row + ((c ^ sw) << 4)), "r"(w[4 * c]),
                 "r"(w[4 * c + 1]), "r"(w[4 * c + 2]), "r"(w[4 * c + 3])
                 : "memory");
}

// Bounded wait of the fused kernel: the waiting thread asks to be suspended
// (up to 20 us per try) until the phase completes, so that spinning warps do
// not take issue slots from the working ones on the same scheduler; gives up
// after FZ_WAIT_NS of wall time (global timer) or when *abort is raised,
// raising it itself on the time limit.
constexpr uint64_t FZ_WAIT_NS = 200000000ull;  // 0.2 s
__device__ __forceinline__ uint64_t fz_now() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool fz_wait(uint32_t bar, uint32_t parity, volatile int* abort) {
  uint64_t t0 = 0;
  for (uint32_t it = 0; it < (1u << 26); ++it) {  // the iteration bound backs up the time limit
    uint32_t ok = 0;
    asm volatile(
        "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2, 20000;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (it == 0) t0 = fz_now();
    if ((it & 15) == 15) {
      if (*abort) return false;
      if (fz_now() - t0 > FZ_WAIT_NS) break;
    }
  }
  *abort = 1;
  return false;
}

// tensor-memory column (within a layer's 128) of the accumulator of output row
// r: four slots, r & 3 = 3, 2, 1, 0 at columns 0, 32, 64, 96, so that rows
// r + 2, r + 1, r (which one input row feeds) lie at increasing columns
__device__ __forceinline__ int fz_col(int r) { return 32 * (3 - (r & 3)); }

// 32 zero columns of tensor memory at taddr for this warp's 32 lanes
__device__ __forceinline__ void fz_tmem_zero32(uint32_t taddr) {
  const uint32_t z = 0u;
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,"
      "%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
      "r"(z)
      : "memory");
}

// Reads the finished accumulator of output row rho of layer j + 2 (32 columns,
// this warp's lanes; tlane = TMEM address of lane 32 (warp % 4), column 0)
// into v, then starts zeroing its slot for row rho + 4 (all four slots of the
// layer at a unit's last step, which leaves no partial sums to the next unit);
// fz_release completes it.  okw (warp-uniform) false: nothing is read, v = 0.
__device__ __forceinline__ void fz_take(uint32_t tlane, int j, int rho, bool okw, bool last, uint32_t (&v)[NC]) {
  const uint32_t tacc = tlane + (uint32_t)(j * 128 + fz_col(rho));
  if (okw) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
          "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(tacc));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (last) {
      for (int c = 0; c < 128; c += 32) fz_tmem_zero32(tlane + (uint32_t)(j * 128 + c));
    } else {
      fz_tmem_zero32(tacc);
    }
  } else {
#pragma unroll
    for (int c = 0; c < NC; ++c) v[c] = 0u;
  }
}

// after fz_take: the zeroing stores are complete and the slot is released to
// the MMAs (whose next write to it comes two steps on)
__device__ __forceinline__ void fz_release(uint32_t tempty) {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncwarp();
  if ((threadIdx.x & 31) == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tempty) : "memory");
}

// Packed FP32 pairs: fma.rn.f32x2 is two round-to-nearest FMAs in one
// instruction, so each lane's result is the scalar __fmaf_rn's while the
// fused kernel's CUDA-core layers issue half the FMA instructions.
__device__ __forceinline__ uint64_t fz_pk(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void fz_upk(uint64_t v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ void fz_fma2(uint64_t& acc, uint64_t w, uint64_t x) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(w), "l"(x));
}
// (a0 + b0, a1 + b1), each rounded to nearest as a scalar addition
__device__ __forceinline__ void fz_add2(float a0, float a1, float b0, float b1, float& r0, float& r1) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(fz_pk(a0, a1)), "l"(fz_pk(b0, b1)));
  fz_upk(r, r0, r1);
}

// the 3 x 3 input window of pixel x in row tau of image img (0 outside the image)
__device__ __forceinline__ void fz_window(const FzArgs& a, int img, int tau, int x, float2 (&v)[9]) {
  const bool in = tau >= 0 && tau < a.im.R && x >= 0 && x < a.im.W;
#pragma unroll
  for (int d = 0; d < 9; ++d) {
    const int xx = x + d % 3 - 1, rr = tau + d / 3 - 1;
    v[d] = (in && xx >= 0 && xx < a.im.W && rr >= 0 && rr < a.im.R)
               ? __ldg(a.in + ((int64_t)img * a.im.R + rr) * a.im.W + xx)
               : make_float2(0.f, 0.f);
  }
}

__device__ __forceinline__ void fz_unit(const FzArgs& a, int64_t u, int& img, int& r0, int& r1, int& x0) {
  const int strip = (int)(u % a.strips);
  const int64_t q = u / a.strips;
  const int seg = (int)(q % a.segs);
  img = (int)(q / a.segs);
  x0 = strip * FZ_OUT;
  r0 = seg * a.seg_rows;
  r1 = min(r0 + a.seg_rows, a.im.R);
}

__global__ void __launch_bounds__(FZ_THREADS, 1) k_net_fwd(const __grid_constant__ FzArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t base = smem_addr(smem_raw);
  const uint32_t bars = base + FZ_BAR;
  auto rdy = [&](int j, int b) { return bars + 8 * (2 * j + b); };
  auto mdone = [&](int j, int b) { return bars + 8 * (8 + 2 * j + b); };
  auto tempty = [&](int j, int b) { return bars + 8 * (16 + 2 * j + b); };
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem_raw + FZ_BAR + 8 * FZ_NBAR);
  volatile int* abort = reinterpret_cast<volatile int*>(smem_raw + FZ_BAR + 8 * FZ_NBAR + 8);
  float* sT = reinterpret_cast<float*>(smem_raw + FZ_T);
  float* sW1 = reinterpret_cast<float*>(smem_raw + FZ_W1);
  float* sW6 = reinterpret_cast<float*>(smem_raw + FZ_W6);
  float* sBM = reinterpret_cast<float*>(smem_raw + FZ_BM);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const Image& im = a.im;

  // rings and T start at 0 (slots 0 and 129 of every ring row stay 0)
  for (int i = tid; i < FZ_W / 16; i += FZ_THREADS) reinterpret_cast<int4*>(smem_raw)[i] = make_int4(0, 0, 0, 0);
  for (int i = tid; i < FZ_TRING * FZ_TROW; i += FZ_THREADS) sT[i] = 0.0f;
  for (int i = tid; i < NMID * 9 * NC * 4; i += FZ_THREADS) {  // B operands, as in k_conv32_tma
    // [dx][channel group g][dy * 32 + n][8 k]: one horizontal tap's three tap rows side by side in N
    const int g = i & 3, n = (i >> 2) % NC, d = ((i >> 2) / NC) % 9, l = (i >> 2) / (NC * 9);
    const int dy = d / 3, dx = d % 3;
    *reinterpret_cast<int4*>(smem_raw + FZ_W + l * TC_W + dx * FZ_WDX + g * (96 * 16) + (dy * NC + n) * 16) =
        *reinterpret_cast<const int4*>(a.wf + (int64_t)l * WM_N + (d * NC + n) * NC + g * 8);
  }
  // layer 1: weight (tap d, input ci) of the 32 outputs contiguous, so that a
  // thread feeds eight output channels' FMA chains from two float4 loads
  for (int i = tid; i < 18 * NC; i += FZ_THREADS) {
    const int co = i % NC, q = i / NC;
    sW1[i] = a.P[OFF_W1 + co * 18 + q];
  }
  for (int i = tid; i < NC; i += FZ_THREADS) sW1[18 * NC + i] = a.P[OFF_W1 + W1_N + i];
  // layer 6: the nine taps of input channel c contiguous (padded to 12)
  for (int i = tid; i < NC * 12; i += FZ_THREADS) {
    const int c = i / 12, d = i % 12;
    sW6[i] = d < 9 ? a.P[OFF_W6 + d * NC + c] : 0.0f;
  }
  if (tid == 0) sW6[NC * 12] = a.P[OFF_W6 + W6_N];
  for (int i = tid; i < NMID * NC; i += FZ_THREADS) sBM[i] = a.P[off_wm(i / NC) + WM_N + i % NC];
  if (tid == 0) {
    for (int b = 0; b < FZ_NBAR; ++b) {
      const uint32_t cnt = (b >= 8 && b < 16) ? 1u : 4u;  // mdone: one commit; rdy, tempty: four warps
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bars + 8 * b), "r"(cnt));
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_addr(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;");  // zeroed rings and weights are read by the tensor cores
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  // every MMA accumulates: the output-row slots of tensor memory start at 0
  if (warp < 4) {
    for (int c = 0; c < 512; c += 32) fz_tmem_zero32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c);
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");

  if (warp >= 12) {
    // layer 5's epilogue, layer 6 and the tap partials (warps 12-15): thread t
    // = TMEM lane t = pixel slot t + 1 (warp w reads lanes 32 (w - 12) ..)
    const int t = tid - 384;
    const uint32_t tlane = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    int64_t k = 0;
    for (int64_t u = blockIdx.x; u < a.units; u += gridDim.x) {
      int img, r0, r1, x0;
      fz_unit(a, u, img, r0, r1, x0);
      const int nsteps = r1 - r0 + 15;
      const int x = x0 - 6 + t;
      for (int st = 0; st < nsteps; ++st, ++k) {
        const int tau = r0 - 5 + st;
        // layer 6 writes row tau - 10 at the end of the step: its mask value now
        const int r6 = tau - 10;
        const bool out6 = r6 >= r0 && r6 < r1 && t >= 6 && t < 6 + FZ_OUT && x < im.W;
        const int64_t p6 = ((int64_t)img * im.R + r6) * im.W + x;
        const float m6 = out6 ? __ldg(a.in + p6).y : 0.0f;
        // layer 5 (row tau - 8): its values, bf16-rounded as layer 6 reads them
        const int j = NMID - 1, b = (int)(k & 1);
        const bool okl = fz_wait(mdone(j, b), (uint32_t)(k >> 1) & 1u, abort) && !*abort;
        const bool okw = __all_sync(0xffffffffu, okl);  // tcgen05.ld is warp-collective
        const int rho = tau - 2 * (j + 1);
        uint32_t v5[NC];
        fz_take(tlane, j, rho, okw, st == nsteps - 1, v5);
        const bool in_img = okw && rho >= 0 && rho < im.R && x >= 0 && x < im.W;
        fz_release(tempty(j, b));
        // layer 6 at row tau - 10 from the tap partials of earlier steps
        asm volatile("bar.sync 2, 128;" ::: "memory");
        if (!*abort && out6) {
          float acc = sW6[NC * 12];
#pragma unroll
          for (int d = 0; d < 9; ++d) {
            const int dy = d / 3, dx = d % 3;
            acc = __fadd_rn(acc, sT[((r6 - 1 + dy) & 3) * FZ_TROW + d * TC_PIX + t + dx]);
          }
          a.out[p6] = m6 * acc;
        }
        asm volatile("bar.sync 2, 128;" ::: "memory");
        // tap partials of layer 5's row rho
        const float* bj = sBM + j * NC;
        float f[NC];
#pragma unroll
        for (int c = 0; c < NC; c += 2) {
          float s0, s1;
          fz_add2(__uint_as_float(v5[c]), __uint_as_float(v5[c + 1]), bj[c], bj[c + 1], s0, s1);
          f[c] = in_img ? __bfloat162float(__float2bfloat16_rn(fmaxf(s0, 0.0f))) : 0.0f;
          f[c + 1] = in_img ? __bfloat162float(__float2bfloat16_rn(fmaxf(s1, 0.0f))) : 0.0f;
        }
        // nine chains over c = 0 .. 31, side by side (taps in pairs)
        uint64_t tp[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) tp[q] = fz_pk(0.0f, 0.0f);
        float t8 = 0.0f;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const float4 wa = *reinterpret_cast<const float4*>(sW6 + c * 12);
          const float4 wb = *reinterpret_cast<const float4*>(sW6 + c * 12 + 4);
          const float wc = sW6[c * 12 + 8];
          const uint64_t f2 = fz_pk(f[c], f[c]);
          fz_fma2(tp[0], fz_pk(wa.x, wa.y), f2);
          fz_fma2(tp[1], fz_pk(wa.z, wa.w), f2);
          fz_fma2(tp[2], fz_pk(wb.x, wb.y), f2);
          fz_fma2(tp[3], fz_pk(wb.z, wb.w), f2);
          t8 = __fmaf_rn(wc, f[c], t8);
        }
        float* tr = sT + (rho & 3) * FZ_TROW + t + 1;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float ta, tb;
          fz_upk(tp[q], ta, tb);
          tr[(2 * q) * TC_PIX] = ta;
          tr[(2 * q + 1) * TC_PIX] = tb;
        }
        tr[8 * TC_PIX] = t8;
      }
    }
  } else if (warp >= 8) {
    // warp 8 + j issues the MMAs of layer j + 2 (ring j in): one issuing thread
    // per layer, so that the four layers' MMAs of a step overlap on the tensor
    // cores (an issuing thread waits out each MMA's operand fetch)
    if (lane == 0) {
      const int j = warp - 8;
      int64_t k = 0;
      uint32_t last_bar = 0, last_par = 0;
      bool ok = true;
      for (int64_t u = blockIdx.x; u < a.units && ok; u += gridDim.x) {
        int img, r0, r1, x0;
        fz_unit(a, u, img, r0, r1, x0);
        const int nsteps = r1 - r0 + 15;
        for (int st = 0; st < nsteps && ok; ++st, ++k) {
          const int tau = r0 - 5 + st, b = (int)(k & 1);
          {
            if (k >= 1 && !fz_wait(rdy(j, (int)((k - 1) & 1)), (uint32_t)((k - 1) >> 1) & 1u, abort)) {
              ok = false;
              break;
            }
            // slots are reused four rows later: the epilogue of step k - 2 has read and
            // zeroed the slot written first here; the first step of a unit also waits
            // for the step before, whose epilogue cleared the previous unit's slots
            if (st == 0 && k >= 1) {
              if (!fz_wait(tempty(j, (int)((k - 1) & 1)), (uint32_t)((k - 1) >> 1) & 1u, abort)) {
                ok = false;
                break;
              }
            } else if (k >= 2 && !fz_wait(tempty(j, b), (uint32_t)((k - 2) >> 1) & 1u, abort)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            // input row rho + 1 (the newest) enters output rows rho + 2, rho + 1 and
            // rho (tap rows dy = 0, 1, 2): runs of those whose slots are adjacent
            // in tensor memory take one MMA per (dx, kh), N = 32 x run length
            const int rho = tau - 2 * (j + 1);
            const uint32_t row = base + (uint32_t)(j * FZ_RINGB + ((rho + 1) & 1) * FZ_ROW);
            const uint32_t wl = base + (uint32_t)(FZ_W + j * TC_W);
            for (int dy = 0; dy < 3;) {
              const int c0 = fz_col(rho + 2 - dy);
              int n = 1;
              while (dy + n < 3 && fz_col(rho + 2 - dy - n) == c0 + 32 * n) ++n;
              const uint32_t idesc = tc_idesc(128, 32 * n);
#pragma unroll 1
              for (int q = 0; q < 6; ++q) {
                const int dx = q >> 1, kh = q & 1;
                const uint64_t da = tc_desc_sw64(row + dx * 64 + kh * 32);
                const uint64_t db =
                    tc_desc(wl + (uint32_t)(dx * FZ_WDX + (2 * kh) * (96 * 16) + dy * NC * 16), 96 * 16, 128);
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(
                        tmem + (uint32_t)(j * 128 + c0)),
                    "l"(da), "l"(db), "r"(idesc), "r"(1u));
              }
              dy += n;
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             mdone(j, b))
                         : "memory");
            last_bar = mdone(j, b);
            last_par = (uint32_t)(k >> 1) & 1u;
          }
        }
      }
      if (last_bar) {  // the last commit covers every MMA this thread issued: they finish before TMEM is freed
        volatile int never = 0;
        fz_wait(last_bar, last_par, &never);
      }
    }
  } else if (warp >= 4) {
    // layer 1 (warps 4-7): thread t = pixel slot t + 1 of ring 0
    const int t = tid - 128;
    int64_t k = 0;
    for (int64_t u = blockIdx.x; u < a.units; u += gridDim.x) {
      int img, r0, r1, x0;
      fz_unit(a, u, img, r0, r1, x0);
      const int nsteps = r1 - r0 + 15;
      const int x = x0 - 6 + t;
      float2 vn[9];
      fz_window(a, img, r0 - 5, x, vn);
      for (int st = 0; st < nsteps; ++st, ++k) {
        const int tau = r0 - 5 + st;
        // the input window of this step, loaded one step ahead; the next step's now
        const bool l1_in = tau >= 0 && tau < im.R && x >= 0 && x < im.W;
        float2 v[9];
#pragma unroll
        for (int d = 0; d < 9; ++d) v[d] = vn[d];
        if (st + 1 < nsteps) fz_window(a, img, tau + 1, x, vn);
        bool ok = true;
        if (k >= 1) ok = fz_wait(mdone(0, (int)((k - 1) & 1)), (uint32_t)((k - 1) >> 1) & 1u, abort);
        uint32_t o[NC / 2];
#pragma unroll
        for (int c = 0; c < NC / 2; ++c) o[c] = 0u;
        if (ok && !*abort && l1_in) {
          // eight output channels at a time, each one FMA chain in k_l1_fwd's order
#pragma unroll
          for (int cg = 0; cg < NC; cg += 8) {
            uint64_t acc[4];  // channel pairs (cg + 2q, cg + 2q + 1)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fz_pk(sW1[18 * NC + cg + 2 * q], sW1[18 * NC + cg + 2 * q + 1]);
#pragma unroll
            for (int e = 0; e < 18; ++e) {
              const float4 wa = *reinterpret_cast<const float4*>(sW1 + e * NC + cg);
              const float4 wb = *reinterpret_cast<const float4*>(sW1 + e * NC + cg + 4);
              const float xv = (e & 1) ? v[e >> 1].y : v[e >> 1].x;
              const uint64_t x2 = fz_pk(xv, xv);
              fz_fma2(acc[0], fz_pk(wa.x, wa.y), x2);
              fz_fma2(acc[1], fz_pk(wa.z, wa.w), x2);
              fz_fma2(acc[2], fz_pk(wb.x, wb.y), x2);
              fz_fma2(acc[3], fz_pk(wb.z, wb.w), x2);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              float a0, a1;
              fz_upk(acc[q], a0, a1);
              const __nv_bfloat162 hv = __floats2bfloat162_rn(fmaxf(a0, 0.0f), fmaxf(a1, 0.0f));
              o[cg / 2 + q] = *reinterpret_cast<const uint32_t*>(&hv);
            }
          }
        }
        fz_st_row(base + (uint32_t)((tau & 1) * FZ_ROW + (t + 1) * 64), o);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(rdy(0, (int)(k & 1))) : "memory");
      }
    }
  } else {
    // epilogues of layers 2-4 (warps 0-3): thread i = TMEM lane i = pixel slot i + 1
    const int i = tid;
    const uint32_t tlane = tmem + ((uint32_t)(warp * 32) << 16);
    int64_t k = 0;
    for (int64_t u = blockIdx.x; u < a.units; u += gridDim.x) {
      int img, r0, r1, x0;
      fz_unit(a, u, img, r0, r1, x0);
      const int nsteps = r1 - r0 + 15;
      const int x = x0 - 6 + i;
      for (int st = 0; st < nsteps; ++st, ++k) {
        const int tau = r0 - 5 + st, b = (int)(k & 1);
#pragma unroll 1
        for (int j = 0; j < NMID - 1; ++j) {
          const bool okl = fz_wait(mdone(j, b), (uint32_t)(k >> 1) & 1u, abort) && !*abort;
          const bool okw = __all_sync(0xffffffffu, okl);  // tcgen05.ld is warp-collective
          const int rho = tau - 2 * (j + 1);
          uint32_t v[NC];
          fz_take(tlane, j, rho, okw, st == nsteps - 1, v);
          fz_release(tempty(j, b));
          const bool in_img = okw && rho >= 0 && rho < im.R && x >= 0 && x < im.W;
          const float* bj = sBM + j * NC;
          uint32_t o[NC / 2];
#pragma unroll
          for (int c = 0; c < NC; c += 2) {
            float s0, s1;
            fz_add2(__uint_as_float(v[c]), __uint_as_float(v[c + 1]), bj[c], bj[c + 1], s0, s1);
            const float f0 = in_img ? fmaxf(s0, 0.0f) : 0.0f;
            const float f1 = in_img ? fmaxf(s1, 0.0f) : 0.0f;
            const __nv_bfloat162 hv = __floats2bfloat162_rn(f0, f1);
            o[c / 2] = *reinterpret_cast<const uint32_t*>(&hv);
          }
          // the row overwritten here was read by layer j + 3's MMAs of the step
          // before: layers 3 and 4 were waited for above at that step, layer 5's
          // completion (waited by warps 4-7) is waited for here
          if (j == NMID - 2 && k >= 1)
            fz_wait(mdone(NMID - 1, (int)((k - 1) & 1)), (uint32_t)((k - 1) >> 1) & 1u, abort);
          fz_st_row(base + (uint32_t)((j + 1) * FZ_RINGB + (rho & 1) * FZ_ROW + (i + 1) * 64), o);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(rdy(j + 1, b)) : "memory");
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid == 0 && *abort) atomicExch(a.err, 1);
  if (warp == 8) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
}

// ----------------------------------------------------------- backward
// g6 = dout * m; dy5[p][ci] = (sum_d W6[d][ci] g6[p - off(d)]) * (y5[p][ci] > 0)
__global__ void k_l6_bwd(Image im, const float* __restrict__ dout, const float2* __restrict__ in,
                         const bf16* __restrict__ y5, const float* __restrict__ P, bf16* __restrict__ dy5) {
  __shared__ float w[W6_N];
  for (int i = threadIdx.x; i < W6_N; i += blockDim.x) w[i] = P[OFF_W6 + i];
  __syncthreads();
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= im.npx()) return;
  const int x = (int)(p % im.W), r = (int)(p / im.W);
  const int lo = (r / im.R) * im.R, hi = lo + im.R;
  float g[9];
#pragma unroll
  for (int d = 0; d < 9; ++d) {
    const int xx = x - (d % 3 - 1), rr = r - (d / 3 - 1);
    const int64_t q = (int64_t)rr * im.W + xx;
    g[d] = (xx >= 0 && xx < im.W && rr >= lo && rr < hi) ? dout[q] * in[q].y : 0.0f;
  }
  __align__(16) bf16 yv[NC];
  __align__(16) bf16 ov[NC];
#pragma unroll
  for (int q = 0; q < 4; ++q) reinterpret_cast<int4*>(yv)[q] = reinterpret_cast<const int4*>(y5 + p * NC)[q];
#pragma unroll 4
  for (int ci = 0; ci < NC; ++ci) {
    float a = 0.0f;
#pragma unroll
    for (int d = 0; d < 9; ++d) a += w[d * NC + ci] * g[d];
    ov[ci] = __float2bfloat16_rn(__bfloat162float(yv[ci]) > 0.0f ? a : 0.0f);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) reinterpret_cast<int4*>(dy5 + p * NC)[q] = reinterpret_cast<const int4*>(ov)[q];
}

// pixels [p0, p1) of CTA b out of nb over n pixels
__device__ __forceinline__ void chunk_of(int64_t n, int b, int nb, int64_t& p0, int64_t& p1) {
  const int64_t c = (n + nb - 1) / nb;
  p0 = (int64_t)b * c < n ? (int64_t)b * c : n;
  p1 = p0 + c < n ? p0 + c : n;
}

// layer 6 gradient partials: slot d * 32 + ci: sum g6[p] y5[p + off(d)][ci]; slot 288: sum g6[p].
// A warp walks pixels of the CTA's chunk (lane = input channel, 9 tap sums in
// registers); the 8 warps' sums are added in a fixed order.
__global__ void __launch_bounds__(256) k_l6_wgrad(Image im, const float* __restrict__ dout,
                                                  const float2* __restrict__ in, const bf16* __restrict__ y5,
                                                  float* __restrict__ part) {
  __shared__ float sm[8][W6_N + B6_N];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t p0, p1;
  chunk_of(im.npx(), blockIdx.x, gridDim.x, p0, p1);
  float acc[9], bacc = 0.0f;
#pragma unroll
  for (int d = 0; d < 9; ++d) acc[d] = 0.0f;
  // 4 pixels per step, their loads issued before the sums (latency hiding)
  for (int64_t pb = p0 + w; pb < p1; pb += 32) {
    float g[4], v[4][9];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t p = pb + 8 * u;
      g[u] = p < p1 ? dout[p] * in[p].y : 0.0f;
      const int x = (int)(p % im.W), r = (int)(p / im.W);
      const int lo = (r / im.R) * im.R, hi = lo + im.R;
#pragma unroll
      for (int d = 0; d < 9; ++d) {
        const int xx = x + d % 3 - 1, rr = r + d / 3 - 1;
        v[u][d] = (p < p1 && xx >= 0 && xx < im.W && rr >= lo && rr < hi)
                      ? __bfloat162float(y5[((int64_t)rr * im.W + xx) * NC + lane])
                      : 0.0f;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      bacc += g[u];
#pragma unroll
      for (int d = 0; d < 9; ++d) acc[d] += g[u] * v[u][d];
    }
  }
#pragma unroll
  for (int d = 0; d < 9; ++d) sm[w][d * NC + lane] = acc[d];
  if (lane == 0) sm[w][W6_N] = bacc;
  __syncthreads();
  for (int i = threadIdx.x; i < W6_N + B6_N; i += blockDim.x) {
    float t = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += sm[k][i];
    part[(int64_t)blockIdx.x * (W6_N + B6_N) + i] = t;
  }
}

// layer 1 gradient partials: slot (co * 9 + d) * 2 + ci: sum dy1[p][co] in[p + off(d)][ci];
// slot 576 + co: sum dy1[p][co].  A warp walks pixels (lane = output channel).
__global__ void __launch_bounds__(256) k_l1_wgrad(Image im, const bf16* __restrict__ dy1,
                                                  const float2* __restrict__ in, float* __restrict__ part) {
  __shared__ float sm[8][W1_N + B1_N];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t p0, p1;
  chunk_of(im.npx(), blockIdx.x, gridDim.x, p0, p1);
  float acc[9][2], bacc = 0.0f;
#pragma unroll
  for (int d = 0; d < 9; ++d) acc[d][0] = acc[d][1] = 0.0f;
  // 4 pixels per step, their loads issued before the sums (latency hiding)
  for (int64_t pb = p0 + w; pb < p1; pb += 32) {
    float g[4];
    float2 v[4][9];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t p = pb + 8 * u;
      g[u] = p < p1 ? __bfloat162float(dy1[p * NC + lane]) : 0.0f;
      const int x = (int)(p % im.W), r = (int)(p / im.W);
      const int lo = (r / im.R) * im.R, hi = lo + im.R;
#pragma unroll
      for (int d = 0; d < 9; ++d) {
        const int xx = x + d % 3 - 1, rr = r + d / 3 - 1;
        v[u][d] = (p < p1 && xx >= 0 && xx < im.W && rr >= lo && rr < hi) ? in[(int64_t)rr * im.W + xx]
                                                                            : make_float2(0.0f, 0.0f);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      bacc += g[u];
#pragma unroll
      for (int d = 0; d < 9; ++d) {
        acc[d][0] += g[u] * v[u][d].x;
        acc[d][1] += g[u] * v[u][d].y;
      }
    }
  }
#pragma unroll
  for (int d = 0; d < 9; ++d) {
    sm[w][(lane * 9 + d) * 2] = acc[d][0];
    sm[w][(lane * 9 + d) * 2 + 1] = acc[d][1];
  }
  sm[w][W1_N + lane] = bacc;
  __syncthreads();
  for (int i = threadIdx.x; i < W1_N + B1_N; i += blockDim.x) {
    float t = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += sm[k][i];
    part[(int64_t)blockIdx.x * (W1_N + B1_N) + i] = t;
  }
}

// 32 -> 32 weight-gradient partials on the tensor cores (mma.sync fragments):
// part[cta][d][k = ci][n = co] = sum_p x[p + off(d)][ci] dy[p][co].
// Warp w owns the 16 x 16 quadrant (ci block w >> 1, co block w & 1) of all 9
// taps: per 16-pixel step it loads one dy fragment and 9 shifted x fragments.
__global__ void __launch_bounds__(128) k_conv32_wgrad(Image im, const bf16* __restrict__ x,
                                                      const bf16* __restrict__ dy, float* __restrict__ part) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  bf16* sIn = reinterpret_cast<bf16*>(smem_raw);  // [3][TPX + 2][LDA]
  bf16* sDy = sIn + 3 * (TPX + 2) * LDA;          // [TPX][LDA]
  const int segs = (im.W + TPX - 1) / TPX;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int kb = warp >> 1, nb = warp & 1;
  wm::fragment<wm::accumulator, 16, 16, 16, float> acc[9];
#pragma unroll
  for (int d = 0; d < 9; ++d) wm::fill_fragment(acc[d], 0.0f);
  const int64_t jobs = (int64_t)segs * im.H;
  for (int64_t job = blockIdx.x; job < jobs; job += gridDim.x) {
    const int r = (int)(job / segs), x0 = (int)(job % segs) * TPX;
    __syncthreads();
    stage_rows(im, x, r, x0, sIn);
    for (int i = tid; i < TPX * 4; i += blockDim.x) {
      const int q = i & 3, px = i >> 2, gx = x0 + px;
      int4 v = make_int4(0, 0, 0, 0);
      if (gx < im.W) v = *reinterpret_cast<const int4*>(dy + ((int64_t)r * im.W + gx) * NC + q * 8);
      *reinterpret_cast<int4*>(sDy + px * LDA + q * 8) = v;
    }
    __syncthreads();
#pragma unroll 1
    for (int ks = 0; ks < TPX / 16; ++ks) {
      wm::fragment<wm::matrix_b, 16, 16, 16, bf16, wm::row_major> fb;
      wm::load_matrix_sync(fb, sDy + (16 * ks) * LDA + nb * 16, LDA);
#pragma unroll
      for (int d = 0; d < 9; ++d) {
        wm::fragment<wm::matrix_a, 16, 16, 16, bf16, wm::col_major> fa;
        wm::load_matrix_sync(fa, sIn + ((d / 3) * (TPX + 2) + 16 * ks + d % 3) * LDA + kb * 16, LDA);
        wm::mma_sync(acc[d], fa, fb, acc[d]);
      }
    }
  }
  float* out = part + (int64_t)blockIdx.x * WM_N;
#pragma unroll
  for (int d = 0; d < 9; ++d)
    wm::store_matrix_sync(out + (d * NC + 16 * kb) * NC + 16 * nb, acc[d], NC, wm::mem_row_major);
}

// bias-gradient partials of a 32-channel gradient: part[cta][c] = sum over the CTA's pixels
__global__ void __launch_bounds__(256) k_bias_grad(int64_t npx, const bf16* __restrict__ dy,
                                                   float* __restrict__ part) {
  __shared__ float sm[8][NC];
  const int c = threadIdx.x & 31, row = threadIdx.x >> 5;
  int64_t p0, p1;
  chunk_of(npx, blockIdx.x, gridDim.x, p0, p1);
  float a = 0.0f;
  for (int64_t p = p0 + row; p < p1; p += 8) a += __bfloat162float(dy[p * NC + c]);
  sm[row][c] = a;
  __syncthreads();
  if (row == 0) {
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += sm[i][c];
    part[(int64_t)blockIdx.x * NC + c] = s;
  }
}

// out[i] = sum over parts of part[c][i] (fixed order)
__global__ void k_sum_parts(const float* __restrict__ part, int nparts, int n, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.0f;
  for (int c = 0; c < nparts; ++c) s += part[(int64_t)c * n + i];
  out[i] = s;
}

// middle-layer weight gradient: G[(co 9 + d) 32 + ci] = sum over parts of part[c][(d 32 + ci) 32 + co]
__global__ void k_sum_wgrad(const float* __restrict__ part, int nparts, float* __restrict__ G) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= WM_N) return;
  float s = 0.0f;
  for (int c = 0; c < nparts; ++c) s += part[(int64_t)c * WM_N + j];
  const int co = j % NC, ci = (j / NC) % NC, d = j / (NC * NC);
  G[(co * 9 + d) * NC + ci] = s;
}

// ------------------------------------------------------------- weights
// B operands of k_conv32_tma, [tap][n][k]:
// forward: wf[l][d][n = co][k = ci] = W_l[co][d][ci]
// data gradient: wb[l][8 - d][n = ci][k = co] = W_l[co][d][ci]
__global__ void k_pack_weights(const float* __restrict__ P, bf16* __restrict__ wf, bf16* __restrict__ wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NMID * WM_N) return;
  const int l = i / WM_N, rem = i % WM_N;
  const int co = rem / (9 * NC), d = (rem / NC) % 9, ci = rem % NC;
  const bf16 w = __float2bfloat16_rn(P[off_wm(l) + rem]);
  wf[(int64_t)l * WM_N + (d * NC + co) * NC + ci] = w;
  wb[(int64_t)l * WM_N + ((8 - d) * NC + ci) * NC + co] = w;
}

__global__ void k_adam(int n, float* __restrict__ P, const float* __restrict__ G, float* __restrict__ m,
                       float* __restrict__ v, float lr, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float g = G[i];
  const float mi = b1 * m[i] + (1.0f - b1) * g;
  const float vi = b2 * v[i] + (1.0f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ----------------------------------------------------------------- loss
// Gathers batch image k from the pair store: input (s_hat, m), node codes,
// diagonal and c.
__global__ void k_gather(Image im, const float* __restrict__ s_store, const double* __restrict__ c_store,
                         const int32_t* __restrict__ geo_of, const uint8_t* __restrict__ code_store,
                         const float* __restrict__ diag_store, const int32_t* __restrict__ pick,
                         float2* __restrict__ in, uint8_t* __restrict__ code, float* __restrict__ diag,
                         double* __restrict__ cimg) {
  const int64_t per = (int64_t)im.W * im.R;
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= im.npx()) return;
  const int k = (int)(p / per);
  const int64_t q = p - (int64_t)k * per;
  const int64_t s = pick[k];
  const int64_t g = geo_of[s];
  const uint8_t c = code_store[g * per + q];
  const bool cp = (c & CODE_CP) != 0;
  in[p] = make_float2(cp ? s_store[s * per + q] : 0.0f, cp ? 1.0f : 0.0f);
  code[p] = c;
  diag[p] = diag_store[g * per + q];
  if (q == 0) cimg[k] = c_store[s];
}

// Per image k (grid.y): per-CTA sums of o'A~o - 2 o's_hat (double);
// dout = (2 / batch) (A~ o - s_hat) / c_k at the CPs, 0 elsewhere.
__global__ void __launch_bounds__(256) k_loss(Image im, const uint8_t* __restrict__ code,
                                              const float* __restrict__ diag, const float2* __restrict__ in,
                                              const float* __restrict__ o, const double* __restrict__ cimg,
                                              float inv_batch, float* __restrict__ dout, double* __restrict__ part) {
  const int k = blockIdx.y;
  const int64_t per = (int64_t)im.W * im.R;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double contrib = 0.0;
  if (q < per) {
    const int64_t p = (int64_t)k * per + q;
    const uint8_t c = code[p];
    float g = 0.0f;
    if (c & CODE_CP) {
      const int x = (int)(q % im.W), r = (int)(q / im.W);
      const float oc = o[p];
      float sum = 0.0f;
      if (!(c & 1) && x > 0) sum += o[p - 1];
      if (!(c & 2) && x + 1 < im.W) sum += o[p + 1];
      if (!(c & 4) && r > 0) sum += o[p - im.W];
      if (!(c & 8) && r + 1 < im.R) sum += o[p + im.W];
      const float Ao = diag[p] * oc - sum;
      const float sh = in[p].x;
      contrib = (double)oc * Ao - 2.0 * (double)oc * sh;
      g = 2.0f * inv_batch * (Ao - sh) / (float)cimg[k];
    }
    dout[p] = g;
  }
  __shared__ double sm[256];
  sm[threadIdx.x] = contrib;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(int64_t)k * gridDim.x + blockIdx.x] = sm[0];
}

// loss[k] = (sum of part[k][*] + c_k) / c_k; loss[batch] = their mean
__global__ void k_loss_reduce(const double* __restrict__ part, int nblk, int batch, const double* __restrict__ cimg,
                              float* __restrict__ loss) {
  __shared__ double sl[256];
  double acc = 0.0;
  for (int k = threadIdx.x; k < batch; k += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)k * nblk + b];
    const double L = (s + cimg[k]) / cimg[k];
    loss[k] = (float)L;
    acc += L;
  }
  sl[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) t += sl[i];
    loss[batch] = (float)(t / batch);
  }
}

// ------------------------------------------------ full-grid operator helpers
// (sigma I + A) x at the CP node p; only CP neighbours are read (mask bits of the code)
struct GridOp {
  int dim;
  int64_t st[3];
  double inv_h2, sigma;
};

template <class T>
__device__ __forceinline__ double op_at(const GridOp& G, const uint8_t c, const double* diag, const T* x, int64_t p) {
  double sum = 0.0;
  for (int s = 0; s < 2 * G.dim; ++s)
    if (!(c & (1u << s))) sum += (double)x[p + ((s & 1) ? G.st[s >> 1] : -G.st[s >> 1])];
  return (G.sigma + diag[p] * G.inv_h2) * (double)x[p] - sum * G.inv_h2;
}

// per-CTA sums of a and b into out2[0..1] (blockDim.x = 256)
__device__ __forceinline__ void block_sum2(double a, double b, double* out2) {
  __shared__ double s0[256], s1[256];
  s0[threadIdx.x] = a;
  s1[threadIdx.x] = b;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s0[threadIdx.x] += s0[threadIdx.x + w];
      s1[threadIdx.x] += s1[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out2[0] = s0[0];
    out2[1] = s1[0];
  }
}

// r = b - (sigma I + A) x at the CPs, 0 elsewhere
__global__ void __launch_bounds__(256) k_pr_resid(GridOp G, int64_t nn, const uint8_t* __restrict__ code,
                                                  const double* __restrict__ diag, const double* __restrict__ b,
                                                  const double* __restrict__ x, double* __restrict__ r) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nn; p += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t c = code[p];
    r[p] = (c & CODE_CP) ? b[p] - op_at(G, c, diag, x, p) : 0.0;
  }
}

// x += z; e = x* - x at the CPs (e = 0 elsewhere)
__global__ void k_pr_update(int64_t nn, const uint8_t* __restrict__ code, const double* __restrict__ z,
                            const double* __restrict__ xs, double* __restrict__ x, double* __restrict__ e) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nn; p += (int64_t)gridDim.x * blockDim.x) {
    if (code[p] & CODE_CP) {
      const double xv = x[p] + z[p];
      x[p] = xv;
      e[p] = xs[p] - xv;
    } else {
      e[p] = 0.0;
    }
  }
}

// t = h^2 (sigma I + A) e at the CPs; per-CTA partials (sum t^2, sum e t)
__global__ void __launch_bounds__(256) k_pr_unit(GridOp G, double h2, int64_t nn, const uint8_t* __restrict__ code,
                                                 const double* __restrict__ diag, const double* __restrict__ e,
                                                 double* __restrict__ t, double* __restrict__ part) {
  double a = 0.0, b = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nn; p += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t c = code[p];
    double tv = 0.0;
    if (c & CODE_CP) {
      tv = h2 * op_at(G, c, diag, e, p);
      a += tv * tv;
      b += e[p] * tv;
    }
    t[p] = tv;
  }
  block_sum2(a, b, part + 2 * blockIdx.x);
}

// rho = rms(t) over the CPs; scal = (1 / rho, c = sum e t / rho^2), c also into c_out
__global__ void k_pr_norm(const double* __restrict__ part, int nblk, double ncp, double* __restrict__ scal,
                          double* __restrict__ c_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < nblk; ++i) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
  const double rho = sqrt(a / ncp);
  const double inv = rho > 0.0 ? 1.0 / rho : 0.0;
  scal[0] = inv;
  scal[1] = b * inv * inv;
  *c_out = b * inv * inv;
}

__global__ void k_pr_write(int64_t nn, const double* __restrict__ t, const double* __restrict__ e,
                           const double* __restrict__ scal, float* __restrict__ s_out, double* __restrict__ e_out) {
  const double inv = scal[0];
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nn; p += (int64_t)gridDim.x * blockDim.x) {
    s_out[p] = (float)(t[p] * inv);
    if (e_out) e_out[p] = e[p] * inv;
  }
}

// ------------------------------------------------------ stage in the PCG
// s = r - (sigma I + A) z at the CPs; per-CTA sums of s^2
__global__ void __launch_bounds__(256) k_st_resid(GridOp G, int64_t nn, const uint8_t* __restrict__ code,
                                                  const double* __restrict__ diag, const double* __restrict__ r,
                                                  const double* __restrict__ z, double* __restrict__ s,
                                                  double* __restrict__ part) {
  double a = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nn; p += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t c = code[p];
    double v = 0.0;
    if (c & CODE_CP) {
      v = r[p] - op_at(G, c, diag, z, p);
      a += v * v;
    }
    s[p] = v;
  }
  block_sum2(a, 0.0, part + 2 * blockIdx.x);
}

// scal = (1 / rms(s), or 0 when s = 0; h^2 rms(s))
__global__ void k_st_norm(const double* __restrict__ part, int nblk, double ncp, double h2,
                          double* __restrict__ scal) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 0.0;
  for (int i = 0; i < nblk; ++i) a += part[2 * i];
  const double rms = sqrt(a / ncp);
  scal[0] = rms > 0.0 ? 1.0 / rms : 0.0;
  scal[1] = h2 * rms;
}

__global__ void k_st_input(int64_t nn, const uint8_t* __restrict__ code, const double* __restrict__ s,
                           const double* __restrict__ scal, float2* __restrict__ in) {
  const double inv = scal[0];
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nn; p += (int64_t)gridDim.x * blockDim.x) {
    const bool cp = (code[p] & CODE_CP) != 0;
    in[p] = make_float2(cp ? (float)(s[p] * inv) : 0.0f, cp ? 1.0f : 0.0f);
  }
}

// energy-optimal step: per-CTA sums of o's_hat and o'A~o, A~ = h^2 (sigma I + A)
__global__ void __launch_bounds__(256) k_st_energy(GridOp G, double h2, int64_t nn, const uint8_t* __restrict__ code,
                                                   const double* __restrict__ diag, const float2* __restrict__ in,
                                                   const float* __restrict__ o, double* __restrict__ part) {
  double a = 0.0, b = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nn; p += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t c = code[p];
    if (c & CODE_CP) {
      const double ov = (double)o[p];
      a += ov * (double)in[p].x;
      b += ov * h2 * op_at(G, c, diag, o, p);
    }
  }
  block_sum2(a, b, part + 2 * blockIdx.x);
}

// scal[1] *= omega = (o's_hat) / (o'A~o), 0 when o'A~o <= 0
__global__ void k_st_omega(const double* __restrict__ part, int nblk, double* __restrict__ scal) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < nblk; ++i) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
  scal[1] *= b > 0.0 ? a / b : 0.0;
}

__global__ void k_st_correct(int64_t nn, const uint8_t* __restrict__ code, const float* __restrict__ o,
                             const double* __restrict__ scal, double* __restrict__ z) {
  const double a = scal[1];
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nn; p += (int64_t)gridDim.x * blockDim.x)
    if (code[p] & CODE_CP) z[p] += a * (double)o[p];
}

// ---------------------------------------------------------------- host
struct NN {
  float* P = nullptr;  // FP32 master parameters
  float* G = nullptr;  // gradient
  float* m = nullptr;  // Adam moments
  float* v = nullptr;
  int* err = nullptr;  // set by a convolution whose tensor-core wait gave up
  // optional CUDA-event timing of the 32 -> 32 convolution launches of forward()
  bool prof = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev;
  int prof_n = 0;
  bf16* wf = nullptr;  // packed forward weights of the middle layers
  bf16* wb = nullptr;  // packed data-gradient weights
  int64_t steps = 0;
  cudaStream_t home = 0;
  bool fused = true;  // nn_forward and the PCG stage: k_net_fwd (else the layer-by-layer launches)
  // activations (grown to the largest stack seen)
  int64_t cap_px = 0;
  bf16* act[6] = {};  // act[1..5]: outputs of layers 1..5
  bf16* gA = nullptr;
  bf16* gB = nullptr;
  float* out = nullptr;
  float* dout = nullptr;
  float2* in = nullptr;     // gathered / staged input
  uint8_t* code = nullptr;  // gathered batch geometry
  float* diag = nullptr;
  // reductions
  float* part = nullptr;
  int64_t cap_part = 0;
  double* lpart = nullptr;
  int64_t cap_lpart = 0;
  double* cimg = nullptr;
  float* loss = nullptr;
  int cap_batch = 0;
  // stage in the PCG
  int64_t cap_nodes = 0;
  double* s64 = nullptr;
  double* spart = nullptr;
  double* scal = nullptr;
  int snblk = 0;
};

static size_t wgrad_smem() { return (size_t)(3 * (TPX + 2) * LDA + TPX * LDA) * sizeof(bf16); }

static void set_attrs() {
  static bool done = false;
  if (done) return;
  EB_CUDA(cudaFuncSetAttribute(k_conv32_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CP_SMEM));
  EB_CUDA(cudaFuncSetAttribute(k_conv32_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wgrad_smem()));
  EB_CUDA(cudaFuncSetAttribute(k_net_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FZ_SMEM));
  done = true;
}

// Tensor map of a BF16 NHWC activation stack for k_conv32_tma: dimensions
// (32 channels, pixel, row in image, image), strides 64 B, W * 64 B,
// R * W * 64 B; box (32, 130, 3, 1) written in the 64-byte swizzled layout;
// out-of-range elements read as zero.
static CUtensorMap conv_map(const bf16* x, const Image& im) {
  EB_REQUIRE(((uintptr_t)x & 15) == 0, EB_ERR_INVALID, "conv: activations not 16-byte aligned");
  EB_REQUIRE(im.R > 0 && im.H % im.R == 0, EB_ERR_INVALID, "conv: rows are not whole images");
  CUtensorMap m;
  const cuuint64_t dims[4] = {(cuuint64_t)NC, (cuuint64_t)im.W, (cuuint64_t)im.R, (cuuint64_t)(im.H / im.R)};
  const cuuint64_t strides[3] = {(cuuint64_t)NC * 2, (cuuint64_t)im.W * NC * 2, (cuuint64_t)im.R * im.W * NC * 2};
  const cuuint32_t box[4] = {(cuuint32_t)NC, (cuuint32_t)TC_PIX, 3, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = tensor_map_encoder()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(x), dims,
                                          strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                          CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  EB_REQUIRE(r == CUDA_SUCCESS, EB_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return m;
}

// y = conv(x; wk) (+ bias, ReLU, mask) through k_conv32_tma
static void conv32(const Image& im, const bf16* x, const bf16* wk, const float* bias, bf16* y, int relu,
                   const bf16* mask_ref, int* err, cudaStream_t s) {
  const CUtensorMap m = conv_map(x, im);
  const int64_t jobs = (int64_t)((im.W + TPX - 1) / TPX) * im.H;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(jobs, (int64_t)num_sms() * 3));
  k_conv32_tma<<<grid, CP_THREADS, CP_SMEM, s>>>(m, im, wk, bias, y, relu, mask_ref, err);
}

static void ensure_act(NN& N, int64_t px, cudaStream_t s) {
  if (px <= N.cap_px) return;
  for (int l = 1; l <= 5; ++l) dfree(N.act[l], s);
  dfree(N.gA, s); dfree(N.gB, s); dfree(N.out, s); dfree(N.dout, s); dfree(N.in, s); dfree(N.code, s);
  dfree(N.diag, s);
  N.cap_px = 0;
  for (int l = 1; l <= 5; ++l) N.act[l] = dalloc<bf16>((size_t)px * NC, s, false);
  N.gA = dalloc<bf16>((size_t)px * NC, s, false);
  N.gB = dalloc<bf16>((size_t)px * NC, s, false);
  N.out = dalloc<float>(px, s, false);
  N.dout = dalloc<float>(px, s, false);
  N.in = dalloc<float2>(px, s, false);
  N.code = dalloc<uint8_t>(px, s, false);
  N.diag = dalloc<float>(px, s, false);
  N.cap_px = px;
}

static float* ensure_part(NN& N, int64_t n, cudaStream_t s) {
  if (n > N.cap_part) {
    dfree(N.part, s);
    N.cap_part = 0;
    N.part = dalloc<float>(n, s, false);
    N.cap_part = n;
  }
  return N.part;
}

static unsigned conv_grid(const Image& im, int per_sm) {
  const int64_t jobs = (int64_t)((im.W + TPX - 1) / TPX) * im.H;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(jobs, (int64_t)num_sms() * per_sm));
}

static int64_t npx_of(const Image& im) { return (int64_t)im.W * im.H; }

static void pack(NN& N, cudaStream_t s, int64_t& nl) {
  k_pack_weights<<<blocks_for(NMID * WM_N, 256), 256, 0, s>>>(N.P, N.wf, N.wb);
  ++nl;
}

// out = N(in) over the stack; the activations stay for backward.  prof (may be
// NULL): a solver timing the 32 -> 32 convolution launches.
static void forward(NN& N, const Image& im, const float2* in, float* out, cudaStream_t s, int64_t& nl,
                    Solver* prof = nullptr) {
  const int64_t npx = npx_of(im);
  const int64_t npairs = (int64_t)((im.W + 1) / 2) * im.H;  // layer 1: two pixels per thread
  k_l1_fwd<<<blocks_for(npairs, 128), 128, 0, s>>>(im, in, N.P, N.act[1]);
  for (int l = 0; l < NMID; ++l) {
    const bool own = N.prof && !prof;  // events of the handle (not inside a solver's graph)
    if (own) {
      if (N.prof_n >= (int)N.prof_ev.size()) {
        cudaEvent_t a, b;
        EB_CUDA(cudaEventCreate(&a));
        EB_CUDA(cudaEventCreate(&b));
        N.prof_ev.push_back({a, b});
      }
      EB_CUDA(cudaEventRecord(N.prof_ev[N.prof_n].first, s));
    }
    if (prof) prof->prof_mark(s, true, PROF_CONV);
    conv32(im, N.act[l + 1], N.wf + (int64_t)l * WM_N, N.P + off_wm(l) + WM_N, N.act[l + 2], 1, nullptr, N.err, s);
    if (prof) prof->prof_mark(s, false, PROF_CONV);
    if (own) EB_CUDA(cudaEventRecord(N.prof_ev[N.prof_n++].second, s));
  }
  k_l6_fwd<<<blocks_for(npx, 128), 128, 0, s>>>(im, N.act[5], N.P, in, out);
  nl += 6;
  EB_CUDA(cudaGetLastError());
}

// The work units of k_net_fwd: strips of FZ_OUT columns x runs of rows of
// one image.  A run of n rows takes n + 15 steps; the run length minimises
// (waves of units over the SMs) x (steps per unit).
static FzArgs fz_plan(const Image& im) {
  FzArgs a{};
  a.im = im;
  a.strips = (im.W + FZ_OUT - 1) / FZ_OUT;
  const int64_t nimg = im.H / im.R;
  const int64_t nsm = num_sms();
  int64_t best = -1;
  for (int sg = 1; sg <= im.R; ++sg) {
    const int rows = (im.R + sg - 1) / sg;
    const int segs = (im.R + rows - 1) / rows;
    const int64_t units = (int64_t)a.strips * nimg * segs;
    const int64_t cost = ((units + nsm - 1) / nsm) * (rows + 15);
    if (best < 0 || cost < best) {
      best = cost;
      a.segs = segs;
      a.seg_rows = rows;
      a.units = units;
    }
    if (units > 4 * nsm) break;
  }
  return a;
}

// out = N(in) in one launch of k_net_fwd
static void forward_fused(NN& N, const Image& im, const float2* in, float* out, cudaStream_t s, int64_t& nl,
                          Solver* prof = nullptr) {
  EB_REQUIRE(im.R > 0 && im.H % im.R == 0, EB_ERR_INVALID, "forward: rows are not whole images");
  FzArgs a = fz_plan(im);
  a.in = in;
  a.out = out;
  a.P = N.P;
  a.wf = N.wf;
  a.err = N.err;
  const bool own = N.prof && !prof;
  if (own) {
    if (N.prof_n >= (int)N.prof_ev.size()) {
      cudaEvent_t e0, e1;
      EB_CUDA(cudaEventCreate(&e0));
      EB_CUDA(cudaEventCreate(&e1));
      N.prof_ev.push_back({e0, e1});
    }
    EB_CUDA(cudaEventRecord(N.prof_ev[N.prof_n].first, s));
  }
  if (prof) prof->prof_mark(s, true, PROF_CONV);
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(a.units, num_sms()));
  k_net_fwd<<<grid, FZ_THREADS, FZ_SMEM, s>>>(a);
  if (prof) prof->prof_mark(s, false, PROF_CONV);
  if (own) EB_CUDA(cudaEventRecord(N.prof_ev[N.prof_n++].second, s));
  nl += 1;
  EB_CUDA(cudaGetLastError());
}

// the inference forward: fused unless the handle asks for the layer-by-layer path
static void forward_infer(NN& N, const Image& im, const float2* in, float* out, cudaStream_t s, int64_t& nl,
                          Solver* prof = nullptr) {
  if (N.fused) forward_fused(N, im, in, out, s, nl, prof);
  else forward(N, im, in, out, s, nl, prof);
}

// gradient of sum(dout * out) into N.G (forward ran on the same input)
static void backward(NN& N, const Image& im, const float2* in, const float* dout, cudaStream_t s, int64_t& nl) {
  const int64_t npx = npx_of(im);
  const int nsm = num_sms();
  {
    const int nb = nsm * 4;
    float* part = ensure_part(N, (int64_t)nb * (W6_N + B6_N), s);
    k_l6_wgrad<<<nb, 256, 0, s>>>(im, dout, in, N.act[5], part);
    k_sum_parts<<<blocks_for(W6_N + B6_N, 256), 256, 0, s>>>(part, nb, W6_N + B6_N, N.G + OFF_W6);
    k_l6_bwd<<<blocks_for(npx, 128), 128, 0, s>>>(im, dout, in, N.act[5], N.P, N.gA);
    nl += 3;
  }
  bf16* cur = N.gA;
  bf16* nxt = N.gB;
  for (int l = NMID - 1; l >= 0; --l) {
    const unsigned gw = conv_grid(im, 4);
    const int nbb = nsm * 4;
    float* part = ensure_part(N, std::max<int64_t>((int64_t)gw * WM_N, (int64_t)nbb * NC), s);
    k_conv32_wgrad<<<gw, 128, wgrad_smem(), s>>>(im, N.act[l + 1], cur, part);
    k_sum_wgrad<<<blocks_for(WM_N, 256), 256, 0, s>>>(part, (int)gw, N.G + off_wm(l));
    k_bias_grad<<<nbb, 256, 0, s>>>(npx, cur, part);
    k_sum_parts<<<1, 32, 0, s>>>(part, nbb, NC, N.G + off_wm(l) + WM_N);
    conv32(im, cur, N.wb + (int64_t)l * WM_N, nullptr, nxt, 0, N.act[l + 1], N.err, s);
    std::swap(cur, nxt);
    nl += 5;
  }
  {
    const int nb = nsm * 4;
    float* part = ensure_part(N, (int64_t)nb * (W1_N + B1_N), s);
    k_l1_wgrad<<<nb, 256, 0, s>>>(im, cur, in, part);
    k_sum_parts<<<blocks_for(W1_N + B1_N, 256), 256, 0, s>>>(part, nb, W1_N + B1_N, N.G + OFF_W1);
    nl += 2;
  }
  EB_CUDA(cudaGetLastError());
}

static GridOp grid_op(const EBHandle& eb, double sigma) {
  GridOp G;
  G.dim = eb.g.dim;
  G.st[0] = 1;
  G.st[1] = eb.g.n0;
  G.st[2] = (int64_t)eb.g.n0 * eb.g.n1;
  G.inv_h2 = 1.0 / (eb.g.h * eb.g.h);
  G.sigma = sigma;
  return G;
}

static unsigned grid_blocks(int64_t nn) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((nn + 255) / 256, (int64_t)num_sms() * 8));
}

}  // namespace ebk

struct nn_handle {
  ebk::NN n;
};

namespace ebk {

void nn_stage_prepare(nn_handle* h, const EBHandle& eb, cudaStream_t s) {
  NN& N = h->n;
  EB_REQUIRE(eb.g.dim == 2, EB_ERR_INVALID, "learned stage: 2D grids only");
  const int64_t nn = eb.g.num_nodes;
  ensure_act(N, nn, s);
  if (nn > N.cap_nodes) {
    dfree(N.s64, s);
    dfree(N.spart, s);
    N.cap_nodes = 0;
    N.snblk = (int)grid_blocks(nn);
    N.s64 = dalloc<double>(nn, s, false);
    N.spart = dalloc<double>(2 * (int64_t)N.snblk, s, false);
    N.cap_nodes = nn;
  }
  if (!N.scal) N.scal = dalloc<double>(2, s);
}

// z = z1 + omega h^2 rms(s) N(s / rms(s), m) with s = r - (sigma I + A) z1 and z1 = z on
// entry; omega = 1 (EB_NN_PLAIN) or the energy-optimal step (EB_NN_ENERGY)
void nn_stage_apply(nn_handle* h, const EBHandle& eb, double shift, int mode, const double* r, double* z,
                    int64_t& nl, Solver* prof, cudaStream_t s) {
  NN& N = h->n;
  const int64_t nn = eb.g.num_nodes;
  const unsigned nb = grid_blocks(nn);
  EB_REQUIRE(nn <= N.cap_nodes && (int)nb <= N.snblk && N.scal, EB_ERR_INVALID, "learned stage: not prepared");
  const GridOp G = grid_op(eb, shift);
  k_st_resid<<<nb, 256, 0, s>>>(G, nn, eb.code, eb.diag, r, z, N.s64, N.spart);
  k_st_norm<<<1, 32, 0, s>>>(N.spart, (int)nb, (double)eb.num_cp, eb.g.h * eb.g.h, N.scal);
  k_st_input<<<nb, 256, 0, s>>>(nn, eb.code, N.s64, N.scal, N.in);
  const Image im{eb.g.n0, eb.g.n1, eb.g.n1};
  forward_infer(N, im, N.in, N.out, s, nl, prof);
  if (mode == EB_NN_ENERGY) {
    k_st_energy<<<nb, 256, 0, s>>>(G, eb.g.h * eb.g.h, nn, eb.code, eb.diag, N.in, N.out, N.spart);
    k_st_omega<<<1, 32, 0, s>>>(N.spart, (int)nb, N.scal);
    nl += 2;
  }
  k_st_correct<<<nb, 256, 0, s>>>(nn, eb.code, N.out, N.scal, z);
  nl += 4;
}

}  // namespace ebk

using namespace ebk;

static int check_shape(int width, int height, int images) {
  if (width < 1 || height < 1 || images < 1 || (int64_t)height * images >= ((int64_t)1 << 30)) {
    set_error("nn: width, height and images must be >= 1 and height x images < 2^30");
    return EB_ERR_INVALID;
  }
  return EB_OK;
}

extern "C" {

int nn_create(nn_handle** out, cudaStream_t stream) {
  if (!out) {
    set_error("nn_create: NULL argument");
    return EB_ERR_INVALID;
  }
  *out = nullptr;
  nn_handle* h = new (std::nothrow) nn_handle();
  if (!h) {
    set_error("nn_create: host allocation failed");
    return EB_ERR_OOM;
  }
  h->n.home = stream;
  int st = guarded([&] {
    NN& N = h->n;
    set_attrs();
    N.P = dalloc<float>(NPARAM, stream);
    N.G = dalloc<float>(NPARAM, stream);
    N.m = dalloc<float>(NPARAM, stream);
    N.v = dalloc<float>(NPARAM, stream);
    N.wf = dalloc<bf16>(NMID * WM_N, stream);
    N.wb = dalloc<bf16>(NMID * WM_N, stream);
    N.err = dalloc<int>(1, stream);
    EB_CUDA(cudaStreamSynchronize(stream));
  });
  if (st != EB_OK) {
    nn_destroy(h);
    return st;
  }
  *out = h;
  return EB_OK;
}

void nn_destroy(nn_handle* h) {
  if (!h) return;
  NN& N = h->n;
  cudaStream_t s = N.home;
  dfree(N.P, s); dfree(N.G, s); dfree(N.m, s); dfree(N.v, s); dfree(N.wf, s); dfree(N.wb, s); dfree(N.err, s);
  for (int l = 1; l <= 5; ++l) dfree(N.act[l], s);
  dfree(N.gA, s); dfree(N.gB, s); dfree(N.out, s); dfree(N.dout, s); dfree(N.in, s); dfree(N.code, s);
  dfree(N.diag, s); dfree(N.part, s); dfree(N.lpart, s); dfree(N.cimg, s); dfree(N.loss, s);
  dfree(N.s64, s); dfree(N.spart, s); dfree(N.scal, s);
  cudaStreamSynchronize(s);
  for (auto& e : N.prof_ev) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  delete h;
}

int nn_num_params(void) { return NPARAM; }

int nn_set_profile(nn_handle* h, int on) {
  if (!h) {
    set_error("nn_set_profile: NULL handle");
    return EB_ERR_INVALID;
  }
  h->n.prof = on != 0;
  h->n.prof_n = 0;
  return EB_OK;
}

int nn_set_fused(nn_handle* h, int on) {
  if (!h) {
    set_error("nn_set_fused: NULL handle");
    return EB_ERR_INVALID;
  }
  h->n.fused = on != 0;
  return EB_OK;
}

int nn_profile(nn_handle* h, double* ms, int* launches, cudaStream_t stream) {
  if (!h || !ms || !launches) {
    set_error("nn_profile: NULL argument");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    NN& N = h->n;
    EB_CUDA(cudaStreamSynchronize(stream));
    double t = 0.0;
    for (int i = 0; i < N.prof_n; ++i) {
      float m = 0.0f;
      EB_CUDA(cudaEventElapsedTime(&m, N.prof_ev[i].first, N.prof_ev[i].second));
      t += m;
    }
    *ms = t;
    *launches = N.prof_n;
    N.prof_n = 0;
  });
}

int nn_status(nn_handle* h, cudaStream_t stream) {
  if (!h) {
    set_error("nn_status: NULL handle");
    return EB_ERR_INVALID;
  }
  int flag = 0;
  int st = guarded([&] {
    EB_CUDA(cudaMemcpyAsync(&flag, h->n.err, sizeof(int), cudaMemcpyDeviceToHost, stream));
    EB_CUDA(cudaMemsetAsync(h->n.err, 0, sizeof(int), stream));
    EB_CUDA(cudaStreamSynchronize(stream));
  });
  if (st != EB_OK) return st;
  if (flag) {
    set_error("nn: a tensor-core wait in a convolution gave up (results of that call are invalid)");
    return EB_ERR_TIMEOUT;
  }
  return EB_OK;
}

int nn_set_params(nn_handle* h, const float* params_host, cudaStream_t stream) {
  if (!h || !params_host) {
    set_error("nn_set_params: NULL argument");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    NN& N = h->n;
    int64_t nl = 0;
    EB_CUDA(cudaMemcpyAsync(N.P, params_host, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, stream));
    EB_CUDA(cudaMemsetAsync(N.m, 0, sizeof(float) * NPARAM, stream));
    EB_CUDA(cudaMemsetAsync(N.v, 0, sizeof(float) * NPARAM, stream));
    pack(N, stream, nl);
    N.steps = 0;
    EB_CUDA(cudaStreamSynchronize(stream));
  });
}

int nn_get_params(const nn_handle* h, float* params_host, float* grad_host, cudaStream_t stream) {
  if (!h) {
    set_error("nn_get_params: NULL handle");
    return EB_ERR_INVALID;
  }
  if (int ns = nn_status(const_cast<nn_handle*>(h), stream)) return ns;
  return guarded([&] {
    const NN& N = h->n;
    if (params_host)
      EB_CUDA(cudaMemcpyAsync(params_host, N.P, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, stream));
    if (grad_host) EB_CUDA(cudaMemcpyAsync(grad_host, N.G, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, stream));
    EB_CUDA(cudaStreamSynchronize(stream));
  });
}

int nn_forward(nn_handle* h, int width, int height, int images, const float* in_dev, float* out_dev,
               cudaStream_t stream) {
  if (!h || !in_dev || !out_dev) {
    set_error("nn_forward: NULL argument");
    return EB_ERR_INVALID;
  }
  if (int st = check_shape(width, height, images)) return st;
  if (reinterpret_cast<uintptr_t>(in_dev) % 8) {
    set_error("nn_forward: in must be 8-byte aligned");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    NN& N = h->n;
    const Image im{width, height * images, height};
    if (!N.fused) ensure_act(N, npx_of(im), stream);
    int64_t nl = 0;
    forward_infer(N, im, reinterpret_cast<const float2*>(in_dev), out_dev, stream, nl);
  });
}

int nn_backward(nn_handle* h, int width, int height, int images, const float* in_dev, const float* dout_dev,
                cudaStream_t stream) {
  if (!h || !in_dev || !dout_dev) {
    set_error("nn_backward: NULL argument");
    return EB_ERR_INVALID;
  }
  if (int st = check_shape(width, height, images)) return st;
  if (reinterpret_cast<uintptr_t>(in_dev) % 8) {
    set_error("nn_backward: in must be 8-byte aligned");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    NN& N = h->n;
    const Image im{width, height * images, height};
    ensure_act(N, npx_of(im), stream);
    int64_t nl = 0;
    const float2* in = reinterpret_cast<const float2*>(in_dev);
    forward(N, im, in, N.out, stream, nl);
    backward(N, im, in, dout_dev, stream, nl);
  });
}

int nn_geometry(const eb_handle* eb, uint8_t* code_dev, float* diag_dev, cudaStream_t stream) {
  if (!eb || !code_dev || !diag_dev) {
    set_error("nn_geometry: NULL argument");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    const EBHandle& E = eb->h;
    EB_REQUIRE(!E.has_beta(), EB_ERR_NOT_IMPLEMENTED, "nn_geometry: the learned stage needs beta = 1");
    EB_CUDA(cudaMemcpyAsync(code_dev, E.code, (size_t)E.g.num_nodes, cudaMemcpyDeviceToDevice, stream));
    EB_CUDA(cudaMemcpyAsync(diag_dev, E.diag32, sizeof(float) * E.g.num_nodes, cudaMemcpyDeviceToDevice, stream));
  });
}

int nn_pairs(const amg_handle* amg, const double* b_dev, const double* xstar_dev, int count, float* s_hat_dev,
             double* c_dev, double* e_hat_dev, cudaStream_t stream) {
  if (!amg || !b_dev || !xstar_dev || !s_hat_dev || !c_dev || count < 0) {
    set_error("nn_pairs: NULL argument or count < 0");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    Solver& S = const_cast<Solver&>(amg->s);
    EB_REQUIRE(S.H != nullptr, EB_ERR_INVALID, "nn_pairs: handle has no hierarchy");
    EB_REQUIRE(!S.eb->has_beta(), EB_ERR_NOT_IMPLEMENTED, "nn_pairs: the learned stage needs beta = 1");
    const EBHandle& eb = *S.eb;
    const int64_t nn = eb.g.num_nodes;
    const unsigned nb = grid_blocks(nn);
    const GridOp G = grid_op(eb, S.shift);
    double *x = nullptr, *r = nullptr, *z = nullptr, *e = nullptr, *t = nullptr, *part = nullptr, *scal = nullptr;
    auto release = [&] {
      dfree(x, stream); dfree(r, stream); dfree(z, stream); dfree(e, stream); dfree(t, stream);
      dfree(part, stream); dfree(scal, stream);
    };
    try {
      x = dalloc<double>(nn, stream);
      r = dalloc<double>(nn, stream);
      z = dalloc<double>(nn, stream);
      e = dalloc<double>(nn, stream);
      t = dalloc<double>(nn, stream);
      part = dalloc<double>(2 * (int64_t)nb, stream);
      scal = dalloc<double>(2, stream);
      for (int k = 0; k < count; ++k) {
        k_pr_resid<<<nb, 256, 0, stream>>>(G, nn, eb.code, eb.diag, b_dev, x, r);
        amg_vcycle_grid(S, r, z, stream);
        k_pr_update<<<nb, 256, 0, stream>>>(nn, eb.code, z, xstar_dev, x, e);
        k_pr_unit<<<nb, 256, 0, stream>>>(G, eb.g.h * eb.g.h, nn, eb.code, eb.diag, e, t, part);
        k_pr_norm<<<1, 32, 0, stream>>>(part, (int)nb, (double)eb.num_cp, scal, c_dev + k);
        k_pr_write<<<nb, 256, 0, stream>>>(nn, t, e, scal, s_hat_dev + (int64_t)k * nn,
                                           e_hat_dev ? e_hat_dev + (int64_t)k * nn : nullptr);
        EB_CUDA(cudaGetLastError());
      }
      EB_CUDA(cudaStreamSynchronize(stream));
    } catch (...) {
      release();
      throw;
    }
    release();
  });
}

int nn_train_step(nn_handle* h, int width, int height, int batch, const float* s_hat_dev, const double* c_dev,
                  const int32_t* geo_of_dev, const uint8_t* code_dev, const float* diag_dev, const int32_t* pick_dev,
                  float lr, float* loss_dev, cudaStream_t stream) {
  if (!h || !s_hat_dev || !c_dev || !geo_of_dev || !code_dev || !diag_dev || !pick_dev) {
    set_error("nn_train_step: NULL argument");
    return EB_ERR_INVALID;
  }
  if (int st = check_shape(width, height, batch)) return st;
  if (!(lr > 0.0f)) {
    set_error("nn_train_step: lr must be > 0");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    NN& N = h->n;
    const Image im{width, height * batch, height};
    const int64_t npx = npx_of(im);
    ensure_act(N, npx, stream);
    const int64_t per = (int64_t)width * height;
    const int lnb = (int)((per + 255) / 256);
    if ((int64_t)batch * lnb > N.cap_lpart) {
      dfree(N.lpart, stream);
      N.cap_lpart = 0;
      N.lpart = dalloc<double>((int64_t)batch * lnb, stream, false);
      N.cap_lpart = (int64_t)batch * lnb;
    }
    if (batch > N.cap_batch) {
      dfree(N.cimg, stream);
      dfree(N.loss, stream);
      N.cap_batch = 0;
      N.cimg = dalloc<double>(batch, stream);
      N.loss = dalloc<float>(batch + 1, stream);
      N.cap_batch = batch;
    }
    int64_t nl = 0;
    k_gather<<<blocks_for(npx, 256), 256, 0, stream>>>(im, s_hat_dev, c_dev, geo_of_dev, code_dev, diag_dev,
                                                       pick_dev, N.in, N.code, N.diag, N.cimg);
    forward(N, im, N.in, N.out, stream, nl);
    k_loss<<<dim3((unsigned)lnb, (unsigned)batch), 256, 0, stream>>>(im, N.code, N.diag, N.in, N.out, N.cimg,
                                                                      1.0f / (float)batch, N.dout, N.lpart);
    k_loss_reduce<<<1, 256, 0, stream>>>(N.lpart, lnb, batch, N.cimg, loss_dev ? loss_dev : N.loss);
    backward(N, im, N.in, N.dout, stream, nl);
    N.steps += 1;
    const float c1 = (float)(1.0 - std::pow(0.9, (double)N.steps));
    const float c2 = (float)(1.0 - std::pow(0.999, (double)N.steps));
    k_adam<<<blocks_for(NPARAM, 256), 256, 0, stream>>>(NPARAM, N.P, N.G, N.m, N.v, lr, c1, c2);
    pack(N, stream, nl);
    EB_CUDA(cudaGetLastError());
  });
}

int nn_precondition(const amg_handle* amg, nn_handle* nn, int mode, const double* r_dev, double* z_dev,
                    cudaStream_t stream) {
  if (!amg || !nn || !r_dev || !z_dev) {
    set_error("nn_precondition: NULL argument");
    return EB_ERR_INVALID;
  }
  if (mode != EB_NN_PLAIN && mode != EB_NN_ENERGY) {
    set_error("nn_precondition: mode must be EB_NN_PLAIN or EB_NN_ENERGY");
    return EB_ERR_INVALID;
  }
  return guarded([&] {
    Solver& S = const_cast<Solver&>(amg->s);
    EB_REQUIRE(S.H != nullptr, EB_ERR_INVALID, "nn_precondition: handle has no hierarchy");
    EB_REQUIRE(!S.eb->has_beta(), EB_ERR_NOT_IMPLEMENTED, "nn_precondition: the learned stage needs beta = 1");
    nn_stage_prepare(nn, *S.eb, stream);
    int64_t nl = 0;
    amg_vcycle_grid(S, r_dev, z_dev, stream);
    nn_stage_apply(nn, *S.eb, S.shift, mode, r_dev, z_dev, nl, nullptr, stream);
    EB_CUDA(cudaGetLastError());
  });
}

int pcg_solve_nn(const amg_handle* amg, nn_handle* nn, int mode, const double* b_dev, double* x_dev, double rtol,
                 int maxit, const pcg_opts* opts, pcg_stats* stats, cudaStream_t stream) {
  if (!amg || !nn || !b_dev || !x_dev) {
    set_error("pcg_solve_nn: NULL argument");
    return EB_ERR_INVALID;
  }
  if (mode != EB_NN_PLAIN && mode != EB_NN_ENERGY) {
    set_error("pcg_solve_nn: mode must be EB_NN_PLAIN or EB_NN_ENERGY");
    return EB_ERR_INVALID;
  }
  pcg_opts o{EB_PC_AMG_NN, 1, 1, 0};
  if (opts) o = *opts;
  o.precond = EB_PC_AMG_NN;
  int rc = EB_OK;
  int st = guarded([&] {
    Solver& S = const_cast<Solver&>(amg->s);
    EB_REQUIRE(S.H != nullptr, EB_ERR_INVALID, "pcg_solve_nn: handle has no hierarchy");
    EB_REQUIRE(!S.eb->has_beta(), EB_ERR_NOT_IMPLEMENTED, "pcg_solve_nn: the learned stage needs beta = 1");
    nn_stage_prepare(nn, *S.eb, stream);
    S.nn = nn;
    S.nn_mode = mode;
    try {
      rc = S.pcg(b_dev, x_dev, rtol, maxit, o, stats, stream);
    } catch (...) {
      S.nn = nullptr;
      throw;
    }
    S.nn = nullptr;
  });
  if (st != EB_OK) return st;
  const int ns = nn_status(nn, stream);
  return ns != EB_OK ? ns : rc;
}

}  // extern "C"
