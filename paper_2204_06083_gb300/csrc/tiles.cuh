// Active-tile traversal shared by every grid kernel.
//
// The grid is cut into tiles of 256 nodes, x fastest; the extents are powers
// of two chosen at run time (default 2D: 32 x 8, 3D: 16 x 4 x 4; eb_retile /
// the autotuner pick others).  Only tiles that hold a CP are listed.  For each
// listed tile the build stores the node index of its corner and its extents
// (ragged at the high ends of the grid), so a thread finds its nodes with
// shifts and one multiply-add -- no integer division in the hot loops.
//
// Hot kernels work on PAIRS of x-adjacent nodes (n0 even, tile origins even,
// so a pair is 16-byte aligned in FP64): 128 threads cover a tile and a CTA of
// 256 threads covers two tiles per iteration of a grid-stride loop.
#pragma once

#include <stdint.h>

namespace ebk {

constexpr int TILE_NODES = 256;
// flag in the DIM template argument of a grid kernel: the variable-coefficient
// stencil (beta of eq. 3 read from the view); dim_of strips it
constexpr int DIM_VB = 8;
// flag in the DIM template argument: the view has a CP pair list and EB_SWEEP
// visits its pairs, one per thread and grid-stride, with no tile-mode code
constexpr int DIM_LIST = 16;
__host__ __device__ constexpr int dim_of(int d) { return d & 3; }
constexpr int PAIR_THREADS = 128;  // threads per tile in the pair layout

// default tile extents
template <int DIM>
struct TileShape;
template <>
struct TileShape<2> {
  static constexpr int X = 32, Y = 8, Z = 1;
};
template <>
struct TileShape<3> {
  static constexpr int X = 16, Y = 4, Z = 4;
};

struct TileView {
  const int32_t* base;  // node index of the tile's (0,0,0) corner
  const int32_t* lim;   // extents: x | y << 8 | z << 16
  int64_t ntiles;
  int32_t sy, sz;       // node strides of y and z
  int32_t nn;           // number of grid nodes (even)
  // batched grids only (null for one grid): per-tile shift sigma and
  // 1 / (sigma + 2 dim) of the unit-spacing operator, FP64 and FP32 copies
  const double2* tshift64 = nullptr;
  const float2* tshift32 = nullptr;
  int32_t bx = 5, by = 3;  // log2 of the tile extents in x and y (z = 256 >> (bx + by))
  // single grids: the pairs of the tiles that hold a CP (EBHandle::pairs), in
  // tile order; null for batched views
  const int32_t* pair_node = nullptr;
  int64_t npairs = 0;
  // variable coefficient of eq. 3 (null for beta = 1): beta at the half point
  // node + h/2 e_a of every node, per axis a, FP64 and FP32 copies
  const double* beta64[3] = {nullptr, nullptr, nullptr};
  const float* beta32[3] = {nullptr, nullptr, nullptr};
};

// Node of this thread in listed tile tt (one node per thread, 256 threads).
template <int DIM>
__device__ __forceinline__ bool tile_node(const TileView& tv, int64_t tt, int32_t& node) {
  const int l = threadIdx.x;
  const int lx = l & ((1 << tv.bx) - 1), ly = (l >> tv.bx) & ((1 << tv.by) - 1), lz = l >> (tv.bx + tv.by);
  const int32_t lim = __ldg(tv.lim + tt);
  node = __ldg(tv.base + tt) + lx + ly * tv.sy + lz * tv.sz;
  return lx < (lim & 0xFF) && ly < ((lim >> 8) & 0xFF) && lz < ((lim >> 16) & 0xFF);
}

// First node of this thread's pair in listed tile tt (pair layout).
template <int DIM>
__device__ __forceinline__ bool tile_pair(const TileView& tv, int64_t tt, int t, int32_t& node) {
  const int bp = tv.bx - 1;  // pairs per tile row: 2^(bx - 1)
  const int px = t & ((1 << bp) - 1), ly = (t >> bp) & ((1 << tv.by) - 1), lz = t >> (bp + tv.by);
  const int32_t lim = __ldg(tv.lim + tt);
  node = __ldg(tv.base + tt) + 2 * px + ly * tv.sy + lz * tv.sz;
  return 2 * px < (lim & 0xFF) && ly < ((lim >> 8) & 0xFF) && lz < ((lim >> 16) & 0xFF);
}

// The node pairs of the tile view (pair layout, first node even) that hold
// at least one CP, in tile order and, within a tile, in pair order.
struct PairList {
  const int32_t* node = nullptr;
  int64_t n = 0;
};

}  // namespace ebk

// for (each listed tile of this CTA) if (this thread's node is in the grid) body
#define EB_TILE_LOOP(DIM, tv, node)                                    \
  for (int64_t tt_ = blockIdx.x; tt_ < (tv).ntiles; tt_ += gridDim.x) \
    if (int32_t node = 0; ::ebk::tile_node<DIM>((tv), tt_, node))

// pair layout: node and node + 1 belong to this thread
#define EB_PAIR_LOOP(DIM, tv, node)                                                                      \
  for (int64_t tt_ = 2 * (int64_t)blockIdx.x + (threadIdx.x >> 7); tt_ < (tv).ntiles; tt_ += 2 * (int64_t)gridDim.x) \
    if (int32_t node = 0; ::ebk::tile_pair<DIM>((tv), tt_, threadIdx.x & 127, node))

// for (each pair of the list given to this thread: grid-stride) body; node
// and node + 1 belong to this thread
#define EB_LIST_LOOP(pl, node)                                                                              \
  for (int64_t li_ = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; li_ < (pl).n;                          \
       li_ += (int64_t)gridDim.x * blockDim.x)                                                              \
    if (const int32_t node = __ldg((pl).node + li_); true)

namespace ebk {
// item it_ of EB_SWEEP: a CP pair of the list, or pair t of listed tile it_
template <int DIM>
__device__ __forceinline__ bool sweep_pair(const TileView& tv, int64_t it, int t, int32_t& node) {
  if ((DIM & DIM_LIST) != 0 || tv.pair_node) {
    node = __ldg(tv.pair_node + it);
    return true;
  }
  return tile_pair<DIM>(tv, it, t, node);
}
// first item, end and stride of EB_SWEEP
template <int DIM>
__device__ __forceinline__ bool sweep_list(const TileView& tv) {
  return (DIM & DIM_LIST) != 0 || tv.pair_node != nullptr;
}
template <int DIM>
__device__ __forceinline__ int64_t sweep_begin(const TileView& tv) {
  return sweep_list<DIM>(tv) ? (int64_t)blockIdx.x * blockDim.x + threadIdx.x
                             : 2 * (int64_t)blockIdx.x + (threadIdx.x >> 7);
}
template <int DIM>
__device__ __forceinline__ int64_t sweep_end(const TileView& tv) {
  return sweep_list<DIM>(tv) ? tv.npairs : tv.ntiles;
}
template <int DIM>
__device__ __forceinline__ int64_t sweep_step(const TileView& tv) {
  return sweep_list<DIM>(tv) ? (int64_t)gridDim.x * blockDim.x : 2 * (int64_t)gridDim.x;
}
}  // namespace ebk

// for (each pair this thread handles) body: the CP pairs of the view's list
// when it has one (values at the nodes of the other pairs are never read at a
// CP) or DIM carries DIM_LIST, else every pair of every listed tile as
// EB_PAIR_LOOP (tt_ is then the tile; with a list it is the list index and the
// view has no per-tile shifts)
#define EB_SWEEP(DIM, tv, node)                                                                             \
  for (int64_t tt_ = ::ebk::sweep_begin<DIM>(tv), end_ = ::ebk::sweep_end<DIM>(tv),                         \
               step_ = ::ebk::sweep_step<DIM>(tv);                                                          \
       tt_ < end_; tt_ += step_)                                                                            \
    if (int32_t node = 0; ::ebk::sweep_pair<DIM>((tv), tt_, threadIdx.x & 127, node))
