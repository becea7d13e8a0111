// Host helper for tensor-memory-access (TMA) copies: the tiled tensor-map
// encoder, fetched from the driver through the runtime (no link to libcuda).
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include "eb_internal.cuh"

namespace ebk {

inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    EB_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    EB_REQUIRE(q == cudaDriverEntryPointSuccess && p, EB_ERR_CUDA, "cuTensorMapEncodeTiled not available");
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

}  // namespace ebk
