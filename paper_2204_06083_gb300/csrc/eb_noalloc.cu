// wave_step_noalloc: the leapfrog steps of wave_step for callers that must
// not allocate during the call.
//
// wave_step runs whole chunks of steps as a CUDA graph cached on the handle;
// building that graph (on the first call for a set of fields, or after they
// change) creates and instantiates a graph, which may allocate.  Some callers
// cannot allow that: code that runs while a larger CUDA graph is being
// captured around it, loops with a fixed memory budget that must not touch the
// allocator after start-up, and processes whose device memory is owned by
// another framework's pool.  This variant launches every step directly on the
// stream: no cudaMalloc / cudaFree, no graph, no allocating library routine.
// The fields and the eb handle are the caller's, created beforehand.
#include "eb_internal.cuh"

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
      rc = launch_leapfrog<double>(h, (double*)u_prev_dev, (double*)u_cur_dev, nsteps, dt, stream, false);
    else if (prec == EB_F32)
      rc = launch_leapfrog<float>(h, (float*)u_prev_dev, (float*)u_cur_dev, nsteps, dt, stream, false);
    else
      throw Failure{EB_ERR_INVALID, "wave_step_noalloc: precision must be EB_F64 or EB_F32"};
  });
  return st != EB_OK ? st : rc;
}
