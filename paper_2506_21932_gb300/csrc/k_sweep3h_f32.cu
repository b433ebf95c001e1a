// F32 instantiations of the two-warp wavefront sweeps (sweep3h.cuh).
#include "sweep3h.cuh"

using namespace sweep3;

cudaError_t sweep3h_launch_k32(int ns, int W, int kind, int dir, const Sweep3Params& P, cudaStream_t st) {
  if (W == 2) {
    if (ns == 27) return launch_kind_h<K32, 27, 2, 1>(kind, dir, P, st);
    if (ns == 19) return launch_kind_h<K32, 19, 2, 1>(kind, dir, P, st);
    return cudaErrorNotSupported;
  }
  if (ns == 27) return launch_kind_h<K32, 27, 1, 1>(kind, dir, P, st);
  if (ns == 19) return launch_kind_h<K32, 19, 1, 1>(kind, dir, P, st);
  return cudaErrorNotSupported;
}
