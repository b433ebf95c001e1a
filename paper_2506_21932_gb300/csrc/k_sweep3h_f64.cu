// FP64 instantiations of the two-warp wavefront sweeps (sweep3h.cuh).
#include "sweep3h.cuh"

using namespace sweep3;

cudaError_t sweep3h_launch_k64(int ns, int W, int kind, int dir, const Sweep3Params& P, cudaStream_t st) {
  if (W == 2) {
    if (ns == 27) return launch_kind_h<K64, 27, 2, 0>(kind, dir, P, st);
    if (ns == 19) return launch_kind_h<K64, 19, 2, 0>(kind, dir, P, st);
    return cudaErrorNotSupported;
  }
  if (ns == 27) return launch_kind_h<K64, 27, 1, 0>(kind, dir, P, st);
  if (ns == 19) return launch_kind_h<K64, 19, 1, 0>(kind, dir, P, st);
  return cudaErrorNotSupported;
}
