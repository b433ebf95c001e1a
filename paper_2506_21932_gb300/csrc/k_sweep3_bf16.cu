// BF16 instantiations of the warp-pipelined wavefront sweeps (sweep3.cuh).
#include "sweep3.cuh"

using namespace sweep3;

cudaError_t sweep3_launch_kbf(int ns, int W, int kind, int dir, bool rec, const Sweep3Params& P, cudaStream_t st) {
  if (W == 2) {
    if (ns == 27) return launch_kind<KBF, 27, 2, 1>(kind, dir, rec, P, st);
    if (ns == 7) return launch_kind<KBF, 7, 2, 1>(kind, dir, rec, P, st);
    return launch_kind<KBF, 19, 2, 1>(kind, dir, rec, P, st);
  }
  if (ns == 27) return launch_kind<KBF, 27, 1, 1>(kind, dir, rec, P, st);
  if (ns == 7) return launch_kind<KBF, 7, 1, 1>(kind, dir, rec, P, st);
  return launch_kind<KBF, 19, 1, 1>(kind, dir, rec, P, st);
}
