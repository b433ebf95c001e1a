// Dispatch of the warp-pipelined wavefront sweeps (kernel in sweep3.cuh) and
// the FP64 instantiations.
#include "sweep3.cuh"
#include "sweep3h.cuh"

using namespace sweep3;

namespace {

// Whether the library picks the two-warp sweeps where they apply.
constexpr bool kHelperByDefault = true;

int planes_per_cta(const LevelView& L) {
  const int NW = (L.g.ny + 31) / 32;
  return (L.pk != K64 && (2 * NW + 2) * 32 <= kMaxThreads) ? 2 : 1;
}


}  // namespace

cudaError_t sweep3_launch_k64(int ns, int kind, int dir, bool rec, const Sweep3Params& P, cudaStream_t st) {
  if (ns == 27) return launch_kind<K64, 27, 1, 0>(kind, dir, rec, P, st);
  if (ns == 7) return launch_kind<K64, 7, 1, 0>(kind, dir, rec, P, st);
  return launch_kind<K64, 19, 1, 0>(kind, dir, rec, P, st);
}

bool sweep3_supported(const LevelView& L, int kind) {
  const int ns = L.s.ns;
  if (L.B != 1) return false;
  if (!((ns == 27 && canonical<27>(L.s)) || (ns == 7 && canonical<7>(L.s)) || (ns == 19 && canonical<19>(L.s))))
    return false;
  const int NW = (L.g.ny + 31) / 32;
  const int W = planes_per_cta(L);
  const int maxt = L.pk != K64 ? kMaxThreads
                               : (kind == SW_GS_FULL ? max_threads<K64, SW_GS_FULL>() : max_threads<K64, SW_ILU_L>());
  if (NW > kMaxWarpsPerPlane || (W * NW + 2) * 32 > maxt) return false;
  return (size_t)((L.g.nx + W - 1) / W) * NW <= (size_t)kProgSlots;
}

// Planes per CTA of the two-warp kernel: two when both fit.
static int helper_planes(const LevelView& L) {
  const int NW = (L.g.ny + 31) / 32;
  return NW <= kHelperMaxStrips / 2 ? 2 : 1;
}

int sweep3_warps(const LevelView& L, int kind, bool rec, const SweepCfg& cfg) {
  if (!sweep3_supported(L, kind)) return 0;
  const bool want = cfg.warps == 2 || (cfg.warps == 0 && kHelperByDefault);
  return (rec && want && helper_applies(L.pk, L.s.ns, L.g.nx, L.g.ny, helper_planes(L), kind)) ? 2 : 1;
}

// Planes per CTA: FP64 sweeps are bound by the FP64 pipe, so one plane per
// CTA keeps the per-SM work at one plane; FP32 / BF16 sweeps are bound by
// synchronisation latency, so two planes share a CTA and every other plane
// hand-off stays inside the SM.  rec: M is the sweep's records and b, u are
// vectors, all in the skewed layout (ilurec.cuh); otherwise M is the matrix
// or ILU factors [n][NS] and the vectors are in natural order (FP64 only).
cudaError_t launch_sweep3(const LevelView& L, int kind, int dir, const void* M, const float* sc1, const float* sc2,
                          const void* dinv, double w, const void* b, void* u, SweepWs* ws, int* err,
                          const SweepCfg& cfg, cudaStream_t st, bool rec) {
  if (!sweep3_supported(L, kind)) return cudaErrorNotSupported;
  const int ns = L.s.ns;
  const int W = planes_per_cta(L);
  Sweep3Params P;
  P.g = L.g;
  P.budget_ns = cfg.budget_ns;
  P.M = M;
  P.scale = kind == SW_ILU_U ? sc2 : sc1;
  P.dinv = dinv;
  P.w = w;
  P.b = b;
  P.u = u;
  P.ws = ws;
  P.err = err;
  for (int e = 0; e < 27; ++e) P.lin[e] = L.s.lin[e];
  cudaError_t e = cudaErrorNotSupported;
  // two warps per strip (sweep3h.cuh) where they apply and are asked for
  if (sweep3_warps(L, kind, rec, cfg) == 2) {
    const int Wh = helper_planes(L);
    if (L.pk == K64) e = sweep3h_launch_k64(ns, Wh, kind, dir, P, st);
    else if (L.pk == K32) e = sweep3h_launch_k32(ns, Wh, kind, dir, P, st);
    else e = sweep3h_launch_kbf(ns, Wh, kind, dir, P, st);
    if (e != cudaErrorNotSupported) {
      smg_count_launch(1);
      return e;
    }
  }
  if (L.pk == K64) e = sweep3_launch_k64(ns, kind, dir, rec, P, st);
  else if (L.pk == K32) e = sweep3_launch_k32(ns, W, kind, dir, rec, P, st);
  else e = sweep3_launch_kbf(ns, W, kind, dir, rec, P, st);
  if (e != cudaErrorNotSupported) smg_count_launch(1);
  return e;
}
