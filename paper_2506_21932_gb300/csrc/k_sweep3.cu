// Warp-pipelined wavefront sweeps (exact lexicographic order) for the
// 7/19/27-point masks with one unknown per point.
//
// Same global schedule as k_sweep.cu / k_sweep2.cu: point (i,j,k) runs at
// t = SA*i + SB*j + k.  What changes is who waits for whom:
//  * A CTA owns W consecutive x-planes.  Each plane is split into warps of
//    32 y-columns; every warp runs its own time loop.  A warp may run local
//    step s once its left neighbour warp has finished step s-1 and the three
//    warps of the previous plane whose columns it reads (w-1, w, w+1) have
//    finished global time t+1 (values two steps ahead are loaded early).
//    These conditions are read from per-warp progress counters in shared
//    memory (CTA-scope acquire/release), so no CTA-wide barrier is taken per
//    step and a warp waits only for the warps it really depends on -- not
//    for the slowest warp of the previous plane.
//  * One extra warp talks to the other CTAs: lane w publishes the progress
//    of warp w of the CTA's last plane with a GPU-scope release store and
//    polls warp w of the previous CTA (relaxed loads, one acquire fence per
//    batch of new values), forwarding it into shared memory.  Compute warps
//    never execute a GPU-scope fence.
//  * At most one CTA runs per SM (the launch reserves more than half of the
//    SM's shared memory) and the grid is capped at the SM count: CTAs take
//    plane groups by ticket, so no plane shares its SM's FP64 pipe with a
//    plane that is still waiting for its turn.
// Inside a warp the step body is the software pipeline of k_sweep2.cu:
// finish point k from a partial sum prepared one step earlier plus the own
// column (register) and neighbour column (shared ring) terms of the previous
// step; pre-sum point k+1 from operands loaded one step earlier; load the
// operands of point k+2.  Every wait is bounded.
#include <algorithm>
#include <climits>

#include "shapes.cuh"
#include "smg_internal.cuh"

namespace {

enum { C_SKIP = 0, C_OWN = 1, C_LATE = 2, C_EARLY = 3, C_MEM = 4 };

template <int NS, int KIND, int DIR>
__host__ __device__ constexpr int cls(int e) {
  using S = Shape<NS>;
  const int sx = DIR * S::o(e, 0), sy = DIR * S::o(e, 1), sz = DIR * S::o(e, 2);
  if (e == S::EC) return C_SKIP;
  const bool is_new = sx < 0 || (sx == 0 && (sy < 0 || (sy == 0 && sz < 0)));
  if (!(KIND == SW_GS_FULL || is_new)) return C_SKIP;
  if (sx == 0 && sy == 0 && sz == -1) return C_OWN;
  if (sx == 0 && sy == -1) return sz == S::SB - 1 ? C_LATE : C_EARLY;
  return C_MEM;
}

struct Sweep3Params {
  Grid g;
  unsigned long long budget_ns;
  const void* M;
  const float* scale;
  const void* dinv;
  double w;
  const void* b;  // may alias u
  void* u;
  SweepWs* ws;    // prog[] indexed by plane group
  int* err;
  int lin[27];
};

constexpr int kMaxWarpsPerPlane = 16;  // ny <= 512
constexpr int kMaxThreads = 576;       // 16 compute + 2 communication warps
constexpr int kPrefetch = 10;
constexpr int kDone = INT_MAX / 2;
constexpr size_t kOneCtaPerSmSmem = 120 * 1024;
constexpr unsigned kPublishGapNs = 300;
// Shared ring of the last kRing values of every column.  A column's value
// at point k is overwritten by point k + kRing.  A warp publishes step s
// once point k is stored, before it reads the ring for point k+1, so its
// left-hand neighbour may run at most kRing - SB - 2 steps ahead of the
// published step without overwriting a value still to be read.
constexpr int kRing = 16;

__device__ __forceinline__ int ld_acq_cta(const int* p) {
  int v;
  asm volatile("ld.acquire.cta.shared.s32 %0, [%1];" : "=r"(v) : "r"((unsigned)__cvta_generic_to_shared(p)) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel_cta(int* p, int v) {
  asm volatile("st.release.cta.shared.s32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "r"(v) : "memory");
}
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

template <int W>
struct Shared3 {
  int wdone[W][kMaxWarpsPerPlane];  // per compute warp: all local steps < value are finished
  int avail[kMaxWarpsPerPlane];     // previous CTA's last plane, per warp: global time finished
  int abort;
  int group;
};

// FP64 sweeps that use every stencil entry hold twice the operands of the
// others; they get 10 warps (ny <= 256) and the registers that leaves.
template <int PK, int KIND>
__host__ __device__ constexpr int max_threads() {
  return (PK == K64 && KIND == SW_GS_FULL) ? 320 : kMaxThreads;
}

template <int PK, int NS, int KIND, int DIR, int W>
__global__ void __launch_bounds__(max_threads<PK, KIND>(), 1) k_sweep3(Sweep3Params P) {
  using V = typename Prec<PK>::vec;
  using Val = typename Prec<PK>::val;
  using S = Shape<NS>;
  constexpr int SA = S::SA, SB = S::SB;
  extern __shared__ unsigned char dyn_smem[];
  __shared__ Shared3<W> sh;

  const Grid g = P.g;
  const int NW = (g.ny + 31) >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ncompute = W * NW;  // warps ncompute and ncompute + 1 talk to the other CTAs
  constexpr int LEAD = kRing - SB - 2;  // largest lead over the right-hand warp
  // shared value ring: hist[plane][k % kRing][column]
  V* hist = (V*)dyn_smem;
  const int ngroups = (g.nx + W - 1) / W;

  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      sh.group = atomicAdd(&P.ws->ticket, 1);
      sh.abort = 0;
    }
    __syncthreads();
    const int I = sh.group;
    if (I >= ngroups) break;
    const int nplanes = min(W, g.nx - I * W);
    if (threadIdx.x < W * kMaxWarpsPerPlane) {
      const int p = threadIdx.x / kMaxWarpsPerPlane, w = threadIdx.x % kMaxWarpsPerPlane;
      // a warp has trivially finished every step before its first one
      sh.wdone[p][w] = (p < nplanes && w < NW) ? SB * 32 * w - 2 : kDone;
    }
    // nothing precedes the first plane; 0 is below every time a later plane asks for
    if (threadIdx.x < kMaxWarpsPerPlane) sh.avail[threadIdx.x] = (I == 0) ? kDone : 0;
    __syncthreads();

    if (warp == ncompute) {
      // ---- publisher warp: lane w publishes the progress of warp w of the
      // CTA's last plane with a GPU-scope release store whenever it grows
      const int plast = nplanes - 1;
      const int gt0 = SA * (I * W + plast);
      const bool mine = lane < NW;
      int* out_slot = P.ws->prog + (size_t)I * NW + lane;
      int published = INT_MIN;
      for (;;) {
        const int T = mine ? ld_acq_cta(&sh.wdone[plast][lane]) : kDone;
        if (__any_sync(0xffffffffu, mine && T != published)) {
          // one release (one GPU-scope fence) covers every lane's value; a
          // fence also stalls the SM's other memory traffic, so they are
          // spaced by a fraction of a step
          if (mine) st_release(out_slot, T >= kDone ? kDone : gt0 + T);
          published = T;
          if (__all_sync(0xffffffffu, T >= kDone)) break;
          __nanosleep(kPublishGapNs);
        } else {
          __nanosleep(32);
        }
        if (__any_sync(0xffffffffu, ld_acq_cta(&sh.abort) != 0)) {
          // release everything downstream; the error word is already set
          if (mine) st_release(out_slot, kDone);
          break;
        }
      }
    } else if (warp == ncompute + 1) {
      // ---- poller warp: lane w forwards the progress of warp w of the
      // previous CTA's last plane into shared memory (GPU-scope acquire loads)
      const bool mine = lane < NW;
      const int* in_slot = P.ws->prog + (size_t)(I - 1) * NW + lane;
      int seen = (I == 0 || !mine) ? kDone : 0;
      unsigned long long t_wait = 0;
      unsigned iter = 0;
      while (__any_sync(0xffffffffu, seen < kDone)) {
        int v = seen;
        if (seen < kDone) asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(in_slot) : "memory");
        const bool fresh = v > seen;
        bool stop = false;
        if (__any_sync(0xffffffffu, fresh)) {
          if (fresh) {
            seen = v;
            st_rel_cta(&sh.avail[lane], v);
          }
          t_wait = 0;
        } else if (lane == 0) {
          // bounded: the previous CTA must make progress within the budget
          const unsigned long long now = globaltimer_ns();
          if (t_wait == 0) t_wait = now;
          else if (now - t_wait > P.budget_ns) {
            atomicCAS(P.err, 0, DEV_ERR_TIMEOUT);
            stop = true;
          }
        }
        if ((++iter & 63u) == 0 && lane == 0) stop = stop || ld_relaxed(P.err) != 0 || ld_acq_cta(&sh.abort) != 0;
        if (__shfl_sync(0xffffffffu, stop, 0)) {
          if (lane == 0) st_rel_cta(&sh.abort, 1);
          break;
        }
      }
    } else if (warp < W * NW) {
      // ---- compute warp (p, w)
      const int p = warp / NW, w = warp % NW;
      if (p < nplanes) {
        const Val* __restrict__ M = (const Val*)P.M;
        const V* b = (const V*)P.b;
        V* u = (V*)P.u;
        const V* __restrict__ dinv = (const V*)P.dinv;
        const bool relax = P.w != 1.0;
        const V wv = (V)P.w;
        const int Ip = I * W + p;  // schedule plane
        const int i = DIR > 0 ? Ip : g.nx - 1 - Ip;
        const int J = 32 * w + lane;
        const bool colok = J < g.ny;
        const int j = DIR > 0 ? J : g.ny - 1 - J;
        const int jlast = min(32 * w + 31, g.ny - 1);
        const int s_begin = SB * 32 * w - 2;
        const int s_end = SB * jlast + g.nz - 1;
        const int gt0 = SA * Ip;
        V* hp = hist + (size_t)p * kRing * (NW * 32);
        int have_left = (w == 0) ? kDone : INT_MIN;        // cached progress of the left warp
        int have_right = (w + 1 == NW) ? kDone : INT_MIN;  // cached progress of the right warp
        int have_up = INT_MIN;                             // cached progress of the previous plane
        Val cB[NS];
        V mB[NS];
        V bB = V(0), dB = V(0), uoB = V(0);
        float sB = 1.0f;
        V accA = V(0), bA = V(0), dA = V(0), uoA = V(0);
        Val cOwnA = Val(0), cLateA = Val(0);
        float sA = 1.0f;
        V carry = V(0);
#pragma unroll
        for (int e = 0; e < NS; ++e) {
          cB[e] = Val(0);
          mB[e] = V(0);
        }
        bool aborted = false;
        for (int s = s_begin; s <= s_end; ++s) {
          // -- dependencies, checked by lane 0 against cached counters
          if (lane == 0) {
            unsigned long long t_start = 0;
            for (;;) {
              bool ok = true;
              if (have_left < s) {
                have_left = ld_acq_cta(&sh.wdone[p][w - 1]);
                ok = have_left >= s;
              }
              if (ok && have_right < s - LEAD) {
                have_right = ld_acq_cta(&sh.wdone[p][w + 1]);
                ok = have_right >= s - LEAD;
              }
              if (ok) {
                // the previous plane's points this warp reads (loads run two
                // steps ahead) lie in columns 32w-1 .. 32w+32: warps w-1..w+1
                const int need = (p == 0) ? gt0 + s + 2 : s + SA + 2;
                if (have_up < need) {
                  const int* src = (p == 0) ? sh.avail : sh.wdone[p - 1];
                  int T = kDone;
                  for (int ww = max(w - 1, 0); ww <= min(w + 1, NW - 1); ++ww) T = min(T, ld_acq_cta(&src[ww]));
                  have_up = T;
                  ok = have_up >= need;
                }
              }
              if (ok) break;
              if (ld_acq_cta(&sh.abort)) { aborted = true; break; }
              const unsigned long long now = globaltimer_ns();
              if (t_start == 0) t_start = now;
              else if (now - t_start > P.budget_ns) {
                atomicCAS(P.err, 0, DEV_ERR_TIMEOUT);
                st_rel_cta(&sh.abort, 1);
                aborted = true;
                break;
              }
            }
          }
          aborted = __shfl_sync(0xffffffffu, aborted, 0);
          if (aborted) break;
          __syncwarp();
          const int K = s - SB * J;

          // (1) finish point K
          if (colok && K >= 0 && K < g.nz) {
            // FOLD (FP64 / FP32): the partial sum of point k started from b and
            // subtracted its terms, so accA = b - (partial sum): fewer FP64
            // operations per point.  BF16 keeps b apart (the row scale
            // multiplies the sum only).
            constexpr bool FOLD = PK != KBF;
            constexpr V sg = FOLD ? V(-1) : V(1);
            V sacc = accA;
#pragma unroll
            for (int e = 0; e < NS; ++e) {
              if (cls<NS, KIND, DIR>(e) == C_OWN) sacc = fma(sg * (V)to_c(cOwnA), carry, sacc);
              if (cls<NS, KIND, DIR>(e) == C_LATE) {
                const int kk = K + DIR * S::o(e, 2);
                const V v = (J > 0 && kk >= 0 && kk < g.nz) ? hp[(kk & (kRing - 1)) * (NW * 32) + J - 1] : V(0);
                sacc = fma(sg * (V)to_c(cLateA), v, sacc);
              }
            }
            if (PK == KBF) sacc = (V)sA * sacc;
            V r;
            if (KIND == SW_ILU_L) {
              r = FOLD ? sacc : bA - sacc;
            } else {
              r = (FOLD ? sacc : bA - sacc) * dA;
              if (KIND != SW_ILU_U && relax) r = (KIND == SW_GS_ZERO) ? wv * r : (V(1) - wv) * uoA + wv * r;
            }
            const int k = DIR > 0 ? K : g.nz - 1 - K;
            u[((long long)i * g.ny + j) * g.nz + k] = r;
            hp[(K & (kRing - 1)) * (NW * 32) + J] = r;
            carry = r;
          }
          // -- point K is stored: publish step s before the loads of K+2 are
          // issued, so the release does not wait for them
          __syncwarp();
          if (lane == 0) st_rel_cta(&sh.wdone[p][w], s + 1);

          // (2) partial sum of point K+1
          const int K1 = K + 1;
          if (colok && K1 >= 0 && K1 < g.nz) {
            constexpr bool FOLD = PK != KBF;
            constexpr V sg = FOLD ? V(-1) : V(1);
            V a0 = FOLD ? bB : V(0), a1 = V(0), a2 = V(0), a3 = V(0);
            int q = 0;
#pragma unroll
            for (int e = 0; e < NS; ++e) {
              const int c = cls<NS, KIND, DIR>(e);
              V tv = V(0);
              bool has = false;
              if (c == C_MEM) {
                tv = mB[e];
                has = true;
              } else if (c == C_EARLY) {
                const int kk = K1 + DIR * S::o(e, 2);
                tv = (J > 0 && kk >= 0 && kk < g.nz) ? hp[(kk & (kRing - 1)) * (NW * 32) + J - 1] : V(0);
                has = true;
              }
              if (has) {
                const V cv = sg * (V)to_c(cB[e]);
                if ((q & 1) == 0) a0 = fma(cv, tv, a0);
                else a1 = fma(cv, tv, a1);
                ++q;
              }
              if (c == C_OWN) cOwnA = cB[e];
              if (c == C_LATE) cLateA = cB[e];
            }
            accA = a0 + a1;
            bA = bB;
            dA = dB;
            sA = sB;
            uoA = uoB;
          }

          // (3) loads of point K+2
          const int K2 = K + 2;
          if (colok && K2 >= 0 && K2 < g.nz) {
            const int k2 = DIR > 0 ? K2 : g.nz - 1 - K2;
            const long long p2 = ((long long)i * g.ny + j) * g.nz + k2;
            const Val* a = M + p2 * NS;
#pragma unroll
            for (int e = 0; e < NS; ++e) {
              const int c = cls<NS, KIND, DIR>(e);
              if (c != C_SKIP) cB[e] = a[e];
              if (c == C_MEM) {
                const int ox = S::o(e, 0), oy = S::o(e, 1), oz = S::o(e, 2);
                const bool in = (unsigned)(i + ox) < (unsigned)g.nx && (unsigned)(j + oy) < (unsigned)g.ny &&
                                (unsigned)(k2 + oz) < (unsigned)g.nz;
                V v = V(0);
                if (in) {
                  // the previous schedule plane of another CTA: read through L2;
                  // everything else (this CTA's planes, old values) through L1
                  const bool other_cta = (DIR * ox < 0) && p == 0;
                  v = other_cta ? __ldcg(u + p2 + P.lin[e]) : u[p2 + P.lin[e]];
                }
                mB[e] = v;
              }
            }
            bB = b[p2];
            if (KIND != SW_ILU_L) dB = dinv[p2];
            if (PK == KBF) sB = P.scale[p2];
            if (KIND == SW_GS_FULL && relax) uoB = u[p2];
            if (K2 + kPrefetch < g.nz) {
              const char* pf = (const char*)(M + (p2 + DIR * kPrefetch) * NS);
              prefetch_l2(pf);
              if (NS * sizeof(Val) > 128) prefetch_l2(pf + 128);
            }
          }
        }
        if (lane == 0) st_rel_cta(&sh.wdone[p][w], kDone);
      }
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    sh.group = (atomicAdd(&P.ws->finished, 1) == (int)gridDim.x - 1);
  }
  __syncthreads();
  if (sh.group) {
    for (int q = threadIdx.x; q < ngroups * NW; q += blockDim.x) P.ws->prog[q] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
      P.ws->ticket = 0;
      __threadfence();
      P.ws->finished = 0;
    }
  }
}

template <int NS>
bool canonical(const Stencil& s) {
  if (s.ns != NS) return false;
  for (int e = 0; e < NS; ++e)
    for (int d = 0; d < 3; ++d)
      if (s.off[e][d] != Shape<NS>::o(e, d)) return false;
  return true;
}

template <int PK, int NS, int W>
cudaError_t launch_kind(int kind, int dir, const Sweep3Params& P, cudaStream_t st) {
  using V = typename Prec<PK>::vec;
  const int NW = (P.g.ny + 31) / 32;
  const int nthr = (W * NW + 2) * 32;
  // the value ring needs <= 64 KB (ny <= 512); reserving more than half of
  // the SM's 228 KB keeps a second CTA off the SM
  const size_t smem = std::max(sizeof(V) * kRing * (size_t)(NW * 32) * W, kOneCtaPerSmSmem);
  int dev = 0, nsm = 0;
  cudaError_t ae = cudaGetDevice(&dev);
  if (ae == cudaSuccess) ae = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (ae != cudaSuccess) return ae;
  const int grid = std::min((P.g.nx + W - 1) / W, nsm);
  auto go = [&](auto kern) {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    kern<<<grid, nthr, smem, st>>>(P);
    return cudaGetLastError();
  };
  if (kind == SW_GS_ZERO) return go(k_sweep3<PK, NS, SW_GS_ZERO, 1, W>);
  if (kind == SW_ILU_L) return go(k_sweep3<PK, NS, SW_ILU_L, 1, W>);
  if (kind == SW_ILU_U) return go(k_sweep3<PK, NS, SW_ILU_U, -1, W>);
  if (dir > 0) return go(k_sweep3<PK, NS, SW_GS_FULL, 1, W>);
  return go(k_sweep3<PK, NS, SW_GS_FULL, -1, W>);
}

}  // namespace

// Planes per CTA: FP64 sweeps are bound by the FP64 pipe, so one plane per
// CTA keeps the per-SM work at one plane; FP32 / BF16 sweeps are bound by
// synchronisation latency, so two planes share a CTA and every other plane
// hand-off stays inside the SM.
cudaError_t launch_sweep3(const LevelView& L, int kind, int dir, const void* M, const float* sc1, const float* sc2,
                          const void* dinv, double w, const void* b, void* u, SweepWs* ws, int* err,
                          const SweepCfg& cfg, cudaStream_t st) {
  const int ns = L.s.ns;
  if (L.B != 1) return cudaErrorNotSupported;
  if (!((ns == 27 && canonical<27>(L.s)) || (ns == 7 && canonical<7>(L.s)) || (ns == 19 && canonical<19>(L.s))))
    return cudaErrorNotSupported;
  const int NW = (L.g.ny + 31) / 32;
  // two planes per CTA only off FP64: an FP64 plane already keeps its SM's
  // FP64 pipe busy enough that a second one slows both (measured)
  const int W = (L.pk != K64 && (2 * NW + 2) * 32 <= kMaxThreads) ? 2 : 1;
  const int maxt = (L.pk == K64 && kind == SW_GS_FULL) ? max_threads<K64, SW_GS_FULL>() : kMaxThreads;
  if (NW > kMaxWarpsPerPlane || (W * NW + 2) * 32 > maxt) return cudaErrorNotSupported;
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
  cudaError_t e;
#define DISPATCH(PK, WW)                                                   \
  do {                                                                     \
    if (ns == 27) e = launch_kind<PK, 27, WW>(kind, dir, P, st);           \
    else if (ns == 7) e = launch_kind<PK, 7, WW>(kind, dir, P, st);        \
    else e = launch_kind<PK, 19, WW>(kind, dir, P, st);                    \
  } while (0)
  if (L.pk == K64) DISPATCH(K64, 1);
  else if (L.pk == K32) {
    if (W == 2) DISPATCH(K32, 2);
    else DISPATCH(K32, 1);
  } else {
    if (W == 2) DISPATCH(KBF, 2);
    else DISPATCH(KBF, 1);
  }
#undef DISPATCH
  smg_count_launch(1);
  return e;
}
