// Software-pipelined wavefront sweeps for the standard masks (7, 19 and 27
// points, one unknown per point): the same exact lexicographic order and the
// same plane-per-CTA schedule as k_sweep.cu (t = SA*i + SB*j + k), with the
// per-step critical path cut to the few dependencies produced in the step
// just before.
//
// Each stencil entry of the point a thread finishes at step t falls in one
// class, fixed at compile time from the mask and the sweep direction:
//   own    the column's previous point (t-1): carried in a register;
//   late   the neighbour column's point finished at t-1: read from a shared
//          memory ring of the last four values of every column;
//   early  neighbour-column points finished at t-2 or before: shared ring;
//   mem    everything else -- the previous plane's new values and all old
//          values -- loaded from global memory two steps ahead.
// Step t therefore (1) finishes point k from a partial sum prepared one step
// earlier plus the own and late terms, (2) forms the partial sum of point k+1
// from the registers loaded one step earlier and the early ring values, and
// (3) issues the loads of point k+2.  A plane waits until the previous plane
// has finished global time t+1 before step t, so the values loaded in (3) are
// final.  Coefficient records further ahead are prefetched into L2.
#include <climits>

#include "smg_internal.cuh"

namespace {

template <int NS> struct Shape;
template <> struct Shape<27> {
  static constexpr int SA = 4, SB = 2, EC = 13;
  __host__ __device__ static constexpr int o(int e, int d) {
    return d == 0 ? e / 9 - 1 : (d == 1 ? (e / 3) % 3 - 1 : e % 3 - 1);
  }
};
template <> struct Shape<7> {
  static constexpr int SA = 1, SB = 1, EC = 3;
  __host__ __device__ static constexpr int o(int e, int d) {
    return d == 0 ? (e == 0 ? -1 : (e == 6 ? 1 : 0)) : d == 1 ? (e == 1 ? -1 : (e == 5 ? 1 : 0))
                                                               : (e == 2 ? -1 : (e == 4 ? 1 : 0));
  }
};
template <> struct Shape<19> {
  static constexpr int SA = 3, SB = 2, EC = 9;
  __host__ __device__ static constexpr int o(int e, int d) {
    // offsets with |dx|+|dy|+|dz| <= 2 in lexicographic order
    constexpr int t[19][3] = {{-1, -1, 0}, {-1, 0, -1}, {-1, 0, 0}, {-1, 0, 1}, {-1, 1, 0}, {0, -1, -1}, {0, -1, 0},
                              {0, -1, 1},  {0, 0, -1},  {0, 0, 0},  {0, 0, 1},  {0, 1, -1}, {0, 1, 0},   {0, 1, 1},
                              {1, -1, 0},  {1, 0, -1},  {1, 0, 0},  {1, 0, 1},  {1, 1, 0}};
    return t[e][d];
  }
};

enum { C_SKIP = 0, C_OWN = 1, C_LATE = 2, C_EARLY = 3, C_MEM = 4 };

// Class of entry e for a sweep of kind KIND in direction DIR (schedule
// coordinates are the actual ones mirrored for DIR = -1).
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

struct Sweep2Params {
  Grid g;
  int G;
  unsigned long long budget_ns;
  const void* M;
  const float* scale;  // KBF row scale used by this sweep (A, L or U)
  const void* dinv;
  double w;
  const void* b;  // may alias u (in-place ILU solves)
  void* u;
  SweepWs* ws;
  int* err;
  int lin[27];  // linear index step of every entry on this grid
};

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

constexpr int kMaxThreads = 512;
constexpr int kPrefetch = 10;  // coefficient records prefetched into L2 this many points ahead

template <int PK, int NS, int KIND, int DIR>
__global__ void __launch_bounds__(kMaxThreads, 1) k_sweep2(Sweep2Params P) {
  using V = typename Prec<PK>::vec;
  using Val = typename Prec<PK>::val;
  using S = Shape<NS>;
  constexpr int SA = S::SA, SB = S::SB;
  __shared__ V hist[4][kMaxThreads];
  __shared__ int s_plane, s_abort, s_last;

  const Grid g = P.g;
  const Val* __restrict__ M = (const Val*)P.M;
  const V* b = (const V*)P.b;
  V* u = (V*)P.u;
  const V* __restrict__ dinv = (const V*)P.dinv;
  const int J = threadIdx.x;
  const bool relax = P.w != 1.0;
  const V w = (V)P.w;

  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      s_plane = atomicAdd(&P.ws->ticket, 1);
      s_abort = 0;
    }
    __syncthreads();
    const int I = s_plane;
    if (I >= g.nx) break;
    const int i = DIR > 0 ? I : g.nx - 1 - I;
    const int j = DIR > 0 ? J : g.ny - 1 - J;
    const bool colok = J < g.ny;
    const int t0 = SA * I;
    const int t1 = t0 + SB * (g.ny - 1) + g.nz - 1;
    int avail = (I == 0) ? INT_MAX : 0;
    int last_pub = t0;

    // stage B: raw loads for the point two steps ahead
    Val cB[NS];
    V mB[NS];
    V bB = V(0), dB = V(0), uoB = V(0);
    float sB = 1.0f;
    // stage A: partial sum and late operands of the next point
    V accA = V(0), bA = V(0), dA = V(0), uoA = V(0);
    Val cOwnA = Val(0), cLateA = Val(0);
    float sA = 1.0f;
    V carry = V(0);
#pragma unroll
    for (int e = 0; e < NS; ++e) {
      cB[e] = Val(0);
      mB[e] = V(0);
    }

    for (int t = t0 - 2; t <= t1; ++t) {
      if (threadIdx.x == 0 && avail < t + 2 && !s_abort) {
        int seen = 0;
        if (!wait_ge(&P.ws->prog[I - 1], t + 2, P.err, P.budget_ns, &seen)) s_abort = 1;
        avail = seen;
      }
      __syncthreads();
      if (s_abort) break;
      if (threadIdx.x == 0 && t - last_pub >= P.G) {
        st_release(&P.ws->prog[I], t);
        last_pub = t;
      }
      const int K = t - t0 - SB * J;

      // (1) finish point K
      if (colok && K >= 0 && K < g.nz) {
        V s = accA;
#pragma unroll
        for (int e = 0; e < NS; ++e) {
          if (cls<NS, KIND, DIR>(e) == C_OWN) s = fma((V)to_c(cOwnA), carry, s);
          if (cls<NS, KIND, DIR>(e) == C_LATE) {
            const int kk = K + DIR * S::o(e, 2);  // schedule z of the neighbour
            const V v = (J > 0 && kk >= 0 && kk < g.nz) ? hist[kk & 3][J - 1] : V(0);
            s = fma((V)to_c(cLateA), v, s);
          }
        }
        if (PK == KBF) s = (V)sA * s;
        V r;
        if (KIND == SW_ILU_L) {
          r = bA - s;
        } else {
          r = (bA - s) * dA;
          if (KIND != SW_ILU_U && relax) r = (KIND == SW_GS_ZERO) ? w * r : (V(1) - w) * uoA + w * r;
        }
        const int k = DIR > 0 ? K : g.nz - 1 - K;
        u[((long long)i * g.ny + j) * g.nz + k] = r;
        hist[K & 3][J] = r;
        carry = r;
      }

      // (2) partial sum of point K+1 from stage B and the early ring values
      const int K1 = K + 1;
      if (colok && K1 >= 0 && K1 < g.nz) {
        V a0 = V(0), a1 = V(0), a2 = V(0), a3 = V(0);
        int q = 0;
#pragma unroll
        for (int e = 0; e < NS; ++e) {
          const int c = cls<NS, KIND, DIR>(e);
          V term_v = V(0);
          bool has = false;
          if (c == C_MEM) {
            term_v = mB[e];
            has = true;
          } else if (c == C_EARLY) {
            const int kk = K1 + DIR * S::o(e, 2);
            term_v = (J > 0 && kk >= 0 && kk < g.nz) ? hist[kk & 3][J - 1] : V(0);
            has = true;
          }
          if (has) {
            const V cv = (V)to_c(cB[e]);
            if ((q & 3) == 0) a0 = fma(cv, term_v, a0);
            else if ((q & 3) == 1) a1 = fma(cv, term_v, a1);
            else if ((q & 3) == 2) a2 = fma(cv, term_v, a2);
            else a3 = fma(cv, term_v, a3);
            ++q;
          }
          if (c == C_OWN) cOwnA = cB[e];
          if (c == C_LATE) cLateA = cB[e];
        }
        accA = (a0 + a1) + (a2 + a3);
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
            mB[e] = in ? (ox != 0 ? __ldcg(u + p2 + P.lin[e]) : u[p2 + P.lin[e]]) : V(0);
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
    __syncthreads();
    if (threadIdx.x == 0) st_release(&P.ws->prog[I], INT_MAX / 2);
  }
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = (atomicAdd(&P.ws->finished, 1) == (int)gridDim.x - 1);
  }
  __syncthreads();
  if (s_last) {
    for (int q = threadIdx.x; q < g.nx; q += blockDim.x) P.ws->prog[q] = 0;
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

template <int PK, int NS>
void launch_kind(int kind, int dir, const Sweep2Params& P, int grid, int nthr, cudaStream_t st) {
  if (kind == SW_GS_ZERO) k_sweep2<PK, NS, SW_GS_ZERO, 1><<<grid, nthr, 0, st>>>(P);
  else if (kind == SW_ILU_L) k_sweep2<PK, NS, SW_ILU_L, 1><<<grid, nthr, 0, st>>>(P);
  else if (kind == SW_ILU_U) k_sweep2<PK, NS, SW_ILU_U, -1><<<grid, nthr, 0, st>>>(P);
  else if (dir > 0) k_sweep2<PK, NS, SW_GS_FULL, 1><<<grid, nthr, 0, st>>>(P);
  else k_sweep2<PK, NS, SW_GS_FULL, -1><<<grid, nthr, 0, st>>>(P);
}

}  // namespace

// Returns cudaErrorNotSupported (nothing launched) when the level is not one
// this kernel handles: 3 unknowns per point, ny > 512, or a mask other than
// the lexicographic 7-, 19- or 27-point one.
cudaError_t launch_sweep2(const LevelView& L, int kind, int dir, const void* M, const float* sc1, const float* sc2,
                          const void* dinv, double w, const void* b, void* u, SweepWs* ws, int* err,
                          const SweepCfg& cfg, cudaStream_t st) {
  if (L.B != 1 || L.g.ny > kMaxThreads) return cudaErrorNotSupported;
  const int ns = L.s.ns;
  if (!((ns == 27 && canonical<27>(L.s)) || (ns == 7 && canonical<7>(L.s)) || (ns == 19 && canonical<19>(L.s))))
    return cudaErrorNotSupported;
  Sweep2Params P;
  P.g = L.g;
  P.G = cfg.G;
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
  const int nthr = ((L.g.ny + 31) / 32) * 32;
  const int grid = L.g.nx;
#define DISPATCH(PK)                                                        \
  do {                                                                      \
    if (ns == 27) launch_kind<PK, 27>(kind, dir, P, grid, nthr, st);       \
    else if (ns == 7) launch_kind<PK, 7>(kind, dir, P, grid, nthr, st);    \
    else launch_kind<PK, 19>(kind, dir, P, grid, nthr, st);                \
  } while (0)
  if (L.pk == K64) DISPATCH(K64);
  else if (L.pk == K32) DISPATCH(K32);
  else DISPATCH(KBF);
#undef DISPATCH
  smg_count_launch(1);
  return cudaGetLastError();
}
