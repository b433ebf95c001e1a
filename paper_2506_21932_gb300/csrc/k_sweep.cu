// Dependence-preserving triangular sweeps on structured grids (Sec. 4.4):
// forward / backward Gauss-Seidel, the two ILU(0) triangular solves and the
// ILU(0) factorisation, each producing exactly the lexicographic-order result.
//
// Schedule.  A point (i,j,k) of the sweep (coordinates mirrored for backward
// sweeps) is processed at global time t = SA*i + SB*j + k.  SA and SB are the
// smallest skews for which every lower stencil neighbour has a strictly
// smaller t and every upper one a strictly larger t (27-point: SA=4, SB=2;
// 7-point: SA=SB=1), so processing all points of equal t in parallel, in
// increasing t, reads exactly the values the sequential sweep reads.
//
// Mapping.  One CTA owns one x-plane (plane order handed out by an atomic
// ticket, so a CTA only ever waits for planes claimed before it) with one
// thread per y-column; a CTA-wide barrier separates consecutive time steps,
// which orders the in-plane dependencies.  Plane i may run time t only after
// plane i-1 has finished every step below t: plane i-1 publishes its progress
// with a release store every G steps, plane i reads it with acquire loads
// (this is the paper's counter array of Sec. 4.4, at plane granularity).
// Every wait is bounded; on expiry the error word is set and all CTAs drain.
#include <climits>

#include "smg_internal.cuh"

namespace {

struct SweepParams {
  Grid g;
  Stencil s;
  int SA, SB, G;
  unsigned long long budget_ns;
  const void* M;       // matrix (GS) or LU factors (ILU)
  const float* sc1;    // KBF: row scale of M (GS) / of L (ILU_L)
  const float* sc2;    // KBF: row scale of U (ILU_U)
  const void* dinv;    // inverse diagonal: double (K64), float (K32/KBF); 3x3 blocks when B == 3
  double w;            // relaxation weight (GS)
  const void* b;       // right-hand side (GS), r (ILU_L), y (ILU_U)
  void* u;             // iterate (GS, in place), y (ILU_L), x (ILU_U)
  SweepWs* ws;
  int* err;
};

template <typename V>
__device__ __forceinline__ V ld_other_plane(const V* p) {
  return __ldcg(p);
}

// Claims planes, runs the time loop, publishes progress and resets the
// workspace when the last CTA leaves.  Body(I, t) computes one step.
template <typename Body>
__device__ __forceinline__ void plane_pipeline(const SweepParams& P, Body body) {
  __shared__ int s_plane, s_abort, s_last;
  const Grid& g = P.g;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      s_plane = atomicAdd(&P.ws->ticket, 1);
      s_abort = 0;
    }
    __syncthreads();
    const int I = s_plane;
    if (I >= g.nx) break;
    const int t0 = P.SA * I;
    const int t1 = t0 + P.SB * (g.ny - 1) + g.nz - 1;
    int avail = (I == 0) ? INT_MAX : 0;
    int last_pub = t0;
    for (int t = t0; t <= t1; ++t) {
      if (threadIdx.x == 0 && avail < t && !s_abort) {
        int seen = 0;
        if (!wait_ge(&P.ws->prog[I - 1], t, P.err, P.budget_ns, &seen)) s_abort = 1;
        avail = seen;
      }
      __syncthreads();
      if (s_abort) break;
      if (threadIdx.x == 0 && t - last_pub >= P.G) {
        st_release(&P.ws->prog[I], t);
        last_pub = t;
      }
      body(I, t - t0);
    }
    __syncthreads();
    if (threadIdx.x == 0) st_release(&P.ws->prog[I], INT_MAX / 2);
  }
  // the last CTA out resets the workspace for the next sweep on this stream
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

// Scalar sweep.  KIND: SW_GS_FULL (all neighbours, D^{-1}, weight w),
// SW_GS_ZERO (forward from u = 0: lower neighbours only), SW_ILU_L (unit
// lower solve), SW_ILU_U (upper solve times 1/u_pp).  DIR +1 / -1.
template <int PK, int NS, int KIND, int DIR>
__global__ void __launch_bounds__(1024) k_sweep1(SweepParams P) {
  using V = typename Prec<PK>::vec;
  using Val = typename Prec<PK>::val;
  const Grid g = P.g;
  const Val* __restrict__ M = (const Val*)P.M;
  const V* b = (const V*)P.b;  // may alias u (in-place ILU solves)
  V* u = (V*)P.u;
  const V* __restrict__ dinv = (const V*)P.dinv;
  const int J = threadIdx.x;
  constexpr int EC = NS / 2;
  constexpr int E0 = (KIND == SW_ILU_U) ? EC + 1 : 0;
  constexpr int E1 = (KIND == SW_GS_ZERO || KIND == SW_ILU_L) ? EC : NS;
  plane_pipeline(P, [&](int I, int tl) {
    const int K = tl - P.SB * J;
    if (J >= g.ny || K < 0 || K >= g.nz) return;
    const int i = DIR > 0 ? I : g.nx - 1 - I;
    const int j = DIR > 0 ? J : g.ny - 1 - J;
    const int k = DIR > 0 ? K : g.nz - 1 - K;
    const long long p = ((long long)i * g.ny + j) * g.nz + k;
    const Val* a = M + p * NS;
    V acc = 0;
#pragma unroll
    for (int e = E0; e < E1; ++e) {
      if (e == EC) continue;
      const int dx = P.s.off[e][0], dy = P.s.off[e][1], dz = P.s.off[e][2];
      const bool in = (unsigned)(i + dx) < (unsigned)g.nx && (unsigned)(j + dy) < (unsigned)g.ny &&
                      (unsigned)(k + dz) < (unsigned)g.nz;
      V xv = V(0);
      if (in) xv = dx != 0 ? ld_other_plane(u + p + P.s.lin[e]) : u[p + P.s.lin[e]];
      acc = fma((V)to_c(a[e]), xv, acc);
    }
    V r;
    if (KIND == SW_ILU_L) {
      if (PK == KBF) acc = (V)P.sc1[p] * acc;
      r = b[p] - acc;
    } else if (KIND == SW_ILU_U) {
      if (PK == KBF) acc = (V)P.sc2[p] * acc;
      r = (b[p] - acc) * dinv[p];
    } else {
      if (PK == KBF) acc = (V)P.sc1[p] * acc;
      r = (b[p] - acc) * dinv[p];
      if (P.w != 1.0) {
        V w = (V)P.w;
        r = (KIND == SW_GS_ZERO) ? w * r : (V(1) - w) * u[p] + w * r;
      }
    }
    u[p] = r;
  });
}

// Point-block (3 unknowns) Gauss-Seidel: u_p = D_p^{-1}(b_p - sum A_pe u_q).
template <typename V, int KIND, int DIR>
__global__ void __launch_bounds__(1024) k_sweep3(SweepParams P) {
  const Grid g = P.g;
  const V* __restrict__ M = (const V*)P.M;
  const V* b = (const V*)P.b;  // may alias u (in-place ILU solves)
  V* u = (V*)P.u;
  const V* __restrict__ dinv = (const V*)P.dinv;
  const int J = threadIdx.x;
  const int NS = P.s.ns, EC = P.s.ec;
  const int E1 = (KIND == SW_GS_ZERO) ? EC : NS;
  plane_pipeline(P, [&](int I, int tl) {
    const int K = tl - P.SB * J;
    if (J >= g.ny || K < 0 || K >= g.nz) return;
    const int i = DIR > 0 ? I : g.nx - 1 - I;
    const int j = DIR > 0 ? J : g.ny - 1 - J;
    const int k = DIR > 0 ? K : g.nz - 1 - K;
    const long long p = ((long long)i * g.ny + j) * g.nz + k;
    V a0 = 0, a1 = 0, a2 = 0;
    for (int e = 0; e < E1; ++e) {
      if (e == EC) continue;
      const int dx = P.s.off[e][0], dy = P.s.off[e][1], dz = P.s.off[e][2];
      if (!((unsigned)(i + dx) < (unsigned)g.nx && (unsigned)(j + dy) < (unsigned)g.ny &&
            (unsigned)(k + dz) < (unsigned)g.nz))
        continue;
      const V* q = u + (p + P.s.lin[e]) * 3;
      V x0, x1, x2;
      if (dx != 0) { x0 = __ldcg(q); x1 = __ldcg(q + 1); x2 = __ldcg(q + 2); }
      else { x0 = q[0]; x1 = q[1]; x2 = q[2]; }
      const V* blk = M + (p * NS + e) * 9;
      a0 = fma(blk[0], x0, fma(blk[1], x1, fma(blk[2], x2, a0)));
      a1 = fma(blk[3], x0, fma(blk[4], x1, fma(blk[5], x2, a1)));
      a2 = fma(blk[6], x0, fma(blk[7], x1, fma(blk[8], x2, a2)));
    }
    const V s0 = b[p * 3] - a0, s1 = b[p * 3 + 1] - a1, s2 = b[p * 3 + 2] - a2;
    const V* D = dinv + p * 9;
    V r0 = fma(D[0], s0, fma(D[1], s1, D[2] * s2));
    V r1 = fma(D[3], s0, fma(D[4], s1, D[5] * s2));
    V r2 = fma(D[6], s0, fma(D[7], s1, D[8] * s2));
    if (P.w != 1.0) {
      V w = (V)P.w;
      if (KIND == SW_GS_ZERO) { r0 *= w; r1 *= w; r2 *= w; }
      else {
        r0 = (V(1) - w) * u[p * 3] + w * r0;
        r1 = (V(1) - w) * u[p * 3 + 1] + w * r1;
        r2 = (V(1) - w) * u[p * 3 + 2] + w * r2;
      }
    }
    u[p * 3] = r0;
    u[p * 3 + 1] = r1;
    u[p * 3 + 2] = r2;
  });
}

// ILU(0) factorisation, row by row in lexicographic order (IKJ elimination
// restricted to the mask): for every lower entry k of row p, l = a_pk / u_qq
// (q = p + o_k), then a_pj -= l * u_{q, o_j - o_k} for the later entries j of
// row p whose offset difference is in the mask.  `upd` lists, per lower entry
// k, the pairs (j, index of o_j - o_k): kstart[k] .. kstart[k+1].
struct IluParams {
  SweepParams base;
  const int* kstart;  // [ec + 1]
  const int2* pairs;  // {j, jq}
  double* LU;
  double* udinv;
};

__global__ void __launch_bounds__(1024) k_ilu_factor(IluParams Q) {
  const SweepParams& P = Q.base;
  const Grid g = P.g;
  const int J = threadIdx.x;
  const int EC = P.s.ec, NS = P.s.ns;
  double* LU = Q.LU;
  plane_pipeline(P, [&](int I, int tl) {
    const int K = tl - P.SB * J;
    if (J >= g.ny || K < 0 || K >= g.nz) return;
    const int i = I, j = J, k = K;
    const long long p = ((long long)i * g.ny + j) * g.nz + k;
    double* row = LU + p * NS;
    for (int ek = 0; ek < EC; ++ek) {
      const int dx = P.s.off[ek][0], dy = P.s.off[ek][1], dz = P.s.off[ek][2];
      if (!((unsigned)(i + dx) < (unsigned)g.nx && (unsigned)(j + dy) < (unsigned)g.ny &&
            (unsigned)(k + dz) < (unsigned)g.nz))
        continue;
      const long long q = p + P.s.lin[ek];
      const double* rowq = LU + q * NS;
      const double uq = dx != 0 ? __ldcg(Q.udinv + q) : Q.udinv[q];
      const double l = row[ek] * uq;
      row[ek] = l;
      for (int t = Q.kstart[ek]; t < Q.kstart[ek + 1]; ++t) {
        const int2 pr = Q.pairs[t];
        const int ej = pr.x, eq = pr.y;
        if (!((unsigned)(i + P.s.off[ej][0]) < (unsigned)g.nx && (unsigned)(j + P.s.off[ej][1]) < (unsigned)g.ny &&
              (unsigned)(k + P.s.off[ej][2]) < (unsigned)g.nz))
          continue;
        const double uqv = dx != 0 ? __ldcg(rowq + eq) : rowq[eq];
        row[ej] = fma(-l, uqv, row[ej]);
      }
    }
    const double piv = row[EC];
    if (!(piv > 0.0)) atomicCAS(P.err, 0, SMG_EBREAKDOWN);
    Q.udinv[p] = 1.0 / piv;
  });
}

int sweep_threads(const Grid& g) { return ((g.ny + 31) / 32) * 32; }

// One bounded wait on a flag that nothing sets: exercises the timeout path of
// wait_ge (it records DEV_ERR_TIMEOUT and returns).
__global__ void k_wait_selftest(const int* flag, int* err, unsigned long long budget_ns) {
  int seen = 0;
  wait_ge(flag, 1, err, budget_ns, &seen);
}

}  // namespace

cudaError_t launch_wait_selftest(const int* flag, int* err, unsigned long long budget_ns, cudaStream_t st) {
  k_wait_selftest<<<1, 1, 0, st>>>(flag, err, budget_ns);
  smg_count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_sweep(const LevelView& L, int kind, int dir, const void* M, const float* sc1, const float* sc2,
                         const void* dinv, double w, const void* b, void* u, SweepWs* ws, int* err,
                         const SweepCfg& cfg, cudaStream_t st) {
  {
    cudaError_t e3 = launch_sweep3(L, kind, dir, M, sc1, sc2, dinv, w, b, u, ws, err, cfg, st, false);
    if (e3 != cudaErrorNotSupported) return e3;
    cudaError_t e2 = launch_sweep2(L, kind, dir, M, sc1, sc2, dinv, w, b, u, ws, err, cfg, st);
    if (e2 != cudaErrorNotSupported) return e2;
  }
  SweepParams P;
  P.g = L.g;
  P.s = L.s;
  P.SA = cfg.SA;
  P.SB = cfg.SB;
  P.G = cfg.G;
  P.budget_ns = cfg.budget_ns;
  P.M = M;
  P.sc1 = sc1;
  P.sc2 = sc2;
  P.dinv = dinv;
  P.w = w;
  P.b = b;
  P.u = u;
  P.ws = ws;
  P.err = err;
  const int nthr = sweep_threads(L.g);
  const int grid = L.g.nx;
  if (L.B == 3) {
    cudaError_t eb = launch_bsweep3(L, kind, dir, M, dinv, w, b, u, ws, err, cfg, st);
    if (eb != cudaErrorNotSupported) return eb;
#define S3(V, KD, DR) k_sweep3<V, KD, DR><<<grid, nthr, 0, st>>>(P)
    if (L.pk == K64) {
      if (kind == SW_GS_ZERO) S3(double, SW_GS_ZERO, 1);
      else if (dir > 0) S3(double, SW_GS_FULL, 1);
      else S3(double, SW_GS_FULL, -1);
    } else {
      if (kind == SW_GS_ZERO) S3(float, SW_GS_ZERO, 1);
      else if (dir > 0) S3(float, SW_GS_FULL, 1);
      else S3(float, SW_GS_FULL, -1);
    }
#undef S3
    return cudaGetLastError();
  }
#define S1(PK, NS)                                                                \
  do {                                                                            \
    if (kind == SW_GS_ZERO) k_sweep1<PK, NS, SW_GS_ZERO, 1><<<grid, nthr, 0, st>>>(P); \
    else if (kind == SW_ILU_L) k_sweep1<PK, NS, SW_ILU_L, 1><<<grid, nthr, 0, st>>>(P); \
    else if (kind == SW_ILU_U) k_sweep1<PK, NS, SW_ILU_U, -1><<<grid, nthr, 0, st>>>(P); \
    else if (dir > 0) k_sweep1<PK, NS, SW_GS_FULL, 1><<<grid, nthr, 0, st>>>(P);  \
    else k_sweep1<PK, NS, SW_GS_FULL, -1><<<grid, nthr, 0, st>>>(P);              \
  } while (0)
#define SPK(PK)                       \
  do {                                \
    if (L.s.ns == 27) S1(PK, 27);     \
    else if (L.s.ns == 7) S1(PK, 7);  \
    else if (L.s.ns == 19) S1(PK, 19); \
    else return cudaErrorInvalidValue; \
  } while (0)
  if (L.pk == K64) SPK(K64);
  else if (L.pk == K32) SPK(K32);
  else SPK(KBF);
#undef SPK
#undef S1
  smg_count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_ilu_factor(Grid g, const Stencil& s, const double* A, double* LU, double* udinv, const int* upd,
                              int nupd, SweepWs* ws, int* err, const SweepCfg& cfg, cudaStream_t st) {
  (void)nupd;
  cudaError_t e = cudaMemcpyAsync(LU, A, sizeof(double) * g.n * s.ns, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  e = launch_ilu_factor3(g, s, LU, udinv, ws, err, cfg.budget_ns, st);
  if (e != cudaErrorNotSupported) return e;
  IluParams Q;
  Q.base.g = g;
  Q.base.s = s;
  Q.base.SA = cfg.SA;
  Q.base.SB = cfg.SB;
  Q.base.G = cfg.G;
  Q.base.budget_ns = cfg.budget_ns;
  Q.base.ws = ws;
  Q.base.err = err;
  Q.kstart = upd;
  Q.pairs = (const int2*)(upd + (s.ec + 1 + 1) / 2 * 2);
  Q.LU = LU;
  Q.udinv = udinv;
  k_ilu_factor<<<g.nx, sweep_threads(g), 0, st>>>(Q);
  smg_count_launch(1);
  return cudaGetLastError();
}
