// Point-block Gauss-Seidel (three coupled unknowns per point, Sec. 4.4
// formulas with 3x3 blocks) for the canonical 7/19/27-point masks, on the
// per-warp wavefront engine (wavefront.cuh):
//   u_p = D_p^{-1} (b_p - sum_{e != centre} A_pe u_{p+o_e}),
// lower neighbours already updated, upper ones old (GS_FULL), or only the
// lower ones from u = 0 (GS_ZERO).  Point (i,j,k) runs at t = SA*i + SB*j + k
// in schedule coordinates (mirrored for the backward sweep); one lane per
// y-column, warps of 32 columns with their own step loops, one x-plane per
// CTA.  Operands are read in the step that uses them: neighbours in the
// previous schedule plane (another CTA's) through L2, the others through L1.
// The arithmetic order per point is that of the plane-per-CTA block kernel.
#include <utility>

#include "shapes.cuh"
#include "smg_internal.cuh"
#include "wavefront.cuh"

namespace {

struct BSweepParams {
  Grid g;
  WfCtl C;
  const void* M;     // [n][NS][3][3]
  const void* dinv;  // [n][3][3]
  double w;
  const void* b;  // [n][3]
  void* u;        // [n][3]
  int lin[27];
};

// Contribution of entry E: acc += A_pE u_q, if E is read by this sweep and
// its neighbour is on the grid.
template <typename V, int NS, int KIND, int DIR, int E>
__device__ __forceinline__ void block_term(V (&acc)[3], long long p, const V* M, const V* u, const int* lin,
                                           unsigned xymask, unsigned zmask) {
  using S = Shape<NS>;
  constexpr int ox = S::o(E, 0), oy = S::o(E, 1), oz = S::o(E, 2);
  constexpr int sx = DIR * ox, sy = DIR * oy, sz = DIR * oz;
  constexpr bool lower = sx < 0 || (sx == 0 && (sy < 0 || (sy == 0 && sz < 0)));
  if (E == S::EC || (KIND == SW_GS_ZERO && !lower)) return;
  if (!(((xymask >> ((ox + 1) * 3 + (oy + 1))) & 1u) && ((zmask >> (oz + 1)) & 1u))) return;
  const V* q = u + (p + lin[E]) * 3;
  V x0, x1, x2;
  if (sx < 0) {  // the previous schedule plane: another CTA's, read through L2
    x0 = __ldcg(q);
    x1 = __ldcg(q + 1);
    x2 = __ldcg(q + 2);
  } else {
    x0 = q[0];
    x1 = q[1];
    x2 = q[2];
  }
  const V* blk = M + (p * NS + E) * 9;
  acc[0] = fma(blk[0], x0, fma(blk[1], x1, fma(blk[2], x2, acc[0])));
  acc[1] = fma(blk[3], x0, fma(blk[4], x1, fma(blk[5], x2, acc[1])));
  acc[2] = fma(blk[6], x0, fma(blk[7], x1, fma(blk[8], x2, acc[2])));
}

template <typename V, int NS, int KIND, int DIR, int... Es>
__device__ __forceinline__ void block_sum(V (&acc)[3], long long p, const V* M, const V* u, const int* lin,
                                          unsigned xymask, unsigned zmask, std::integer_sequence<int, Es...>) {
  (block_term<V, NS, KIND, DIR, Es>(acc, p, M, u, lin, xymask, zmask), ...);
}

template <typename V, int NS, int KIND, int DIR>
__global__ void __launch_bounds__(kWfMaxThreads, 1) k_bsweep3(BSweepParams P) {
  using S = Shape<NS>;
  constexpr int SA = S::SA, SB = S::SB;
  __shared__ WfShared sh;
  const Grid g = P.g;
  const V* __restrict__ M = (const V*)P.M;
  const V* __restrict__ dinv = (const V*)P.dinv;
  const V* b = (const V*)P.b;
  V* u = (V*)P.u;
  wf_run(sh, P.C, [&](int I) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int J = 32 * w + lane;
    const bool colok = J < g.ny;
    const int i = DIR > 0 ? I : g.nx - 1 - I;
    const int j = DIR > 0 ? J : g.ny - 1 - J;
    const int jlast = min(32 * w + 31, g.ny - 1);
    const int s_begin = SB * 32 * w, s_end = SB * jlast + g.nz - 1;
    const int gt0 = SA * I;
    unsigned xymask = 0;
#pragma unroll
    for (int a = -1; a <= 1; ++a)
#pragma unroll
      for (int c = -1; c <= 1; ++c)
        if ((unsigned)(i + a) < (unsigned)g.nx && (unsigned)(j + c) < (unsigned)g.ny)
          xymask |= 1u << ((a + 1) * 3 + (c + 1));
    const long long colbase = ((long long)i * g.ny + j) * g.nz;
    int have_left = (w == 0) ? kWfDone : INT_MIN, have_up = INT_MIN;
    for (int s = s_begin; s <= s_end; ++s) {
      // points of the previous plane read here end at its local step s + SA - 1
      if (wf_wait(sh, P.C, w, s, gt0 + s, have_left, have_up, lane)) break;
      const int K = s - SB * J;
      if (colok && K >= 0 && K < g.nz) {
        const int k = DIR > 0 ? K : g.nz - 1 - K;
        const long long p = colbase + k;
        const unsigned zmask = (k > 0 ? 1u : 0u) | 2u | (k + 1 < g.nz ? 4u : 0u);
        V acc[3] = {V(0), V(0), V(0)};
        block_sum<V, NS, KIND, DIR>(acc, p, M, u, P.lin, xymask, zmask, std::make_integer_sequence<int, NS>{});
        const V s0 = b[p * 3] - acc[0], s1 = b[p * 3 + 1] - acc[1], s2 = b[p * 3 + 2] - acc[2];
        const V* D = dinv + p * 9;
        V r0 = fma(D[0], s0, fma(D[1], s1, D[2] * s2));
        V r1 = fma(D[3], s0, fma(D[4], s1, D[5] * s2));
        V r2 = fma(D[6], s0, fma(D[7], s1, D[8] * s2));
        if (P.w != 1.0) {
          const V wv = (V)P.w;
          if (KIND == SW_GS_ZERO) {
            r0 *= wv;
            r1 *= wv;
            r2 *= wv;
          } else {
            r0 = (V(1) - wv) * u[p * 3] + wv * r0;
            r1 = (V(1) - wv) * u[p * 3 + 1] + wv * r1;
            r2 = (V(1) - wv) * u[p * 3 + 2] + wv * r2;
          }
        }
        u[p * 3] = r0;
        u[p * 3 + 1] = r1;
        u[p * 3 + 2] = r2;
      }
      wf_done(sh, w, s + 1, lane);  // point stored
    }
    if (lane == 0) wf_st_rel_cta(&sh.wdone[w], kWfDone);
  });
}

template <int NS>
bool canonical_mask(const Stencil& s) {
  if (s.ns != NS) return false;
  for (int e = 0; e < NS; ++e)
    for (int d = 0; d < 3; ++d)
      if (s.off[e][d] != Shape<NS>::o(e, d)) return false;
  return true;
}

template <typename V, int NS>
cudaError_t launch_ns(int kind, int dir, BSweepParams& P, int grid, int nthr, cudaStream_t st) {
  P.C.SA = Shape<NS>::SA;
  P.C.SB = Shape<NS>::SB;
  auto go = [&](auto kern) {
    cudaError_t a = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWfOneCtaPerSmSmem);
    if (a != cudaSuccess) return a;
    kern<<<grid, nthr, kWfOneCtaPerSmSmem, st>>>(P);
    return cudaGetLastError();
  };
  if (kind == SW_GS_ZERO) return go(k_bsweep3<V, NS, SW_GS_ZERO, 1>);
  if (dir > 0) return go(k_bsweep3<V, NS, SW_GS_FULL, 1>);
  return go(k_bsweep3<V, NS, SW_GS_FULL, -1>);
}

}  // namespace

cudaError_t launch_bsweep3(const LevelView& L, int kind, int dir, const void* M, const void* dinv, double w,
                           const void* b, void* u, SweepWs* ws, int* err, const SweepCfg& cfg, cudaStream_t st) {
  if (L.B != 3 || L.pk == KBF || (kind != SW_GS_ZERO && kind != SW_GS_FULL)) return cudaErrorNotSupported;
  const bool c7 = canonical_mask<7>(L.s), c19 = canonical_mask<19>(L.s), c27 = canonical_mask<27>(L.s);
  if (!(c7 || c19 || c27)) return cudaErrorNotSupported;
  int grid = 0, nthr = 0;
  cudaError_t e = wf_launch_shape(L.g, &grid, &nthr);
  if (e != cudaSuccess) return e;
  BSweepParams P;
  P.g = L.g;
  P.C = WfCtl{L.g.nx, (L.g.ny + 31) / 32, 0, 0, cfg.budget_ns, ws, err};
  P.M = M;
  P.dinv = dinv;
  P.w = w;
  P.b = b;
  P.u = u;
  for (int t = 0; t < 27; ++t) P.lin[t] = L.s.lin[t];
  if (L.pk == K64) {
    if (c7) e = launch_ns<double, 7>(kind, dir, P, grid, nthr, st);
    else if (c19) e = launch_ns<double, 19>(kind, dir, P, grid, nthr, st);
    else e = launch_ns<double, 27>(kind, dir, P, grid, nthr, st);
  } else {
    if (c7) e = launch_ns<float, 7>(kind, dir, P, grid, nthr, st);
    else if (c19) e = launch_ns<float, 19>(kind, dir, P, grid, nthr, st);
    else e = launch_ns<float, 27>(kind, dir, P, grid, nthr, st);
  }
  smg_count_launch(1);
  return e;
}
