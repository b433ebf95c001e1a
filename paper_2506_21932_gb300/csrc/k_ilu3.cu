// ILU(0) factorisation (Sec. 4.4 ILU formula, on the matrix mask of
// Sec. 4.2) for the canonical 7/19/27-point masks with one unknown per point,
// on the warp-pipelined wavefront of k_sweep3.cu.
//
// Row p of the factors depends on the finished rows of its lower
// neighbours, exactly like a forward triangular solve, so it runs on the same
// schedule t = SA*i + SB*j + k: one CTA per x-plane (taken by ticket), one
// lane per y-column, warps of 32 columns with their own time loops, a warp
// waits only for its left neighbour and for warps w-1..w+1 of the previous
// plane, and one publisher and one poller warp carry the per-warp progress
// between CTAs.  A step factors one row per lane:
//   for every lower entry k (in column order): l = a_pk / u_qq with q the
//   neighbour, then a_pj -= l * u_qj' for every later entry j of row p whose
//   offset difference o_j - o_k is an entry j' of row q (fill outside the
//   mask is dropped);  finally 1 / u_pp.
// The update pairs (j, j') of every k are derived at compile time from the
// mask, so the row lives in registers and every loop is unrolled.  Rows of
// the previous plane belong to another CTA and are read through L2.
#include <algorithm>
#include <climits>
#include <utility>

#include "shapes.cuh"
#include "smg_internal.cuh"
#include "wavefront.cuh"

namespace {

template <int NS>
struct IluPairs {
  int kstart[NS + 1];
  int ej[128];
  int eq[128];
};

// For lower entry k (k < EC) the pairs kstart[k] .. kstart[k+1]-1 list every
// later entry j of the row with o_j - o_k in the mask (entry eq).
template <int NS>
__host__ __device__ constexpr IluPairs<NS> make_pairs() {
  using S = Shape<NS>;
  IluPairs<NS> t{};
  int n = 0;
  for (int ek = 0; ek < S::EC; ++ek) {
    t.kstart[ek] = n;
    for (int ej = ek + 1; ej < NS; ++ej) {
      int eq = -1;
      for (int e = 0; e < NS; ++e)
        if (S::o(e, 0) == S::o(ej, 0) - S::o(ek, 0) && S::o(e, 1) == S::o(ej, 1) - S::o(ek, 1) &&
            S::o(e, 2) == S::o(ej, 2) - S::o(ek, 2))
          eq = e;
      if (eq >= 0) {
        t.ej[n] = ej;
        t.eq[n] = eq;
        ++n;
      }
    }
  }
  for (int e = S::EC; e <= NS; ++e) t.kstart[e] = n;
  return t;
}

template <int NS>
struct IluTab {
  static constexpr IluPairs<NS> v = make_pairs<NS>();
};

// In-grid test of entry e for a point whose neighbour columns are described
// by xymask (bit (dx+1)*3 + dy+1) and whose z neighbours by zmask (bit dz+1).
template <int NS, int E>
__device__ __forceinline__ bool in_grid(unsigned xymask, unsigned zmask) {
  constexpr int ox = Shape<NS>::o(E, 0), oy = Shape<NS>::o(E, 1), oz = Shape<NS>::o(E, 2);
  return ((xymask >> ((ox + 1) * 3 + (oy + 1))) & 1u) && ((zmask >> (oz + 1)) & 1u);
}

// a_pj -= l * u_qj' for pair T of the table
template <int NS, int T>
__device__ __forceinline__ void pair_update(double (&row)[NS], double l, const double* rowq, bool other_cta,
                                            unsigned xymask, unsigned zmask) {
  constexpr int ej = IluTab<NS>::v.ej[T], eq = IluTab<NS>::v.eq[T];
  if (!in_grid<NS, ej>(xymask, zmask)) return;
  const double uv = other_cta ? __ldcg(rowq + eq) : rowq[eq];
  row[ej] = fma(-l, uv, row[ej]);
}

template <int NS, int EK, int... Ts>
__device__ __forceinline__ void pair_updates(double (&row)[NS], double l, const double* rowq, bool other_cta,
                                             unsigned xymask, unsigned zmask, std::integer_sequence<int, Ts...>) {
  (pair_update<NS, IluTab<NS>::v.kstart[EK] + Ts>(row, l, rowq, other_cta, xymask, zmask), ...);
}

// Elimination of lower entry EK of row p: l = a_pk / u_qq, then its updates.
template <int NS, int EK>
__device__ __forceinline__ void eliminate(double (&row)[NS], long long p, const double* LU, const double* udinv,
                                          const int* lin, unsigned xymask, unsigned zmask) {
  if (!in_grid<NS, EK>(xymask, zmask)) return;
  constexpr bool other_cta = Shape<NS>::o(EK, 0) < 0;  // the previous plane is another CTA's
  const long long q = p + lin[EK];
  const double* rowq = LU + q * NS;
  const double uq = other_cta ? __ldcg(udinv + q) : udinv[q];
  const double l = row[EK] * uq;
  row[EK] = l;
  constexpr int npairs = IluTab<NS>::v.kstart[EK + 1] - IluTab<NS>::v.kstart[EK];
  pair_updates<NS, EK>(row, l, rowq, other_cta, xymask, zmask, std::make_integer_sequence<int, npairs>{});
}

template <int NS, int... Ks>
__device__ __forceinline__ void factor_row(double (&row)[NS], long long p, const double* LU, const double* udinv,
                                           const int* lin, unsigned xymask, unsigned zmask,
                                           std::integer_sequence<int, Ks...>) {
  (eliminate<NS, Ks>(row, p, LU, udinv, lin, xymask, zmask), ...);
}

struct Ilu3Params {
  Grid g;
  WfCtl C;
  double* LU;     // in: A, out: factors (same layout)
  double* udinv;  // out: 1 / u_pp
  int lin[27];
};

template <int NS>
__global__ void __launch_bounds__(kWfMaxThreads, 1) k_ilu3(Ilu3Params P) {
  using S = Shape<NS>;
  constexpr int SA = S::SA, SB = S::SB, EC = S::EC;
  __shared__ WfShared sh;
  const Grid g = P.g;
  wf_run(sh, P.C, [&](int I) {
    // compute warp w: columns 32w .. 32w+31 of plane I
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = I, j = 32 * w + lane;
    const bool colok = j < g.ny;
    const int jlast = min(32 * w + 31, g.ny - 1);
    const int s_begin = SB * 32 * w, s_end = SB * jlast + g.nz - 1;
    const int gt0 = SA * I;
    // in-grid mask of the (dx, dy) neighbour columns of this column
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
      // the rows of the previous plane this row reads end at local step s + SA - 1
      if (wf_wait(sh, P.C, w, s, gt0 + s, have_left, have_up, lane)) break;
      const int k = s - SB * j;
      if (colok && k >= 0 && k < g.nz) {
        const long long p = colbase + k;
        const unsigned zmask = (k > 0 ? 1u : 0u) | 2u | (k + 1 < g.nz ? 4u : 0u);
        double row[NS];
        const double* src = P.LU + p * NS;
#pragma unroll
        for (int e = 0; e < NS; ++e) row[e] = src[e];
        factor_row<NS>(row, p, P.LU, P.udinv, P.lin, xymask, zmask, std::make_integer_sequence<int, EC>{});
        const double piv = row[EC];
        if (!(piv > 0.0)) atomicCAS(P.C.err, 0, SMG_EBREAKDOWN);
        double* dst = P.LU + p * NS;
#pragma unroll
        for (int e = 0; e < NS; ++e) dst[e] = row[e];
        P.udinv[p] = 1.0 / piv;
      }
      wf_done(sh, w, s + 1, lane);  // row stored
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

}  // namespace

cudaError_t launch_ilu_factor3(Grid g, const Stencil& s, double* LU, double* udinv, SweepWs* ws, int* err,
                               unsigned long long budget_ns, cudaStream_t st) {
  int grid = 0, nthr = 0;
  cudaError_t e = wf_launch_shape(g, &grid, &nthr);
  if (e != cudaSuccess) return e;
  Ilu3Params P;
  P.g = g;
  P.LU = LU;
  P.udinv = udinv;
  for (int t = 0; t < 27; ++t) P.lin[t] = s.lin[t];
  auto go = [&](auto kern, int SA, int SB) {
    P.C = WfCtl{g.nx, (g.ny + 31) / 32, SA, SB, budget_ns, ws, err};
    cudaError_t a = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWfOneCtaPerSmSmem);
    if (a != cudaSuccess) return a;
    kern<<<grid, nthr, kWfOneCtaPerSmSmem, st>>>(P);
    return cudaGetLastError();
  };
  if (canonical_mask<27>(s)) e = go(k_ilu3<27>, Shape<27>::SA, Shape<27>::SB);
  else if (canonical_mask<19>(s)) e = go(k_ilu3<19>, Shape<19>::SA, Shape<19>::SB);
  else if (canonical_mask<7>(s)) e = go(k_ilu3<7>, Shape<7>::SA, Shape<7>::SB);
  else return cudaErrorNotSupported;
  smg_count_launch(1);
  return e;
}
