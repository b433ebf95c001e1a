// Two-warp form of the skewed-layout wavefront sweeps of sweep3.cuh (same
// schedule, same records, same rounding), included by one translation unit
// per working precision (k_sweep3h*.cu).
#pragma once
// Why: one SM sub-partition issues one FP64 warp instruction per 64 cycles
// however many lanes are active, and a warp's instructions issue in order,
// so in the one-warp sweep the FMAs of the early partial sum of point K+1
// and the loads and unpacking of its records sit on the same instruction
// stream as the dependent finish of point K.  Here every 32-column strip of
// a plane has two warps, placed on different sub-partitions:
//  * the helper warp owns the operands: it waits for the previous plane,
//    loads that plane's rows into the strip's row ring, loads the records,
//    forms the partial sum of every term that is final early (the terms
//    sweep3.cuh pre-sums) and hands the sum, the finish coefficients and the
//    point's constants to the main warp through a two-slot shared buffer;
//  * the main warp only finishes points: the late terms (own column, left
//    column, the previous plane's latest rows), the store, the publish.
// The helper of step s runs while the main warp finishes step s - 1.
// Sums are formed in the same order as in sweep3.cuh, so both kernels give
// bitwise equal results.  Every wait is bounded like in sweep3.cuh.
#include "sweep3.cuh"

namespace sweep3 {

template <int W>
struct Shared3h {
  int wdone[W][kMaxWarpsPerPlane];  // main warps: all local steps < value are finished
  int hrdy[W][kMaxWarpsPerPlane];   // helper warps: operands of all local steps < value are handed over
  int avail[kMaxWarpsPerPlane];     // previous CTA's last plane, per strip: global time finished
  int abort;
  int group;
};

// 8 strips x 2 warps + the two communication warps.  FP64 ILU(0) solves on
// planes of 9 to 12 strips (one per CTA) get an 832-thread instantiation
// (72 registers a thread); FP32 / BF16 sweeps there measured no faster than
// the one-warp kernel (BF16 2% slower at 384^3), which keeps them.
constexpr int kHelperThreads = 576;
constexpr int kHelperMaxStrips = 8;
constexpr int kHelperWideThreads = 832;
constexpr int kHelperWideStrips = 12;

// finish terms of point K (the ones the main warp adds)
template <int NS, int KIND, int DIR, int X>
__host__ __device__ constexpr bool is_fin(int e) {
  const int us = use<NS, KIND, DIR, X>(e);
  return us == U_FIN0 || us == U_FIN1 || us == U_FINR;
}
template <int NS, int KIND, int DIR, int X>
__host__ __device__ constexpr int fin_index(int e) {
  int n = 0;
  for (int q = 0; q < e; ++q) n += is_fin<NS, KIND, DIR, X>(q) ? 1 : 0;
  return n;
}
template <int NS, int KIND, int DIR, int X>
__host__ __device__ constexpr int nfin() {
  return fin_index<NS, KIND, DIR, X>(NS);
}

// hand-over slot fields, each 32 values wide (one per lane)
enum { F_ACC = 0, F_B = 1, F_D = 2, F_S = 3, F_UO = 4, F_CF = 5 };
template <int NS, int KIND, int DIR, int X>
__host__ __device__ constexpr int nfields() {
  return F_CF + nfin<NS, KIND, DIR, X>();
}

template <typename V, int NS, int KIND, int DIR, int X>
__host__ __device__ constexpr size_t helper_smem_bytes(int NW, int W) {
  return sizeof(V) * ((size_t)kRing * NW * 32 * W + (size_t)kRowRing * kRowCols * NW * W +
                      (size_t)2 * nfields<NS, KIND, DIR, X>() * 32 * NW * W);
}

template <int PK, int NS, int KIND, int DIR, int W, int X, int MT>
__global__ void __launch_bounds__(MT, 1) k_sweep3h(Sweep3Params P) {
  using V = typename Prec<PK>::vec;
  using Val = typename Prec<PK>::val;
  using S = Shape<NS>;
  constexpr int SA = S::SA, SB = S::SB;
  using R = SweepRec<PK, NS, KIND == SW_ILU_L ? 0 : (KIND == SW_ILU_U ? 1 : 2)>;
  constexpr bool FOLD = PK != KBF;
  constexpr V sg = FOLD ? V(-1) : V(1);
  constexpr int NFLD = nfields<NS, KIND, DIR, X>();
  extern __shared__ unsigned char dyn_smem[];
  __shared__ Shared3h<W> sh;

  const Grid g = P.g;
  const int NW = (g.ny + 31) >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nstrip = W * NW;
  const int ncompute = 2 * nstrip;  // warps ncompute and ncompute + 1 talk to the other CTAs
  constexpr int LEAD = kRing - SB - 2;
  V* hist = (V*)dyn_smem;
  V* prow_all = hist + (size_t)W * kRing * NW * 32;
  V* slot_all = prow_all + (size_t)nstrip * kRowRing * kRowCols;
  const int ngroups = (g.nx + W - 1) / W;
  for (int t = threadIdx.x; t < W * kRing * NW * 32; t += blockDim.x) hist[t] = V(0);

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
      const int v0 = (p < nplanes && w < NW) ? SB * 32 * w - 2 : kDone;
      sh.wdone[p][w] = v0;
      sh.hrdy[p][w] = v0;
    }
    if (threadIdx.x < kMaxWarpsPerPlane) sh.avail[threadIdx.x] = (I == 0) ? kDone : 0;
    __syncthreads();

    if (warp == ncompute) {
      publisher_warp(sh, sh.wdone[nplanes - 1], P, I, NW, SA * (I * W + nplanes - 1), lane);
    } else if (warp == ncompute + 1) {
      poller_warp(sh, P, I, NW, lane);
    } else if (warp < ncompute) {
      // strip c has warps 2c and 2c + 1; which of them is the main warp
      // alternates every two strips, so each sub-partition (warp % 4) gets
      // as many main warps as helpers
      const int c = warp >> 1;
      const bool is_main = (warp & 1) == ((c >> 1) & 1);
      const int p = c / NW, w = c % NW;
      if (p < nplanes) {
        const V* b = (const V*)P.b;
        V* u = (V*)P.u;
        const bool relax = P.w != 1.0;
        const V wv = (V)P.w;
        const int Ip = I * W + p;
        const int i = DIR > 0 ? Ip : g.nx - 1 - Ip;
        const int J = 32 * w + lane;
        const bool colok = J < g.ny;
        const int j = DIR > 0 ? J : g.ny - 1 - J;
        const int jlast = min(32 * w + 31, g.ny - 1);
        const int s_begin = SB * 32 * w - 2;
        const int s_end = SB * jlast + g.nz - 1;
        const int gt0 = SA * Ip;
        V* hp = hist + (size_t)p * kRing * (NW * 32);
        V* prw = prow_all + (size_t)c * (kRowRing * kRowCols);
        V* slots = slot_all + (size_t)c * (2 * NFLD * 32);
        const int rback = (g.nz - 1 + SB * (g.ny - 1)) % g.nz;
        auto row_of = [&](int t) -> int {
          const int r = (DIR > 0 ? t : rback - t) % g.nz;
          return r < 0 ? r + g.nz : r;
        };
        auto step_off = [&](int d) -> int {
          const int r = (DIR * d) % g.nz;
          return r < 0 ? r + g.nz : r;
        };
        auto radd = [&](int r, int off) -> int {
          r += off;
          return r >= g.nz ? r - g.nz : r;
        };
        // previous-plane neighbour (sweep offsets sy, sz) of the point of step sp
        auto prev = [&](int sp, int e) -> V {
          const int sy = DIR * S::o(e, 1), sz = DIR * S::o(e, 2);
          return prw[((sp + SB * sy + sz) & (kRowRing - 1)) * kRowCols + lane + sy + 1];
        };
        // value of the left column's point kk from the shared value ring
        auto ring = [&](int kk) -> V { return hp[(kk & (kRing - 1)) * (NW * 32) + (J > 0 ? J - 1 : 0)]; };
        const int off1 = step_off(1);
        const long long vbase = (long long)i * g.nz * g.ny + j;  // + row * ny
        int rs = row_of(s_begin) - off1;
        rs = rs < 0 ? rs + g.nz : rs;
        bool aborted = false;
        // bounded poll until ok() holds; false if this CTA gives up
        auto wait_until = [&](auto&& refresh, auto&& ok) -> bool {
          unsigned long long t_start = 0;
          bool gave_up = false;
          for (;;) {
            refresh();
            if (ok()) break;
            if (ld_acq_cta(&sh.abort)) { gave_up = true; break; }
            const unsigned long long now = globaltimer_ns();
            if (t_start == 0) t_start = now;
            else if (now - t_start > P.budget_ns) {
              if (lane == 0) {
                atomicCAS(P.err, 0, DEV_ERR_TIMEOUT);
                st_rel_cta(&sh.abort, 1);
              }
              gave_up = true;
              break;
            }
          }
          // lanes leave the loop together unless one gave up: agree
          return !__any_sync(0xffffffffu, gave_up);
        };

        if (is_main) {
          // ---- main warp: finish point K of step s
          int have_left = (w == 0) ? kDone : INT_MIN;
          int have_right = (w + 1 == NW) ? kDone : INT_MIN;
          int have_h = INT_MIN;
          V carry = V(0);
          for (int s = s_begin; s <= s_end; ++s) {
            rs = radd(rs, off1);
            if (__any_sync(0xffffffffu, have_left < s || have_right < s - LEAD || have_h <= s)) {
              const bool ok = wait_until(
                  [&] {
                    if (have_left < s) have_left = ld_acq_cta(&sh.wdone[p][w - 1]);
                    if (have_right < s - LEAD) have_right = ld_acq_cta(&sh.wdone[p][w + 1]);
                    if (have_h <= s) have_h = ld_acq_cta(&sh.hrdy[p][w]);
                  },
                  [&] { return have_left >= s && have_right >= s - LEAD && have_h > s; });
              if (!ok) {
                aborted = true;
                break;
              }
            }
            const int K = s - SB * J;
            if (colok && K >= 0 && K < g.nz) {
              const V* sl = slots + (s & 1) * (NFLD * 32) + lane;
              V a = sl[F_ACC * 32];
#pragma unroll
              for (int e = 0; e < NS; ++e) {
                if (!is_fin<NS, KIND, DIR, X>(e)) continue;
                V tv;
                if (cls<NS, KIND, DIR>(e) == T_OWN) tv = carry;
                else if (cls<NS, KIND, DIR>(e) == T_Y) tv = ring(K + DIR * S::o(e, 2));
                else tv = prev(s, e);
                a = fma(sg * sl[(F_CF + fin_index<NS, KIND, DIR, X>(e)) * 32], tv, a);
              }
              if (PK == KBF) a = mul_rn(sl[F_S * 32], a);
              V r;
              if (KIND == SW_ILU_L) {
                r = FOLD ? a : sl[F_B * 32] - a;
              } else {
                r = (FOLD ? a : sl[F_B * 32] - a) * sl[F_D * 32];
                if (KIND != SW_ILU_U && relax)
                  r = (KIND == SW_GS_ZERO) ? wv * r : fma(wv, r, mul_rn(V(1) - wv, sl[F_UO * 32]));
              }
              u[vbase + (long long)rs * g.ny] = r;
              hp[(K & (kRing - 1)) * (NW * 32) + J] = r;
              carry = r;
            }
            __syncwarp();
            if (lane == 0) st_rel_cta(&sh.wdone[p][w], s + 1);
          }
          if (lane == 0) st_rel_cta(&sh.wdone[p][w], kDone);
        } else {
          // ---- helper warp: the operands and the early partial sum of step s
          const bool has_prev = DIR > 0 ? i > 0 : i + 1 < g.nx;
          auto load_row = [&](int t, int r, V& v0, V& v1) {
            const long long base = ((long long)(i - DIR) * g.nz + r) * g.ny;
            auto val = [&](int Jc) -> V {
              V v = V(0);
              const int Kc = t - SB * Jc;
              if (has_prev && Jc >= 0 && Jc < g.ny && Kc >= 0 && Kc < g.nz) {
                const V* q = u + base + (DIR > 0 ? Jc : g.ny - 1 - Jc);
                v = (W == 1 || p == 0) ? __ldcg(q) : *q;
              }
              return v;
            };
            v0 = val(32 * w - 1 + lane);
            v1 = lane < 2 ? val(32 * w + 31 + lane) : V(0);
          };
          auto commit_row = [&](int t, V v0, V v1) {
            V* rw = prw + (t & (kRowRing - 1)) * kRowCols;
            rw[lane] = v0;
            if (lane < 2) rw[32 + lane] = v1;
          };
          const int br0 = (SB * j) % g.nz;
          auto vslot = [&](int dx, int dy, int kk) -> long long {
            int r = br0 + SB * dy + kk;
            r = r >= g.nz ? r - g.nz : r;
            r = r >= g.nz ? r - g.nz : r;
            r = r < 0 ? r + g.nz : r;
            return ((long long)(i + dx) * g.nz + r) * g.ny + (j + dy);
          };
          // old value of neighbour e of the point at grid index kk (Gauss-Seidel
          // upper terms); off the grid the coefficient is zero and the point's
          // own right-hand side is read instead
          auto nb = [&](int e, int kk) -> V {
            const int ox = S::o(e, 0), oy = S::o(e, 1), oz = S::o(e, 2);
            const bool in = (unsigned)(i + ox) < (unsigned)g.nx && (unsigned)(j + oy) < (unsigned)g.ny &&
                            (unsigned)(kk + oz) < (unsigned)g.nz;
            return *(in ? u + vslot(ox, oy, kk + oz) : b + vslot(0, 0, kk));
          };
          int have_left = (w == 0) ? kDone : INT_MIN;
          int have_own = INT_MIN;
          int have_up = INT_MIN;
          V pend0 = V(0), pend1 = V(0);
          // operands of the point of step s, loaded at iteration s - 1
          uint4 q2[R::CHUNKS];
          V x2[NS];
          V b2 = V(0), uo2 = V(0);
#pragma unroll
          for (int cc = 0; cc < R::CHUNKS; ++cc) q2[cc] = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
          for (int e = 0; e < NS; ++e) x2[e] = V(0);
          auto coef2 = [&](int e) -> Val { return rec_val<Val>(q2, R::slot(e)); };
          const int offpf = step_off(1 + kPrefetch), offrow = step_off(SA - 1 + X);
          const long long rbase = (long long)i * g.nz * R::CHUNKS * g.ny + j;
          for (int s = s_begin; s <= s_end; ++s) {
            rs = radd(rs, off1);
            // the previous plane SA + X steps ahead (its rows up to s+SA-1+X);
            // the own and left main warps past step s - 2 (the left-column
            // values of the partial sum, and the slot about to be refilled)
            const int need = (p == 0) ? gt0 + s + X : s + SA + X;
            if (__any_sync(0xffffffffu, have_up < need || have_own < s - 1 || have_left < s - 1)) {
              const bool ok = wait_until(
                  [&] {
                    if (have_own < s - 1) have_own = ld_acq_cta(&sh.wdone[p][w]);
                    if (have_left < s - 1) have_left = ld_acq_cta(&sh.wdone[p][w - 1]);
                    if (have_up < need) {
                      const int* src = (p == 0) ? sh.avail : sh.wdone[p - 1];
                      int T = kDone;
                      for (int ww = max(w - 1, 0); ww <= min(w + 1, NW - 1); ++ww) T = min(T, ld_acq_cta(&src[ww]));
                      have_up = T;
                    }
                  },
                  [&] { return have_up >= need && have_own >= s - 1 && have_left >= s - 1; });
              if (!ok) {
                aborted = true;
                break;
              }
            }
            // rows s-SB-1 .. s+SA-2+X in the ring before the partial sum; row
            // s+SA-1 (read by the main warp's finish of step s) committed
            // before the hand-over.  X = 0 loads it here; X = 1 loaded it
            // after the previous hand-over (the first iteration prefills it),
            // so the release below never waits for a load in flight.
            if (s == s_begin) {
              for (int t = s - SB - 1; t <= s + SA - 2 + X; ++t) {
                V v0, v1;
                load_row(t, row_of(t), v0, v1);
                commit_row(t, v0, v1);
              }
            } else if (X == 1) {
              commit_row(s + SA - 1, pend0, pend1);
            }
            if (X == 0) load_row(s + SA - 1, radd(rs, offrow), pend0, pend1);
            __syncwarp();
            const int K = s - SB * J;
            if (colok && K >= 0 && K < g.nz) {
              V a = FOLD ? b2 : V(0);
#pragma unroll
              for (int e = 0; e < NS; ++e) {
                if (use<NS, KIND, DIR, X>(e) != U_PRE) continue;
                V tv;
                if (cls<NS, KIND, DIR>(e) == T_Y) tv = ring(K + DIR * S::o(e, 2));
                else if (cls<NS, KIND, DIR>(e) == T_X) tv = prev(s, e);
                else tv = x2[e];
                a = fma(sg * (V)to_c(coef2(e)), tv, a);
              }
              V* sl = slots + (s & 1) * (NFLD * 32) + lane;
              sl[F_ACC * 32] = a;
              sl[F_B * 32] = b2;
              if constexpr (R::HAS_D) sl[F_D * 32] = rec_vec<V>(q2, R::D_OFF);
              if constexpr (R::HAS_S) sl[F_S * 32] = (V)__uint_as_float(rec_word(q2, R::S_OFF / 4));
              sl[F_UO * 32] = uo2;
#pragma unroll
              for (int e = 0; e < NS; ++e)
                if (is_fin<NS, KIND, DIR, X>(e)) sl[(F_CF + fin_index<NS, KIND, DIR, X>(e)) * 32] = (V)to_c(coef2(e));
            }
            if (X == 0) commit_row(s + SA - 1, pend0, pend1);
            __syncwarp();
            if (lane == 0) st_rel_cta(&sh.hrdy[p][w], s + 1);

            // X = 1: row s+SA, committed at the start of the next iteration
            // (the wait above covered it)
            if (X == 1) load_row(s + SA, radd(rs, offrow), pend0, pend1);

            // operands of the point of step s + 1
            const int K1 = K + 1;
            if (colok && K1 >= 0 && K1 < g.nz) {
              const int k1 = DIR > 0 ? K1 : g.nz - 1 - K1;
              const int r1 = radd(rs, off1);
              const long long p1 = vbase + (long long)r1 * g.ny;
              const uint4* rp = (const uint4*)P.M + rbase + (long long)r1 * (R::CHUNKS * g.ny);
#pragma unroll
              for (int cc = 0; cc < R::CHUNKS; ++cc) q2[cc] = __ldg(rp + (long long)cc * g.ny);
              if (K1 + kPrefetch < g.nz) {
                const uint4* pf = (const uint4*)P.M + rbase + (long long)radd(rs, offpf) * (R::CHUNKS * g.ny);
#pragma unroll
                for (int cc = 0; cc < R::CHUNKS; ++cc) prefetch_l2(pf + (long long)cc * g.ny);
              }
#pragma unroll
              for (int e = 0; e < NS; ++e)
                if (use<NS, KIND, DIR, X>(e) == U_PRE && cls<NS, KIND, DIR>(e) == T_OLD) x2[e] = nb(e, k1);
              b2 = b[p1];
              if (KIND == SW_GS_FULL && relax) uo2 = u[p1];
            }
          }
          if (lane == 0) st_rel_cta(&sh.hrdy[p][w], kDone);
        }
        (void)aborted;
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

// Whether the two-warp kernel takes a sweep: 19 / 27-point masks (the 7-point
// mask has no early terms to hand over), at most kHelperMaxStrips strips per
// CTA except for the FP64 Gauss-Seidel sweep with old values (it would
// spill), or, for the FP64 ILU(0) solves, one plane of at most
// kHelperWideStrips strips.  The caller checks that records and vectors are
// in the skewed layout.
inline bool helper_applies(int pk, int ns, int nx, int ny, int W, int kind) {
  const int NW = (ny + 31) / 32;
  const bool fits = (W * NW <= kHelperMaxStrips && !(pk == K64 && kind == SW_GS_FULL)) ||
                    (pk == K64 && W == 1 && NW <= kHelperWideStrips && (kind == SW_ILU_L || kind == SW_ILU_U));
  return (ns == 19 || ns == 27) && fits && (size_t)((nx + W - 1) / W) * NW <= (size_t)kProgSlots;
}

template <int PK, int NS, int W, int X>
cudaError_t launch_kind_h(int kind, int dir, const Sweep3Params& P, cudaStream_t st) {
  using V = typename Prec<PK>::vec;
  const int NW = (P.g.ny + 31) / 32;
  if (!helper_applies(PK, NS, P.g.nx, P.g.ny, W, kind)) return cudaErrorNotSupported;
  const int nthr = (2 * W * NW + 2) * 32;
  const bool wide = W * NW > kHelperMaxStrips;  // the 832-thread instantiation
  int dev = 0, nsm = 0;
  cudaError_t ae = cudaGetDevice(&dev);
  if (ae == cudaSuccess) ae = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (ae != cudaSuccess) return ae;
  const int grid = std::min((P.g.nx + W - 1) / W, nsm);
  auto go = [&](auto kern, size_t need) {
    // reserving more than half of the SM's shared memory keeps a second CTA off the SM
    const size_t smem = std::max(need, kOneCtaPerSmSmem);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, nthr, smem, st>>>(P);
    return cudaGetLastError();
  };
  if (wide) {
    if constexpr (W == 1 && PK == K64) {
      constexpr int T = kHelperWideThreads;
      if (kind == SW_ILU_L)
        return go(k_sweep3h<PK, NS, SW_ILU_L, 1, 1, X, T>, helper_smem_bytes<V, NS, SW_ILU_L, 1, X>(NW, 1));
      if (kind == SW_ILU_U)
        return go(k_sweep3h<PK, NS, SW_ILU_U, -1, 1, X, T>, helper_smem_bytes<V, NS, SW_ILU_U, -1, X>(NW, 1));
    }
    return cudaErrorNotSupported;
  }
  constexpr int T = kHelperThreads;
  if (kind == SW_GS_ZERO)
    return go(k_sweep3h<PK, NS, SW_GS_ZERO, 1, W, X, T>, helper_smem_bytes<V, NS, SW_GS_ZERO, 1, X>(NW, W));
  if (kind == SW_GS_FULL) {
    // FP64 with every old-value term in flight needs more registers than
    // 576 threads leave (it would spill): the one-warp kernel runs it
    if constexpr (PK == K64) {
      return cudaErrorNotSupported;
    } else {
      if (dir > 0)
        return go(k_sweep3h<PK, NS, SW_GS_FULL, 1, W, X, T>, helper_smem_bytes<V, NS, SW_GS_FULL, 1, X>(NW, W));
      return go(k_sweep3h<PK, NS, SW_GS_FULL, -1, W, X, T>, helper_smem_bytes<V, NS, SW_GS_FULL, -1, X>(NW, W));
    }
  }
  if (kind == SW_ILU_L)
    return go(k_sweep3h<PK, NS, SW_ILU_L, 1, W, X, T>, helper_smem_bytes<V, NS, SW_ILU_L, 1, X>(NW, W));
  return go(k_sweep3h<PK, NS, SW_ILU_U, -1, W, X, T>, helper_smem_bytes<V, NS, SW_ILU_U, -1, X>(NW, W));
}

}  // namespace sweep3

// One entry per working precision, each compiled in its own translation unit.
cudaError_t sweep3h_launch_k64(int ns, int W, int kind, int dir, const sweep3::Sweep3Params& P, cudaStream_t st);
cudaError_t sweep3h_launch_k32(int ns, int W, int kind, int dir, const sweep3::Sweep3Params& P, cudaStream_t st);
cudaError_t sweep3h_launch_kbf(int ns, int W, int kind, int dir, const sweep3::Sweep3Params& P, cudaStream_t st);
