// Kernel template of the warp-pipelined wavefront sweeps, included by one
// translation unit per working precision (k_sweep3*.cu).
#pragma once
// Warp-pipelined wavefront sweeps (exact lexicographic order) for the
// 7/19/27-point masks with one unknown per point: Gauss-Seidel (zero-guess
// and full, both directions) and the two ILU(0) triangular solves (Sec. 4.4).
//
// Schedule: point (i,j,k) runs at global time t = SA*i + SB*j + k (the
// smallest skews that put every lower neighbour strictly earlier).
//  * A CTA owns W consecutive x-planes (handed out by an atomic ticket, so a
//    CTA only ever waits on planes that running CTAs own).  Each plane is cut
//    into warps of 32 y-columns, one lane per column, and every warp runs its
//    own loop over local steps s = t - SA*plane; lane J treats point
//    K = s - SB*J of its column at step s.
//  * A neighbour of the lower triangle is older than its point by a fixed
//    number of steps, its slack (SA*dx' + SB*dy' + dz' in sweep coordinates).
//    With a lookahead of X steps a warp of the next plane needs the previous
//    plane to be SA + X steps ahead.  X = 0 for FP64, whose long FMA issue
//    time covers one load issued and consumed in the same step; X = 1 for
//    FP32 / BF16.
//  * Skewed layout (records and vectors, ilurec.cuh): what one plane
//    finishes at its local step t is one row of the vector (row t mod nz),
//    contiguous over j.  Each compute warp keeps the previous plane's last
//    kRowRing rows over its 32 columns and one on either side in shared
//    memory: a step issues one coalesced row load (row s + SA - 1 + X) and
//    commits it before the finish (X = 0) or a step later (X = 1), and every
//    previous-plane term is a shared-memory read at a constant offset.
//  * Natural layout (the context-free entry point): previous-plane values
//    are loaded one by one, as late as their slack allows: a term of slack
//    sigma is loaded min(2, sigma+X-1) steps before its point is finished.
//  * Inside a step: wait for the three counters it depends on (left warp,
//    right warp for the shared value ring, previous plane), issue the loads
//    whose slack is one step, pre-sum point K+1 (every term that is already
//    final), finish point K (own column, left column, the late
//    previous-plane terms), store it, publish the step, then load the
//    operands of K+1 and K+2.  The pre-sum of K+1 runs while the in-step
//    loads are in flight.
//  * Counters are per warp in shared memory (CTA-scope acquire/release); one
//    publisher warp copies the last plane's counters to global memory
//    (GPU-scope release) and one poller warp copies the previous CTA's into
//    shared memory (GPU-scope acquire), so compute warps never execute a
//    GPU-scope fence.  One CTA per SM (the launch reserves more than half of
//    the shared memory) and the grid is capped at the SM count.
//  * The ILU solves read split, 16-byte-aligned records (ilurec.cuh): a lower
//    solve streams only L, an upper solve only U and 1/u_pp.
// Every wait is bounded; on expiry the error word is set and all CTAs drain.
#include <algorithm>
#include <climits>

#include "ilurec.cuh"
#include "shapes.cuh"
#include "smg_internal.cuh"

namespace sweep3 {

// Term classes, relative to the sweep direction.
enum { T_SKIP = 0, T_OWN = 1, T_Y = 2, T_X = 3, T_OLD = 4 };

template <int NS, int KIND, int DIR>
__host__ __device__ constexpr int cls(int e) {
  using S = Shape<NS>;
  const int sx = DIR * S::o(e, 0), sy = DIR * S::o(e, 1), sz = DIR * S::o(e, 2);
  if (e == S::EC) return T_SKIP;
  const bool is_new = sx < 0 || (sx == 0 && (sy < 0 || (sy == 0 && sz < 0)));
  if (!is_new) return KIND == SW_GS_FULL ? T_OLD : T_SKIP;
  if (sx == 0 && sy == 0) return T_OWN;  // (0, 0, -1)
  if (sx == 0) return T_Y;               // (0, -1, *): the left column
  return T_X;                            // (-1, *, *): the previous plane
}

// Steps between a new neighbour and its point.
template <int NS, int DIR>
__host__ __device__ constexpr int slack(int e) {
  using S = Shape<NS>;
  return -(S::SA * DIR * S::o(e, 0) + S::SB * DIR * S::o(e, 1) + DIR * S::o(e, 2));
}

// When an operand is consumed: in the pre-sum of K+1 (loaded two steps
// ahead), or in the finish of K (loaded one step ahead, or in the step).
enum { U_NONE = 0, U_PRE = 1, U_FIN1 = 2, U_FIN0 = 3, U_FINR = 4 };

template <int NS, int KIND, int DIR, int X>
__host__ __device__ constexpr int use(int e) {
  const int c = cls<NS, KIND, DIR>(e);
  if (c == T_SKIP) return U_NONE;
  if (c == T_OLD) return U_PRE;
  if (c == T_OWN) return U_FINR;
  const int sg = slack<NS, DIR>(e);
  if (c == T_Y) return sg >= 2 ? U_PRE : U_FINR;  // left column, from the shared ring
  const int m = sg + X - 1 < 2 ? sg + X - 1 : 2;  // previous plane
  return m == 2 ? U_PRE : (m == 1 ? U_FIN1 : U_FIN0);
}

struct Sweep3Params {
  Grid g;
  unsigned long long budget_ns;
  const void* M;       // GS: matrix [n][NS]; ILU: split records (REC) or the factors [n][NS]
  const float* scale;  // KBF row scale of M (GS and unsplit ILU)
  const void* dinv;    // GS: inverse diagonal; ILU_U: 1/u_pp where the record has none
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
constexpr unsigned kPublishGapNs = 100;
// Shared ring of the last kRing values of every column.  A column's value
// at point k is overwritten by point k + kRing.  A warp publishes step s
// once point k is stored, before it reads the ring for point k+1, so its
// left-hand neighbour may run at most kRing - SB - 2 steps ahead of the
// published step without overwriting a value still to be read.
constexpr int kRing = 16;
// Skewed layout: ring of the previous plane's last kRowRing rows (one row per
// step of that plane), 34 columns (the warp's 32 and one on either side) per
// compute warp.  A step reads rows s-SB-1 .. s+SA-1 and loads row s+SA-1+X.
constexpr int kRowRing = 8;
constexpr int kRowCols = 34;

__device__ __forceinline__ int ld_acq_cta(const int* p) {
  int v;
  asm volatile("ld.acquire.cta.shared.s32 %0, [%1];" : "=r"(v) : "r"((unsigned)__cvta_generic_to_shared(p)) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel_cta(int* p, int v) {
  asm volatile("st.release.cta.shared.s32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "r"(v) : "memory");
}
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// 32-bit word wi of a record held in registers (wi a compile-time constant
// after unrolling, so this is a register selection), and value `slot`.
// Products that must not be contracted into a following add: the point
// update rounds them on their own, the same in every sweep kernel.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

template <int CH>
__device__ __forceinline__ unsigned rec_word(const uint4 (&q)[CH], int wi) {
  const uint4 v = q[wi >> 2];
  const int c = wi & 3;
  return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}
template <typename Val, int CH>
__device__ __forceinline__ Val rec_val(const uint4 (&q)[CH], int slot) {
  if constexpr (sizeof(Val) == 8) {
    return __hiloint2double((int)rec_word(q, 2 * slot + 1), (int)rec_word(q, 2 * slot));
  } else if constexpr (sizeof(Val) == 4) {
    return __uint_as_float(rec_word(q, slot));
  } else {
    const unsigned wd = rec_word(q, slot >> 1);
    return __ushort_as_bfloat16((unsigned short)((slot & 1) ? (wd >> 16) : (wd & 0xffffu)));
  }
}

// A vector-type value (double or float) at byte offset OFF of a record.
template <typename Vv, int CH>
__device__ __forceinline__ Vv rec_vec(const uint4 (&q)[CH], int off) {
  if constexpr (sizeof(Vv) == 8) return __hiloint2double((int)rec_word(q, off / 4 + 1), (int)rec_word(q, off / 4));
  else return __uint_as_float(rec_word(q, off / 4));
}

template <int W>
struct Shared3 {
  int wdone[W][kMaxWarpsPerPlane];  // per compute warp: all local steps < value are finished
  int avail[kMaxWarpsPerPlane];     // previous CTA's last plane, per warp: global time finished
  int abort;
  int group;
};

// Publisher warp: lane w publishes the progress of warp w of the CTA's last
// plane (wd: that plane's counters, local steps) as global time gt0 + T with
// a GPU-scope release store whenever it grows.
template <class SH>
__device__ __forceinline__ void publisher_warp(SH& sh, const int* wd, const Sweep3Params& P, int I, int NW, int gt0,
                                               int lane) {
  const bool mine = lane < NW;
  int* out_slot = P.ws->prog + (size_t)I * NW + lane;
  int published = INT_MIN;
  for (;;) {
    const int T = mine ? ld_acq_cta(&wd[lane]) : kDone;
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
}

// Poller warp: lane w forwards the progress of warp w of the previous CTA's
// last plane into sh.avail (GPU-scope acquire loads).  Bounded: the previous
// CTA must make progress within the budget, else the error word and the
// CTA's abort flag are set.
template <class SH>
__device__ __forceinline__ void poller_warp(SH& sh, const Sweep3Params& P, int I, int NW, int lane) {
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
}

// FP64 sweeps hold their operands in register pairs: they get at most 12
// compute warps (ny <= 384) and the registers that leaves, 8 (ny <= 256)
// when they use every stencil entry; FP32 / BF16 sweeps up to 16.
template <int PK, int KIND>
__host__ __device__ constexpr int max_threads() {
  return PK == K64 ? (KIND == SW_GS_FULL ? 320 : 448) : kMaxThreads;
}

template <int PK, int NS, int KIND, int DIR, int W, int X, int REC>
__global__ void __launch_bounds__(max_threads<PK, KIND>(), 1) k_sweep3(Sweep3Params P) {
  using V = typename Prec<PK>::vec;
  using Val = typename Prec<PK>::val;
  using S = Shape<NS>;
  constexpr int SA = S::SA, SB = S::SB, EC = S::EC;
  // REC: records and vectors in the skewed layout (ilurec.cuh); otherwise
  // the matrix [n][NS] and vectors in natural order
  constexpr bool SPLIT = REC;
  using R = SweepRec<PK, NS, KIND == SW_ILU_L ? 0 : (KIND == SW_ILU_U ? 1 : 2)>;
  // FOLD (FP64 / FP32): the sum of a point starts from b and subtracts its
  // terms.  BF16 keeps b apart (the row scale multiplies the sum only).
  constexpr bool FOLD = PK != KBF;
  constexpr V sg = FOLD ? V(-1) : V(1);
  constexpr bool NEED_D = KIND != SW_ILU_L;
  extern __shared__ unsigned char dyn_smem[];
  __shared__ Shared3<W> sh;

  const Grid g = P.g;
  const int NW = (g.ny + 31) >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ncompute = W * NW;  // warps ncompute and ncompute + 1 talk to the other CTAs
  constexpr int LEAD = kRing - SB - 2;  // largest lead over the right-hand warp
  // shared value ring: hist[plane][k % kRing][column]
  V* hist = (V*)dyn_smem;
  V* prow_all = hist + (size_t)W * kRing * NW * 32;
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
      // a warp has trivially finished every step before its first one
      sh.wdone[p][w] = (p < nplanes && w < NW) ? SB * 32 * w - 2 : kDone;
    }
    // nothing precedes the first plane; 0 is below every time a later plane asks for
    if (threadIdx.x < kMaxWarpsPerPlane) sh.avail[threadIdx.x] = (I == 0) ? kDone : 0;
    __syncthreads();

    if (warp == ncompute) {
      publisher_warp(sh, sh.wdone[nplanes - 1], P, I, NW, SA * (I * W + nplanes - 1), lane);
    } else if (warp == ncompute + 1) {
      poller_warp(sh, P, I, NW, lane);
    } else if (warp < W * NW) {
      // ---- compute warp (p, w)
      const int p = warp / NW, w = warp % NW;
      if (p < nplanes) {
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
        // the previous schedule plane (skewed layout): it writes one row per
        // step, the row of its local step t being t mod nz (forward) or
        // (nz - 1 + SB (ny - 1) - t) mod nz (backward), the same for all its
        // columns
        V* prw = prow_all + (size_t)(p * NW + w) * (kRowRing * kRowCols);
        const bool has_prev = DIR > 0 ? i > 0 : i + 1 < g.nx;
        const int rback = (g.nz - 1 + SB * (g.ny - 1)) % g.nz;
        V pend0 = V(0), pend1 = V(0);  // the row loaded one step ago, not yet in the ring
        // lane's value of producer step t in ring order: its column 32w-1+lane,
        // and columns 32w+31, 32w+32 for lanes 0, 1 (zero off the grid, where
        // the coefficient is zero too)
        auto row_of = [&](int t) -> int {
          const int r = (DIR > 0 ? t : rback - t) % g.nz;
          return r < 0 ? r + g.nz : r;
        };
        // row_of(t + d) = row_of(t) + step_off(d), reduced once below nz
        auto step_off = [&](int d) -> int {
          const int r = (DIR * d) % g.nz;
          return r < 0 ? r + g.nz : r;
        };
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
        // previous-plane neighbour (sweep offsets sy, sz) of the point of step sp
        auto prev = [&](int sp, int e) -> V {
          const int sy = DIR * S::o(e, 1), sz = DIR * S::o(e, 2);
          return prw[((sp + SB * sy + sz) & (kRowRing - 1)) * kRowCols + lane + sy + 1];
        };
        int have_left = (w == 0) ? kDone : INT_MIN;        // cached progress of the left warp
        int have_right = (w + 1 == NW) ? kDone : INT_MIN;  // cached progress of the right warp
        int have_up = INT_MIN;                             // cached progress of the previous plane
        // vector index of (i + dx, j + dy, kk): natural order, or the skewed
        // layout (row (kk + SB*(j + dy)) mod nz, from the lane's row base)
        const int br0 = SPLIT ? (SB * j) % g.nz : 0;
        auto vslot = [&](int dx, int dy, int kk) -> long long {
          if constexpr (SPLIT) {
            int r = br0 + SB * dy + kk;
            r = r >= g.nz ? r - g.nz : r;
            r = r >= g.nz ? r - g.nz : r;
            r = r < 0 ? r + g.nz : r;
            return ((long long)(i + dx) * g.nz + r) * g.ny + (j + dy);
          } else {
            return ((long long)(i + dx) * g.ny + (j + dy)) * g.nz + kk;
          }
        };

        // stage 2: operands of point K+2, loaded at step s, pre-summed at s+1.
        // A split record stays as loaded (q2) and is unpacked where it is
        // used, so no instruction waits on a load in the step that issues it.
        Val c2[NS];
        uint4 q2[SPLIT ? R::CHUNKS : 1];
        V x2[NS];
        V b2 = V(0), d2 = V(0), uo2 = V(0);
        float s2 = 1.0f;
        // finish operands of point K (pre-summed at s-1) and of point K+1
        Val cfK[NS], cfN[NS];
        V accK = V(0), bK = V(0), dK = V(0), uoK = V(0);
        float sK = 1.0f;
        V x1[NS];  // previous-plane terms of point K loaded one step ahead
        V carry = V(0);
#pragma unroll
        for (int e = 0; e < NS; ++e) {
          c2[e] = Val(0);
          cfK[e] = cfN[e] = Val(0);
          x2[e] = x1[e] = V(0);
        }
#pragma unroll
        for (int c = 0; c < (SPLIT ? R::CHUNKS : 1); ++c) q2[c] = make_uint4(0u, 0u, 0u, 0u);
        // coefficient e of the stage-2 point (unpacked at use)
        auto coef2 = [&](int e) -> Val {
          if constexpr (SPLIT) return rec_val<Val>(q2, R::slot(e));
          else return c2[e];
        };

        // value of neighbour e of sweep point KK (grid index k of KK given).
        // The load is issued unconditionally: a neighbour off the grid has a
        // coefficient of exactly zero (zero padding), so it reads the point's
        // own right-hand side instead (finite, in bounds) and the term adds
        // zero -- no select has to wait for the load.
        auto nb = [&](int e, int kk) -> V {
          const int ox = S::o(e, 0), oy = S::o(e, 1), oz = S::o(e, 2);
          const bool in = (unsigned)(i + ox) < (unsigned)g.nx && (unsigned)(j + oy) < (unsigned)g.ny &&
                          (unsigned)(kk + oz) < (unsigned)g.nz;
          const V* q = in ? u + vslot(ox, oy, kk + oz) : b + vslot(0, 0, kk);
          // the previous schedule plane of another CTA: read through L2;
          // everything else (this CTA's planes, old values) through L1 (the
          // choice is uniform per warp, and known at compile time for W == 1)
          return (DIR * ox < 0 && (W == 1 || p == 0)) ? __ldcg(q) : *q;
        };
        // value of the left column's point kk from the shared ring; the ring
        // starts zeroed, so a slot read off the grid (coefficient zero) is finite
        auto ring = [&](int kk) -> V { return hp[(kk & (kRing - 1)) * (NW * 32) + (J > 0 ? J - 1 : 0)]; };

        // skewed layout: every vector and record access of step s is in row
        // rs = row_of(s) (point K), rs + off2 (point K+2), rs + offpf (the
        // prefetch) or rs + offrow (the previous plane's row), the same for
        // all lanes; rs advances by one row per step
        const int off1 = SPLIT ? step_off(1) : 0, off2 = SPLIT ? step_off(2) : 0;
        const int offpf = SPLIT ? step_off(2 + kPrefetch) : 0, offrow = SPLIT ? step_off(SA - 1 + X) : 0;
        const long long vbase = (long long)i * g.nz * g.ny + j;                // + row * ny
        const long long rbase = (long long)i * g.nz * R::CHUNKS * g.ny + j;    // + row * CHUNKS * ny
        int rs = 0;
        if constexpr (SPLIT) {
          rs = row_of(s_begin) - off1;
          rs = rs < 0 ? rs + g.nz : rs;
        }
        auto radd = [&](int r, int off) -> int {
          r += off;
          return r >= g.nz ? r - g.nz : r;
        };
        bool aborted = false;
        for (int s = s_begin; s <= s_end; ++s) {
          if constexpr (SPLIT) rs = radd(rs, off1);
          // -- dependencies, against counters cached in registers.  Every
          // lane checks them (the same values in all lanes, so the warp does
          // not diverge); only when the cache is stale do the lanes poll the
          // shared counters, each with its own acquire load (one broadcast).
          {
            // the previous plane's points this warp reads lie in columns
            // 32w-1 .. 32w+32: warps w-1..w+1, SA + X steps ahead
            const int need = (p == 0) ? gt0 + s + X : s + SA + X;
            // the caches agree across lanes in practice; the vote makes the
            // entry (and the barrier-like votes below) uniform regardless
            if (__any_sync(0xffffffffu, have_left < s || have_right < s - LEAD || have_up < need)) {
              unsigned long long t_start = 0;
              for (;;) {
                if (have_left < s) have_left = ld_acq_cta(&sh.wdone[p][w - 1]);
                if (have_right < s - LEAD) have_right = ld_acq_cta(&sh.wdone[p][w + 1]);
                if (have_up < need) {
                  const int* src = (p == 0) ? sh.avail : sh.wdone[p - 1];
                  int T = kDone;
                  for (int ww = max(w - 1, 0); ww <= min(w + 1, NW - 1); ++ww) T = min(T, ld_acq_cta(&src[ww]));
                  have_up = T;
                }
                if (have_left >= s && have_right >= s - LEAD && have_up >= need) break;
                if (ld_acq_cta(&sh.abort)) { aborted = true; break; }
                const unsigned long long now = globaltimer_ns();
                if (t_start == 0) t_start = now;
                else if (now - t_start > P.budget_ns) {
                  if (lane == 0) {
                    atomicCAS(P.err, 0, DEV_ERR_TIMEOUT);
                    st_rel_cta(&sh.abort, 1);
                  }
                  aborted = true;
                  break;
                }
              }
              // lanes leave the loop together unless one gave up: agree
              aborted = __any_sync(0xffffffffu, aborted);
              if (aborted) break;
            }
          }
          if constexpr (SPLIT) {
            // rows s-SB-1 .. s+SA-2+X must be in the ring now: the first step
            // of the plane loads them, later steps (X = 1) commit the row
            // loaded one step ago.  Row s+SA-1+X is loaded here; with X = 0
            // it is committed before the finish of K, which reads it.
            if (s == s_begin) {
              for (int t = s - SB - 1; t <= s + SA - 2 + X; ++t) {
                V v0, v1;
                load_row(t, row_of(t), v0, v1);
                commit_row(t, v0, v1);
              }
            } else if (X == 1) {
              commit_row(s + SA - 1, pend0, pend1);
            }
            load_row(s + SA - 1 + X, radd(rs, offrow), pend0, pend1);
            __syncwarp();
          }
          const int K = s - SB * J;
          const bool okK = colok && K >= 0 && K < g.nz;
          const bool okK1 = colok && K + 1 >= 0 && K + 1 < g.nz;
          const int kK = DIR > 0 ? K : g.nz - 1 - K;

          // (a) previous-plane terms of K whose slack is one step: loaded now
          V x0[NS];
#pragma unroll
          for (int e = 0; e < NS; ++e) {
            x0[e] = V(0);
            if (!SPLIT && use<NS, KIND, DIR, X>(e) == U_FIN0 && okK) x0[e] = nb(e, kK);
          }

          // (b) pre-sum of point K+1: every term that is final by now
          V accN = V(0), bN = V(0), dN = V(0), uoN = V(0);
          float sN = 1.0f;
          if (okK1) {
            V a = FOLD ? b2 : V(0);
#pragma unroll
            for (int e = 0; e < NS; ++e) {
              if (use<NS, KIND, DIR, X>(e) != U_PRE) continue;
              V tv;
              if (cls<NS, KIND, DIR>(e) == T_Y) {
                tv = ring(K + 1 + DIR * S::o(e, 2));  // sweep index of the left column's point
              } else if (SPLIT && cls<NS, KIND, DIR>(e) == T_X) {
                tv = prev(s + 1, e);
              } else {
                tv = x2[e];
              }
              a = fma(sg * (V)to_c(coef2(e)), tv, a);
            }
            accN = a;
            bN = b2;
            if constexpr (SPLIT && R::HAS_D) dN = rec_vec<V>(q2, R::D_OFF);
            else dN = d2;
            if constexpr (SPLIT && R::HAS_S) sN = __uint_as_float(rec_word(q2, R::S_OFF / 4));
            else sN = s2;
            uoN = uo2;
          }
#pragma unroll
          for (int e = 0; e < NS; ++e) {
            const int us = use<NS, KIND, DIR, X>(e);
            if (us == U_FIN0 || us == U_FIN1 || us == U_FINR) cfN[e] = coef2(e);
          }

          if constexpr (SPLIT && X == 0) {
            commit_row(s + SA - 1, pend0, pend1);
            __syncwarp();
          }

          // (c) finish point K
          if (okK) {
            V a = accK;
#pragma unroll
            for (int e = 0; e < NS; ++e) {
              const int us = use<NS, KIND, DIR, X>(e);
              if (us != U_FIN0 && us != U_FIN1 && us != U_FINR) continue;
              V tv;
              if (cls<NS, KIND, DIR>(e) == T_OWN) {
                tv = carry;
              } else if (cls<NS, KIND, DIR>(e) == T_Y) {
                tv = ring(K + DIR * S::o(e, 2));
              } else if (SPLIT) {
                tv = prev(s, e);
              } else {
                tv = us == U_FIN0 ? x0[e] : x1[e];
              }
              a = fma(sg * (V)to_c(cfK[e]), tv, a);
            }
            if (PK == KBF) a = mul_rn((V)sK, a);
            V r;
            if (KIND == SW_ILU_L) {
              r = FOLD ? a : bK - a;
            } else {
              r = (FOLD ? a : bK - a) * dK;
              if (KIND != SW_ILU_U && relax) r = (KIND == SW_GS_ZERO) ? wv * r : fma(wv, r, mul_rn(V(1) - wv, uoK));
            }
            u[SPLIT ? vbase + (long long)rs * g.ny : vslot(0, 0, kK)] = r;
            hp[(K & (kRing - 1)) * (NW * 32) + J] = r;
            carry = r;
          }
          // -- point K is stored: publish step s before the loads below are
          // issued, so the release does not wait for them
          __syncwarp();
          if (lane == 0) st_rel_cta(&sh.wdone[p][w], s + 1);
          accK = accN;
          bK = bN;
          dK = dN;
          sK = sN;
          uoK = uoN;
#pragma unroll
          for (int e = 0; e < NS; ++e) cfK[e] = cfN[e];

          // (d) previous-plane terms of K+1 whose slack allows one step
          if (okK1) {
            const int k1 = DIR > 0 ? K + 1 : g.nz - 2 - K;
#pragma unroll
            for (int e = 0; e < NS; ++e)
              if (!SPLIT && use<NS, KIND, DIR, X>(e) == U_FIN1) x1[e] = nb(e, k1);
          }

          // (e) operands of point K+2
          const int K2 = K + 2;
          if (colok && K2 >= 0 && K2 < g.nz) {
            const int k2 = DIR > 0 ? K2 : g.nz - 1 - K2;
            const long long p2 = SPLIT ? vbase + (long long)radd(rs, off2) * g.ny : vslot(0, 0, k2);
            if constexpr (SPLIT) {
              const uint4* rp = (const uint4*)P.M + rbase + (long long)radd(rs, off2) * (R::CHUNKS * g.ny);
#pragma unroll
              for (int c = 0; c < R::CHUNKS; ++c) q2[c] = __ldg(rp + (long long)c * g.ny);
              if (K2 + kPrefetch < g.nz) {
                const uint4* pf = (const uint4*)P.M + rbase + (long long)radd(rs, offpf) * (R::CHUNKS * g.ny);
#pragma unroll
                for (int c = 0; c < R::CHUNKS; ++c) prefetch_l2(pf + (long long)c * g.ny);
              }
            } else {
              const Val* __restrict__ a = (const Val*)P.M + p2 * NS;
#pragma unroll
              for (int e = 0; e < NS; ++e)
                if (use<NS, KIND, DIR, X>(e) != U_NONE) c2[e] = a[e];
              if (NEED_D) d2 = dinv[p2];
              if (PK == KBF) s2 = P.scale[p2];
              if (K2 + kPrefetch < g.nz) {
                constexpr int RB = NS * (int)sizeof(Val);
                const char* pf = (const char*)P.M + (p2 + DIR * kPrefetch) * RB;
                prefetch_l2(pf);
                prefetch_l2(pf + RB - 1);
              }
            }
#pragma unroll
            for (int e = 0; e < NS; ++e)
              if (use<NS, KIND, DIR, X>(e) == U_PRE && cls<NS, KIND, DIR>(e) != T_Y &&
                  !(SPLIT && cls<NS, KIND, DIR>(e) == T_X))
                x2[e] = nb(e, k2);
            b2 = b[p2];
            if (KIND == SW_GS_FULL && relax) uo2 = u[p2];
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

template <int PK, int NS, int W, int X>
cudaError_t launch_kind(int kind, int dir, bool rec, const Sweep3Params& P, cudaStream_t st) {
  using V = typename Prec<PK>::vec;
  const int NW = (P.g.ny + 31) / 32;
  const int nthr = (W * NW + 2) * 32;
  // the value ring needs <= 64 KB (ny <= 512); reserving more than half of
  // the SM's 228 KB keeps a second CTA off the SM
  const size_t smem = std::max(sizeof(V) * ((size_t)kRing * NW * 32 + (size_t)kRowRing * kRowCols * NW) * W,
                               kOneCtaPerSmSmem);
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
  // rec: records and vectors in the skewed layout.  The natural layout (the
  // matrix [n][NS], vectors in natural order) is kept for FP64 only, where
  // the context-free entry point uses it.
  if constexpr (PK == K64) {
    if (!rec) {
      if (kind == SW_GS_ZERO) return go(k_sweep3<PK, NS, SW_GS_ZERO, 1, W, X, 0>);
      if (kind == SW_GS_FULL) {
        if (dir > 0) return go(k_sweep3<PK, NS, SW_GS_FULL, 1, W, X, 0>);
        return go(k_sweep3<PK, NS, SW_GS_FULL, -1, W, X, 0>);
      }
      if (kind == SW_ILU_L) return go(k_sweep3<PK, NS, SW_ILU_L, 1, W, X, 0>);
      return go(k_sweep3<PK, NS, SW_ILU_U, -1, W, X, 0>);
    }
  } else {
    if (!rec) return cudaErrorNotSupported;
  }
  if (kind == SW_GS_ZERO) return go(k_sweep3<PK, NS, SW_GS_ZERO, 1, W, X, 1>);
  if (kind == SW_GS_FULL) {
    if (dir > 0) return go(k_sweep3<PK, NS, SW_GS_FULL, 1, W, X, 1>);
    return go(k_sweep3<PK, NS, SW_GS_FULL, -1, W, X, 1>);
  }
  if (kind == SW_ILU_L) return go(k_sweep3<PK, NS, SW_ILU_L, 1, W, X, 1>);
  return go(k_sweep3<PK, NS, SW_ILU_U, -1, W, X, 1>);
}

}  // namespace sweep3

// One entry per working precision, each compiled in its own translation unit.
cudaError_t sweep3_launch_k64(int ns, int kind, int dir, bool rec, const sweep3::Sweep3Params& P, cudaStream_t st);
cudaError_t sweep3_launch_k32(int ns, int W, int kind, int dir, bool rec, const sweep3::Sweep3Params& P,
                              cudaStream_t st);
cudaError_t sweep3_launch_kbf(int ns, int W, int kind, int dir, bool rec, const sweep3::Sweep3Params& P,
                              cudaStream_t st);
