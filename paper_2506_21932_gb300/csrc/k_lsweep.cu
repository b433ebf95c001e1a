// Line Gauss-Seidel along z (Sec. 4.4, LGS): the points of a z-column (i, j)
// are updated together.  The column's right-hand side is b minus every
// coupling to another column (columns earlier in the sweep already new,
// later ones old, none of the later ones from a zero guess), and the
// tridiagonal system of the offsets (0,0,-1), (0,0,0), (0,0,+1) is solved
// exactly.  Columns run in lexicographic (i, j) order (reversed for the
// backward sweep), scheduled like the point sweeps: one x-plane per CTA at a
// time (atomic ticket), column j of plane i after column j + 1 (or j for a
// 7-point mask) of plane i - 1, progress published by the wavefront engine's
// publisher / poller warps.
//
// A column is solved by four warps, one per SM sub-partition (each of which
// issues about one FP64 warp instruction per 64 cycles on GB300).  The serial
// Thomas recurrence of the paper would put 2 nz dependent FP64 operations on
// the critical path, so the column is cut into 128 chunks of m rows, one per
// thread (partition method): every thread eliminates its rows 2..m in terms
// of its own first unknown P_c and the next chunk's first unknown P_{c+1},
// the 128 chunk-first unknowns form a tridiagonal system solved by parallel
// cyclic reduction through shared memory, and each thread then recovers its
// rows.  Everything that depends only on the matrix (reciprocal pivots,
// elimination multipliers, the reduced system's PCR multipliers) is computed
// once at set-up, so a sweep does no division.  In exact arithmetic the
// result is the Thomas solution; the rounding differs.  All eight compute
// warps assemble the right-hand side and store the column; the next
// column's matrix rows, right-hand side and factors are copied to shared
// memory by bulk copies (one thread, mbarrier completion) while the current
// column is worked on.
#include <cstdint>
#include <utility>

#include "shapes.cuh"
#include "smg_internal.cuh"
#include "wavefront.cuh"

namespace {

constexpr int kLgsWarps = 8;                       // compute warps of a CTA
constexpr int kLgsThreads = (kLgsWarps + 2) * 32;  // + publisher + poller
constexpr int kLgsSolveWarps = 4;                  // warps solving a column (warps 0..3)
constexpr int kLgsChunks = 32 * kLgsSolveWarps;    // chunks of a column, one per solving thread
constexpr int kLgsPcr = 7;                         // PCR steps: log2(kLgsChunks)
constexpr int kLgsMaxM = 8;                        // rows per chunk: nz <= 1024

// Column block of the line factors, in doubles, every field kLgsChunks wide:
// for chunk rows r = 1..m-1 the fields F_W (a_r / den_r), F_INV (1 / den_r),
// F_CP (c_r / den_r), F_G, F_H (x_r = e_r - g_r P_{c+1} - h_r P_c); then per
// chunk C_A0, C_C0 (the couplings of its first row), C_AL + t, C_GA + t (the
// PCR multipliers of step t, stride 2^t) and C_INVB (1 / final pivot).
enum { F_W, F_INV, F_CP, F_G, F_H, F_N };
enum { C_A0 = 0, C_C0 = 1, C_AL = 2, C_GA = 2 + kLgsPcr, C_INVB = 2 + 2 * kLgsPcr, C_N = 3 + 2 * kLgsPcr };
__host__ __device__ inline int lgs_row(int r, int f) { return ((r - 1) * F_N + f) * kLgsChunks; }
__host__ __device__ inline int lgs_chunk(int m, int f) { return ((m - 1) * F_N + f) * kLgsChunks; }

__device__ __forceinline__ void lgs_bar() {
  asm volatile("bar.sync 1, %0;" ::"n"(kLgsWarps * 32) : "memory");
}
// barrier of the solving warps only
__device__ __forceinline__ void lgs_bar_solve() {
  asm volatile("bar.sync 2, %0;" ::"n"(kLgsChunks) : "memory");
}

struct LineIdx {
  int sub, diag, sup;  // stencil entries of (0,0,-1), (0,0,0), (0,0,+1); -1 if absent
};

// Tridiagonal coefficients of row k of column col (identity beyond nz).
__device__ __forceinline__ void line_coef(const Grid& g, int ns, const LineIdx& e, const double* A, long long col,
                                          int k, double& a, double& b, double& c) {
  if (k >= g.nz) {
    a = 0.0;
    b = 1.0;
    c = 0.0;
    return;
  }
  const long long p = col * g.nz + k;
  a = (k > 0 && e.sub >= 0) ? A[p * ns + e.sub] : 0.0;
  b = A[p * ns + e.diag];
  c = (k + 1 < g.nz && e.sup >= 0) ? A[p * ns + e.sup] : 0.0;
}

// The oracle's breakdown rule: every Thomas pivot of every column positive.
__global__ void k_lgs_pivots(Grid g, int ns, LineIdx e, const double* __restrict__ A, int* err) {
  const long long col = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= (long long)g.nx * g.ny) return;
  double cprev = 0.0;
  for (int k = 0; k < g.nz; ++k) {
    double a, b, c;
    line_coef(g, ns, e, A, col, k, a, b, c);
    const double piv = b - a * cprev;
    if (!(piv > 0.0)) {
      atomicCAS(err, 0, SMG_EBREAKDOWN);
      return;
    }
    cprev = c / piv;
  }
}

// One block of kLgsChunks threads per column, thread c = chunk c: the
// partitioned elimination of rows c*m + 1 .. c*m + m-1 and the reduced
// system's PCR multipliers (neighbour values through shared memory).
__global__ void __launch_bounds__(kLgsChunks) k_lgs_factor(Grid g, int ns, LineIdx e, const double* __restrict__ A,
                                                           double* __restrict__ Fo, int m, long long blk, int* err) {
  __shared__ double xa[kLgsChunks], xb[kLgsChunks], xc[kLgsChunks];
  const long long col = blockIdx.x;
  const int c = threadIdx.x;
  double* F = Fo + col * blk;
  double cp[kLgsMaxM], fp[kLgsMaxM];
  bool bad = false;
  for (int r = 1; r < m; ++r) {
    double a, b, cc;
    line_coef(g, ns, e, A, col, c * m + r, a, b, cc);
    const double den = r == 1 ? b : b - a * cp[r - 1];
    bad |= !(den > 0.0);
    const double inv = 1.0 / den;
    cp[r] = cc * inv;
    fp[r] = (r == 1 ? a : -a * fp[r - 1]) * inv;
    F[lgs_row(r, F_W) + c] = a * inv;
    F[lgs_row(r, F_INV) + c] = inv;
    F[lgs_row(r, F_CP) + c] = cp[r];
  }
  double gg = cp[m - 1], hh = fp[m - 1];
  const double glast = gg, hlast = hh;
  F[lgs_row(m - 1, F_G) + c] = gg;
  F[lgs_row(m - 1, F_H) + c] = hh;
  for (int r = m - 2; r >= 1; --r) {
    hh = fp[r] - cp[r] * hh;
    gg = -cp[r] * gg;
    F[lgs_row(r, F_G) + c] = gg;
    F[lgs_row(r, F_H) + c] = hh;
  }
  // reduced row of chunk c in P_{c-1}, P_c, P_{c+1}
  double a0, b0, c0;
  line_coef(g, ns, e, A, col, c * m, a0, b0, c0);
  xa[c] = glast;
  xb[c] = hlast;
  __syncthreads();
  const double gl = c > 0 ? xa[c - 1] : 0.0, hl = c > 0 ? xb[c - 1] : 0.0;
  double Ar = -a0 * hl;
  double Br = b0 - a0 * gl - c0 * hh;  // hh, gg now hold h_1, g_1
  double Cr = -c0 * gg;
  F[lgs_chunk(m, C_A0) + c] = a0;
  F[lgs_chunk(m, C_C0) + c] = c0;
  for (int t = 0; t < kLgsPcr; ++t) {
    const int s = 1 << t;
    __syncthreads();
    xa[c] = Ar;
    xb[c] = Br;
    xc[c] = Cr;
    __syncthreads();
    const bool lo = c >= s, hi = c + s < kLgsChunks;
    const double Am = lo ? xa[c - s] : 0.0, Bm = lo ? xb[c - s] : 1.0, Cm = lo ? xc[c - s] : 0.0;
    const double Ap = hi ? xa[c + s] : 0.0, Bp = hi ? xb[c + s] : 1.0, Cp = hi ? xc[c + s] : 0.0;
    const double al = lo ? -Ar / Bm : 0.0, ga = hi ? -Cr / Bp : 0.0;
    const double nB = Br + al * Cm + ga * Ap;
    Ar = al * Am;
    Cr = ga * Cp;
    Br = nB;
    F[lgs_chunk(m, C_AL + t) + c] = al;
    F[lgs_chunk(m, C_GA + t) + c] = ga;
  }
  bad |= !(Br > 0.0);
  F[lgs_chunk(m, C_INVB) + c] = 1.0 / Br;
  if (bad) atomicCAS(err, 0, SMG_EBREAKDOWN);
}

struct LsParams {
  Grid g;
  WfCtl C;
  Stencil s;
  const double* A;
  const double* F;
  const double* b;
  double* u;
  int m;          // rows per chunk
  long long blk;  // doubles per column block of F
  int dep;        // previous-plane columns a column reads beyond its own (0 or 1)
};

// Bulk (TMA, non-tensor) global -> shared copies completing on an mbarrier:
// one thread issues a column's copies, the transaction count of the barrier
// tracks their bytes.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the given phase of a copy barrier, bounded by budget_ns; false
// (and DEV_ERR_TIMEOUT in *err) when the budget runs out.
// Bound of the waits that drain a plane's bulk copies after an abort.
constexpr unsigned long long kLgsDrainNs = 100ull * 1000 * 1000;

__device__ __noinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity, unsigned long long budget_ns,
                                               int* err) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > budget_ns) {
      atomicCAS(err, 0, DEV_ERR_TIMEOUT);
      return false;
    }
  }
}

// Shared-memory carve-up (doubles): rhs and x of the current column in the
// chunk layout (chunk L, row r at L * (m + 1) + r), two buffers of the
// column factors, and with STAGE two buffers of the column's matrix rows
// [nz][ns] and right-hand side [nz].
__host__ __device__ inline long long lgs_smem_doubles(int m, long long blk, int nz, int ns, bool stage) {
  return 2LL * kLgsChunks * (m + 1) + kLgsChunks + 2 * blk + (stage ? 2LL * ((long long)nz * ns + nz) : 0);
}

// One off-column term of a point's right-hand side for a canonical mask
// (compile-time offsets): acc -= a_E x_{p + o_E}.  The neighbour is read
// unconditionally at a clamped address (its own point when off the grid, the
// term then dropped), so all loads of a point can be issued together.
template <int NS, int KIND, int DIR, int E>
__device__ __forceinline__ void line_term(double (&acc)[4], const double* __restrict__ arow,
                                          const double* __restrict__ up, const double* __restrict__ xs, int kc,
                                          int kr, int m, int mp, const int* lin, unsigned xymask, unsigned zmask) {
  using S = Shape<NS>;
  constexpr int dx = S::o(E, 0), dy = S::o(E, 1), dz = S::o(E, 2);
  constexpr bool in_column = dx == 0 && dy == 0;
  constexpr bool earlier = DIR * dx < 0 || (dx == 0 && DIR * dy < 0);
  if constexpr (!in_column && (KIND != SW_GS_ZERO || earlier)) {
    const bool ok = ((xymask >> ((dx + 1) * 3 + (dy + 1))) & 1u) && ((zmask >> (dz + 1)) & 1u);
    double x;
    if constexpr (dx == 0 && dy == -DIR) {
      // the previous column of the sweep, still in the x buffer (chunk layout)
      int rc = kc, rr = kr + dz;
      if (rr < 0) { rc -= 1; rr += m; }
      if (rr >= m) { rc += 1; rr -= m; }
      x = xs[ok ? rc * mp + rr : kc * mp + kr];
    } else if constexpr (dx != 0) {
      x = __ldcg(up + (ok ? lin[E] : 0));  // other planes: other CTAs' data, through L2
    } else {
      x = up[ok ? lin[E] : 0];
    }
    acc[E & 3] = fma(-arow[E], ok ? x : 0.0, acc[E & 3]);
  }
}

template <int NS, int KIND, int DIR, int... Es>
__device__ __forceinline__ void line_terms(double (&acc)[4], const double* __restrict__ arow,
                                           const double* __restrict__ up, const double* __restrict__ xs, int kc,
                                           int kr, int m, int mp, const int* lin, unsigned xymask, unsigned zmask,
                                           std::integer_sequence<int, Es...>) {
  (line_term<NS, KIND, DIR, Es>(acc, arow, up, xs, kc, kr, m, mp, lin, xymask, zmask), ...);
}

// Forward and backward elimination of rows 1..m-1 of chunk c, the PCR
// solve of the chunk-first unknowns (through xch, kLgsChunks doubles) and
// the recovery of the rows: x (in the chunk layout) from the right-hand side
// d (overwritten).  Called by the kLgsChunks threads of the solving warps.
// (xch is written and read by different threads between barriers, so it
// carries no __restrict__: its loads must not move across the barriers.)
__device__ __forceinline__ void lgs_solve_column(double* __restrict__ d, double* __restrict__ x,
                                                 const double* __restrict__ fc, double* xch, int m, int c) {
  const int mp = m + 1, base = c * mp;
  double v = 0.0;
  for (int r0 = 1; r0 < m; r0 += 4) {
    double dv[4], iv[4], wv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = r0 + q;
      if (r < m) {
        dv[q] = d[base + r];
        iv[q] = fc[lgs_row(r, F_INV) + c];
        wv[q] = fc[lgs_row(r, F_W) + c];
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = r0 + q;
      if (r < m) {
        // dp_r = d_r / den_r - (a_r / den_r) dp_{r-1}  (no dp_0 term in row 1)
        v = r == 1 ? dv[q] * iv[q] : fma(-wv[q], v, dv[q] * iv[q]);
        d[base + r] = v;
      }
    }
  }
  // backward: e_r = dp_r - c'_r e_{r+1}, from e_{m-1} = dp_{m-1} (= v)
  for (int r0 = m - 2; r0 >= 1; r0 -= 4) {
    double dv[4], cv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = r0 - q;
      if (r >= 1) {
        dv[q] = d[base + r];
        cv[q] = fc[lgs_row(r, F_CP) + c];
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = r0 - q;
      if (r >= 1) {
        v = fma(-cv[q], v, dv[q]);
        d[base + r] = v;
      }
    }
  }
  double al[kLgsPcr], ga[kLgsPcr];
#pragma unroll
  for (int t = 0; t < kLgsPcr; ++t) {
    al[t] = fc[lgs_chunk(m, C_AL + t) + c];
    ga[t] = fc[lgs_chunk(m, C_GA + t) + c];
  }
  const double a0 = fc[lgs_chunk(m, C_A0) + c], c0 = fc[lgs_chunk(m, C_C0) + c];
  const double invb = fc[lgs_chunk(m, C_INVB) + c];
  const double e1 = d[base + 1];
  xch[c] = d[base + m - 1];  // e_{m-1}, read by the next chunk
  lgs_bar_solve();
  double D = fma(-c0, e1, fma(-a0, c > 0 ? xch[c - 1] : 0.0, d[base]));
#pragma unroll
  for (int t = 0; t < kLgsPcr; ++t) {
    const int s = 1 << t;
    lgs_bar_solve();  // every read of xch is done
    xch[c] = D;
    lgs_bar_solve();
    const double Dm = c >= s ? xch[c - s] : 0.0, Dp = c + s < kLgsChunks ? xch[c + s] : 0.0;
    D = fma(al[t], Dm, fma(ga[t], Dp, D));
  }
  const double Pv = D * invb;
  lgs_bar_solve();
  xch[c] = Pv;
  lgs_bar_solve();
  const double Pn = c + 1 < kLgsChunks ? xch[c + 1] : 0.0;
  x[base] = Pv;
  for (int r0 = 1; r0 < m; r0 += 4) {
    double ev[4], gv[4], hv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = r0 + q;
      if (r < m) {
        ev[q] = d[base + r];
        gv[q] = fc[lgs_row(r, F_G) + c];
        hv[q] = fc[lgs_row(r, F_H) + c];
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = r0 + q;
      if (r < m) x[base + r] = fma(-gv[q], Pn, fma(-hv[q], Pv, ev[q]));
    }
  }
}

// STAGE: the next column's matrix rows and right-hand side are copied to
// shared memory while the current one is solved (needs even nz, 16-byte
// aligned A and b, and room); otherwise they are read from global memory.
// NS = 7, 19, 27: the canonical mask of that size (compile-time offsets);
// NS = 0: any mask, offsets read at run time.
template <int NS, int KIND, int DIR, bool STAGE>
__global__ void __launch_bounds__(kLgsThreads, 1) k_lsweep(LsParams P) {
  __shared__ WfShared sh;
  __shared__ int s_abort;
  __shared__ __align__(8) unsigned long long s_bar[2];  // copy barriers of the two buffers
  __shared__ int s_landed, s_broken;
  extern __shared__ __align__(16) double lgs_sm[];
  const Grid g = P.g;
  const int ns = P.s.ns;
  const int m = P.m, mp = m + 1, nzp = kLgsChunks * m;
  const long long blk = P.blk, na = (long long)g.nz * ns;
  // shared-memory offsets (doubles): rhs and x in the chunk layout, the PCR
  // exchange row, two factor buffers, with STAGE two buffers of matrix rows
  // and of b
  const int o_rhs = 0, o_x = kLgsChunks * mp, o_xch = 2 * kLgsChunks * mp;
  const long long o_fac = o_xch + kLgsChunks, o_a = o_fac + 2 * blk, o_b = o_a + 2 * na;
  const double* __restrict__ A = P.A;
  const double* __restrict__ b = P.b;
  double* u = P.u;
  if (threadIdx.x == 0) {
    mbar_init(&s_bar[0]);
    mbar_init(&s_bar[1]);
    s_broken = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // completed phases of each buffer's barrier (the same count in every thread)
  unsigned fills[2] = {0u, 0u};
  wf_run(
      sh, P.C,
      [&](int I) {
        const int tid = threadIdx.x, lane = tid & 31;
        const int i = DIR > 0 ? I : g.nx - 1 - I;
        // bulk copies of column Jn's data into buffer Jn & 1, issued by thread 0
        // (the buffer's previous contents were last read before the barrier
        // that precedes this call)
        auto prefetch = [&](int Jn) {
          if (Jn < g.ny && tid == 0 && !s_broken) {
            const int jn = DIR > 0 ? Jn : g.ny - 1 - Jn;
            const long long coln = (long long)i * g.ny + jn;
            const int sel = Jn & 1;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const unsigned fb = (unsigned)(blk * sizeof(double));
            const unsigned ab = STAGE ? (unsigned)(na * sizeof(double)) : 0u;
            const unsigned bb = STAGE ? (unsigned)(g.nz * sizeof(double)) : 0u;
            mbar_expect_tx(&s_bar[sel], fb + ab + bb);
            bulk_copy_g2s(lgs_sm + o_fac + sel * blk, P.F + coln * blk, fb, &s_bar[sel]);
            if (STAGE) {
              bulk_copy_g2s(lgs_sm + o_a + sel * na, A + coln * na, ab, &s_bar[sel]);
              bulk_copy_g2s(lgs_sm + o_b + sel * g.nz, b + coln * g.nz, bb, &s_bar[sel]);
            }
          }
        };
        if (s_broken) {
          // a drain gave up earlier: the copy barriers' phases are unknown, so
          // this CTA issues no more copies and releases its planes at once
          if (tid == 0) {
            wf_st_rel_cta(&sh.abort_flag, 1);
            wf_st_rel_cta(&sh.wdone[0], kWfDone);
          }
          return;
        }
        prefetch(0);
        int have_left = kWfDone, have_up = INT_MIN;
        for (int J = 0; J < g.ny; ++J) {
          const int j = DIR > 0 ? J : g.ny - 1 - J;
          const int sel = J & 1;
          prefetch(J + 1);
          if (tid < 32) {
            const int ab = wf_wait(sh, P.C, 0, J, min(J + 1 + P.dep, g.ny), have_left, have_up, lane);
            // column J's copies have landed (thread 0 waits, whether or not
            // the dependency wait gave up; the barrier below hands the data on
            // to the other threads)
            if (lane == 0) {
              const bool landed = mbar_wait_bounded(&s_bar[sel], fills[sel] & 1u, P.C.budget_ns, P.C.err);
              s_landed = landed;
              s_abort = ab || !landed;
            }
          }
          lgs_bar();
          if (s_abort) {
            // drain every copy issued before leaving the plane: column J's if
            // its wait gave up, column J + 1's always.  The drain bound does
            // not depend on the wait budget (a copy lands in microseconds).
            if (tid == 0) {
              bool ok = s_landed || mbar_wait_bounded(&s_bar[sel], fills[sel] & 1u, kLgsDrainNs, P.C.err);
              if (J + 1 < g.ny) {
                const int s1 = (J + 1) & 1;
                ok = mbar_wait_bounded(&s_bar[s1], fills[s1] & 1u, kLgsDrainNs, P.C.err) && ok;
              }
              if (!ok) s_broken = 1;
            }
            ++fills[sel];
            if (J + 1 < g.ny) ++fills[(J + 1) & 1];
            lgs_bar();
            break;
          }
          ++fills[sel];
          unsigned xymask = 0;
#pragma unroll
          for (int a = -1; a <= 1; ++a)
#pragma unroll
            for (int c = -1; c <= 1; ++c)
              if ((unsigned)(i + a) < (unsigned)g.nx && (unsigned)(j + c) < (unsigned)g.ny)
                xymask |= 1u << ((a + 1) * 3 + (c + 1));
          const long long colbase = ((long long)i * g.ny + j) * g.nz;
          const long long oa = o_a + sel * na, ob = o_b + sel * g.nz;
          // right-hand side: b minus the couplings to other columns; the
          // previous column of the sweep is still in the x buffer
          for (int k = tid; k < nzp; k += kLgsWarps * 32) {
            double acc[4] = {0.0, 0.0, 0.0, 0.0};
            const int kc = k / m, kr = k - kc * m;
            if (k < g.nz) {
              const long long p = colbase + k;
              acc[0] = STAGE ? lgs_sm[ob + k] : b[p];
              const unsigned zmask = (k > 0 ? 1u : 0u) | 2u | (k + 1 < g.nz ? 4u : 0u);
              if constexpr (NS > 0) {
                const double* arow = STAGE ? lgs_sm + oa + (long long)k * NS : A + p * NS;
                line_terms<NS, KIND, DIR>(acc, arow, u + p, lgs_sm + o_x, kc, kr, m, mp, P.s.lin, xymask, zmask,
                                          std::make_integer_sequence<int, NS>{});
              } else {
#pragma unroll 1
              for (int e = 0; e < ns; ++e) {
                const int dx = P.s.off[e][0], dy = P.s.off[e][1], dz = P.s.off[e][2];
                if (dx == 0 && dy == 0) continue;
                if (KIND == SW_GS_ZERO && !(DIR * dx < 0 || (dx == 0 && DIR * dy < 0))) continue;
                if (!((xymask >> ((dx + 1) * 3 + (dy + 1))) & 1u) || !((zmask >> (dz + 1)) & 1u)) continue;
                double x;
                if (dx == 0 && dy == -DIR) {
                  // row k + dz of the chunk layout: same chunk unless it crosses an edge
                  int rc = kc, rr = kr + dz;
                  if (rr < 0) { rc -= 1; rr += m; }
                  if (rr >= m) { rc += 1; rr -= m; }
                  x = lgs_sm[o_x + rc * mp + rr];
                } else if (dx != 0) {
                  x = __ldcg(u + p + P.s.lin[e]);  // other planes: other CTAs' data, through L2
                } else {
                  x = u[p + P.s.lin[e]];
                }
                const double a = STAGE ? lgs_sm[oa + (long long)k * ns + e] : __ldg(A + p * ns + e);
                acc[e & 3] = fma(-a, x, acc[e & 3]);
              }
              }
            }
            lgs_sm[o_rhs + kc * mp + kr] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
          }
          lgs_bar();
          if (tid < kLgsChunks)
            lgs_solve_column(lgs_sm + o_rhs, lgs_sm + o_x, lgs_sm + o_fac + sel * blk, lgs_sm + o_xch, m, tid);
          lgs_bar();
          for (int k = tid; k < g.nz; k += kLgsWarps * 32) {
            const int kc = k / m;
            u[colbase + k] = lgs_sm[o_x + kc * mp + (k - kc * m)];
          }
          lgs_bar();  // the column's stores precede the release below
          if (tid == 0) wf_st_rel_cta(&sh.wdone[0], J + 1);
        }
        if (tid == 0) wf_st_rel_cta(&sh.wdone[0], kWfDone);
      },
      kLgsWarps);
}

LineIdx line_idx(const Stencil& s) {
  LineIdx e{-1, -1, -1};
  for (int t = 0; t < s.ns; ++t) {
    if (s.off[t][0] != 0 || s.off[t][1] != 0) continue;
    if (s.off[t][2] == -1) e.sub = t;
    if (s.off[t][2] == 0) e.diag = t;
    if (s.off[t][2] == 1) e.sup = t;
  }
  return e;
}

constexpr size_t kLgsMaxSmem = 200 * 1024;

template <int NS>
bool canonical_mask(const Stencil& s) {
  if (s.ns != NS) return false;
  for (int e = 0; e < NS; ++e)
    for (int d = 0; d < 3; ++d)
      if (s.off[e][d] != Shape<NS>::o(e, d)) return false;
  return true;
}

template <int NSMAX, bool STAGE>
cudaError_t launch_ns(int kind, int dir, const LsParams& P, int grid, size_t smem, cudaStream_t st) {
  auto go = [&](auto kern) {
    cudaError_t a = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (a != cudaSuccess) return a;
    kern<<<grid, kLgsThreads, smem, st>>>(P);
    return cudaGetLastError();
  };
  if (kind == SW_GS_ZERO)
    return dir > 0 ? go(k_lsweep<NSMAX, SW_GS_ZERO, 1, STAGE>) : go(k_lsweep<NSMAX, SW_GS_ZERO, -1, STAGE>);
  return dir > 0 ? go(k_lsweep<NSMAX, SW_GS_FULL, 1, STAGE>) : go(k_lsweep<NSMAX, SW_GS_FULL, -1, STAGE>);
}

template <int NSMAX>
cudaError_t launch_stage(bool stage, int kind, int dir, const LsParams& P, int grid, size_t smem, cudaStream_t st) {
  return stage ? launch_ns<NSMAX, true>(kind, dir, P, grid, smem, st)
               : launch_ns<NSMAX, false>(kind, dir, P, grid, smem, st);
}

}  // namespace

int lgs_chunk_rows(int nz) {
  const int m = (nz + kLgsChunks - 1) / kLgsChunks;
  return m < 2 ? 2 : m;
}

long long lgs_block_doubles(int nz) { return (long long)((lgs_chunk_rows(nz) - 1) * F_N + C_N) * kLgsChunks; }

bool lgs_supported(const Grid& g, const Stencil& s) {
  const LineIdx e = line_idx(s);
  return e.diag >= 0 && lgs_chunk_rows(g.nz) <= kLgsMaxM && (size_t)g.nx <= (size_t)kProgSlots;
}

cudaError_t launch_lgs_setup(const Grid& g, const Stencil& s, const double* A, double* F, int* err,
                             cudaStream_t st) {
  if (!lgs_supported(g, s)) return cudaErrorNotSupported;
  const LineIdx e = line_idx(s);
  const long long ncol = (long long)g.nx * g.ny;
  k_lgs_pivots<<<div_up(ncol, 128), 128, 0, st>>>(g, s.ns, e, A, err);
  cudaError_t r = cudaGetLastError();
  if (r != cudaSuccess) return r;
  k_lgs_factor<<<(unsigned)ncol, kLgsChunks, 0, st>>>(g, s.ns, e, A, F, lgs_chunk_rows(g.nz),
                                                       lgs_block_doubles(g.nz), err);
  smg_count_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_lsweep(const Grid& g, const Stencil& s, int kind, int dir, const double* A, const double* F,
                          const double* b, double* u, SweepWs* ws, int* err, unsigned long long budget_ns,
                          cudaStream_t st) {
  if (!lgs_supported(g, s) || (kind != SW_GS_ZERO && kind != SW_GS_FULL)) return cudaErrorNotSupported;
  int dev = 0, nsm = 0;
  cudaError_t r = cudaGetDevice(&dev);
  if (r == cudaSuccess) r = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (r != cudaSuccess) return r;
  LsParams P;
  P.g = g;
  P.C = WfCtl{g.nx, 1, 0, 0, budget_ns, ws, err};
  P.s = s;
  P.A = A;
  P.F = F;
  P.b = b;
  P.u = u;
  P.m = lgs_chunk_rows(g.nz);
  P.blk = lgs_block_doubles(g.nz);
  // previous-plane columns read beyond the current one, in sweep order
  P.dep = 0;
  for (int t = 0; t < s.ns; ++t)
    if (dir * s.off[t][0] == -1) P.dep = std::max(P.dep, dir * s.off[t][1]);
  // stage the matrix rows and right-hand side of the next column in shared
  // memory when the 16-byte copies line up and both buffers fit
  const bool stage = g.nz % 2 == 0 && ((uintptr_t)A % 16) == 0 && ((uintptr_t)b % 16) == 0 &&
                     lgs_smem_doubles(P.m, P.blk, g.nz, s.ns, true) * sizeof(double) <= kLgsMaxSmem;
  // one CTA per SM: the reservation exceeds half of the SM's shared memory
  const size_t smem =
      std::max(kWfOneCtaPerSmSmem, (size_t)lgs_smem_doubles(P.m, P.blk, g.nz, s.ns, stage) * sizeof(double));
  const int grid = std::min(g.nx, nsm);
  if (canonical_mask<7>(s)) r = launch_stage<7>(stage, kind, dir, P, grid, smem, st);
  else if (canonical_mask<19>(s)) r = launch_stage<19>(stage, kind, dir, P, grid, smem, st);
  else if (canonical_mask<27>(s)) r = launch_stage<27>(stage, kind, dir, P, grid, smem, st);
  else r = launch_stage<0>(stage, kind, dir, P, grid, smem, st);
  smg_count_launch(1);
  return r;
}
