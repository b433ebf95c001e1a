// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "smg.h"

#define SMG_MAX_LEVELS 16

// ---------------------------------------------------------------------------
// Precision kinds of a level's stored matrix and V-cycle vectors.
//   K64: double matrix, double vectors, double arithmetic.
//   K32: float matrix, float vectors, float arithmetic.
//   KBF: bf16 matrix values with one float scale per row, float vectors,
//        float accumulation; row result = scale_p * sum_e v_pe x_q.
// ---------------------------------------------------------------------------
enum PrecKind { K64 = 0, K32 = 1, KBF = 2 };

template <int PK> struct Prec;
template <> struct Prec<K64> { using val = double; using vec = double; };
template <> struct Prec<K32> { using val = float; using vec = float; };
template <> struct Prec<KBF> { using val = __nv_bfloat16; using vec = float; };

__device__ __forceinline__ double to_c(double v) { return v; }
__device__ __forceinline__ float to_c(float v) { return v; }
__device__ __forceinline__ float to_c(__nv_bfloat16 v) { return __bfloat162float(v); }

// Grid of one level.
struct Grid {
  int nx, ny, nz;
  long long n;  // nx*ny*nz
};

// Stencil of one level, passed by value: offsets in lexicographic order (so
// for a structurally symmetric mask the entries [0, ec) are the lower ones,
// ec is the centre, (ec, ns) the upper ones), and the linear index step of
// each offset on this level's grid.
struct Stencil {
  int ns, ec;
  int off[27][3];
  int lin[27];
};

// Per-sweep device workspace for the wavefront kernels: progress of every
// plane, a ticket that hands out planes in order, a count of finished CTAs.
// Progress slots: one per x-plane (plane-per-CTA kernels) or one per x-plane
// group and 32-column warp (warp-pipelined kernel): 4096 planes x 16 warps.
constexpr int kProgSlots = 4096 * 16;
struct SweepWs {
  int ticket;
  int finished;
  int pad[2];
  int prog[kProgSlots];  // global time step up to which a plane (or a plane's warp) is done
};

// Kernel-visible error word values (mirror smg_status).
#define DEV_ERR_TIMEOUT SMG_ETIMEOUT

// ---------------------------------------------------------------------------
// Memory-ordering helpers for the cross-CTA progress flags (PTX acquire /
// release at GPU scope) and the bounded wait used everywhere a CTA waits for
// another one.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Wait until *flag >= target.  Gives up (returns false) when the error word is
// set by another CTA or when budget_ns of wall time have passed, in which case
// it records DEV_ERR_TIMEOUT in *err.  Returns the last value read.
// Polls with relaxed loads and issues one GPU-scope fence after the flag is
// seen (relaxed load + fence = acquire), so a poll does not pay for a fence.
__device__ __forceinline__ bool wait_ge(const int* flag, int target, int* err, unsigned long long budget_ns,
                                        int* seen) {
  int v = ld_relaxed(flag);
  if (v >= target) {
    __threadfence();
    *seen = v;
    return true;
  }
  unsigned long long t0 = globaltimer_ns();
  for (;;) {
    __nanosleep(20);
    v = ld_relaxed(flag);
    if (v >= target) {
      __threadfence();
      *seen = v;
      return true;
    }
    if (ld_relaxed(err) != 0) { *seen = v; return false; }
    if (globaltimer_ns() - t0 > budget_ns) {
      atomicCAS(err, 0, DEV_ERR_TIMEOUT);
      *seen = v;
      return false;
    }
  }
}

// ---------------------------------------------------------------------------
// Host helpers
// ---------------------------------------------------------------------------
#define SMG_CUDA_TRY(expr)                                      \
  do {                                                          \
    cudaError_t e_ = (expr);                                    \
    if (e_ != cudaSuccess) {                                    \
      smg_set_last_cuda_error(e_, #expr, __FILE__, __LINE__);   \
      return SMG_ECUDA;                                         \
    }                                                           \
  } while (0)

void smg_set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);

// Counts kernels enqueued by this library (reported by smg_launch_count).
void smg_count_launch(long long k);

static inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// Launchers (all enqueue on `st` and return cudaError_t of the launch).
// `pk` is a PrecKind; B the unknowns per point (1 or 3).
// ---------------------------------------------------------------------------
struct LevelView {
  Grid g;
  Stencil s;
  int B;
  int pk;
  const void* A;        // matrix values (type by pk)
  const float* scale;   // KBF row scales of A (else null)
};

// y = A x (mode 0) or y = b - A x (mode 1).
// fc = R (b - A x) in one pass for scalar levels and the full-weighting or
// 3d8c restriction; cudaErrorNotSupported otherwise (the caller then runs
// launch_spmv and launch_restrict)
cudaError_t launch_resid_restrict(const LevelView& L, int transfer, const void* x, const void* b, void* fc,
                                  cudaStream_t st);
// y = A x (mode 0) or b - A x (mode 1); skew > 0 writes y in the skewed
// plane layout of in-plane skew skew (scalar levels only)
cudaError_t launch_spmv(const LevelView& L, const void* x, const void* b, void* y, int mode, cudaStream_t st,
                        int skew = 0);

// Restriction / prolongation between level (g, B) and its coarse level.
cudaError_t launch_restrict(int transfer, Grid fine, int B, int pk, const void* rf, void* fc, cudaStream_t st);
cudaError_t launch_prolong_add(int transfer, Grid fine, int B, int pk, const void* ec, void* uf, cudaStream_t st);

// Precision casts of vectors.
cudaError_t launch_cast_d2f(const double* a, float* b, long long n, cudaStream_t st);
cudaError_t launch_cast_f2d(const float* a, double* b, long long n, cudaStream_t st);

// Wavefront sweeps (exact lexicographic order).
enum SweepKind { SW_GS_FULL = 0, SW_GS_ZERO = 1, SW_ILU_L = 2, SW_ILU_U = 3 };
struct SweepCfg {
  int SA, SB;  // schedule skews: global time t = SA*i + SB*j + k
  int G;       // publish progress every G steps
  unsigned long long budget_ns;
  int warps = 0;  // warps per 32-column strip of the skewed-layout sweeps: 0 the library's choice, 1, 2
};
cudaError_t launch_sweep(const LevelView& L, int kind, int dir, const void* M, const float* sc1, const float* sc2,
                         const void* dinv, double w, const void* b, void* u, SweepWs* ws, int* err,
                         const SweepCfg& cfg, cudaStream_t st);

// Software-pipelined variant for the lexicographic 7/19/27-point masks with
// one unknown per point; returns cudaErrorNotSupported (nothing launched) for
// any other level, which launch_sweep then runs with the generic kernel.
cudaError_t launch_sweep2(const LevelView& L, int kind, int dir, const void* M, const float* sc1, const float* sc2,
                          const void* dinv, double w, const void* b, void* u, SweepWs* ws, int* err,
                          const SweepCfg& cfg, cudaStream_t st);

// Warp-pipelined variant (same masks, ny <= 512): per-warp time loops synced
// through shared-memory counters, a communication warp for the GPU-scope
// hand-off; returns cudaErrorNotSupported when it does not apply.  rec: M is
// the sweep's records and b, u are vectors, all in the skewed layout of
// ilurec.cuh (FP32 / BF16 sweeps exist only in that form); otherwise M is
// the matrix or ILU factors [n][ns] and the vectors are in natural order.
bool sweep3_supported(const LevelView& L, int kind);
// Warps per 32-column strip launch_sweep3 uses for this sweep: 2 (the
// two-warp kernel), 1 (the one-warp kernel), 0 (not supported).
int sweep3_warps(const LevelView& L, int kind, bool rec, const SweepCfg& cfg);
cudaError_t launch_sweep3(const LevelView& L, int kind, int dir, const void* M, const float* sc1, const float* sc2,
                          const void* dinv, double w, const void* b, void* u, SweepWs* ws, int* err,
                          const SweepCfg& cfg, cudaStream_t st, bool rec);

// Bounded wait on a flag nobody sets (failure-path self-test).
cudaError_t launch_wait_selftest(const int* flag, int* err, unsigned long long budget_ns, cudaStream_t st);

// ILU(0) factorisation (FP64, wavefront over the lower dependencies).
// upd: [kstart (ec+1 ints, padded to an even count)] then int2 pairs.
// Point-block (B == 3) Gauss-Seidel sweeps (GS_ZERO / GS_FULL) on the
// per-warp wavefront engine, for the canonical 7/19/27-point masks, FP64 or
// FP32, ny <= 512; cudaErrorNotSupported (nothing launched) otherwise.
cudaError_t launch_bsweep3(const LevelView& L, int kind, int dir, const void* M, const void* dinv, double w,
                           const void* b, void* u, SweepWs* ws, int* err, const SweepCfg& cfg, cudaStream_t st);
// ILU(0) factorisation of LU in place (LU holds A on entry) on the
// warp-pipelined wavefront, for the canonical 7/19/27-point masks with one
// unknown per point and ny <= 512; cudaErrorNotSupported (nothing launched)
// otherwise.
cudaError_t launch_ilu_factor3(Grid g, const Stencil& s, double* LU, double* udinv, SweepWs* ws, int* err,
                               unsigned long long budget_ns, cudaStream_t st);
cudaError_t launch_ilu_factor(Grid g, const Stencil& s, const double* A, double* LU, double* udinv,
                              const int* upd, int nupd, SweepWs* ws, int* err, const SweepCfg& cfg, cudaStream_t st);

// Line Gauss-Seidel along z (FP64, one unknown per point).  A column of nz
// points is solved by four warps in 128 chunks of lgs_chunk_rows(nz) rows;
// its matrix-only factors take lgs_block_doubles(nz) doubles per column,
// columns in (i, j) order.  lgs_supported: the mask holds the centre and
// nz <= 1024.
int lgs_chunk_rows(int nz);
long long lgs_block_doubles(int nz);
bool lgs_supported(const Grid& g, const Stencil& s);
// Checks every column's Thomas pivots (SMG_EBREAKDOWN in *err unless all are
// positive) and writes the factors F of every column.
cudaError_t launch_lgs_setup(const Grid& g, const Stencil& s, const double* A, double* F, int* err, cudaStream_t st);
// One forward (dir = +1) or backward (dir = -1) line sweep in place on u,
// kind SW_GS_FULL, or SW_GS_ZERO (the later columns are left out).
cudaError_t launch_lsweep(const Grid& g, const Stencil& s, int kind, int dir, const double* A, const double* F,
                          const double* b, double* u, SweepWs* ws, int* err, unsigned long long budget_ns,
                          cudaStream_t st);

// Inverse diagonal (scalar 1/a_pp, or 3x3 block inverse); sets *err to
// SMG_EBREAKDOWN on a zero pivot.
cudaError_t launch_diag_inverse(Grid g, const Stencil& s, int B, const double* A, double* dinv, int* err,
                                cudaStream_t st);

// Galerkin coarse operator from a chain table: chains of coarse entry c are
// [cstart[c], cstart[c+1]); chains[t] = {u offset from the anchor (x,y,z),
// fine stencil entry}; weights[t] = R(I,u) * P(v,J).
cudaError_t launch_rap(int transfer, Grid fine, const Stencil& sf, int B, const double* Af, Grid coarse,
                       const Stencil& sc, const int* cstart, const int4* chains, const double* weights, double* Ac,
                       cudaStream_t st);

// Zero-padding check: counts coefficients with an off-grid neighbour that are
// not exactly zero into *count (device int).
cudaError_t launch_check_padding(Grid g, const Stencil& s, int B, const double* A, int* count, cudaStream_t st);

// Reduced precision copies.
cudaError_t launch_lower_matrix(Grid g, const Stencil& s, const double* A, int pk, int split, void* vals,
                                float* scale, float* scale2, cudaStream_t st);
cudaError_t launch_permute(long long n, int ns, int bb, const int* perm, const double* in, double* out,
                           cudaStream_t st);
cudaError_t launch_d2f_array(const double* a, float* b, long long n, cudaStream_t st);

// Dense coarsest level: assemble, Gauss-Jordan inverse with partial pivoting,
// apply (y = Minv x, double).
cudaError_t launch_assemble_dense(Grid g, const Stencil& s, int B, const double* A, double* M, cudaStream_t st);
// Dense inverse Minv = M^-1 (M destroyed) by Gauss-Jordan elimination with
// partial pivoting.  With scratch (kGjScratchDoubles doubles) one persistent
// cooperative launch whose grid barriers wait at most budget_ns; otherwise
// (or when the device cannot co-schedule the grid) two launches per column.
constexpr int kGjMaxBlocks = 1024;
constexpr int kGjScratchDoubles = 3 * kGjMaxBlocks + 2;
cudaError_t launch_gauss_jordan(int n, double* M, double* Minv, double* colbuf, int* err, cudaStream_t st,
                                double* scratch = nullptr, unsigned long long budget_ns = 0);
cudaError_t launch_dense_matvec(int n, const double* Minv, const double* x, double* y, cudaStream_t st);

// Deterministic reduction workspace of the Krylov kernels: per-block
// partials in fixed order, the last block sums them in fixed order.
struct RedWs {
  double* partial;  // [nblocks * 8]
  unsigned int* counter;
  int nblocks;
};
