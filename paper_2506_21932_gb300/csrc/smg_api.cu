// C ABI of the library: hierarchy set-up, V-cycle sequencing, Krylov loops
// and the level-wise building blocks.  All numerical work runs in the
// kernels of k_*.cu; this file allocates, validates and orders launches.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "chains.h"
#include "cnn.cuh"
#include "ilurec.cuh"
#include "krylov.cuh"
#include "smg_internal.cuh"

// ---------------------------------------------------------------------------
// error reporting
// ---------------------------------------------------------------------------
static thread_local char g_cuda_msg[512];
static std::atomic<long long> g_launches{0};

void smg_set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_cuda_msg, sizeof(g_cuda_msg), "%s (%s) at %s:%d", cudaGetErrorString(e), what, file, line);
}

void smg_count_launch(long long k) { g_launches += k; }

extern "C" long long smg_launch_count(void) { return g_launches.load(); }

extern "C" const char* smg_strerror(int s) {
  switch (s) {
    case SMG_OK: return "ok";
    case SMG_EINVAL: return "invalid argument";
    case SMG_ENOMEM: return "out of device memory";
    case SMG_ECUDA: return g_cuda_msg[0] ? g_cuda_msg : "CUDA error";
    case SMG_EBREAKDOWN: return "numerical breakdown (zero/negative pivot or p^T A p <= 0)";
    case SMG_ENOTCONV: return "not converged within maxit";
    case SMG_ENAN: return "non-finite residual";
    case SMG_ETIMEOUT: return "device-side wait timed out";
    default: return "unknown status";
  }
}

extern "C" const char* smg_version(void) { return "structmg-gb300 0.1 (sm_103a)"; }

#define TRY(expr)                                 \
  do {                                            \
    int rc_ = (expr);                             \
    if (rc_ != SMG_OK) return rc_;                \
  } while (0)

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct Level {
  Grid g{};
  Stencil s{};
  int B = 1;
  double* A = nullptr;      // FP64 matrix [n][ns][B][B]
  double* dinv = nullptr;   // GS: FP64 inverse diagonal [n][B][B]
  double* LU = nullptr;     // ILU(0) factors [n][ns]
  double* udinv = nullptr;  // ILU: 1 / u_pp
  void* Av = nullptr;       // low precision matrix values
  float* As = nullptr;      // BF16 row scale of A
  void* LUv = nullptr;      // low precision ILU factors
  float* Ls = nullptr;      // BF16 row scale of L
  float* Us = nullptr;      // BF16 row scale of U
  void* dinv32 = nullptr;   // float inverse diagonal ([n] or [n][9])
  void* f = nullptr;        // V-cycle vectors in working precision
  void* u = nullptr;
  void* t = nullptr;
  SweepWs* ws = nullptr;
  SweepCfg cfg{};
  int* ilu_upd = nullptr;
  double* lf = nullptr;     // line Gauss-Seidel: per-column factors
  // warp-pipelined sweeps (canonical masks): records of the working
  // precision in the skewed layout (ilurec.cuh) and two skewed vectors
  void* Lrec = nullptr;     // ILU(0) lower solve
  void* Urec = nullptr;     // ILU(0) upper solve
  void* Grec = nullptr;     // Gauss-Seidel
  void* vs0 = nullptr;
  void* vs1 = nullptr;
};

struct smg_ctx {
  smg_options opt{};
  int B = 1, nlev = 0, pk = K64;
  Level L[SMG_MAX_LEVELS];
  int nco = 0;
  double *cinv = nullptr, *cf = nullptr, *cu = nullptr;
  double *kr = nullptr, *kz = nullptr, *kp = nullptr, *kq = nullptr, *kold = nullptr, *sc = nullptr;
  double *gV = nullptr, *gZ = nullptr, *gw = nullptr;
  int gm = 0;
  RedWs rw{};
  int* err = nullptr;
  double* hsc = nullptr;  // pinned host mirror of sc
  int* herr = nullptr;    // pinned host mirror of err
  smg_stats_t stats{};
  std::vector<void*> allocs;
  cudaGraphExec_t vgraph = nullptr;
  const double* g_in = nullptr;
  double* g_out = nullptr;
  cudaStream_t cap = nullptr;  // library-owned stream for graph capture / replay
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int kernels_per_vcycle = 0;
  // learned post-smoother of the finest level (null when detached)
  const double* ls_logk = nullptr;
  // SMG_LEARNED_REPLACE: the network stands in for the finest level's
  // post-smoothing (which the V-cycle then skips while a network is attached
  // and while training pairs are drawn)
  int ls_mode = 0;
  bool ls_sampling = false;
  void* ls_ws = nullptr;
  CnnWork ls_w{};
  double *ls_r = nullptr, *ls_d = nullptr, *ls_t = nullptr;
  double* ls_dinv = nullptr;  // 1 / a_pp of the finest matrix: scales the network output
  // V-cycle profiling (smg_vcycle_profile): an event after every launch
  bool prof_on = false;
  int prof_n = 0;
  std::vector<cudaEvent_t> prof_ev;
  std::vector<int> prof_level, prof_code;
};

// Records a profiling event after the launches of one stage (no-op unless a
// profiled V-cycle is running).
enum { PM_START = 0, PM_PRE1, PM_PRE2, PM_RESID, PM_RESTRICT, PM_COARSE, PM_PROLONG, PM_POST_RESID, PM_POST1,
       PM_POST2, PM_POST_ADD, PM_CAST, PM_LEARNED, PM_PACK, PM_UNPACK };
static void prof_mark(smg_ctx* h, int level, int code, cudaStream_t st) {
  if (!h->prof_on) return;
  if (h->prof_n >= (int)h->prof_ev.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    h->prof_ev.push_back(e);
    h->prof_level.push_back(0);
    h->prof_code.push_back(0);
  }
  cudaEventRecord(h->prof_ev[h->prof_n], st);
  h->prof_level[h->prof_n] = level;
  h->prof_code[h->prof_n] = code;
  ++h->prof_n;
}

static int dev_alloc(smg_ctx* h, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    *p = nullptr;
    return SMG_ENOMEM;
  }
  h->allocs.push_back(*p);
  return SMG_OK;
}
template <typename T>
static int dalloc(smg_ctx* h, T** p, size_t count) {
  return dev_alloc(h, (void**)p, count * sizeof(T));
}

static void free_ctx(smg_ctx* h) {
  if (!h) return;
  if (h->vgraph) cudaGraphExecDestroy(h->vgraph);
  if (h->cap) {
    cudaStreamSynchronize(h->cap);
    cudaStreamDestroy(h->cap);
  }
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  for (cudaEvent_t e : h->prof_ev) cudaEventDestroy(e);
  for (void* p : h->allocs) cudaFree(p);
  if (h->hsc) cudaFreeHost(h->hsc);
  if (h->herr) cudaFreeHost(h->herr);
  delete h;
}

extern "C" void smg_destroy(smg_t h) { free_ctx(h); }

static Grid make_grid(int nx, int ny, int nz) {
  Grid g{nx, ny, nz, (long long)nx * ny * nz};
  return g;
}

static void make_stencil(Stencil& s, const Grid& g, int ns, const int (*off)[3]) {
  s.ns = ns;
  s.ec = -1;
  for (int e = 0; e < 27; ++e) {
    s.off[e][0] = s.off[e][1] = s.off[e][2] = 0;
    s.lin[e] = 0;
  }
  for (int e = 0; e < ns; ++e) {
    for (int t = 0; t < 3; ++t) s.off[e][t] = off[e][t];
    s.lin[e] = (off[e][0] * g.ny + off[e][1]) * g.nz + off[e][2];
    if (off[e][0] == 0 && off[e][1] == 0 && off[e][2] == 0) s.ec = e;
  }
}

static int lex_index(const int* o) { return (o[0] + 1) * 9 + (o[1] + 1) * 3 + (o[2] + 1); }

static size_t vsize(const smg_ctx* h) { return h->pk == K64 ? sizeof(double) : sizeof(float); }

static LevelView view(const smg_ctx* h, const Level& L, bool lowp) {
  LevelView v;
  v.g = L.g;
  v.s = L.s;
  v.B = L.B;
  if (lowp && h->pk != K64) {
    v.pk = h->pk;
    v.A = L.Av;
    v.scale = L.As;
  } else {
    v.pk = K64;
    v.A = L.A;
    v.scale = nullptr;
  }
  return v;
}

// Reads the device error word (synchronising the stream) and resets it.
static int fetch_err(smg_ctx* h, cudaStream_t st) {
  SMG_CUDA_TRY(cudaMemcpyAsync(h->herr, h->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  SMG_CUDA_TRY(cudaStreamSynchronize(st));
  int e = *h->herr;
  if (e) SMG_CUDA_TRY(cudaMemsetAsync(h->err, 0, sizeof(int), st));
  return e;
}

// ---------------------------------------------------------------------------
// smoothing on one level (V-cycle precision)
// ---------------------------------------------------------------------------
static int sweep(smg_ctx* h, Level& L, int kind, int dir, const void* b, void* u, cudaStream_t st) {
  const bool lp = h->pk != K64;
  LevelView v = view(h, L, true);
  const void* M;
  const float *s1 = nullptr, *s2 = nullptr;
  const void* dv;
  if (kind == SW_ILU_L || kind == SW_ILU_U) {
    M = lp ? L.LUv : (const void*)L.LU;
    s1 = L.Ls;
    s2 = L.Us;
    dv = lp ? L.dinv32 : (const void*)L.udinv;
  } else {
    M = lp ? L.Av : (const void*)L.A;
    s1 = L.As;
    dv = lp ? L.dinv32 : (const void*)L.dinv;
  }
  SMG_CUDA_TRY(launch_sweep(v, kind, dir, M, s1, s2, dv, h->opt.relax_w, b, u, L.ws, h->err, L.cfg, st));
  return SMG_OK;
}

// Levels whose sweeps run on the records and vectors of the skewed layout.
static bool skewed(const Level& L) { return L.Lrec || L.Grec; }

// One sweep of a skewed level; b and u are skewed vectors.
static int sweep_rec(smg_ctx* h, Level& L, int kind, int dir, const void* b, void* u, cudaStream_t st) {
  const void* M = kind == SW_ILU_L ? L.Lrec : (kind == SW_ILU_U ? L.Urec : L.Grec);
  SMG_CUDA_TRY(launch_sweep3(view(h, L, true), kind, dir, M, nullptr, nullptr, nullptr, h->opt.relax_w, b, u, L.ws,
                             h->err, L.cfg, st, true));
  return SMG_OK;
}

// Vector between natural order and the level's skewed layout.
static int skew(smg_ctx* h, Level& L, const void* src, void* dst, bool to_skew, bool add, cudaStream_t st) {
  SMG_CUDA_TRY(launch_skew_copy(L.g, L.cfg.SB, (int)vsize(h), to_skew, src, dst, add, st));
  return SMG_OK;
}

// One line Gauss-Seidel sweep (FP64 hierarchy only).
static int lsweep(smg_ctx* h, Level& L, int kind, int dir, const void* b, void* u, cudaStream_t st) {
  SMG_CUDA_TRY(launch_lsweep(L.g, L.s, kind, dir, L.A, L.lf, (const double*)b, (double*)u, L.ws, h->err,
                             L.cfg.budget_ns, st));
  return SMG_OK;
}

static int smooth_pre(smg_ctx* h, Level& L, int l, const void* f, void* u, cudaStream_t st) {
  if (skewed(L)) {
    // f -> vs0; the first sweep writes vs1 from zero, the second updates it
    TRY(skew(h, L, f, L.vs0, true, false, st));
    prof_mark(h, l, PM_PACK, st);
    const bool ilu = h->opt.smoother == SMG_SMOOTHER_ILU0;
    TRY(sweep_rec(h, L, ilu ? SW_ILU_L : SW_GS_ZERO, +1, L.vs0, L.vs1, st));
    prof_mark(h, l, PM_PRE1, st);
    TRY(sweep_rec(h, L, ilu ? SW_ILU_U : SW_GS_FULL, -1, ilu ? L.vs1 : L.vs0, L.vs1, st));
    prof_mark(h, l, PM_PRE2, st);
    TRY(skew(h, L, L.vs1, u, false, false, st));
    prof_mark(h, l, PM_UNPACK, st);
    return SMG_OK;
  }
  if (h->opt.smoother == SMG_SMOOTHER_LGS) {
    TRY(lsweep(h, L, SW_GS_ZERO, +1, f, u, st));
    prof_mark(h, l, PM_PRE1, st);
    TRY(lsweep(h, L, SW_GS_FULL, -1, f, u, st));
  } else if (h->opt.smoother == SMG_SMOOTHER_SGS) {
    TRY(sweep(h, L, SW_GS_ZERO, +1, f, u, st));
    prof_mark(h, l, PM_PRE1, st);
    TRY(sweep(h, L, SW_GS_FULL, -1, f, u, st));
  } else {
    TRY(sweep(h, L, SW_ILU_L, +1, f, u, st));
    prof_mark(h, l, PM_PRE1, st);
    TRY(sweep(h, L, SW_ILU_U, -1, u, u, st));
  }
  prof_mark(h, l, PM_PRE2, st);
  return SMG_OK;
}

static int smooth_post(smg_ctx* h, Level& L, int l, const void* f, void* u, cudaStream_t st) {
  if (skewed(L)) {
    if (h->opt.smoother == SMG_SMOOTHER_ILU0) {
      // u += U^-1 L^-1 (f - A u): the residual computed in natural order
      // and written in the skewed layout, the solves on skewed vectors, the
      // correction added while unpacking
      SMG_CUDA_TRY(launch_spmv(view(h, L, true), u, f, L.vs0, 1, st, L.cfg.SB));
      prof_mark(h, l, PM_POST_RESID, st);
      TRY(sweep_rec(h, L, SW_ILU_L, +1, L.vs0, L.vs1, st));
      prof_mark(h, l, PM_POST1, st);
      TRY(sweep_rec(h, L, SW_ILU_U, -1, L.vs1, L.vs1, st));
      prof_mark(h, l, PM_POST2, st);
      TRY(skew(h, L, L.vs1, u, false, true, st));
      prof_mark(h, l, PM_POST_ADD, st);
    } else {
      TRY(skew(h, L, f, L.vs0, true, false, st));
      TRY(skew(h, L, u, L.vs1, true, false, st));
      prof_mark(h, l, PM_PACK, st);
      TRY(sweep_rec(h, L, SW_GS_FULL, +1, L.vs0, L.vs1, st));
      prof_mark(h, l, PM_POST1, st);
      TRY(sweep_rec(h, L, SW_GS_FULL, -1, L.vs0, L.vs1, st));
      prof_mark(h, l, PM_POST2, st);
      TRY(skew(h, L, L.vs1, u, false, false, st));
      prof_mark(h, l, PM_UNPACK, st);
    }
    return SMG_OK;
  }
  if (h->opt.smoother == SMG_SMOOTHER_LGS) {
    TRY(lsweep(h, L, SW_GS_FULL, +1, f, u, st));
    prof_mark(h, l, PM_POST1, st);
    TRY(lsweep(h, L, SW_GS_FULL, -1, f, u, st));
    prof_mark(h, l, PM_POST2, st);
  } else if (h->opt.smoother == SMG_SMOOTHER_SGS) {
    TRY(sweep(h, L, SW_GS_FULL, +1, f, u, st));
    prof_mark(h, l, PM_POST1, st);
    TRY(sweep(h, L, SW_GS_FULL, -1, f, u, st));
    prof_mark(h, l, PM_POST2, st);
  } else {
    SMG_CUDA_TRY(launch_spmv(view(h, L, true), u, f, L.t, 1, st));
    prof_mark(h, l, PM_POST_RESID, st);
    TRY(sweep(h, L, SW_ILU_L, +1, L.t, L.t, st));
    prof_mark(h, l, PM_POST1, st);
    TRY(sweep(h, L, SW_ILU_U, -1, L.t, L.t, st));
    prof_mark(h, l, PM_POST2, st);
    SMG_CUDA_TRY(vec_add(L.g.n * L.B, L.t, u, h->pk == K64, h->rw, st));
    prof_mark(h, l, PM_POST_ADD, st);
  }
  return SMG_OK;
}

static int coarse_solve(smg_ctx* h, const void* f, void* u, cudaStream_t st) {
  if (h->pk == K64) {
    SMG_CUDA_TRY(launch_dense_matvec(h->nco, h->cinv, (const double*)f, (double*)u, st));
  } else {
    SMG_CUDA_TRY(launch_cast_f2d((const float*)f, h->cf, h->nco, st));
    SMG_CUDA_TRY(launch_dense_matvec(h->nco, h->cinv, h->cf, h->cu, st));
    SMG_CUDA_TRY(launch_cast_d2f(h->cu, (float*)u, h->nco, st));
  }
  return SMG_OK;
}

// Learned post-smoother on the finest level (not in the paper), applied to
// the V-cycle's result z: r' = r - A z, s = rms(r'),
// delta = s D^-1 f(r'/s, logk) with D the diagonal of A,
// z += delta only if ||r' - A delta|| < ||r'||.  The decision is taken on the
// device from the two norms; nothing is read back.
static int learned_post_smooth(smg_ctx* h, const double* r, double* z, cudaStream_t st) {
  const Level& L0 = h->L[0];
  const long long n = L0.g.n;
  const LevelView A0 = view(h, L0, false);
  CnnDims d{L0.g.nx, L0.g.ny, L0.g.nz};
  SMG_CUDA_TRY(launch_spmv(A0, z, r, h->ls_r, 1, st));
  SMG_CUDA_TRY(kry_dot(n, h->ls_r, h->ls_r, h->sc, SC_LS_RR, h->rw, st));
  SMG_CUDA_TRY(
      cnn_post_glue(0, n, nullptr, nullptr, nullptr, h->sc + SC_LS_RR, nullptr, nullptr, h->sc + SC_LS_INVS, st));
  SMG_CUDA_TRY(cnn_pack_input(n, h->ls_r, h->ls_logk, h->sc + SC_LS_INVS, 0.0, h->ls_w.a0, st));
  SMG_CUDA_TRY(cnn_forward_packed(d, h->ls_w, st));
  SMG_CUDA_TRY(cnn_post_glue(1, n, h->ls_w.y, nullptr, h->ls_d, h->sc + SC_LS_S, nullptr, h->ls_dinv, nullptr, st));
  SMG_CUDA_TRY(launch_spmv(A0, h->ls_d, h->ls_r, h->ls_t, 1, st));
  SMG_CUDA_TRY(kry_dot(n, h->ls_t, h->ls_t, h->sc, SC_LS_WW, h->rw, st));
  SMG_CUDA_TRY(cnn_post_glue(2, n, nullptr, z, h->ls_d, h->sc + SC_LS_WW, h->sc + SC_LS_RR, nullptr, nullptr, st));
  if (h->ls_mode == SMG_LEARNED_REPLACE) {
    // the correction stood in for the post-smoothing: when the test above
    // rejected it (z unchanged), run the skipped post-smoothing, so z is the
    // plain V-cycle's result
    double nrm[2];
    SMG_CUDA_TRY(cudaMemcpyAsync(&nrm[0], h->sc + SC_LS_WW, sizeof(double), cudaMemcpyDeviceToHost, st));
    SMG_CUDA_TRY(cudaMemcpyAsync(&nrm[1], h->sc + SC_LS_RR, sizeof(double), cudaMemcpyDeviceToHost, st));
    SMG_CUDA_TRY(cudaStreamSynchronize(st));
    if (!(nrm[0] < nrm[1])) TRY(smooth_post(h, h->L[0], 0, r, z, st));
  }
  return SMG_OK;
}

// z = M^{-1} r, one V(1,1)-cycle (Sec. 2): pre-smooth from zero, residual,
// restrict; direct solve on the coarsest level; prolong, correct, post-smooth.
static int vcycle_body(smg_ctx* h, const double* r, double* z, cudaStream_t st) {
  const int nl = h->nlev;
  Level& L0 = h->L[0];
  const long long n0 = L0.g.n * h->B;
  const void* f0;
  void* u0;
  prof_mark(h, 0, PM_START, st);
  if (h->pk == K64) {
    f0 = r;
    u0 = z;
  } else {
    SMG_CUDA_TRY(launch_cast_d2f(r, (float*)L0.f, n0, st));
    prof_mark(h, 0, PM_CAST, st);
    f0 = L0.f;
    u0 = L0.u;
  }
  auto F = [&](int l) -> const void* { return l == 0 ? f0 : h->L[l].f; };
  auto U = [&](int l) -> void* { return l == 0 ? u0 : h->L[l].u; };
  for (int l = 0; l < nl - 1; ++l) {
    Level& L = h->L[l];
    TRY(smooth_pre(h, L, l, F(l), U(l), st));
    // f_{l+1} = R (f - A u): one fused pass where the level allows it
    const cudaError_t rr = h->opt.fuse_restrict
                               ? launch_resid_restrict(view(h, L, true), h->opt.transfer, U(l), F(l), h->L[l + 1].f, st)
                               : cudaErrorNotSupported;
    if (rr == cudaSuccess) {
      prof_mark(h, l, PM_RESID, st);
    } else if (rr == cudaErrorNotSupported) {
      SMG_CUDA_TRY(launch_spmv(view(h, L, true), U(l), F(l), L.t, 1, st));
      prof_mark(h, l, PM_RESID, st);
      SMG_CUDA_TRY(launch_restrict(h->opt.transfer, L.g, h->B, h->pk, L.t, h->L[l + 1].f, st));
    } else {
      SMG_CUDA_TRY(rr);
    }
    prof_mark(h, l, PM_RESTRICT, st);
  }
  TRY(coarse_solve(h, F(nl - 1), U(nl - 1), st));
  prof_mark(h, nl - 1, PM_COARSE, st);
  for (int l = nl - 2; l >= 0; --l) {
    Level& L = h->L[l];
    SMG_CUDA_TRY(launch_prolong_add(h->opt.transfer, L.g, h->B, h->pk, h->L[l + 1].u, U(l), st));
    prof_mark(h, l, PM_PROLONG, st);
    const bool replaced = l == 0 && h->ls_mode == SMG_LEARNED_REPLACE && (h->ls_logk || h->ls_sampling);
    if (!replaced) TRY(smooth_post(h, L, l, F(l), U(l), st));
  }
  if (h->pk != K64) {
    SMG_CUDA_TRY(launch_cast_f2d((const float*)u0, z, n0, st));
    prof_mark(h, 0, PM_CAST, st);
  }
  if (h->ls_logk) {
    TRY(learned_post_smooth(h, r, z, st));
    prof_mark(h, 0, PM_LEARNED, st);
  }
  return SMG_OK;
}

// With use_graph the V-cycle is captured once per (r, z) pair on a stream the
// library owns (the legacy default stream cannot be captured) and replayed
// there, ordered after and before the caller's stream by events.  If the
// caller's stream is itself being captured, the launches go straight into
// the caller's graph instead.
static int vcycle_run(smg_ctx* h, const double* r, double* z, cudaStream_t user) {
  if (!h->opt.use_graph) return vcycle_body(h, r, z, user);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  SMG_CUDA_TRY(cudaStreamIsCapturing(user, &cs));
  if (cs != cudaStreamCaptureStatusNone) return vcycle_body(h, r, z, user);
  if (!h->cap) {
    SMG_CUDA_TRY(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
    SMG_CUDA_TRY(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
    SMG_CUDA_TRY(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
  }
  cudaStream_t st = h->cap;
  SMG_CUDA_TRY(cudaEventRecord(h->ev_in, user));
  SMG_CUDA_TRY(cudaStreamWaitEvent(st, h->ev_in, 0));
  if (!h->vgraph || h->g_in != r || h->g_out != z) {
    if (h->vgraph) {
      cudaGraphExecDestroy(h->vgraph);
      h->vgraph = nullptr;
    }
    cudaGraph_t graph;
    SMG_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const long long c0 = g_launches.load();
    int rc = vcycle_body(h, r, z, st);
    // captured launches do not run now; they are counted on every replay
    h->kernels_per_vcycle = (int)(g_launches.load() - c0);
    g_launches -= h->kernels_per_vcycle;
    cudaError_t ce = cudaStreamEndCapture(st, &graph);
    if (rc != SMG_OK) {
      if (ce == cudaSuccess) cudaGraphDestroy(graph);
      return rc;
    }
    SMG_CUDA_TRY(ce);
    cudaError_t ie = cudaGraphInstantiate(&h->vgraph, graph, 0);
    cudaGraphDestroy(graph);
    SMG_CUDA_TRY(ie);
    h->g_in = r;
    h->g_out = z;
  }
  SMG_CUDA_TRY(cudaGraphLaunch(h->vgraph, st));
  g_launches += h->kernels_per_vcycle;
  SMG_CUDA_TRY(cudaEventRecord(h->ev_out, st));
  SMG_CUDA_TRY(cudaStreamWaitEvent(user, h->ev_out, 0));
  return SMG_OK;
}

// ---------------------------------------------------------------------------
// setup
// ---------------------------------------------------------------------------
static int validate_mask(int ns, const int* off) {
  if (ns < 1 || ns > 27 || !off) return SMG_EINVAL;
  bool seen[27] = {false};
  for (int e = 0; e < ns; ++e) {
    for (int t = 0; t < 3; ++t)
      if (off[3 * e + t] < -1 || off[3 * e + t] > 1) return SMG_EINVAL;
    int li = lex_index(off + 3 * e);
    if (seen[li]) return SMG_EINVAL;
    seen[li] = true;
  }
  if (!seen[13]) return SMG_EINVAL;
  for (int li = 0; li < 27; ++li)
    if (seen[li] && !seen[26 - li]) return SMG_EINVAL;
  return SMG_OK;
}

// Coarsening schedule: halve every dimension while all are even and the
// smallest is at least 8 (full coarsening), or only x and y under the same
// rule for the x-y semi-coarsening transfer.
static int plan_levels(const int d[3], int maxl, int transfer, int dims[][3]) {
  const bool semi = transfer == SMG_TRANSFER_C16C_XY;
  int c[3] = {d[0], d[1], d[2]};
  int L = 0;
  for (;;) {
    dims[L][0] = c[0];
    dims[L][1] = c[1];
    dims[L][2] = c[2];
    ++L;
    const int mn = semi ? std::min(c[0], c[1]) : std::min(c[0], std::min(c[1], c[2]));
    const bool odd = (c[0] & 1) || (c[1] & 1) || (!semi && (c[2] & 1));
    if (L >= maxl || mn < 8 || odd) break;
    c[0] /= 2;
    c[1] /= 2;
    if (!semi) c[2] /= 2;
  }
  return L;
}

// ILU(0) factors and 1/u_pp in the V-cycle precision (FP32 / BF16 levels of
// an ILU(0) hierarchy): lower entries scaled by Ls, upper ones by Us.
// Idempotent; a no-op for FP64 and for the other smoothers.
static int lower_factors(smg_ctx* h, Level& L, cudaStream_t st) {
  if (h->pk == K64 || !L.LU || L.LUv) return SMG_OK;
  const long long n = L.g.n;
  const size_t vb = h->pk == K32 ? sizeof(float) : sizeof(__nv_bfloat16);
  void *luv = nullptr, *dv = nullptr;
  float *ls = nullptr, *us = nullptr;
  TRY(dev_alloc(h, &luv, n * L.s.ns * vb));
  TRY(dalloc(h, &ls, n));
  TRY(dalloc(h, &us, n));
  TRY(dev_alloc(h, &dv, n * sizeof(float)));
  SMG_CUDA_TRY(launch_lower_matrix(L.g, L.s, L.LU, h->pk, 1, luv, ls, us, st));
  SMG_CUDA_TRY(launch_d2f_array(L.udinv, (float*)dv, n, st));
  L.LUv = luv;
  L.Ls = ls;
  L.Us = us;
  L.dinv32 = dv;
  return SMG_OK;
}

static int setup_level_smoother(smg_ctx* h, Level& L, cudaStream_t st) {
  const long long n = L.g.n;
  const int B = L.B;
  int SA, SB;
  smg_host::schedule_skews(L.s.ns, L.s.off, &SA, &SB);
  L.cfg.SA = SA;
  L.cfg.SB = SB;
  // progress is published every G time steps: a release store stalls the
  // plane's CTA for about one L2 round trip, so it is amortised over G steps
  // (at the price of a G-step larger lag between consecutive planes)
  L.cfg.G = 4;
  L.cfg.budget_ns = (unsigned long long)h->opt.spin_budget_ms * 1000000ull;
  L.cfg.warps = h->opt.sweep_warps;
  TRY(dalloc(h, &L.ws, 1));
  SMG_CUDA_TRY(cudaMemsetAsync(L.ws, 0, sizeof(SweepWs), st));
  if (h->opt.smoother == SMG_SMOOTHER_LGS) {
    if (!lgs_supported(L.g, L.s)) return SMG_EINVAL;
    TRY(dalloc(h, &L.lf, (long long)L.g.nx * L.g.ny * lgs_block_doubles(L.g.nz)));
    SMG_CUDA_TRY(launch_lgs_setup(L.g, L.s, L.A, L.lf, h->err, st));
  } else if (h->opt.smoother == SMG_SMOOTHER_SGS) {
    TRY(dalloc(h, &L.dinv, n * B * B));
    SMG_CUDA_TRY(launch_diag_inverse(L.g, L.s, B, L.A, L.dinv, h->err, st));
  } else {
    std::vector<int> kstart, pairs;
    smg_host::build_ilu_updates(L.s.ns, L.s.off, L.s.ec, kstart, pairs);
    const int kpad = (L.s.ec + 1 + 1) / 2 * 2;
    std::vector<int> upd(kpad + pairs.size(), 0);
    for (int t = 0; t <= L.s.ec; ++t) upd[t] = kstart[t];
    for (size_t t = 0; t < pairs.size(); ++t) upd[kpad + t] = pairs[t];
    TRY(dalloc(h, &L.ilu_upd, upd.size()));
    SMG_CUDA_TRY(cudaMemcpyAsync(L.ilu_upd, upd.data(), upd.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    SMG_CUDA_TRY(cudaStreamSynchronize(st));  // upd is a host temporary
    TRY(dalloc(h, &L.LU, n * L.s.ns));
    TRY(dalloc(h, &L.udinv, n));
    SMG_CUDA_TRY(launch_ilu_factor(L.g, L.s, L.A, L.LU, L.udinv, L.ilu_upd, (int)pairs.size() / 2, L.ws, h->err,
                                   L.cfg, st));
  }
  if (h->pk != K64) {
    const size_t vb = h->pk == K32 ? sizeof(float) : sizeof(__nv_bfloat16);
    if (B == 1) {
      TRY(dev_alloc(h, &L.Av, n * L.s.ns * vb));
      TRY(dalloc(h, &L.As, n));
      SMG_CUDA_TRY(launch_lower_matrix(L.g, L.s, L.A, h->pk, 0, L.Av, L.As, nullptr, st));
    } else {
      TRY(dev_alloc(h, &L.Av, n * L.s.ns * 9 * sizeof(float)));
      SMG_CUDA_TRY(launch_d2f_array(L.A, (float*)L.Av, n * L.s.ns * 9, st));
    }
    if (h->opt.smoother == SMG_SMOOTHER_SGS) {
      TRY(dev_alloc(h, &L.dinv32, n * B * B * sizeof(float)));
      SMG_CUDA_TRY(launch_d2f_array(L.dinv, (float*)L.dinv32, n * B * B, st));
    }
  }
  // point smoothers on the warp-pipelined kernel read records of the skewed
  // layout (ilurec.cuh), on skewed vectors
  const bool ilu = h->opt.smoother == SMG_SMOOTHER_ILU0, sgs = h->opt.smoother == SMG_SMOOTHER_SGS;
  const LevelView lv = view(h, L, true);
  if (B == 1 && ((ilu && sweep3_supported(lv, SW_ILU_L)) ||
                 (sgs && sweep3_supported(lv, SW_GS_ZERO) && sweep3_supported(lv, SW_GS_FULL)))) {
    const size_t unit = 16 * (size_t)n;
    if (ilu) {
      TRY(dev_alloc(h, &L.Lrec, unit * sweep_rec_chunks(h->pk, L.s.ns, 0)));
      TRY(dev_alloc(h, &L.Urec, unit * sweep_rec_chunks(h->pk, L.s.ns, 1)));
      SMG_CUDA_TRY(launch_ilu_records(L.g, L.s.ns, L.cfg.SB, h->pk, L.LU, L.udinv, L.Lrec, L.Urec, st));
    } else {
      TRY(dev_alloc(h, &L.Grec, unit * sweep_rec_chunks(h->pk, L.s.ns, 2)));
      SMG_CUDA_TRY(launch_gs_records(L.g, L.s.ns, L.cfg.SB, h->pk, L.A, L.dinv, L.Grec, st));
    }
    TRY(dev_alloc(h, &L.vs0, (size_t)n * vsize(h)));
    TRY(dev_alloc(h, &L.vs1, (size_t)n * vsize(h)));
  }
  // the natural-order sweeps read the factors in the V-cycle precision; the
  // skewed levels' records were built from the FP64 factors directly
  if (!skewed(L)) TRY(lower_factors(h, L, st));
  return SMG_OK;
}

static void compute_stats(smg_ctx* h) {
  smg_stats_t& S = h->stats;
  S.levels = h->nlev;
  double n0 = (double)h->L[0].g.n, z0 = n0 * h->L[0].s.ns;
  double sn = 0, sz = 0, bytes = 0, flops = 0;
  const double c = h->pk == K64 ? 8.0 : (h->pk == K32 ? 4.0 : 2.0);  // matrix value bytes
  const double v = h->pk == K64 ? 8.0 : 4.0;                          // vector bytes
  const double s = h->pk == KBF ? 4.0 : 0.0;                          // row scale bytes
  const double cd = h->pk == K64 ? 8.0 : 4.0;                         // inverse diagonal bytes
  const int B = h->B;
  const double bb = (double)B * B;
  for (int l = 0; l < h->nlev; ++l) {
    const Level& L = h->L[l];
    for (int t = 0; t < 3; ++t) S.dims[l][t] = (&L.g.nx)[t];
    S.nstencil[l] = L.s.ns;
    const double n = (double)L.g.n;
    sn += n;
    sz += n * L.s.ns;
    if (l == h->nlev - 1) {
      bytes += (double)h->nco * h->nco * 8.0 + 2.0 * h->nco * 8.0;
      flops += 2.0 * h->nco * h->nco;
      continue;
    }
    const int ns = L.s.ns, nlow = L.s.ec, nup = ns - 1 - L.s.ec;
    // per point, each array touched once per kernel
    double bpt = 0, fpt = 0;
    if (h->opt.smoother == SMG_SMOOTHER_LGS) {
      // four line sweeps: the matrix row, the column factors, b, u read + write
      const double fpt_bytes = 8.0 * (double)lgs_block_doubles(L.g.nz) / L.g.nz;
      bpt += 4 * (ns * c + fpt_bytes + 3 * v);
      fpt += 4 * (2 * (ns - 3) + 10);
    } else if (h->opt.smoother == SMG_SMOOTHER_SGS) {
      bpt += nlow * c * bb + cd * bb + 2 * v * B + s;                    // GS_ZERO forward
      bpt += 3 * ((ns - 1) * c * bb + cd * bb + 3 * v * B + s);          // three full sweeps
      fpt += 2 * (nlow * bb + bb) + 3 * 2 * ((ns - 1) * bb + bb);
    } else {
      bpt += nlow * c + 2 * v + s + nup * c + cd + 2 * v + s;             // pre: L and U solves
      bpt += ns * c + 3 * v + s;                                          // post residual
      bpt += nlow * c + 2 * v + s + nup * c + cd + 2 * v + s + 3 * v;     // post solves + add
      fpt += 2 * (nlow + nup + 1) * 2 + 2 * ns;
    }
    bpt += ns * c * bb + 3 * v * B + s;                                   // residual before restriction
    fpt += 2 * ns * bb;
    const double cf = (double)h->L[l + 1].g.n / n;                        // coarse / fine points
    bpt += v * B + v * B * cf;                                            // restriction
    bpt += 2 * v * B + v * B * cf;                                        // prolongation + correction
    fpt += 2 * 27.0 / 8.0 * B * 2;
    bytes += bpt * n;
    flops += fpt * n;
  }
  S.grid_complexity = sn / n0;
  S.operator_complexity = sz / z0;
  S.vcycle_bytes = bytes;
  S.vcycle_fp64_flops = h->pk == K64 ? flops : 2.0 * h->nco * h->nco;
  S.precision = h->pk;
  S.smoother = h->opt.smoother;
  S.transfer = h->opt.transfer;
  S.block = h->B;
}

static int do_setup(smg_ctx* h, const int dims[3], int ns, const int* offsets, const double* coeffs,
                    cudaStream_t st) {
  const int B = h->B;
  int pd[SMG_MAX_LEVELS][3];
  const int maxl = h->opt.max_levels > 0 ? std::min(h->opt.max_levels, SMG_MAX_LEVELS) : SMG_MAX_LEVELS;
  h->nlev = plan_levels(dims, maxl, h->opt.transfer, pd);
  TRY(dalloc(h, &h->err, 4));
  SMG_CUDA_TRY(cudaMemsetAsync(h->err, 0, 4 * sizeof(int), st));
  SMG_CUDA_TRY(cudaMallocHost(&h->hsc, SC_COUNT * sizeof(double)));
  SMG_CUDA_TRY(cudaMallocHost(&h->herr, 4 * sizeof(int)));
  // level 0: canonical (lexicographic) stencil order
  {
    Level& L = h->L[0];
    L.g = make_grid(dims[0], dims[1], dims[2]);
    L.B = B;
    std::vector<int> order(ns);
    for (int e = 0; e < ns; ++e) order[e] = e;
    std::sort(order.begin(), order.end(),
              [&](int a, int b) { return lex_index(offsets + 3 * a) < lex_index(offsets + 3 * b); });
    int off[27][3];
    for (int e = 0; e < ns; ++e)
      for (int t = 0; t < 3; ++t) off[e][t] = offsets[3 * order[e] + t];
    make_stencil(L.s, L.g, ns, off);
    TRY(dalloc(h, &L.A, L.g.n * ns * B * B));
    bool ident = true;
    for (int e = 0; e < ns; ++e) ident = ident && order[e] == e;
    if (ident) {
      SMG_CUDA_TRY(cudaMemcpyAsync(L.A, coeffs, sizeof(double) * L.g.n * ns * B * B, cudaMemcpyDeviceToDevice, st));
    } else {
      int* dperm;
      TRY(dalloc(h, &dperm, ns));
      SMG_CUDA_TRY(cudaMemcpyAsync(dperm, order.data(), ns * sizeof(int), cudaMemcpyHostToDevice, st));
      SMG_CUDA_TRY(launch_permute(L.g.n, ns, B * B, dperm, coeffs, L.A, st));
      SMG_CUDA_TRY(cudaStreamSynchronize(st));
    }
    SMG_CUDA_TRY(launch_check_padding(L.g, L.s, B, L.A, h->err + 1, st));
    SMG_CUDA_TRY(cudaMemcpyAsync(h->herr, h->err, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    SMG_CUDA_TRY(cudaStreamSynchronize(st));
    if (h->herr[1] != 0) return SMG_EINVAL;
  }
  // coarse operators by the stencil Galerkin product
  for (int l = 0; l + 1 < h->nlev; ++l) {
    Level& F = h->L[l];
    Level& C = h->L[l + 1];
    smg_host::RapTable T;
    if (smg_host::build_rap_table(h->opt.transfer, F.s.ns, F.s.off, T) < 0) return SMG_EINVAL;
    C.g = make_grid(pd[l + 1][0], pd[l + 1][1], pd[l + 1][2]);
    C.B = B;
    make_stencil(C.s, C.g, T.ns_c, T.off_c);
    if (C.s.ec < 0) return SMG_EINVAL;
    int* dstart;
    int4* dent;
    double* dw;
    TRY(dalloc(h, &dstart, T.start.size()));
    TRY(dalloc(h, &dent, std::max<size_t>(1, T.entries.size())));
    TRY(dalloc(h, &dw, std::max<size_t>(1, T.weights.size())));
    std::vector<int4> ent(T.entries.size());
    for (size_t t = 0; t < ent.size(); ++t) ent[t] = make_int4(T.entries[t].rx, T.entries[t].ry, T.entries[t].rz,
                                                               T.entries[t].a);
    SMG_CUDA_TRY(cudaMemcpyAsync(dstart, T.start.data(), T.start.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    SMG_CUDA_TRY(cudaMemcpyAsync(dent, ent.data(), ent.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    SMG_CUDA_TRY(cudaMemcpyAsync(dw, T.weights.data(), T.weights.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    TRY(dalloc(h, &C.A, C.g.n * C.s.ns * B * B));
    SMG_CUDA_TRY(launch_rap(h->opt.transfer, F.g, F.s, B, F.A, C.g, C.s, dstart, dent, dw, C.A, st));
    SMG_CUDA_TRY(cudaStreamSynchronize(st));  // host tables go out of scope
  }
  // smoothers and vectors
  for (int l = 0; l < h->nlev; ++l) {
    Level& L = h->L[l];
    // smoother data on every level above the coarsest; a one-level hierarchy
    // keeps it too, so the level-wise sweeps stay available
    if (l + 1 < h->nlev || h->nlev == 1) TRY(setup_level_smoother(h, L, st));
    const size_t nv = (size_t)L.g.n * B;
    TRY(dev_alloc(h, &L.f, nv * vsize(h)));
    TRY(dev_alloc(h, &L.u, nv * vsize(h)));
    TRY(dev_alloc(h, &L.t, nv * vsize(h)));
  }
  // coarsest level: dense inverse by Gauss-Jordan with partial pivoting
  {
    Level& Lc = h->L[h->nlev - 1];
    h->nco = (int)(Lc.g.n * B);
    if (h->nco > 8192) return SMG_EINVAL;
    double *M, *colbuf, *gjs;
    TRY(dalloc(h, &M, (size_t)h->nco * h->nco));
    TRY(dalloc(h, &h->cinv, (size_t)h->nco * h->nco));
    TRY(dalloc(h, &colbuf, h->nco));
    TRY(dalloc(h, &gjs, kGjScratchDoubles));
    TRY(dalloc(h, &h->cf, h->nco));
    TRY(dalloc(h, &h->cu, h->nco));
    SMG_CUDA_TRY(launch_assemble_dense(Lc.g, Lc.s, B, Lc.A, M, st));
    SMG_CUDA_TRY(launch_gauss_jordan(h->nco, M, h->cinv, colbuf, h->err, st, gjs,
                                     (unsigned long long)h->opt.spin_budget_ms * 1000000ull));
  }
  // Krylov storage
  const long long n0 = h->L[0].g.n * B;
  TRY(dalloc(h, &h->kr, n0));
  TRY(dalloc(h, &h->kz, n0));
  TRY(dalloc(h, &h->kp, n0));
  TRY(dalloc(h, &h->kq, n0));
  TRY(dalloc(h, &h->kold, n0));
  TRY(dalloc(h, &h->sc, SC_COUNT));
  SMG_CUDA_TRY(cudaMemsetAsync(h->sc, 0, SC_COUNT * sizeof(double), st));
  int dev = 0, nsm = 0;
  SMG_CUDA_TRY(cudaGetDevice(&dev));
  SMG_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  h->rw.nblocks = std::max(1, 2 * nsm);
  TRY(dalloc(h, &h->rw.partial, (size_t)h->rw.nblocks * RED_STRIDE));
  TRY(dalloc(h, &h->rw.counter, 1));
  SMG_CUDA_TRY(cudaMemsetAsync(h->rw.counter, 0, sizeof(unsigned int), st));
  if (h->opt.krylov == SMG_KRYLOV_FGMRES) {
    h->gm = h->opt.restart;
    TRY(dalloc(h, &h->gV, (size_t)n0 * (h->gm + 1)));
    TRY(dalloc(h, &h->gZ, (size_t)n0 * h->gm));
    TRY(dalloc(h, &h->gw, n0));
  }
  int e = fetch_err(h, st);
  if (e) return e;
  compute_stats(h);
  return SMG_OK;
}

extern "C" int smg_setup(smg_t* out, const int dims[3], int nstencil, const int* offsets, const double* coeffs,
                         int block, const smg_options* opt, void* stream) {
  if (!out) return SMG_EINVAL;
  *out = nullptr;
  if (!dims || !coeffs) return SMG_EINVAL;
  for (int t = 0; t < 3; ++t)
    if (dims[t] < 1 || dims[t] > 4096) return SMG_EINVAL;
  if (dims[1] > 1024) return SMG_EINVAL;
  if (block != 1 && block != 3) return SMG_EINVAL;
  TRY(validate_mask(nstencil, offsets));
  smg_options o{};
  if (opt) o = *opt;
  if (o.smoother < 0 || o.smoother > 2 || o.transfer < 0 || o.transfer > 3 || o.precision < 0 || o.precision > 2 ||
      o.krylov < 0 || o.krylov > 2)
    return SMG_EINVAL;
  if (o.restart == 0) o.restart = 30;
  if (o.restart < 1 || o.restart > 64) return SMG_EINVAL;
  if (o.relax_w == 0.0) o.relax_w = 1.0;
  if (!(o.relax_w > 0.0 && o.relax_w < 2.0)) return SMG_EINVAL;
  if (o.max_levels < 0) return SMG_EINVAL;
  if (o.spin_budget_ms <= 0) o.spin_budget_ms = 1000;
  if (o.fuse_restrict < 0 || o.fuse_restrict > 1) return SMG_EINVAL;
  if (o.sweep_warps < 0 || o.sweep_warps > 2) return SMG_EINVAL;
  if (block == 3 && (o.smoother != SMG_SMOOTHER_SGS || o.precision == SMG_PREC_BF16)) return SMG_EINVAL;
  if (o.smoother == SMG_SMOOTHER_ILU0 && nstencil != 7 && nstencil != 19 && nstencil != 27) return SMG_EINVAL;
  // line Gauss-Seidel: scalar FP64 hierarchy, weight 1, columns of at most 1024 points
  if (o.smoother == SMG_SMOOTHER_LGS &&
      (block != 1 || o.precision != SMG_PREC_FP64 || o.relax_w != 1.0 || dims[2] > 1024))
    return SMG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  smg_ctx* h = new smg_ctx();
  h->opt = o;
  h->B = block;
  h->pk = o.precision == SMG_PREC_FP64 ? K64 : (o.precision == SMG_PREC_FP32 ? K32 : KBF);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  int rc = do_setup(h, dims, nstencil, offsets, coeffs, st);
  if (rc == SMG_OK) {
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    h->stats.setup_ms = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != SMG_OK) {
    cudaStreamSynchronize(st);
    (void)cudaGetLastError();
    free_ctx(h);
    return rc;
  }
  *out = h;
  return SMG_OK;
}

extern "C" int smg_stats(smg_t h, smg_stats_t* out) {
  if (!h || !out) return SMG_EINVAL;
  *out = h->stats;
  return SMG_OK;
}

extern "C" int smg_vcycle_profile(smg_t h, const double* r, double* z, int cap, int* count, int* levels,
                                  int* stages, float* ms, void* stream) {
  if (!h || !r || !z || r == z || !count || cap < 0 || (cap > 0 && (!levels || !stages || !ms))) return SMG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  h->prof_on = true;
  h->prof_n = 0;
  const int rc = vcycle_body(h, r, z, st);
  h->prof_on = false;
  TRY(rc);
  SMG_CUDA_TRY(cudaStreamSynchronize(st));
  const int n = h->prof_n - 1;
  *count = n;
  for (int t = 0; t < n && t < cap; ++t) {
    levels[t] = h->prof_level[t + 1];
    stages[t] = h->prof_code[t + 1];
    SMG_CUDA_TRY(cudaEventElapsedTime(&ms[t], h->prof_ev[t], h->prof_ev[t + 1]));
  }
  return fetch_err(h, st);
}

extern "C" int smg_vcycle(smg_t h, const double* r, double* z, void* stream) {
  if (!h || !r || !z || r == z) return SMG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  TRY(vcycle_run(h, r, z, st));
  return fetch_err(h, st);
}

// ---------------------------------------------------------------------------
// Krylov solvers
// ---------------------------------------------------------------------------
static int read_scalars(smg_ctx* h, cudaStream_t st, int* errv) {
  SMG_CUDA_TRY(cudaMemcpyAsync(h->hsc, h->sc, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, st));
  SMG_CUDA_TRY(cudaMemcpyAsync(h->herr, h->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  SMG_CUDA_TRY(cudaStreamSynchronize(st));
  *errv = *h->herr;
  if (*errv) SMG_CUDA_TRY(cudaMemsetAsync(h->err, 0, sizeof(int), st));
  return SMG_OK;
}

static int true_relres(smg_ctx* h, const double* b, const double* x, double bn2, double* relres, cudaStream_t st) {
  const long long n = h->L[0].g.n * h->B;
  SMG_CUDA_TRY(launch_spmv(view(h, h->L[0], false), x, b, h->kr, 1, st));
  SMG_CUDA_TRY(kry_dot(n, h->kr, h->kr, h->sc, SC_WW, h->rw, st));
  int ev = 0;
  TRY(read_scalars(h, st, &ev));
  if (ev) return ev;
  if (relres) *relres = bn2 > 0 ? std::sqrt(h->hsc[SC_WW] / bn2) : 0.0;
  return SMG_OK;
}

static int solve_pcg(smg_ctx* h, const double* b, double* x, double tol, int maxit, int* iters, double* relres,
                     cudaStream_t st) {
  const long long n = h->L[0].g.n * h->B;
  const bool flex = h->opt.krylov == SMG_KRYLOV_FPCG;
  const LevelView A0 = view(h, h->L[0], false);
  SMG_CUDA_TRY(launch_spmv(A0, x, b, h->kr, 1, st));
  SMG_CUDA_TRY(kry_rr_bb(n, h->kr, b, h->sc, h->rw, st));
  int ev = 0;
  TRY(read_scalars(h, st, &ev));
  if (ev) return ev;
  const double bb = h->hsc[SC_BB];
  int it = 0, status = SMG_ENOTCONV;
  if (bb == 0.0) {
    SMG_CUDA_TRY(cudaMemsetAsync(x, 0, n * sizeof(double), st));
    SMG_CUDA_TRY(cudaStreamSynchronize(st));
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    return SMG_OK;
  }
  const double bn = std::sqrt(bb);
  double rel = std::sqrt(h->hsc[SC_RR]) / bn;
  if (rel != rel) return SMG_ENAN;
  if (rel < tol) {
    status = SMG_OK;
  } else {
    TRY(vcycle_run(h, h->kr, h->kz, st));
    SMG_CUDA_TRY(kry_rz_beta(n, h->kr, h->kz, nullptr, h->sc, 1, h->rw, st));
    SMG_CUDA_TRY(kry_update_p(n, h->kp, h->kz, h->sc, 0, h->rw, st));
    for (it = 1; it <= maxit; ++it) {
      SMG_CUDA_TRY(launch_spmv(A0, h->kp, nullptr, h->kq, 0, st));
      SMG_CUDA_TRY(kry_pq_alpha(n, h->kp, h->kq, h->sc, h->err, h->rw, st));
      SMG_CUDA_TRY(kry_update_xr(n, x, h->kp, h->kr, h->kq, flex ? h->kold : nullptr, h->sc, h->rw, st));
      TRY(read_scalars(h, st, &ev));
      if (ev) return ev;
      rel = std::sqrt(h->hsc[SC_RR]) / bn;
      if (rel != rel) return SMG_ENAN;
      if (rel < tol) { status = SMG_OK; break; }
      if (it == maxit) break;
      TRY(vcycle_run(h, h->kr, h->kz, st));
      SMG_CUDA_TRY(kry_rz_beta(n, h->kr, h->kz, flex ? h->kold : nullptr, h->sc, 0, h->rw, st));
      SMG_CUDA_TRY(kry_update_p(n, h->kp, h->kz, h->sc, 1, h->rw, st));
    }
    if (it > maxit) it = maxit;
  }
  if (iters) *iters = it;
  TRY(true_relres(h, b, x, bb, relres, st));
  return status;
}

// Right-preconditioned flexible GMRES(m), classical Gram-Schmidt applied
// twice, Givens rotations on the host (the (m+1) x m Hessenberg matrix is
// tiny), true residual recomputed at every restart.
static int solve_fgmres(smg_ctx* h, const double* b, double* x, double tol, int maxit, int* iters, double* relres,
                        cudaStream_t st) {
  const long long n = h->L[0].g.n * h->B;
  const int m = h->gm;
  const LevelView A0 = view(h, h->L[0], false);
  int ev = 0;
  SMG_CUDA_TRY(launch_spmv(A0, x, b, h->gw, 1, st));
  SMG_CUDA_TRY(kry_rr_bb(n, h->gw, b, h->sc, h->rw, st));
  TRY(read_scalars(h, st, &ev));
  if (ev) return ev;
  const double bb = h->hsc[SC_BB];
  if (bb == 0.0) {
    SMG_CUDA_TRY(cudaMemsetAsync(x, 0, n * sizeof(double), st));
    SMG_CUDA_TRY(cudaStreamSynchronize(st));
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    return SMG_OK;
  }
  const double bn = std::sqrt(bb);
  double beta = std::sqrt(h->hsc[SC_RR]);
  std::vector<double> H((m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  int total = 0;
  while (beta / bn >= tol && total < maxit) {
    if (beta != beta) return SMG_ENAN;
    SMG_CUDA_TRY(kry_scale_rsqrt(n, h->gw, h->gV, h->sc, SC_RR, h->rw, st));
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jdone = 0;
    for (int j = 0; j < m && total < maxit; ++j) {
      double* vj = h->gV + (size_t)j * n;
      double* zj = h->gZ + (size_t)j * n;
      TRY(vcycle_run(h, vj, zj, st));
      SMG_CUDA_TRY(launch_spmv(A0, zj, nullptr, h->gw, 0, st));
      SMG_CUDA_TRY(kry_multidot(n, j + 1, h->gV, n, h->gw, h->sc + SC_H, h->rw, st));
      SMG_CUDA_TRY(kry_multiaxpy(n, j + 1, h->gV, n, h->sc + SC_H, h->gw, h->rw, st));
      SMG_CUDA_TRY(kry_multidot(n, j + 1, h->gV, n, h->gw, h->sc + SC_H2, h->rw, st));
      SMG_CUDA_TRY(kry_multiaxpy(n, j + 1, h->gV, n, h->sc + SC_H2, h->gw, h->rw, st));
      SMG_CUDA_TRY(kry_dot(n, h->gw, h->gw, h->sc, SC_WW, h->rw, st));
      SMG_CUDA_TRY(kry_scale_rsqrt(n, h->gw, h->gV + (size_t)(j + 1) * n, h->sc, SC_WW, h->rw, st));
      TRY(read_scalars(h, st, &ev));
      if (ev) return ev;
      for (int i = 0; i <= j; ++i) H[i * m + j] = h->hsc[SC_H + i] + h->hsc[SC_H2 + i];
      const double hn = std::sqrt(std::max(0.0, h->hsc[SC_WW]));
      H[(j + 1) * m + j] = hn;
      for (int i = 0; i < j; ++i) {
        const double a = H[i * m + j], c = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * c;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      const double a = H[j * m + j], c = H[(j + 1) * m + j];
      const double den = std::sqrt(a * a + c * c);
      cs[j] = den == 0.0 ? 1.0 : a / den;
      sn[j] = den == 0.0 ? 0.0 : c / den;
      H[j * m + j] = cs[j] * a + sn[j] * c;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++total;
      jdone = j + 1;
      if (std::fabs(g[j + 1]) / bn < tol || hn == 0.0) break;
    }
    for (int i = jdone - 1; i >= 0; --i) {
      double s = g[i];
      for (int t = i + 1; t < jdone; ++t) s -= H[i * m + t] * y[t];
      y[i] = s / H[i * m + i];
    }
    for (int i = 0; i < jdone; ++i) h->hsc[SC_H + i] = y[i];
    SMG_CUDA_TRY(cudaMemcpyAsync(h->sc + SC_H, h->hsc + SC_H, jdone * sizeof(double), cudaMemcpyHostToDevice, st));
    SMG_CUDA_TRY(kry_combine(n, jdone, h->gZ, n, h->sc + SC_H, x, h->rw, st));
    SMG_CUDA_TRY(launch_spmv(A0, x, b, h->gw, 1, st));
    SMG_CUDA_TRY(kry_dot(n, h->gw, h->gw, h->sc, SC_RR, h->rw, st));
    TRY(read_scalars(h, st, &ev));
    if (ev) return ev;
    beta = std::sqrt(h->hsc[SC_RR]);
  }
  if (iters) *iters = total;
  if (relres) *relres = beta / bn;
  if (beta != beta) return SMG_ENAN;
  return beta / bn < tol ? SMG_OK : SMG_ENOTCONV;
}

extern "C" int smg_solve(smg_t h, const double* b, double* x, double tol, int maxit, int* iters, double* relres,
                         void* stream) {
  if (!h || !b || !x || b == x || !(tol > 0.0) || maxit < 0) return SMG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = h->opt.krylov == SMG_KRYLOV_FGMRES ? solve_fgmres(h, b, x, tol, maxit, iters, relres, st)
                                              : solve_pcg(h, b, x, tol, maxit, iters, relres, st);
  if (rc == SMG_ECUDA) return rc;
  int ev = fetch_err(h, st);
  if (ev > 0 && ev != SMG_OK) return ev;
  return rc;
}

// ---------------------------------------------------------------------------
// level-wise building blocks
// ---------------------------------------------------------------------------
extern "C" int smg_level_count(smg_t h) { return h ? h->nlev : 0; }

extern "C" int smg_level_sweep_warps(smg_t h, int l, int op) {
  if (!h || l < 0 || l >= h->nlev) return -SMG_EINVAL;
  int kind;
  switch (op) {
    case SMG_OP_GS_FORWARD:
    case SMG_OP_GS_BACKWARD: kind = SW_GS_FULL; break;
    case SMG_OP_GS_ZERO: kind = SW_GS_ZERO; break;
    case SMG_OP_ILU_LOWER: kind = SW_ILU_L; break;
    case SMG_OP_ILU_UPPER: kind = SW_ILU_U; break;
    default: return -SMG_EINVAL;
  }
  Level& L = h->L[l];
  const bool ilu_op = kind == SW_ILU_L || kind == SW_ILU_U;
  if (ilu_op != (h->opt.smoother == SMG_SMOOTHER_ILU0) || h->opt.smoother == SMG_SMOOTHER_LGS) return 0;
  // the warp-pipelined kernels run a level's point sweeps exactly when its
  // records are in the skewed layout
  return skewed(L) ? sweep3_warps(view(h, L, true), kind, true, L.cfg) : 0;
}

extern "C" int smg_level_info(smg_t h, int l, int dims[3], int* nstencil, int* offsets) {
  if (!h || l < 0 || l >= h->nlev) return SMG_EINVAL;
  const Level& L = h->L[l];
  if (dims) {
    dims[0] = L.g.nx;
    dims[1] = L.g.ny;
    dims[2] = L.g.nz;
  }
  if (nstencil) *nstencil = L.s.ns;
  if (offsets)
    for (int e = 0; e < L.s.ns; ++e)
      for (int t = 0; t < 3; ++t) offsets[3 * e + t] = L.s.off[e][t];
  return SMG_OK;
}

extern "C" int smg_level_copy(smg_t h, int l, int which, void* dst, size_t bytes, size_t* needed, void* stream) {
  if (!h || l < 0 || l >= h->nlev) return SMG_EINVAL;
  Level& L = h->L[l];
  const long long n = L.g.n;
  const size_t vb = h->pk == K32 ? 4 : 2;
  const void* src = nullptr;
  size_t sz = 0;
  cudaStream_t st = (cudaStream_t)stream;
  // skewed levels keep no lowered factors; they are made on first request
  if (which >= 5 && which <= 8) TRY(lower_factors(h, L, st));
  switch (which) {
    case 0: src = L.A; sz = n * L.s.ns * L.B * L.B * 8; break;
    case 1: src = L.LU; sz = n * L.s.ns * 8; break;
    case 2: src = L.dinv ? (const void*)L.dinv : (const void*)L.udinv; sz = L.dinv ? n * L.B * L.B * 8 : n * 8; break;
    case 3: src = L.Av; sz = L.B == 1 ? n * L.s.ns * vb : n * L.s.ns * 9 * 4; break;
    case 4: src = L.As; sz = n * 4; break;
    case 5: src = L.LUv; sz = n * L.s.ns * vb; break;
    case 6: src = L.Ls; sz = n * 4; break;
    case 7: src = L.Us; sz = n * 4; break;
    case 8: src = L.dinv32; sz = n * L.B * L.B * 4; break;
    default: return SMG_EINVAL;
  }
  if (!src) return SMG_EINVAL;
  if (needed) *needed = sz;
  if (!dst) return SMG_OK;
  if (bytes < sz) return SMG_EINVAL;
  SMG_CUDA_TRY(cudaMemcpyAsync(dst, src, sz, cudaMemcpyDeviceToDevice, st));
  SMG_CUDA_TRY(cudaStreamSynchronize(st));
  return SMG_OK;
}

extern "C" int smg_level_apply(smg_t h, int l, int op, const void* x, const void* b, void* y, void* stream) {
  if (!h || l < 0 || l >= h->nlev) return SMG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  Level& L = h->L[l];
  const bool coarsest = l == h->nlev - 1;
  const bool has_sm = !coarsest || h->nlev == 1;
  switch (op) {
    case SMG_OP_SPMV:
    case SMG_OP_RESIDUAL:
      if (!x || !y || (op == SMG_OP_RESIDUAL && !b)) return SMG_EINVAL;
      if (h->pk != K64 && !L.Av) return SMG_EINVAL;
      SMG_CUDA_TRY(launch_spmv(view(h, L, true), x, b, y, op == SMG_OP_RESIDUAL, st));
      break;
    case SMG_OP_GS_FORWARD:
    case SMG_OP_GS_BACKWARD:
    case SMG_OP_GS_ZERO:
      if (!has_sm || h->opt.smoother != SMG_SMOOTHER_SGS || !x || !b) return SMG_EINVAL;
      if (skewed(L)) {
        TRY(skew(h, L, b, L.vs0, true, false, st));
        if (op != SMG_OP_GS_ZERO) TRY(skew(h, L, x, L.vs1, true, false, st));
        TRY(sweep_rec(h, L, op == SMG_OP_GS_ZERO ? SW_GS_ZERO : SW_GS_FULL, op == SMG_OP_GS_BACKWARD ? -1 : +1,
                      L.vs0, L.vs1, st));
        TRY(skew(h, L, L.vs1, (void*)x, false, false, st));
        break;
      }
      TRY(sweep(h, L, op == SMG_OP_GS_ZERO ? SW_GS_ZERO : SW_GS_FULL, op == SMG_OP_GS_BACKWARD ? -1 : +1, b,
                (void*)x, st));
      break;
    case SMG_OP_LGS_FORWARD:
    case SMG_OP_LGS_BACKWARD:
    case SMG_OP_LGS_ZERO:
      if (!has_sm || h->opt.smoother != SMG_SMOOTHER_LGS || !x || !b) return SMG_EINVAL;
      TRY(lsweep(h, L, op == SMG_OP_LGS_ZERO ? SW_GS_ZERO : SW_GS_FULL, op == SMG_OP_LGS_BACKWARD ? -1 : +1, b,
                 (void*)x, st));
      break;
    case SMG_OP_ILU_APPLY:
      if (!has_sm || h->opt.smoother != SMG_SMOOTHER_ILU0 || !b || !y) return SMG_EINVAL;
      if (skewed(L)) {
        TRY(skew(h, L, b, L.vs0, true, false, st));
        TRY(sweep_rec(h, L, SW_ILU_L, +1, L.vs0, L.vs1, st));
        TRY(sweep_rec(h, L, SW_ILU_U, -1, L.vs1, L.vs1, st));
        TRY(skew(h, L, L.vs1, y, false, false, st));
        break;
      }
      TRY(sweep(h, L, SW_ILU_L, +1, b, y, st));
      TRY(sweep(h, L, SW_ILU_U, -1, y, y, st));
      break;
    case SMG_OP_RESTRICT:
      if (coarsest || !x || !y) return SMG_EINVAL;
      SMG_CUDA_TRY(launch_restrict(h->opt.transfer, L.g, h->B, h->pk, x, y, st));
      break;
    case SMG_OP_PROLONG_ADD:
      if (coarsest || !x || !y) return SMG_EINVAL;
      SMG_CUDA_TRY(launch_prolong_add(h->opt.transfer, L.g, h->B, h->pk, x, y, st));
      break;
    case SMG_OP_COARSE_SOLVE:
      if (!coarsest || !b || !y) return SMG_EINVAL;
      SMG_CUDA_TRY(launch_dense_matvec(h->nco, h->cinv, (const double*)b, (double*)y, st));
      break;
    case SMG_OP_ILU_LOWER:
    case SMG_OP_ILU_UPPER:
      if (!has_sm || h->opt.smoother != SMG_SMOOTHER_ILU0 || !b || !y) return SMG_EINVAL;
      if (skewed(L)) {
        TRY(skew(h, L, b, L.vs0, true, false, st));
        TRY(sweep_rec(h, L, op == SMG_OP_ILU_LOWER ? SW_ILU_L : SW_ILU_U, op == SMG_OP_ILU_LOWER ? +1 : -1, L.vs0,
                      L.vs1, st));
        TRY(skew(h, L, L.vs1, y, false, false, st));
        break;
      }
      TRY(sweep(h, L, op == SMG_OP_ILU_LOWER ? SW_ILU_L : SW_ILU_U, op == SMG_OP_ILU_LOWER ? +1 : -1, b, y, st));
      break;
    default:
      return SMG_EINVAL;
  }
  return fetch_err(h, st);
}

static int ensure_ls_buffers(smg_ctx* h, cudaStream_t st) {
  if (h->ls_ws) return SMG_OK;
  const Level& L0 = h->L[0];
  const long long n = L0.g.n;
  CnnDims d{L0.g.nx, L0.g.ny, L0.g.nz};
  TRY(dev_alloc(h, &h->ls_ws, cnn_workspace_bytes(d)));
  TRY(dalloc(h, &h->ls_r, n));
  TRY(dalloc(h, &h->ls_d, n));
  TRY(dalloc(h, &h->ls_t, n));
  TRY(dalloc(h, &h->ls_dinv, n));
  cnn_carve(d, h->ls_ws, h->ls_w);
  SMG_CUDA_TRY(launch_diag_inverse(L0.g, L0.s, 1, L0.A, h->ls_dinv, h->err, st));
  return fetch_err(h, st);
}

extern "C" int smg_learned_sample(smg_t h, const double* e0, const double* logk, float* in2, float* target,
                                  void* stream) {
  if (!h || !e0 || !logk || !in2 || !target || h->B != 1) return SMG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  TRY(ensure_ls_buffers(h, st));
  const Level& L0 = h->L[0];
  const long long n = L0.g.n;
  const LevelView A0 = view(h, L0, false);
  SMG_CUDA_TRY(launch_spmv(A0, e0, e0, h->ls_r, 0, st));  // r0 = A e0
  const double* saved = h->ls_logk;
  h->ls_logk = nullptr;  // the plain V-cycle (without the finest post-smoothing in replace mode)
  h->ls_sampling = true;
  const int rc = vcycle_body(h, h->ls_r, h->ls_d, st);
  h->ls_sampling = false;
  h->ls_logk = saved;
  TRY(rc);
  SMG_CUDA_TRY(cnn_sample_glue(0, n, e0, h->ls_d, h->ls_t, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, st));
  SMG_CUDA_TRY(launch_spmv(A0, h->ls_t, h->ls_t, h->ls_r, 0, st));  // r' = A e1
  SMG_CUDA_TRY(kry_dot(n, h->ls_r, h->ls_r, h->sc, SC_LS_RR, h->rw, st));
  SMG_CUDA_TRY(
      cnn_post_glue(0, n, nullptr, nullptr, nullptr, h->sc + SC_LS_RR, nullptr, nullptr, h->sc + SC_LS_INVS, st));
  SMG_CUDA_TRY(cnn_sample_glue(1, n, nullptr, nullptr, h->ls_t, h->ls_r, logk, h->sc + SC_LS_INVS, h->ls_dinv, in2,
                               target, st));
  return fetch_err(h, st);
}

extern "C" int smg_learned_loss_grad(smg_t h, const float* theta, const float* in2, const float* target, int kind,
                                     float* grad, float* loss, void* ws, size_t ws_bytes, void* stream) {
  if (!h || !theta || !in2 || !grad || !loss || !ws || h->B != 1) return SMG_EINVAL;
  if (kind != SMG_LOSS_ERROR && kind != SMG_LOSS_RESIDUAL) return SMG_EINVAL;
  const Level& L0 = h->L[0];
  const int dims[3] = {L0.g.nx, L0.g.ny, L0.g.nz};
  if (kind == SMG_LOSS_ERROR) return smg_cnn_loss_grad(dims, theta, in2, target, grad, loss, ws, ws_bytes, stream);
  CnnDims d{L0.g.nx, L0.g.ny, L0.g.nz};
  if (ws_bytes < cnn_workspace_bytes(d)) return SMG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  TRY(ensure_ls_buffers(h, st));
  const long long n = L0.g.n;
  const LevelView A0 = view(h, L0, false);
  CnnWork w;
  cnn_carve(d, ws, w);
  SMG_CUDA_TRY(cnn_pack(theta, w.pk, st));
  SMG_CUDA_TRY(cnn_pack_input_f32(n, in2, w.a0, st));
  SMG_CUDA_TRY(cnn_forward_packed(d, w, st));
  // q = A D^-1 y - rhat, loss += |q|^2 / n, output gradient 2 D^-1 A q / n
  // (A symmetric, D its diagonal)
  SMG_CUDA_TRY(cnn_resid_glue(3, n, nullptr, w.y, h->ls_dinv, h->ls_d, nullptr, nullptr, st));
  SMG_CUDA_TRY(launch_spmv(A0, h->ls_d, h->ls_d, h->ls_t, 0, st));
  SMG_CUDA_TRY(cnn_resid_glue(0, n, h->ls_t, in2, nullptr, h->ls_r, nullptr, nullptr, st));
  SMG_CUDA_TRY(kry_dot(n, h->ls_r, h->ls_r, h->sc, SC_LS_RR, h->rw, st));
  SMG_CUDA_TRY(cnn_resid_glue(1, n, h->sc + SC_LS_RR, nullptr, nullptr, nullptr, loss, nullptr, st));
  SMG_CUDA_TRY(launch_spmv(A0, h->ls_r, h->ls_r, h->ls_t, 0, st));
  SMG_CUDA_TRY(cnn_resid_glue(2, n, h->ls_t, nullptr, h->ls_dinv, nullptr, nullptr, w.g3, st));
  SMG_CUDA_TRY(cnn_backward(d, w, grad, st));
  return SMG_OK;
}

extern "C" int smg_set_learned_smoother(smg_t h, const float* theta, const double* logk, void* stream) {
  if (!h) return SMG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (!theta) {
    h->ls_logk = nullptr;
    if (h->vgraph) {
      cudaGraphExecDestroy(h->vgraph);
      h->vgraph = nullptr;
    }
    return SMG_OK;
  }
  if (!logk || h->B != 1 || h->opt.krylov == SMG_KRYLOV_PCG) return SMG_EINVAL;
  TRY(ensure_ls_buffers(h, st));
  SMG_CUDA_TRY(cnn_pack(theta, h->ls_w.pk, st));
  h->ls_logk = logk;
  // a captured V-cycle graph does not contain the post-smoother yet
  if (h->vgraph) {
    cudaGraphExecDestroy(h->vgraph);
    h->vgraph = nullptr;
  }
  SMG_CUDA_TRY(cudaStreamSynchronize(st));
  return SMG_OK;
}

extern "C" int smg_set_learned_mode(smg_t h, int mode) {
  if (!h || (mode != SMG_LEARNED_AFTER && mode != SMG_LEARNED_REPLACE)) return SMG_EINVAL;
  if (mode == SMG_LEARNED_REPLACE && h->pk != K64) return SMG_EINVAL;
  h->ls_mode = mode;
  if (h->vgraph) {
    cudaGraphExecDestroy(h->vgraph);
    h->vgraph = nullptr;
  }
  return SMG_OK;
}

extern "C" int smg_set_wait_budget_ns(smg_t h, long long budget_ns) {
  if (!h || budget_ns < 0 || budget_ns > 10000000000LL) return SMG_EINVAL;
  for (int l = 0; l < h->nlev; ++l) h->L[l].cfg.budget_ns = (unsigned long long)budget_ns;
  if (h->vgraph) {
    cudaGraphExecDestroy(h->vgraph);
    h->vgraph = nullptr;
  }
  return SMG_OK;
}

extern "C" int smg_selftest_wait(smg_t h, int budget_ms, void* stream) {
  if (!h || budget_ms < 1 || budget_ms > 10000) return SMG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  // h->err[2] is reserved and stays 0: nothing ever sets it
  SMG_CUDA_TRY(launch_wait_selftest(h->err + 2, h->err, (unsigned long long)budget_ms * 1000000ull, st));
  return fetch_err(h, st);
}
