// Allocation-free variant of the wavefront sweep (smg_sweep_noalloc).
//
// Some callers cannot let a library allocate device memory: a host
// application that owns every byte of the GPU through its own pool or arena,
// a real-time or embedded caller with a fixed memory budget decided at build
// time, a plugin whose host forbids stray cudaMalloc calls (they synchronise
// the device and fragment the pool).  For them, one sweep kernel is exposed
// without a context: the caller passes the matrix, the inverse diagonal and
// the vectors, and the only scratch the kernel needs -- the per-plane
// progress counters, the plane ticket and the error word of the wavefront --
// lives in a fixed array in device memory that every GPU using this library
// holds until the process exits.
#include <cstring>
#include <mutex>

#include "chains.h"
#include "smg_internal.cuh"

namespace {

// Largest x-extent the scratch covers: progress counters for up to 16 warps
// of every x-plane.
constexpr int kNoAllocMaxPlanes = 4096;

struct NoAllocScratch {
  SweepWs ws;  // ticket, finished-CTA count, prog[kNoAllocMaxPlanes * 16]
  int err[4];  // err[0]: device error word of the bounded waits
};
static_assert(sizeof(SweepWs) == 16 + 4 * 16 * kNoAllocMaxPlanes, "scratch layout");

// The scratch itself: about 256 KB, zero at module load, shared by every call
// on a device.  In host code this name is only a stand-in for the symbol;
// kernels get its device address from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device, looked up once per
// device (with that device current) and cached.
int scratch_address(NoAllocScratch** out) {
  int dev = 0;
  SMG_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return SMG_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    SMG_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_addr[dev] = p;
  }
  *out = (NoAllocScratch*)g_addr[dev];
  return SMG_OK;
}

}  // namespace

extern "C" int smg_sweep_noalloc(int op, const int dims[3], int nstencil, const int* offsets, const double* M,
                                 const double* dinv, const double* b, double* u, double relax_w, int spin_budget_ms,
                                 void* stream) {
  // ---- validation, before any device work
  if (!dims || !offsets || !M || !b || !u) return SMG_EINVAL;
  int kind, dir;
  switch (op) {
    case SMG_OP_GS_FORWARD: kind = SW_GS_FULL; dir = +1; break;
    case SMG_OP_GS_BACKWARD: kind = SW_GS_FULL; dir = -1; break;
    case SMG_OP_GS_ZERO: kind = SW_GS_ZERO; dir = +1; break;
    case SMG_OP_ILU_LOWER: kind = SW_ILU_L; dir = +1; break;
    case SMG_OP_ILU_UPPER: kind = SW_ILU_U; dir = -1; break;
    default: return SMG_EINVAL;
  }
  if (kind != SW_ILU_L && !dinv) return SMG_EINVAL;
  if (dims[0] < 1 || dims[0] > kNoAllocMaxPlanes || dims[1] < 1 || dims[1] > 1024 || dims[2] < 1 || dims[2] > 4096)
    return SMG_EINVAL;
  if (nstencil < 1 || nstencil > 27) return SMG_EINVAL;
  // offsets must already be in lexicographic order (no reordered copy can be
  // made without allocating), unique, structurally symmetric, with a centre
  int off[27][3];
  bool seen[27] = {false};
  int prev = -1;
  for (int e = 0; e < nstencil; ++e) {
    for (int t = 0; t < 3; ++t) {
      off[e][t] = offsets[3 * e + t];
      if (off[e][t] < -1 || off[e][t] > 1) return SMG_EINVAL;
    }
    const int li = (off[e][0] + 1) * 9 + (off[e][1] + 1) * 3 + (off[e][2] + 1);
    if (li <= prev) return SMG_EINVAL;
    prev = li;
    seen[li] = true;
  }
  if (!seen[13]) return SMG_EINVAL;
  for (int li = 0; li < 27; ++li)
    if (seen[li] && !seen[26 - li]) return SMG_EINVAL;
  if (relax_w == 0.0) relax_w = 1.0;
  if (!(relax_w > 0.0 && relax_w < 2.0)) return SMG_EINVAL;
  if (spin_budget_ms <= 0) spin_budget_ms = 1000;

  // ---- launch on the caller's arrays with the fixed scratch
  NoAllocScratch* S = nullptr;
  {
    int rc = scratch_address(&S);
    if (rc != SMG_OK) return rc;
  }
  cudaStream_t st = (cudaStream_t)stream;
  LevelView L;
  L.g = Grid{dims[0], dims[1], dims[2], (long long)dims[0] * dims[1] * dims[2]};
  L.s.ns = nstencil;
  L.s.ec = -1;
  for (int e = 0; e < 27; ++e) {
    L.s.off[e][0] = L.s.off[e][1] = L.s.off[e][2] = 0;
    L.s.lin[e] = 0;
  }
  for (int e = 0; e < nstencil; ++e) {
    for (int t = 0; t < 3; ++t) L.s.off[e][t] = off[e][t];
    L.s.lin[e] = (off[e][0] * dims[1] + off[e][1]) * dims[2] + off[e][2];
    if (!off[e][0] && !off[e][1] && !off[e][2]) L.s.ec = e;
  }
  L.B = 1;
  L.pk = K64;
  L.A = M;
  L.scale = nullptr;
  SweepCfg cfg;
  smg_host::schedule_skews(nstencil, L.s.off, &cfg.SA, &cfg.SB);
  cfg.G = 2;
  cfg.budget_ns = (unsigned long long)spin_budget_ms * 1000000ull;
  // the progress counters, ticket and error word must start at zero; clear
  // them (and nothing else) for this call
  SMG_CUDA_TRY(cudaMemsetAsync(S, 0, 16 + 4 * 16 * (size_t)dims[0], st));
  SMG_CUDA_TRY(cudaMemsetAsync(S->err, 0, sizeof(S->err), st));
  SMG_CUDA_TRY(launch_sweep(L, kind, dir, M, nullptr, nullptr, dinv, relax_w, b, u, &S->ws, S->err, cfg, st));
  int herr = 0;
  SMG_CUDA_TRY(cudaMemcpyAsync(&herr, S->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  SMG_CUDA_TRY(cudaStreamSynchronize(st));
  return herr;
}
