// Per-warp wavefront engine of the warp-pipelined kernels (ILU(0)
// factorisation, block Gauss-Seidel): the exact lexicographic order of a
// sweep or a factorisation, point (i,j,k) at global time t = SA*i + SB*j + k.
//
//  * A CTA owns one x-plane at a time, taken by an atomic ticket (so a CTA
//    only ever waits on a plane a running CTA owns); the grid is capped at the
//    SM count and the launch reserves more than half of the SM's shared
//    memory, so one CTA runs per SM.
//  * The plane is cut into warps of 32 y-columns (one lane per column); warp
//    w runs its own loop over local steps s = t - SA*i.  Step s may start once
//    the left warp has finished s-1 (wdone[w-1] >= s) and warps w-1..w+1 of
//    the previous plane have finished a caller-given global time.  All
//    counters are per warp, in shared memory, CTA-scope acquire/release.
//  * Warp NW publishes wdone[] of the plane to global memory with GPU-scope
//    release stores; warp NW+1 polls the previous plane's counters with
//    GPU-scope acquire loads and forwards them into avail[].  Compute warps
//    never execute a GPU-scope fence.
//  * Every wait is bounded by the budget; on expiry the error word is set,
//    the CTA's abort flag releases everything downstream and all CTAs drain.
#pragma once
#include <algorithm>
#include <climits>

#include "smg_internal.cuh"

constexpr int kWfMaxWarps = 16;  // ny <= 512
constexpr int kWfMaxThreads = (kWfMaxWarps + 2) * 32;
constexpr int kWfDone = INT_MAX / 2;
constexpr size_t kWfOneCtaPerSmSmem = 120 * 1024;

struct WfShared {
  int wdone[kWfMaxWarps];  // per compute warp: all local steps < value are finished
  int avail[kWfMaxWarps];  // previous plane, per warp: global time finished
  int abort_flag;
  int group;
};

struct WfCtl {
  int nx, NW, SA, SB;  // planes, compute warps per plane, skews
  unsigned long long budget_ns;
  SweepWs* ws;  // prog[] indexed by plane and warp
  int* err;
};

__device__ __forceinline__ int wf_ld_acq_cta(const int* p) {
  int v;
  asm volatile("ld.acquire.cta.shared.s32 %0, [%1];" : "=r"(v) : "r"((unsigned)__cvta_generic_to_shared(p)) : "memory");
  return v;
}
__device__ __forceinline__ void wf_st_rel_cta(int* p, int v) {
  asm volatile("st.release.cta.shared.s32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "r"(v) : "memory");
}
__device__ __forceinline__ int wf_ld_acq_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Publisher warp of plane I: lane w releases gt0 + wdone[w] until all are done.
__device__ __forceinline__ void wf_publish(WfShared& sh, const WfCtl& C, int I, int gt0, int lane) {
  const bool mine = lane < C.NW;
  int* out_slot = C.ws->prog + (size_t)I * C.NW + lane;
  int published = INT_MIN;
  for (;;) {
    const int T = mine ? wf_ld_acq_cta(&sh.wdone[lane]) : kWfDone;
    if (__any_sync(0xffffffffu, mine && T != published)) {
      if (mine) st_release(out_slot, T >= kWfDone ? kWfDone : gt0 + T);
      published = T;
      if (__all_sync(0xffffffffu, T >= kWfDone)) break;
    } else {
      __nanosleep(64);
    }
    if (__any_sync(0xffffffffu, wf_ld_acq_cta(&sh.abort_flag) != 0)) {
      if (mine) st_release(out_slot, kWfDone);
      break;
    }
  }
}

// Poller warp of plane I: lane w forwards the previous plane's warp w.
__device__ __forceinline__ void wf_poll(WfShared& sh, const WfCtl& C, int I, int lane) {
  const bool mine = lane < C.NW;
  const int* in_slot = C.ws->prog + (size_t)(I - 1) * C.NW + lane;
  int seen = (I == 0 || !mine) ? kWfDone : 0;
  unsigned long long t_wait = 0;
  unsigned iter = 0;
  while (__any_sync(0xffffffffu, seen < kWfDone)) {
    const int v = seen < kWfDone ? wf_ld_acq_gpu(in_slot) : seen;
    const bool fresh = v > seen;
    bool stop = false;
    if (__any_sync(0xffffffffu, fresh)) {
      if (fresh) {
        seen = v;
        wf_st_rel_cta(&sh.avail[lane], v);
      }
      t_wait = 0;
    } else if (lane == 0) {
      // bounded: the previous plane must make progress within the budget
      const unsigned long long now = globaltimer_ns();
      if (t_wait == 0) t_wait = now;
      else if (now - t_wait > C.budget_ns) {
        atomicCAS(C.err, 0, DEV_ERR_TIMEOUT);
        stop = true;
      }
    }
    if ((++iter & 63u) == 0 && lane == 0) stop = stop || ld_relaxed(C.err) != 0 || wf_ld_acq_cta(&sh.abort_flag) != 0;
    if (__shfl_sync(0xffffffffu, stop, 0)) {
      if (lane == 0) wf_st_rel_cta(&sh.abort_flag, 1);
      break;
    }
  }
}

// Wait of compute warp w before its step s: the left warp has finished s-1
// and warps w-1..w+1 of the previous plane have reached global time need.
// have_left / have_up cache the last values seen (in every lane).  Every
// lane checks the caches, so the warp does not diverge; only a stale cache
// sends the warp into the polling loop, where each lane takes its own
// acquire load of the same shared word.  Returns nonzero (in every lane)
// when the plane is aborted.
__device__ __forceinline__ int wf_wait(WfShared& sh, const WfCtl& C, int w, int s, int need, int& have_left,
                                       int& have_up, int lane) {
  int aborted = 0;
  if (__any_sync(0xffffffffu, have_left < s || have_up < need)) {
    unsigned long long t_start = 0;
    for (;;) {
      if (have_left < s) have_left = wf_ld_acq_cta(&sh.wdone[w - 1]);
      if (have_up < need) {
        int Tm = kWfDone;
        for (int ww = max(w - 1, 0); ww <= min(w + 1, C.NW - 1); ++ww) Tm = min(Tm, wf_ld_acq_cta(&sh.avail[ww]));
        have_up = Tm;
      }
      if (have_left >= s && have_up >= need) break;
      if (wf_ld_acq_cta(&sh.abort_flag)) {
        aborted = 1;
        break;
      }
      const unsigned long long now = globaltimer_ns();
      if (t_start == 0) t_start = now;
      else if (now - t_start > C.budget_ns) {
        if (lane == 0) {
          atomicCAS(C.err, 0, DEV_ERR_TIMEOUT);
          wf_st_rel_cta(&sh.abort_flag, 1);
        }
        aborted = 1;
        break;
      }
    }
    aborted = __any_sync(0xffffffffu, aborted) ? 1 : 0;
  }
  return aborted;
}

// Step s of warp w is finished (its stores precede the release).
__device__ __forceinline__ void wf_done(WfShared& sh, int w, int s, int lane) {
  __syncwarp();
  if (lane == 0) wf_st_rel_cta(&sh.wdone[w], s);
}

// The persistent plane loop.  compute(I) runs on the compute warps of each
// claimed plane (warps 0..ncompute-1, by default one per progress counter,
// ncompute = NW), the publisher and poller on the next two warps.  The last
// CTA to leave resets the ticket and the counters it used.
template <typename Compute>
__device__ __forceinline__ void wf_run(WfShared& sh, const WfCtl& C, Compute compute, int ncompute = -1) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (ncompute < 0) ncompute = C.NW;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      sh.group = atomicAdd(&C.ws->ticket, 1);
      sh.abort_flag = 0;
    }
    __syncthreads();
    const int I = sh.group;
    if (I >= C.nx) break;
    if (threadIdx.x < kWfMaxWarps) {
      // a warp has trivially finished every step before its first one
      sh.wdone[threadIdx.x] = threadIdx.x < C.NW ? C.SB * 32 * threadIdx.x : kWfDone;
      sh.avail[threadIdx.x] = (I == 0) ? kWfDone : 0;
    }
    __syncthreads();
    if (warp == ncompute) wf_publish(sh, C, I, C.SA * I, lane);
    else if (warp == ncompute + 1) wf_poll(sh, C, I, lane);
    else if (warp < ncompute) compute(I);
  }
  if (threadIdx.x == 0) {
    __threadfence();
    sh.group = (atomicAdd(&C.ws->finished, 1) == (int)gridDim.x - 1);
  }
  __syncthreads();
  if (sh.group) {
    for (int q = threadIdx.x; q < C.nx * C.NW; q += blockDim.x) C.ws->prog[q] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
      C.ws->ticket = 0;
      __threadfence();
      C.ws->finished = 0;
    }
  }
}

// Grid, block and shared-memory reservation of a launch; returns
// cudaErrorNotSupported when the plane does not fit the engine.
__host__ inline cudaError_t wf_launch_shape(const Grid& g, int* grid, int* threads) {
  const int NW = (g.ny + 31) / 32;
  if (NW > kWfMaxWarps || (size_t)g.nx * NW > (size_t)kProgSlots) return cudaErrorNotSupported;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  *grid = std::min(g.nx, nsm);
  *threads = (NW + 2) * 32;
  return cudaSuccess;
}
