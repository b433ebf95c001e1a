// Krylov vector kernels (Sec. 5.2: CG and GMRES as in hypre), FP64, with the
// scalars kept on the device.  Every reduction is deterministic: a fixed grid
// of blocks, each reduces its grid-stride share in a fixed shuffle order and
// writes one partial; the last block to finish sums the partials in block
// order and runs the scalar epilogue (alpha, beta, ...) in one thread.
#include "krylov.cuh"

namespace {

constexpr int RTPB = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide fixed-order sum of NV values; result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (*sh)[RTPB / 32]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < NV; ++t) {
    double s = warp_sum(v[t]);
    if (lane == 0) sh[t][wid] = s;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      double s = lane < RTPB / 32 ? sh[t][lane] : 0.0;
      v[t] = warp_sum(s);
    }
  }
}

// Publishes the block partials; returns true (in every thread) for the last
// block, whose thread 0 then holds the totals in tot[].
template <int NV>
__device__ __forceinline__ bool finish(double (&v)[NV], const RedWs& rw, double (&tot)[NV]) {
  __shared__ double sh[NV][RTPB / 32];
  __shared__ int s_last;
  block_sum<NV>(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int t = 0; t < NV; ++t) rw.partial[blockIdx.x * RED_STRIDE + t] = v[t];
    __threadfence();
    s_last = atomicAdd(rw.counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return false;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int t = 0; t < NV; ++t) tot[t] = 0.0;
    for (int bidx = 0; bidx < (int)gridDim.x; ++bidx)
#pragma unroll
      for (int t = 0; t < NV; ++t) tot[t] += __ldcg(rw.partial + bidx * RED_STRIDE + t);
    *rw.counter = 0;
  }
  return true;
}

// r = b - A x has been formed elsewhere; here ||r||^2 and ||b||^2.
__global__ void __launch_bounds__(RTPB) k_rr_bb(long long n, const double* __restrict__ r,
                                                const double* __restrict__ b, double* sc, RedWs rw) {
  double v[2] = {0.0, 0.0};
  for (long long i = (long long)blockIdx.x * RTPB + threadIdx.x; i < n; i += (long long)gridDim.x * RTPB) {
    v[0] = fma(r[i], r[i], v[0]);
    v[1] = fma(b[i], b[i], v[1]);
  }
  double tot[2];
  if (finish<2>(v, rw, tot) && threadIdx.x == 0) {
    sc[SC_RR] = tot[0];
    sc[SC_BB] = tot[1];
  }
}

// <a, b> into sc[slot]; mode 1 additionally sets rho = <r, z> (slot SC_RHO).
__global__ void __launch_bounds__(RTPB) k_dot(long long n, const double* __restrict__ a, const double* __restrict__ b,
                                              double* sc, int slot, RedWs rw) {
  double v[1] = {0.0};
  for (long long i = (long long)blockIdx.x * RTPB + threadIdx.x; i < n; i += (long long)gridDim.x * RTPB)
    v[0] = fma(a[i], b[i], v[0]);
  double tot[1];
  if (finish<1>(v, rw, tot) && threadIdx.x == 0) sc[slot] = tot[0];
}

// pq = <p, q>; alpha = rho / pq.  A non-positive pq is a CG breakdown.
__global__ void __launch_bounds__(RTPB) k_pq_alpha(long long n, const double* __restrict__ p,
                                                   const double* __restrict__ q, double* sc, int* err, RedWs rw) {
  double v[1] = {0.0};
  for (long long i = (long long)blockIdx.x * RTPB + threadIdx.x; i < n; i += (long long)gridDim.x * RTPB)
    v[0] = fma(p[i], q[i], v[0]);
  double tot[1];
  if (finish<1>(v, rw, tot) && threadIdx.x == 0) {
    const double pq = tot[0];
    sc[SC_PQ] = pq;
    if (!(pq > 0.0)) {
      atomicCAS(err, 0, pq != pq ? SMG_ENAN : SMG_EBREAKDOWN);
      sc[SC_ALPHA] = 0.0;
    } else {
      sc[SC_ALPHA] = sc[SC_RHO] / pq;
    }
  }
}

// x += alpha p; r -= alpha q (rold = r before, if rold != null); rr = <r, r>.
__global__ void __launch_bounds__(RTPB) k_update_xr(long long n, double* __restrict__ x, const double* __restrict__ p,
                                                    double* __restrict__ r, const double* __restrict__ q,
                                                    double* __restrict__ rold, double* sc, RedWs rw) {
  const double alpha = sc[SC_ALPHA];
  double v[1] = {0.0};
  for (long long i = (long long)blockIdx.x * RTPB + threadIdx.x; i < n; i += (long long)gridDim.x * RTPB) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = r[i];
    if (rold) rold[i] = ri;
    const double rn = fma(-alpha, q[i], ri);
    r[i] = rn;
    v[0] = fma(rn, rn, v[0]);
  }
  double tot[1];
  if (finish<1>(v, rw, tot) && threadIdx.x == 0) sc[SC_RR] = tot[0];
}

// rz = <r, z>; flexible: num = <z, r - rold>; beta = num / rho; rho = rz.
// first != 0: only rho = rz (start of the iteration).
__global__ void __launch_bounds__(RTPB) k_rz_beta(long long n, const double* __restrict__ r,
                                                  const double* __restrict__ z, const double* __restrict__ rold,
                                                  double* sc, int first, RedWs rw) {
  double v[2] = {0.0, 0.0};
  for (long long i = (long long)blockIdx.x * RTPB + threadIdx.x; i < n; i += (long long)gridDim.x * RTPB) {
    v[0] = fma(r[i], z[i], v[0]);
    if (rold) v[1] = fma(z[i], r[i] - rold[i], v[1]);
  }
  double tot[2];
  if (finish<2>(v, rw, tot) && threadIdx.x == 0) {
    const double rz = tot[0];
    if (!first) {
      const double num = rold ? tot[1] : rz;
      sc[SC_BETA] = num / sc[SC_RHO];
    }
    sc[SC_RZ] = rz;
    sc[SC_RHO] = rz;
  }
}

// p = z + beta p   (beta from sc[SC_BETA]; use_beta == 0: p = z)
__global__ void __launch_bounds__(RTPB) k_update_p(long long n, double* __restrict__ p, const double* __restrict__ z,
                                                   const double* sc, int use_beta) {
  const double beta = use_beta ? sc[SC_BETA] : 0.0;
  for (long long i = (long long)blockIdx.x * RTPB + threadIdx.x; i < n; i += (long long)gridDim.x * RTPB)
    p[i] = use_beta ? fma(beta, p[i], z[i]) : z[i];
}

// ---- GMRES helpers ----------------------------------------------------------

// out[t] = <V_{c0+t}, w> for t < cnt <= 8 (one chunk of classical
// Gram-Schmidt); V is column-major with leading dimension ld.
__global__ void __launch_bounds__(RTPB) k_dot8(long long n, int c0, int cnt, const double* __restrict__ V,
                                               long long ld, const double* __restrict__ w, double* out, RedWs rw) {
  double v[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (long long i = (long long)blockIdx.x * RTPB + threadIdx.x; i < n; i += (long long)gridDim.x * RTPB) {
    const double wi = w[i];
#pragma unroll
    for (int t = 0; t < 8; ++t)
      if (t < cnt) v[t] = fma(V[(c0 + t) * ld + i], wi, v[t]);
  }
  double tot[8];
  if (finish<8>(v, rw, tot) && threadIdx.x == 0)
    for (int t = 0; t < cnt; ++t) out[c0 + t] = tot[t];
}

// w -= sum_t h[t] V_t ; optionally acc[t] += h[t]
__global__ void __launch_bounds__(RTPB) k_multiaxpy(long long n, int m, const double* __restrict__ V, long long ld,
                                                    const double* __restrict__ h, double* __restrict__ w) {
  for (long long i = (long long)blockIdx.x * RTPB + threadIdx.x; i < n; i += (long long)gridDim.x * RTPB) {
    double s = w[i];
    for (int t = 0; t < m; ++t) s = fma(-h[t], V[t * ld + i], s);
    w[i] = s;
  }
}

// y = x * (1 / sqrt(sc[slot]))  (normalise; a zero norm leaves y = 0)
__global__ void __launch_bounds__(RTPB) k_scale_rsqrt(long long n, const double* __restrict__ x, double* __restrict__ y,
                                                      const double* sc, int slot) {
  const double nn = sc[slot];
  const double s = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
  for (long long i = (long long)blockIdx.x * RTPB + threadIdx.x; i < n; i += (long long)gridDim.x * RTPB)
    y[i] = x[i] * s;
}

// x += sum_t y[t] Z_t
__global__ void __launch_bounds__(RTPB) k_combine(long long n, int m, const double* __restrict__ Z, long long ld,
                                                  const double* __restrict__ y, double* __restrict__ x) {
  for (long long i = (long long)blockIdx.x * RTPB + threadIdx.x; i < n; i += (long long)gridDim.x * RTPB) {
    double s = x[i];
    for (int t = 0; t < m; ++t) s = fma(y[t], Z[t * ld + i], s);
    x[i] = s;
  }
}

__global__ void __launch_bounds__(RTPB) k_add(long long n, const void* src, void* dst, int dbl) {
  for (long long i = (long long)blockIdx.x * RTPB + threadIdx.x; i < n; i += (long long)gridDim.x * RTPB) {
    if (dbl) ((double*)dst)[i] += ((const double*)src)[i];
    else ((float*)dst)[i] += ((const float*)src)[i];
  }
}

}  // namespace

#define KRY_GRID(rw) (rw).nblocks, RTPB, 0, st

cudaError_t kry_rr_bb(long long n, const double* r, const double* b, double* sc, const RedWs& rw, cudaStream_t st) {
  k_rr_bb<<<KRY_GRID(rw)>>>(n, r, b, sc, rw);
  smg_count_launch(1);
  return cudaGetLastError();
}
cudaError_t kry_dot(long long n, const double* a, const double* b, double* sc, int slot, const RedWs& rw,
                    cudaStream_t st) {
  k_dot<<<KRY_GRID(rw)>>>(n, a, b, sc, slot, rw);
  smg_count_launch(1);
  return cudaGetLastError();
}
cudaError_t kry_pq_alpha(long long n, const double* p, const double* q, double* sc, int* err, const RedWs& rw,
                         cudaStream_t st) {
  k_pq_alpha<<<KRY_GRID(rw)>>>(n, p, q, sc, err, rw);
  smg_count_launch(1);
  return cudaGetLastError();
}
cudaError_t kry_update_xr(long long n, double* x, const double* p, double* r, const double* q, double* rold,
                          double* sc, const RedWs& rw, cudaStream_t st) {
  k_update_xr<<<KRY_GRID(rw)>>>(n, x, p, r, q, rold, sc, rw);
  smg_count_launch(1);
  return cudaGetLastError();
}
cudaError_t kry_rz_beta(long long n, const double* r, const double* z, const double* rold, double* sc, int first,
                        const RedWs& rw, cudaStream_t st) {
  k_rz_beta<<<KRY_GRID(rw)>>>(n, r, z, rold, sc, first, rw);
  smg_count_launch(1);
  return cudaGetLastError();
}
cudaError_t kry_update_p(long long n, double* p, const double* z, const double* sc, int use_beta, const RedWs& rw,
                         cudaStream_t st) {
  k_update_p<<<KRY_GRID(rw)>>>(n, p, z, sc, use_beta);
  smg_count_launch(1);
  return cudaGetLastError();
}
cudaError_t kry_multidot(long long n, int m, const double* V, long long ld, const double* w, double* out,
                         const RedWs& rw, cudaStream_t st) {
  for (int c0 = 0; c0 < m; c0 += 8) {
    k_dot8<<<KRY_GRID(rw)>>>(n, c0, m - c0 < 8 ? m - c0 : 8, V, ld, w, out, rw);
    smg_count_launch(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
cudaError_t kry_multiaxpy(long long n, int m, const double* V, long long ld, const double* h, double* w,
                          const RedWs& rw, cudaStream_t st) {
  k_multiaxpy<<<KRY_GRID(rw)>>>(n, m, V, ld, h, w);
  smg_count_launch(1);
  return cudaGetLastError();
}
cudaError_t kry_scale_rsqrt(long long n, const double* x, double* y, const double* sc, int slot, const RedWs& rw,
                            cudaStream_t st) {
  k_scale_rsqrt<<<KRY_GRID(rw)>>>(n, x, y, sc, slot);
  smg_count_launch(1);
  return cudaGetLastError();
}
cudaError_t kry_combine(long long n, int m, const double* Z, long long ld, const double* y, double* x, const RedWs& rw,
                        cudaStream_t st) {
  k_combine<<<KRY_GRID(rw)>>>(n, m, Z, ld, y, x);
  smg_count_launch(1);
  return cudaGetLastError();
}
cudaError_t vec_add(long long n, const void* src, void* dst, int dbl, const RedWs& rw, cudaStream_t st) {
  k_add<<<KRY_GRID(rw)>>>(n, src, dst, dbl);
  smg_count_launch(1);
  return cudaGetLastError();
}
