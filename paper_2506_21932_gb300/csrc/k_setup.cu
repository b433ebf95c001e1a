// Stencil-based Galerkin triple product (Sec. 4.3, Eq. 4-10): one thread per
// (coarse point, coarse stencil entry), summing the influence chains of that
// entry from a table derived once per pattern triple on the host.  The two
// products of R A P are fused, as in the paper's generated kernels, so no
// intermediate A P is stored; one GPU thread per coarse element is also the
// mapping the paper suggests for GPUs (end of Sec. 4.3).
#include "smg_internal.cuh"

namespace {

constexpr int TPB = 256;

// Threads are numbered entry-major (idx = c * n_coarse + P) so the 32 lanes
// of a warp share the coarse entry c and walk the same chain list.
template <int B>
__global__ void __launch_bounds__(TPB) k_rap(Grid f, Grid c, Stencil sc, int nsf, int ashift, int zs,
                                             const int* __restrict__ cstart, const int4* __restrict__ ent,
                                             const double* __restrict__ wt, const double* __restrict__ Af,
                                             double* __restrict__ Ac) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= c.n * sc.ns) return;
  const int ce = (int)(idx / c.n);
  const long long P = idx % c.n;
  const int K = (int)(P % c.nz);
  const long long t2 = P / c.nz;
  const int J = (int)(t2 % c.ny);
  const int I = (int)(t2 / c.ny);
  double acc[B * B];
#pragma unroll
  for (int m = 0; m < B * B; ++m) acc[m] = 0.0;
  const bool jin = (unsigned)(I + sc.off[ce][0]) < (unsigned)c.nx && (unsigned)(J + sc.off[ce][1]) < (unsigned)c.ny &&
                   (unsigned)(K + sc.off[ce][2]) < (unsigned)c.nz;
  if (jin) {
    const int u0 = 2 * I + ashift, u1 = 2 * J + ashift, u2 = zs * K + ashift;
    for (int t = cstart[ce]; t < cstart[ce + 1]; ++t) {
      const int4 e = ent[t];
      const int a = u0 + e.x, b = u1 + e.y, cc = u2 + e.z;
      if ((unsigned)a >= (unsigned)f.nx || (unsigned)b >= (unsigned)f.ny || (unsigned)cc >= (unsigned)f.nz) continue;
      const long long q = ((long long)a * f.ny + b) * f.nz + cc;
      const double* src = Af + (q * nsf + e.w) * (B * B);
      const double w = wt[t];
#pragma unroll
      for (int m = 0; m < B * B; ++m) acc[m] = fma(w, src[m], acc[m]);
    }
  }
  double* dst = Ac + (P * sc.ns + ce) * (B * B);
#pragma unroll
  for (int m = 0; m < B * B; ++m) dst[m] = acc[m];
}

}  // namespace

cudaError_t launch_rap(int transfer, Grid fine, const Stencil& sf, int B, const double* Af, Grid coarse,
                       const Stencil& sc, const int* cstart, const int4* chains, const double* weights, double* Ac,
                       cudaStream_t st) {
  const int ashift = transfer == SMG_TRANSFER_FW27V ? 1 : 0;
  const int zs = transfer == SMG_TRANSFER_C16C_XY ? 1 : 2;  // z stride between coarse and fine
  const long long total = coarse.n * sc.ns;
  const int nb = div_up(total, TPB);
  if (B == 1)
    k_rap<1><<<nb, TPB, 0, st>>>(fine, coarse, sc, sf.ns, ashift, zs, cstart, chains, weights, Af, Ac);
  else
    k_rap<3><<<nb, TPB, 0, st>>>(fine, coarse, sc, sf.ns, ashift, zs, cstart, chains, weights, Af, Ac);
  smg_count_launch(1);
  return cudaGetLastError();
}
