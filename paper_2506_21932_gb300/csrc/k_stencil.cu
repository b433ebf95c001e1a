// Point-parallel stencil kernels: SG-DIA SpMV / residual (Sec. 6.1.1), grid
// transfers (Sec. 2 V-cycle; Table 2 patterns 3d27v, 3d8c and 3d64c, and the
// 2d4c / 2d16c pair of x-y semi-coarsening), precision
// casts and lowering, diagonal inverses and the dense coarsest level.
#include <algorithm>

#include "ilurec.cuh"
#include "smg_internal.cuh"

namespace {

constexpr int TPB = 256;

__device__ __forceinline__ bool inside3(int i, int j, int k, const Grid& g) {
  return (unsigned)i < (unsigned)g.nx && (unsigned)j < (unsigned)g.ny && (unsigned)k < (unsigned)g.nz;
}

__device__ __forceinline__ void coords(long long p, const Grid& g, int& i, int& j, int& k) {
  k = (int)(p % g.nz);
  long long t = p / g.nz;
  j = (int)(t % g.ny);
  i = (int)(t / g.ny);
}

// ---------------------------------------------------------------------------
// SpMV / residual.  One thread per point, all stencil entries unrolled
// (NS known at compile time), one fused multiply-add per coefficient.  With
// skew > 0 the result goes to the point's slot in the skewed plane layout of
// in-plane skew SB = skew (ilurec.cuh) instead of its natural index.
// ---------------------------------------------------------------------------
template <int PK, int NS>
__global__ void __launch_bounds__(TPB) k_spmv1(Grid g, Stencil s, const typename Prec<PK>::val* __restrict__ A,
                                               const float* __restrict__ scale,
                                               const typename Prec<PK>::vec* __restrict__ x,
                                               const typename Prec<PK>::vec* __restrict__ b,
                                               typename Prec<PK>::vec* __restrict__ y, int mode, int skew) {
  using V = typename Prec<PK>::vec;
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.n) return;
  int i, j, k;
  coords(p, g, i, j, k);
  const typename Prec<PK>::val* a = A + p * NS;
  V acc = 0;
#pragma unroll
  for (int e = 0; e < NS; ++e) {
    int a0 = i + s.off[e][0], a1 = j + s.off[e][1], a2 = k + s.off[e][2];
    V xv = inside3(a0, a1, a2, g) ? x[p + s.lin[e]] : V(0);
    acc = fma((V)to_c(a[e]), xv, acc);
  }
  // the row scale multiplies the finished sum, rounded on its own (never
  // contracted into the subtraction below)
  if (PK == KBF) acc = __fmul_rn(scale[p], (float)acc);
  y[skew ? skew_slot(g, skew, i, j, k) : p] = mode ? b[p] - acc : acc;
}

// The same for FP32 levels, bandwidth-bound: the CTA's rows of A (one
// contiguous, 16-byte aligned run: TPB * NS values) are staged in shared
// memory by 16-byte loads, instead of 27 scattered loads per thread
// (residual at 384^3: 1.50 -> 1.42 ms).  BF16 rows (54 bytes) read back at
// that stride conflict in shared memory and measured slower: they keep
// k_spmv1.
template <int PK, int NS>
__global__ void __launch_bounds__(TPB) k_spmv1s(Grid g, Stencil s, const typename Prec<PK>::val* __restrict__ A,
                                                const float* __restrict__ scale,
                                                const typename Prec<PK>::vec* __restrict__ x,
                                                const typename Prec<PK>::vec* __restrict__ b,
                                                typename Prec<PK>::vec* __restrict__ y, int mode, int skew) {
  using V = typename Prec<PK>::vec;
  using Val = typename Prec<PK>::val;
  __shared__ __align__(16) Val sa[TPB * NS];
  const long long p0 = (long long)blockIdx.x * TPB;
  const int rows = (int)min((long long)TPB, g.n - p0);
  const int nval = rows * NS;
  const int nvec = nval * (int)sizeof(Val) / 16;
  const uint4* src = reinterpret_cast<const uint4*>(A + p0 * NS);
  for (int q = threadIdx.x; q < nvec; q += TPB) reinterpret_cast<uint4*>(sa)[q] = src[q];
  for (int q = nvec * 16 / (int)sizeof(Val) + threadIdx.x; q < nval; q += TPB) sa[q] = A[p0 * NS + q];
  __syncthreads();
  if ((int)threadIdx.x >= rows) return;
  const long long p = p0 + threadIdx.x;
  int i, j, k;
  coords(p, g, i, j, k);
  const Val* a = sa + threadIdx.x * NS;
  V acc = 0;
#pragma unroll
  for (int e = 0; e < NS; ++e) {
    int a0 = i + s.off[e][0], a1 = j + s.off[e][1], a2 = k + s.off[e][2];
    V xv = inside3(a0, a1, a2, g) ? x[p + s.lin[e]] : V(0);
    acc = fma((V)to_c(a[e]), xv, acc);
  }
  // the row scale multiplies the finished sum, rounded on its own
  if (PK == KBF) acc = __fmul_rn(scale[p], (float)acc);
  y[skew ? skew_slot(g, skew, i, j, k) : p] = mode ? b[p] - acc : acc;
}

// Runtime stencil size (any mask).
template <int PK>
__global__ void __launch_bounds__(TPB) k_spmv1_any(Grid g, Stencil s, const typename Prec<PK>::val* __restrict__ A,
                                                   const float* __restrict__ scale,
                                                   const typename Prec<PK>::vec* __restrict__ x,
                                                   const typename Prec<PK>::vec* __restrict__ b,
                                                   typename Prec<PK>::vec* __restrict__ y, int mode, int skew) {
  using V = typename Prec<PK>::vec;
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.n) return;
  int i, j, k;
  coords(p, g, i, j, k);
  const typename Prec<PK>::val* a = A + p * s.ns;
  V acc = 0;
  for (int e = 0; e < s.ns; ++e) {
    int a0 = i + s.off[e][0], a1 = j + s.off[e][1], a2 = k + s.off[e][2];
    V xv = inside3(a0, a1, a2, g) ? x[p + s.lin[e]] : V(0);
    acc = fma((V)to_c(a[e]), xv, acc);
  }
  // the row scale multiplies the finished sum, rounded on its own (never
  // contracted into the subtraction below)
  if (PK == KBF) acc = __fmul_rn(scale[p], (float)acc);
  y[skew ? skew_slot(g, skew, i, j, k) : p] = mode ? b[p] - acc : acc;
}

// 3 unknowns per point, BxB blocks (FP64 or FP32 only).
template <typename V>
__global__ void __launch_bounds__(TPB) k_spmv3(Grid g, Stencil s, const V* __restrict__ A, const V* __restrict__ x,
                                               const V* __restrict__ b, V* __restrict__ y, int mode) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.n) return;
  int i, j, k;
  coords(p, g, i, j, k);
  V acc0 = 0, acc1 = 0, acc2 = 0;
  for (int e = 0; e < s.ns; ++e) {
    int a0 = i + s.off[e][0], a1 = j + s.off[e][1], a2 = k + s.off[e][2];
    if (!inside3(a0, a1, a2, g)) continue;
    const V* blk = A + (p * s.ns + e) * 9;
    const V* xq = x + (p + s.lin[e]) * 3;
    V x0 = xq[0], x1 = xq[1], x2 = xq[2];
    acc0 = fma(blk[0], x0, fma(blk[1], x1, fma(blk[2], x2, acc0)));
    acc1 = fma(blk[3], x0, fma(blk[4], x1, fma(blk[5], x2, acc1)));
    acc2 = fma(blk[6], x0, fma(blk[7], x1, fma(blk[8], x2, acc2)));
  }
  if (mode) {
    y[p * 3 + 0] = b[p * 3 + 0] - acc0;
    y[p * 3 + 1] = b[p * 3 + 1] - acc1;
    y[p * 3 + 2] = b[p * 3 + 2] - acc2;
  } else {
    y[p * 3 + 0] = acc0;
    y[p * 3 + 1] = acc1;
    y[p * 3 + 2] = acc2;
  }
}

// ---------------------------------------------------------------------------
// Transfers.  Full weighting (3d27v): coarse I sits on fine 2I+1, 1-D weights
// (1/2, 1, 1/2); R = P^T/8.  Piecewise constant (3d8c): R(I,u) = 1 on
// u in 2I+{0,1}^3, P = R^T.  Cell-centred trilinear (3d64c): the 3d8c
// restriction with the interpolation of k_prolong_c64.  Fine points off the
// grid are skipped.
// ---------------------------------------------------------------------------
template <typename V, int B>
__global__ void __launch_bounds__(TPB) k_restrict_fw(Grid f, Grid c, const V* __restrict__ rf, V* __restrict__ fc) {
  long long P = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (P >= c.n) return;
  int I, J, K;
  coords(P, c, I, J, K);
  const V w1[3] = {V(0.5), V(1), V(0.5)};
  V acc[B];
#pragma unroll
  for (int r = 0; r < B; ++r) acc[r] = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int u0 = 2 * I + a;
    if (u0 >= f.nx) continue;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      int u1 = 2 * J + b;
      if (u1 >= f.ny) continue;
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        int u2 = 2 * K + cc;
        if (u2 >= f.nz) continue;
        V wgt = w1[a] * w1[b] * w1[cc] * V(0.125);
        long long q = ((long long)u0 * f.ny + u1) * f.nz + u2;
#pragma unroll
        for (int r = 0; r < B; ++r) acc[r] = fma(wgt, rf[q * B + r], acc[r]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < B; ++r) fc[P * B + r] = acc[r];
}

// Residual and restriction in one pass (scalar levels): fc = R (b - A u).
// A CTA owns a tile of kRrTJ x kRrTK coarse (j, k) columns and a chunk of
// coarse x-planes [I0, I0 + ci).  It computes the fine residual planes its
// coarse points read, each over the tile's fine (j, k) window, into a ring of
// three planes in shared memory, then restricts from there.  Full weighting
// (FW = true) reads fine planes 2I .. 2I+2 (the plane 2I+2 is kept for the
// next coarse plane) and the window 2T+1 wide; the 3d8c sum reads 2I, 2I+1
// and a window 2T wide, so nothing is computed twice but the one-point
// window edge (full weighting) and the first plane of a chunk.  The residual
// is k_spmv1's expression and the restriction k_restrict_fw's / _pc's, in
// the same order.
constexpr int kRrTJ = 8, kRrTK = 32;
template <int PK, int NS, bool FW>
__global__ void __launch_bounds__(TPB) k_resid_restrict(Grid f, Grid c, Stencil s, const typename Prec<PK>::val* __restrict__ A,
                                                        const float* __restrict__ scale,
                                                        const typename Prec<PK>::vec* __restrict__ x,
                                                        const typename Prec<PK>::vec* __restrict__ b,
                                                        typename Prec<PK>::vec* __restrict__ fc, int ci) {
  using V = typename Prec<PK>::vec;
  constexpr int FJ = FW ? 2 * kRrTJ + 1 : 2 * kRrTJ, FK = FW ? 2 * kRrTK + 1 : 2 * kRrTK;
  __shared__ V rp[3][FJ * FK];
  const int tilesK = (c.nz + kRrTK - 1) / kRrTK, tilesJ = (c.ny + kRrTJ - 1) / kRrTJ;
  const int tile = blockIdx.x % (tilesJ * tilesK), chunk = blockIdx.x / (tilesJ * tilesK);
  const int J0 = (tile / tilesK) * kRrTJ, K0 = (tile % tilesK) * kRrTK;
  const int I0 = chunk * ci, I1 = min(c.nx, I0 + ci);
  if (I0 >= I1) return;
  // fine residual plane fx over the window into ring slot fx % 3 (zero off the grid)
  auto plane = [&](int fx) {
    V* dst = rp[fx % 3];
    for (int q = threadIdx.x; q < FJ * FK; q += blockDim.x) {
      const int fj = 2 * J0 + q / FK, fk = 2 * K0 + q % FK;
      V r = V(0);
      if (fx < f.nx && fj < f.ny && fk < f.nz) {
        const long long p = ((long long)fx * f.ny + fj) * f.nz + fk;
        const typename Prec<PK>::val* a = A + p * NS;
        V acc = 0;
#pragma unroll
        for (int e = 0; e < NS; ++e) {
          const int a0 = fx + s.off[e][0], a1 = fj + s.off[e][1], a2 = fk + s.off[e][2];
          const V xv = inside3(a0, a1, a2, f) ? x[p + s.lin[e]] : V(0);
          acc = fma((V)to_c(a[e]), xv, acc);
        }
        if (PK == KBF) acc = __fmul_rn(scale[p], (float)acc);  // rounded on its own, as in k_spmv1
        r = b[p] - acc;
      }
      dst[q] = r;
    }
  };
  if (FW) plane(2 * I0);
  for (int I = I0; I < I1; ++I) {
    if (FW) {
      plane(2 * I + 1);
      plane(2 * I + 2);
    } else {
      plane(2 * I);
      plane(2 * I + 1);
    }
    __syncthreads();
    const int jj = threadIdx.x / kRrTK, kk = threadIdx.x % kRrTK;
    const int J = J0 + jj, K = K0 + kk;
    if (threadIdx.x < kRrTJ * kRrTK && J < c.ny && K < c.nz) {
      V acc = 0;
      if (FW) {
        const V w1[3] = {V(0.5), V(1), V(0.5)};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (2 * I + a >= f.nx) continue;
          const V* pl = rp[(2 * I + a) % 3];
#pragma unroll
          for (int bb = 0; bb < 3; ++bb) {
            if (2 * J + bb >= f.ny) continue;
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
              if (2 * K + cc >= f.nz) continue;
              const V wgt = w1[a] * w1[bb] * w1[cc] * V(0.125);
              acc = fma(wgt, pl[(2 * jj + bb) * FK + 2 * kk + cc], acc);
            }
          }
        }
      } else {
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int bb = 0; bb < 2; ++bb)
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) acc += rp[(2 * I + a) % 3][(2 * jj + bb) * FK + 2 * kk + cc];
      }
      fc[((long long)I * c.ny + J) * c.nz + K] = acc;
    }
    __syncthreads();
  }
}

template <typename V, int B>
__global__ void __launch_bounds__(TPB) k_restrict_pc(Grid f, Grid c, const V* __restrict__ rf, V* __restrict__ fc) {
  long long P = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (P >= c.n) return;
  int I, J, K;
  coords(P, c, I, J, K);
  V acc[B];
#pragma unroll
  for (int r = 0; r < B; ++r) acc[r] = 0;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        long long q = ((long long)(2 * I + a) * f.ny + (2 * J + b)) * f.nz + (2 * K + cc);
#pragma unroll
        for (int r = 0; r < B; ++r) acc[r] += rf[q * B + r];
      }
#pragma unroll
  for (int r = 0; r < B; ++r) fc[P * B + r] = acc[r];
}

// uf += P ec for full weighting.  Per dimension a fine coordinate v is
// either on a coarse point (v = 2I + 1: weight 1 from I) or between two
// (v = 2I + 2: weights 1/2 from I and I + 1, the one off the coarse grid
// dropped).  One thread owns the fine points 2I + 1 and 2I + 2 of every
// dimension (I = -1 .. nc - 1; each fine point has exactly one owner) and
// forms their values separably from the 2 x 2 x 2 coarse values c(I + a):
// the sums along z, then y, then x, 12 additions for 8 fine points; the
// weight of a fine point is the power of two 2^-(number of even
// coordinates), applied exactly in the one fused multiply-add into uf.
template <typename V, int B>
__global__ void __launch_bounds__(TPB) k_prolong_fw(Grid f, Grid c, const V* __restrict__ ec, V* __restrict__ uf) {
  const int m2 = c.nz + 1, m1 = c.ny + 1;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)(c.nx + 1) * m1 * m2) return;
  const int I2 = (int)(t % m2) - 1;
  t /= m2;
  const int I1 = (int)(t % m1) - 1;
  const int I0 = (int)(t / m1) - 1;
  const int I[3] = {I0, I1, I2};
  const int cn[3] = {c.nx, c.ny, c.nz};
  const int fn[3] = {f.nx, f.ny, f.nz};
  bool cok[3][2], fok[3][2];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      cok[d][h] = (unsigned)(I[d] + h) < (unsigned)cn[d];
      fok[d][h] = (unsigned)(2 * I[d] + 1 + h) < (unsigned)fn[d];
    }
  }
#pragma unroll
  for (int r = 0; r < B; ++r) {
    V cv[2][2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          cv[a][b][h] = V(0);
          if (cok[0][a] && cok[1][b] && cok[2][h])
            cv[a][b][h] = ec[(((long long)(I0 + a) * c.ny + (I1 + b)) * c.nz + (I2 + h)) * B + r];
        }
    // z, then y, then x: index 0 = the odd fine coordinate, 1 = the even one
    V zs[2][2][2], ys[2][2][2], xs[2][2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        zs[a][b][0] = cv[a][b][0];
        zs[a][b][1] = cv[a][b][0] + cv[a][b][1];
      }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int pz = 0; pz < 2; ++pz) {
        ys[a][0][pz] = zs[a][0][pz];
        ys[a][1][pz] = zs[a][0][pz] + zs[a][1][pz];
      }
#pragma unroll
    for (int py = 0; py < 2; ++py)
#pragma unroll
      for (int pz = 0; pz < 2; ++pz) {
        xs[0][py][pz] = ys[0][py][pz];
        xs[1][py][pz] = ys[0][py][pz] + ys[1][py][pz];
      }
#pragma unroll
    for (int px = 0; px < 2; ++px)
#pragma unroll
      for (int py = 0; py < 2; ++py)
#pragma unroll
        for (int pz = 0; pz < 2; ++pz) {
          if (!(fok[0][px] && fok[1][py] && fok[2][pz])) continue;
          const V scale = V(1.0 / (double)(1 << (px + py + pz)));
          const long long q = ((long long)(2 * I0 + 1 + px) * f.ny + (2 * I1 + 1 + py)) * f.nz + (2 * I2 + 1 + pz);
          uf[q * B + r] = fma(scale, xs[px][py][pz], uf[q * B + r]);
        }
  }
}

// uf += P ec for the cell-centred trilinear interpolation (3d64c).  Per
// dimension, fine cell v lies in coarse cell v/2 (weight 3/4) and takes 1/4
// from the coarse cell on its side: v/2 - 1 for even v, v/2 + 1 for odd v.
// Coarse cells off the grid are dropped.  The pair (lower, upper) of coarse
// cells is summed in increasing order in every dimension.
template <typename V, int B>
__global__ void __launch_bounds__(TPB) k_prolong_c64(Grid f, Grid c, const V* __restrict__ ec, V* __restrict__ uf) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= f.n) return;
  int v0, v1, v2;
  coords(q, f, v0, v1, v2);
  const int v[3] = {v0, v1, v2};
  const int cn[3] = {c.nx, c.ny, c.nz};
  // the weight of coarse cell (lo + (a, b, cc)) is 3^m / 64, m the number
  // of dimensions whose factor is 3/4 (exact in any precision; selected in
  // place of the products)
  auto w64 = [](int m) -> V {
    return m == 0 ? V(1.0 / 64) : m == 1 ? V(3.0 / 64) : m == 2 ? V(9.0 / 64) : V(27.0 / 64);
  };
  int lo[3], hi3[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    // 3/4 from the cell the fine cell lies in: the second of the pair for
    // an even v, the first for an odd v
    lo[d] = (v[d] & 1) ? (v[d] >> 1) : (v[d] >> 1) - 1;
    hi3[d] = (v[d] & 1) ? 0 : 1;
  }
  V acc[B];
#pragma unroll
  for (int r = 0; r < B; ++r) acc[r] = 0;
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const int J0 = lo[0] + a;
    if ((unsigned)J0 >= (unsigned)cn[0]) continue;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int J1 = lo[1] + b;
      if ((unsigned)J1 >= (unsigned)cn[1]) continue;
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const int J2 = lo[2] + cc;
        if ((unsigned)J2 >= (unsigned)cn[2]) continue;
        const V wgt = w64((a == hi3[0]) + (b == hi3[1]) + (cc == hi3[2]));
        const long long P = ((long long)J0 * c.ny + J1) * c.nz + J2;
#pragma unroll
        for (int r = 0; r < B; ++r) acc[r] = fma(wgt, ec[P * B + r], acc[r]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < B; ++r) uf[q * B + r] += acc[r];
}

// x-y semi-coarsening (2d4c / 2d16c): fc(I,J,K) = sum of the 2 x 2 fine
// cells (2I + a, 2J + b, K); uf += P ec with the cell-centred bilinear
// weights of k_prolong_c64 in x and y and the same z.
template <typename V, int B>
__global__ void __launch_bounds__(TPB) k_restrict_xy(Grid f, Grid c, const V* __restrict__ rf, V* __restrict__ fc) {
  long long P = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (P >= c.n) return;
  int I, J, K;
  coords(P, c, I, J, K);
  V acc[B];
#pragma unroll
  for (int r = 0; r < B; ++r) acc[r] = 0;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const long long q = ((long long)(2 * I + a) * f.ny + (2 * J + b)) * f.nz + K;
#pragma unroll
      for (int r = 0; r < B; ++r) acc[r] += rf[q * B + r];
    }
#pragma unroll
  for (int r = 0; r < B; ++r) fc[P * B + r] = acc[r];
}

template <typename V, int B>
__global__ void __launch_bounds__(TPB) k_prolong_xy(Grid f, Grid c, const V* __restrict__ ec, V* __restrict__ uf) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= f.n) return;
  int v0, v1, v2;
  coords(q, f, v0, v1, v2);
  const int v[2] = {v0, v1};
  const int cn[2] = {c.nx, c.ny};
  int lo[2];
  V w[2][2];
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    if (v[d] & 1) {
      lo[d] = v[d] >> 1; w[d][0] = V(0.75); w[d][1] = V(0.25);
    } else {
      lo[d] = (v[d] >> 1) - 1; w[d][0] = V(0.25); w[d][1] = V(0.75);
    }
  }
  V acc[B];
#pragma unroll
  for (int r = 0; r < B; ++r) acc[r] = 0;
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const int J0 = lo[0] + a;
    if ((unsigned)J0 >= (unsigned)cn[0]) continue;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int J1 = lo[1] + b;
      if ((unsigned)J1 >= (unsigned)cn[1]) continue;
      const V wgt = w[0][a] * w[1][b];
      const long long P = ((long long)J0 * c.ny + J1) * c.nz + v2;
#pragma unroll
      for (int r = 0; r < B; ++r) acc[r] = fma(wgt, ec[P * B + r], acc[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < B; ++r) uf[q * B + r] += acc[r];
}

template <typename V, int B>
__global__ void __launch_bounds__(TPB) k_prolong_pc(Grid f, Grid c, const V* __restrict__ ec, V* __restrict__ uf) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= f.n) return;
  int v0, v1, v2;
  coords(q, f, v0, v1, v2);
  int J0 = v0 >> 1, J1 = v1 >> 1, J2 = v2 >> 1;
  if (J0 >= c.nx || J1 >= c.ny || J2 >= c.nz) return;
  long long P = ((long long)J0 * c.ny + J1) * c.nz + J2;
#pragma unroll
  for (int r = 0; r < B; ++r) uf[q * B + r] += ec[P * B + r];
}

__global__ void k_cast_d2f(const double* __restrict__ a, float* __restrict__ b, long long n) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = (float)a[t];
}
__global__ void k_cast_f2d(const float* __restrict__ a, double* __restrict__ b, long long n) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = (double)a[t];
}

// Off-grid coefficients must be exactly zero (SG-DIA zero padding).
__global__ void k_check_padding(Grid g, Stencil s, int B, const double* __restrict__ A, int* count) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.n) return;
  int i, j, k;
  coords(p, g, i, j, k);
  int bad = 0;
  for (int e = 0; e < s.ns; ++e) {
    if (inside3(i + s.off[e][0], j + s.off[e][1], k + s.off[e][2], g)) continue;
    const double* blk = A + (p * s.ns + e) * B * B;
    for (int t = 0; t < B * B; ++t) bad |= (blk[t] != 0.0);
  }
  if (bad) atomicAdd(count, 1);
}

// Lowered copy of a scalar matrix.  pk == K32: vals = (float)a.  pk == KBF:
// scale_p = (float)max |a_pe| over all entries, vals = bf16 round-to-
// nearest-even of a / scale_p computed in double; a zero row gets scale 1.
// split != 0 (ILU factors): lower entries (e < ec) use their own scale
// `scale`, centre and upper entries the scale `scale2` of the upper entries.
__device__ __forceinline__ float row_scale(const double* a, int e0, int e1) {
  double mx = 0.0;
  for (int e = e0; e < e1; ++e) mx = fmax(mx, fabs(a[e]));
  return mx > 0.0 ? (float)mx : 1.0f;
}

__global__ void k_lower(Grid g, Stencil s, const double* __restrict__ A, int pk, int split, void* vals, float* scale,
                        float* scale2) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.n) return;
  const double* a = A + p * s.ns;
  if (pk == K32) {
    float* v = (float*)vals + p * s.ns;
    for (int e = 0; e < s.ns; ++e) v[e] = (float)a[e];
    if (scale) scale[p] = 1.0f;
    if (scale2) scale2[p] = 1.0f;
    return;
  }
  __nv_bfloat16* v = (__nv_bfloat16*)vals + p * s.ns;
  if (!split) {
    const float sc = row_scale(a, 0, s.ns);
    scale[p] = sc;
    for (int e = 0; e < s.ns; ++e) v[e] = __double2bfloat16(a[e] / (double)sc);
    return;
  }
  const float sl = row_scale(a, 0, s.ec), su = row_scale(a, s.ec + 1, s.ns);
  scale[p] = sl;
  scale2[p] = su;
  for (int e = 0; e < s.ns; ++e) v[e] = __double2bfloat16(a[e] / (double)(e < s.ec ? sl : su));
}

// Sweep records (ilurec.cuh) of every point, from the FP64 ILU factors or
// matrix, written in the skewed layout.  Values and scales equal those of
// k_lower entry by entry (split = 1 for the ILU triangles, 0 for the matrix).
template <typename R>
struct RecBuf {
  union {
    uint4 q[R::CHUNKS];
    unsigned char b[R::BYTES];
  };
};

__device__ __forceinline__ void grid_ijk(const Grid& g, long long p, int& i, int& j, int& k) {
  k = (int)(p % g.nz);
  j = (int)((p / g.nz) % g.ny);
  i = (int)(p / ((long long)g.ny * g.nz));
}

template <int PK, int NS>
__global__ void k_ilu_records(Grid g, int SB, const double* __restrict__ LU, const double* __restrict__ udinv,
                              uint4* __restrict__ Lrec, uint4* __restrict__ Urec) {
  using Val = typename Prec<PK>::val;
  using Vec = typename Prec<PK>::vec;
  using RL = SweepRec<PK, NS, 0>;
  using RU = SweepRec<PK, NS, 1>;
  constexpr int EC = Shape<NS>::EC;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.n) return;
  const double* a = LU + p * NS;
  RecBuf<RL> L;
  RecBuf<RU> U;
  for (int c = 0; c < RL::CHUNKS; ++c) L.q[c] = make_uint4(0, 0, 0, 0);
  for (int c = 0; c < RU::CHUNKS; ++c) U.q[c] = make_uint4(0, 0, 0, 0);
  Val* lv = (Val*)L.b;
  Val* uv = (Val*)U.b;
  if constexpr (PK == KBF) {
    const float sl = row_scale(a, 0, EC), su = row_scale(a, EC + 1, NS);
    for (int e = 0; e < EC; ++e) lv[e] = __double2bfloat16(a[e] / (double)sl);
    for (int e = EC + 1; e < NS; ++e) uv[RU::slot(e)] = __double2bfloat16(a[e] / (double)su);
    *(float*)(L.b + RL::S_OFF) = sl;
    *(float*)(U.b + RU::S_OFF) = su;
  } else {
    for (int e = 0; e < EC; ++e) lv[e] = (Val)a[e];
    for (int e = EC + 1; e < NS; ++e) uv[RU::slot(e)] = (Val)a[e];
  }
  *(Vec*)(U.b + RU::D_OFF) = (Vec)udinv[p];
  int i, j, k;
  grid_ijk(g, p, i, j, k);
  const long long row = (long long)i * g.nz + skew_row(j, k, SB, g.nz);
  for (int c = 0; c < RL::CHUNKS; ++c) Lrec[(row * RL::CHUNKS + c) * g.ny + j] = L.q[c];
  for (int c = 0; c < RU::CHUNKS; ++c) Urec[(row * RU::CHUNKS + c) * g.ny + j] = U.q[c];
}

template <int PK, int NS>
__global__ void k_gs_records(Grid g, int SB, const double* __restrict__ A, const double* __restrict__ dinv,
                             uint4* __restrict__ Grec) {
  using Val = typename Prec<PK>::val;
  using Vec = typename Prec<PK>::vec;
  using RG = SweepRec<PK, NS, 2>;
  constexpr int EC = Shape<NS>::EC;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.n) return;
  const double* a = A + p * NS;
  RecBuf<RG> G;
  for (int c = 0; c < RG::CHUNKS; ++c) G.q[c] = make_uint4(0, 0, 0, 0);
  Val* v = (Val*)G.b;
  if constexpr (PK == KBF) {
    const float sc = row_scale(a, 0, NS);
    for (int e = 0; e < NS; ++e)
      if (e != EC) v[e] = __double2bfloat16(a[e] / (double)sc);
    *(float*)(G.b + RG::S_OFF) = sc;
  } else {
    for (int e = 0; e < NS; ++e)
      if (e != EC) v[e] = (Val)a[e];
  }
  *(Vec*)(G.b + RG::D_OFF) = (Vec)dinv[p];
  int i, j, k;
  grid_ijk(g, p, i, j, k);
  const long long row = (long long)i * g.nz + skew_row(j, k, SB, g.nz);
  for (int c = 0; c < RG::CHUNKS; ++c) Grec[(row * RG::CHUNKS + c) * g.ny + j] = G.q[c];
}

// Vector between natural order and the skewed layout.
template <typename T>
__global__ void k_skew_copy(Grid g, int SB, int to_skew, const T* __restrict__ src, T* __restrict__ dst, int add) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.n) return;
  int i, j, k;
  grid_ijk(g, p, i, j, k);
  const long long q = skew_slot(g, SB, i, j, k);
  if (to_skew) dst[q] = src[p];
  else dst[p] = add ? dst[p] + src[q] : src[q];
}

// Stencil entries reordered: out[p][e] = in[p][perm[e]] (BxB blocks).
__global__ void k_permute(long long n, int ns, int bb, const int* __restrict__ perm, const double* __restrict__ in,
                          double* __restrict__ out) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long total = n * ns * bb;
  if (t >= total) return;
  long long p = t / (ns * bb);
  int rem = (int)(t % (ns * bb));
  int e = rem / bb, m = rem % bb;
  out[t] = in[(p * ns + perm[e]) * bb + m];
}

__global__ void k_d2f(const double* __restrict__ a, float* __restrict__ b, long long n) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = (float)a[t];
}

// Inverse of the diagonal coefficient (scalar) or of the 3x3 diagonal block
// (Gauss-Jordan with partial pivoting on 3 rows).
__global__ void k_diag_inverse(Grid g, Stencil s, int B, const double* __restrict__ A, double* __restrict__ dinv,
                               int* err) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.n) return;
  if (B == 1) {
    double d = A[p * s.ns + s.ec];
    if (d == 0.0) { atomicCAS(err, 0, SMG_EBREAKDOWN); dinv[p] = 0.0; return; }
    dinv[p] = 1.0 / d;
    return;
  }
  double W[3][6];
  const double* D = A + (p * s.ns + s.ec) * 9;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 6; ++c) W[r][c] = c < 3 ? D[r * 3 + c] : (c - 3 == r ? 1.0 : 0.0);
  for (int col = 0; col < 3; ++col) {
    int piv = col;
    for (int r = col + 1; r < 3; ++r)
      if (fabs(W[r][col]) > fabs(W[piv][col])) piv = r;
    if (W[piv][col] == 0.0) {
      atomicCAS(err, 0, SMG_EBREAKDOWN);
      for (int t = 0; t < 9; ++t) dinv[p * 9 + t] = 0.0;
      return;
    }
    if (piv != col)
      for (int c = 0; c < 6; ++c) { double t = W[col][c]; W[col][c] = W[piv][c]; W[piv][c] = t; }
    double inv = 1.0 / W[col][col];
    for (int c = 0; c < 6; ++c) W[col][c] *= inv;
    for (int r = 0; r < 3; ++r) {
      if (r == col) continue;
      double f = W[r][col];
      for (int c = 0; c < 6; ++c) W[r][c] -= f * W[col][c];
    }
  }
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) dinv[p * 9 + r * 3 + c] = W[r][3 + c];
}

// Dense (n*B)^2 row-major assembly of the coarsest stencil matrix.
__global__ void k_assemble_dense(Grid g, Stencil s, int B, const double* __restrict__ A, double* __restrict__ M) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.n) return;
  int i, j, k;
  coords(p, g, i, j, k);
  long long N = g.n * B;
  for (int e = 0; e < s.ns; ++e) {
    if (!inside3(i + s.off[e][0], j + s.off[e][1], k + s.off[e][2], g)) continue;
    long long q = p + s.lin[e];
    for (int r = 0; r < B; ++r)
      for (int c = 0; c < B; ++c) M[(p * B + r) * N + q * B + c] = A[((p * s.ns + e) * B + r) * B + c];
  }
}

// Gauss-Jordan elimination with partial pivoting on [M | I], one pivot column
// per pair of launches: k_gj_pivot (one block) selects and swaps the pivot
// row, scales it and saves column `col` of the other rows; k_gj_elim updates
// every other row.
__global__ void k_gj_pivot(int n, int col, double* M, double* Minv, double* colbuf, int* err) {
  __shared__ double sv[1024];
  __shared__ int si[1024];
  int t = threadIdx.x;
  double best = -1.0;
  int bi = col;
  for (int r = col + t; r < n; r += blockDim.x) {
    double v = fabs(M[(long long)r * n + col]);
    if (v > best) { best = v; bi = r; }
  }
  sv[t] = best;
  si[t] = bi;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (t < h) {
      if (sv[t + h] > sv[t] || (sv[t + h] == sv[t] && si[t + h] < si[t])) { sv[t] = sv[t + h]; si[t] = si[t + h]; }
    }
    __syncthreads();
  }
  int piv = si[0];
  if (sv[0] <= 0.0) {
    if (t == 0) atomicCAS(err, 0, SMG_EBREAKDOWN);
    return;
  }
  if (piv != col) {
    for (int c = t; c < n; c += blockDim.x) {
      double a = M[(long long)col * n + c]; M[(long long)col * n + c] = M[(long long)piv * n + c];
      M[(long long)piv * n + c] = a;
      double b = Minv[(long long)col * n + c]; Minv[(long long)col * n + c] = Minv[(long long)piv * n + c];
      Minv[(long long)piv * n + c] = b;
    }
  }
  __syncthreads();
  double inv = 1.0 / M[(long long)col * n + col];
  __syncthreads();
  for (int c = t; c < n; c += blockDim.x) {
    M[(long long)col * n + c] *= inv;
    Minv[(long long)col * n + c] *= inv;
  }
  for (int r = t; r < n; r += blockDim.x) colbuf[r] = (r == col) ? 0.0 : M[(long long)r * n + col];
}

__global__ void k_gj_elim(int n, int col, double* M, double* Minv, const double* colbuf, const int* err) {
  if (*err) return;
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long total = (long long)n * 2 * n;
  if (idx >= total) return;
  int r = (int)(idx / (2 * n));
  int c = (int)(idx % (2 * n));
  double f = colbuf[r];
  if (f == 0.0) return;
  if (c < n) {
    if (c == col) { M[(long long)r * n + c] = 0.0; return; }
    // a zero in the pivot row leaves the entry unchanged: skip its read and
    // write (the columns already eliminated, and most of the inverse's
    // columns early on)
    const double pv = M[(long long)col * n + c];
    if (pv == 0.0) return;
    M[(long long)r * n + c] -= f * pv;
  } else {
    c -= n;
    const double pv = Minv[(long long)col * n + c];
    if (pv == 0.0) return;
    Minv[(long long)r * n + c] -= f * pv;
  }
}

// The same Gauss-Jordan elimination in one persistent launch (every CTA
// resident: cooperative launch).  Per column k two grid barriers:
//  (1) every CTA reduces the partial pivot candidates of all CTAs (largest
//      |M[r][k]| over r >= k, the smallest row among equal values: the choice
//      of k_gj_pivot), then swaps rows k and p and scales the new row k by
//      1 / pivot, columns spread over the whole grid;
//  (2) CTA b eliminates column k from its rows r = b, b + G, ... (the same
//      update, expression and skips as k_gj_elim) and leaves the partial
//      pivot candidate of column k + 1 among them.
// The barrier is a counter and a generation word in global memory, waited
// on with a bound; a timeout or a zero pivot ends every CTA at the next
// barrier with the error word set.
struct GjGrid {
  int n;
  double* M;
  double* Minv;
  double* part;   // [3 * gridDim.x]: candidate |value|, row and signed value of each CTA
  unsigned* bar;  // [2]: arrivals, generation (zero before the launch)
  int* err;
  unsigned long long budget_ns;
};

__device__ bool gj_grid_sync(const GjGrid& A, unsigned& gen) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    if (atomicAdd(&A.bar[0], 1u) == gridDim.x - 1) {
      atomicExch(&A.bar[0], 0u);
      __threadfence();
      atomicExch(&A.bar[1], gen + 1);
    } else {
      const unsigned long long t0 = globaltimer_ns();
      for (;;) {
        unsigned g;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(A.bar + 1) : "memory");
        if (g != gen) break;
        if (globaltimer_ns() - t0 > A.budget_ns) {
          atomicCAS(A.err, 0, DEV_ERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    s_ok = ok && ld_relaxed(A.err) == 0;
  }
  __syncthreads();
  ++gen;
  return s_ok != 0;
}

__global__ void __launch_bounds__(TPB) k_gj_persistent(GjGrid A) {
  __shared__ double sv[TPB], sw[TPB];
  __shared__ int si[TPB];
  const int n = A.n, G = gridDim.x, t = threadIdx.x;
  double* M = A.M;
  double* Minv = A.Minv;
  unsigned gen = 0;
  const long long gtid = (long long)blockIdx.x * TPB + t, gstride = (long long)G * TPB;
  for (long long idx = gtid; idx < (long long)n * n; idx += gstride) Minv[idx] = (idx / n == idx % n) ? 1.0 : 0.0;
  // partial pivot candidate of column k among this CTA's rows r >= k
  auto candidate = [&](int k) {
    double best = -1.0, bv = 0.0;
    int bi = n;
    for (int r = blockIdx.x + G * t; r < n; r += G * TPB)
      if (r >= k) {
        const double x = M[(long long)r * n + k], v = fabs(x);
        if (v > best) { best = v; bi = r; bv = x; }
      }
    sv[t] = best;
    si[t] = bi;
    sw[t] = bv;
    __syncthreads();
    for (int h = TPB / 2; h > 0; h >>= 1) {
      if (t < h && (sv[t + h] > sv[t] || (sv[t + h] == sv[t] && si[t + h] < si[t]))) {
        sv[t] = sv[t + h];
        si[t] = si[t + h];
        sw[t] = sw[t + h];
      }
      __syncthreads();
    }
    if (t == 0) {
      A.part[3 * blockIdx.x] = sv[0];
      A.part[3 * blockIdx.x + 1] = (double)si[0];
      A.part[3 * blockIdx.x + 2] = sw[0];
    }
  };
  candidate(0);
  for (int k = 0; k < n; ++k) {
    if (!gj_grid_sync(A, gen)) return;
    // (1) the pivot, from every CTA's candidate (the same answer in every CTA)
    double best = -1.0, pvs = 0.0;
    int p = n;
    for (int q = t; q < G; q += TPB) {
      const double v = A.part[3 * q];
      const int r = (int)A.part[3 * q + 1];
      if (v > best || (v == best && r < p)) { best = v; p = r; pvs = A.part[3 * q + 2]; }
    }
    sv[t] = best;
    si[t] = p;
    sw[t] = pvs;
    __syncthreads();
    for (int h = TPB / 2; h > 0; h >>= 1) {
      if (t < h && (sv[t + h] > sv[t] || (sv[t + h] == sv[t] && si[t + h] < si[t]))) {
        sv[t] = sv[t + h];
        si[t] = si[t + h];
        sw[t] = sw[t + h];
      }
      __syncthreads();
    }
    best = sv[0];
    p = si[0];
    pvs = sw[0];  // the pivot M[p][k] itself (its row is rewritten below)
    __syncthreads();
    if (!(best > 0.0)) {
      if (blockIdx.x == 0 && t == 0) atomicCAS(A.err, 0, SMG_EBREAKDOWN);
      return;
    }
    const double inv = 1.0 / pvs;
    for (long long c = gtid; c < n; c += gstride) {
      const double mk = M[(long long)k * n + c], mp = M[(long long)p * n + c];
      const double ik = Minv[(long long)k * n + c], ip = Minv[(long long)p * n + c];
      M[(long long)k * n + c] = mp * inv;
      Minv[(long long)k * n + c] = ip * inv;
      if (p != k) {
        M[(long long)p * n + c] = mk;
        Minv[(long long)p * n + c] = ik;
      }
    }
    if (!gj_grid_sync(A, gen)) return;
    // (2) eliminate column k from this CTA's rows
    const double* rk = M + (long long)k * n;
    const double* ik = Minv + (long long)k * n;
    for (int r = blockIdx.x; r < n; r += G) {
      if (r == k) continue;
      double* rr = M + (long long)r * n;
      const double f = rr[k];
      if (f == 0.0) continue;
      double* ir = Minv + (long long)r * n;
      __syncthreads();  // every thread has read rr[k] before it is cleared
      for (int c = t; c < n; c += TPB) {
        if (c == k) {
          rr[c] = 0.0;
          continue;
        }
        const double pv = rk[c];
        if (pv == 0.0) continue;
        rr[c] -= f * pv;
      }
      for (int c = t; c < n; c += TPB) {
        const double pv = ik[c];
        if (pv == 0.0) continue;
        ir[c] -= f * pv;
      }
    }
    __syncthreads();
    if (k + 1 < n) candidate(k + 1);
  }
}

__global__ void k_set_identity(int n, double* Minv) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  Minv[idx] = (idx / n == idx % n) ? 1.0 : 0.0;
}

// y = Minv x: one warp per row, coalesced row reads, fixed-order shuffle sum.
__global__ void k_dense_matvec(int n, const double* __restrict__ Minv, const double* __restrict__ x,
                               double* __restrict__ y) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double* row = Minv + (long long)warp * n;
  double acc = 0.0;
  for (int c = lane; c < n; c += 32) acc = fma(row[c], x[c], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) y[warp] = acc;
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
cudaError_t launch_spmv(const LevelView& L, const void* x, const void* b, void* y, int mode, cudaStream_t st,
                        int skew) {
  int nb = div_up(L.g.n, TPB);
  if (L.B == 3) {
    if (skew) return cudaErrorInvalidValue;  // block levels have no skewed layout
    if (L.pk == K64)
      k_spmv3<double><<<nb, TPB, 0, st>>>(L.g, L.s, (const double*)L.A, (const double*)x, (const double*)b,
                                          (double*)y, mode);
    else
      k_spmv3<float><<<nb, TPB, 0, st>>>(L.g, L.s, (const float*)L.A, (const float*)x, (const float*)b, (float*)y,
                                         mode);
    return cudaGetLastError();
  }
  const bool aligned16 = ((uintptr_t)L.A & 15u) == 0;  // the staged kernel copies 16-byte units
#define SPMV_CASE(PK)                                                                                          \
  {                                                                                                            \
    using Val = typename Prec<PK>::val;                                                                        \
    using Vec = typename Prec<PK>::vec;                                                                        \
    if (L.s.ns == 27 && PK == K32 && aligned16)                                                                \
      k_spmv1s<PK, 27><<<nb, TPB, 0, st>>>(L.g, L.s, (const Val*)L.A, L.scale, (const Vec*)x, (const Vec*)b,   \
                                           (Vec*)y, mode, skew);                                               \
    else if (L.s.ns == 7 && PK == K32 && aligned16)                                                            \
      k_spmv1s<PK, 7><<<nb, TPB, 0, st>>>(L.g, L.s, (const Val*)L.A, L.scale, (const Vec*)x, (const Vec*)b,    \
                                          (Vec*)y, mode, skew);                                                \
    else if (L.s.ns == 27)                                                                                     \
      k_spmv1<PK, 27><<<nb, TPB, 0, st>>>(L.g, L.s, (const Val*)L.A, L.scale, (const Vec*)x, (const Vec*)b,    \
                                          (Vec*)y, mode, skew);                                                      \
    else if (L.s.ns == 7)                                                                                      \
      k_spmv1<PK, 7><<<nb, TPB, 0, st>>>(L.g, L.s, (const Val*)L.A, L.scale, (const Vec*)x, (const Vec*)b,     \
                                         (Vec*)y, mode, skew);                                                       \
    else                                                                                                       \
      k_spmv1_any<PK><<<nb, TPB, 0, st>>>(L.g, L.s, (const Val*)L.A, L.scale, (const Vec*)x, (const Vec*)b,    \
                                          (Vec*)y, mode, skew);                                                      \
  }
  if (L.pk == K64) SPMV_CASE(K64)
  else if (L.pk == K32) SPMV_CASE(K32)
  else SPMV_CASE(KBF)
#undef SPMV_CASE
  smg_count_launch(1);
  return cudaGetLastError();
}

static Grid coarse_of(Grid f, int transfer) {
  Grid c{f.nx / 2, f.ny / 2, transfer == SMG_TRANSFER_C16C_XY ? f.nz : f.nz / 2, 0};
  c.n = (long long)c.nx * c.ny * c.nz;
  return c;
}

cudaError_t launch_restrict(int transfer, Grid f, int B, int pk, const void* rf, void* fc, cudaStream_t st) {
  Grid c = coarse_of(f, transfer);
  int nb = div_up(c.n, TPB);
  bool dbl = pk == K64;
#define RCASE(V, BB)                                                                                   \
  if (transfer == SMG_TRANSFER_FW27V)                                                                  \
    k_restrict_fw<V, BB><<<nb, TPB, 0, st>>>(f, c, (const V*)rf, (V*)fc);                              \
  else if (transfer == SMG_TRANSFER_C16C_XY)                                                           \
    k_restrict_xy<V, BB><<<nb, TPB, 0, st>>>(f, c, (const V*)rf, (V*)fc);                              \
  else                                                                                                 \
    k_restrict_pc<V, BB><<<nb, TPB, 0, st>>>(f, c, (const V*)rf, (V*)fc);
  if (dbl) {
    if (B == 1) { RCASE(double, 1) } else { RCASE(double, 3) }
  } else {
    if (B == 1) { RCASE(float, 1) } else { RCASE(float, 3) }
  }
#undef RCASE
  smg_count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_resid_restrict(const LevelView& L, int transfer, const void* x, const void* b, void* fc,
                                  cudaStream_t st) {
  const bool fw = transfer == SMG_TRANSFER_FW27V;
  if (L.B != 1 || !(fw || transfer == SMG_TRANSFER_PC8C || transfer == SMG_TRANSFER_C64C) ||
      !(L.s.ns == 7 || L.s.ns == 19 || L.s.ns == 27))
    return cudaErrorNotSupported;
  const Grid c = coarse_of(L.g, transfer);
  if (!fw && (L.g.nx != 2 * c.nx || L.g.ny != 2 * c.ny || L.g.nz != 2 * c.nz)) return cudaErrorNotSupported;
  const long long tiles = (long long)((c.ny + kRrTJ - 1) / kRrTJ) * ((c.nz + kRrTK - 1) / kRrTK);
  // enough CTAs for two per SM: split the coarse x-planes into chunks
  int dev = 0, nsm = 0;
  cudaError_t ae = cudaGetDevice(&dev);
  if (ae == cudaSuccess) ae = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (ae != cudaSuccess) return ae;
  const long long want = (2LL * nsm + tiles - 1) / tiles;
  const int chunks = (int)std::max(1LL, std::min((long long)c.nx, want));
  const int ci = (c.nx + chunks - 1) / chunks;
  const int nb = (int)(tiles * ((c.nx + ci - 1) / ci));
#define RR_CASE(PK, NSV)                                                                                      \
  {                                                                                                           \
    using Val = typename Prec<PK>::val;                                                                       \
    using Vec = typename Prec<PK>::vec;                                                                       \
    if (fw)                                                                                                   \
      k_resid_restrict<PK, NSV, true><<<nb, TPB, 0, st>>>(L.g, c, L.s, (const Val*)L.A, L.scale, (const Vec*)x,  \
                                                         (const Vec*)b, (Vec*)fc, ci);                        \
    else                                                                                                      \
      k_resid_restrict<PK, NSV, false><<<nb, TPB, 0, st>>>(L.g, c, L.s, (const Val*)L.A, L.scale, (const Vec*)x, \
                                                          (const Vec*)b, (Vec*)fc, ci);                       \
  }
#define RR_NS(PK)                           \
  if (L.s.ns == 27) RR_CASE(PK, 27)         \
  else if (L.s.ns == 19) RR_CASE(PK, 19)    \
  else RR_CASE(PK, 7)
  if (L.pk == K64) { RR_NS(K64) }
  else if (L.pk == K32) { RR_NS(K32) }
  else { RR_NS(KBF) }
#undef RR_NS
#undef RR_CASE
  smg_count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_prolong_add(int transfer, Grid f, int B, int pk, const void* ec, void* uf, cudaStream_t st) {
  Grid c = coarse_of(f, transfer);
  // full weighting: one thread per coarse cell and its far neighbours
  // ((nc + 1)^3 owners of 2 x 2 x 2 fine points); the others one per fine point
  int nb = transfer == SMG_TRANSFER_FW27V ? div_up((long long)(c.nx + 1) * (c.ny + 1) * (c.nz + 1), TPB)
                                          : div_up(f.n, TPB);
  bool dbl = pk == K64;
#define PCASE(V, BB)                                                                                   \
  if (transfer == SMG_TRANSFER_FW27V)                                                                  \
    k_prolong_fw<V, BB><<<nb, TPB, 0, st>>>(f, c, (const V*)ec, (V*)uf);                               \
  else if (transfer == SMG_TRANSFER_C64C)                                                              \
    k_prolong_c64<V, BB><<<nb, TPB, 0, st>>>(f, c, (const V*)ec, (V*)uf);                              \
  else if (transfer == SMG_TRANSFER_C16C_XY)                                                           \
    k_prolong_xy<V, BB><<<nb, TPB, 0, st>>>(f, c, (const V*)ec, (V*)uf);                               \
  else                                                                                                 \
    k_prolong_pc<V, BB><<<nb, TPB, 0, st>>>(f, c, (const V*)ec, (V*)uf);
  if (dbl) {
    if (B == 1) { PCASE(double, 1) } else { PCASE(double, 3) }
  } else {
    if (B == 1) { PCASE(float, 1) } else { PCASE(float, 3) }
  }
#undef PCASE
  smg_count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_cast_d2f(const double* a, float* b, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_cast_d2f<<<div_up(n, TPB), TPB, 0, st>>>(a, b, n);
  smg_count_launch(1);
  return cudaGetLastError();
}
cudaError_t launch_cast_f2d(const float* a, double* b, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_cast_f2d<<<div_up(n, TPB), TPB, 0, st>>>(a, b, n);
  smg_count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_check_padding(Grid g, const Stencil& s, int B, const double* A, int* count, cudaStream_t st) {
  k_check_padding<<<div_up(g.n, TPB), TPB, 0, st>>>(g, s, B, A, count);
  smg_count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_lower_matrix(Grid g, const Stencil& s, const double* A, int pk, int split, void* vals, float* scale,
                                float* scale2, cudaStream_t st) {
  k_lower<<<div_up(g.n, TPB), TPB, 0, st>>>(g, s, A, pk, split, vals, scale, scale2);
  smg_count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_ilu_records(Grid g, int ns, int SB, int pk, const double* LU, const double* udinv, void* Lrec,
                               void* Urec, cudaStream_t st) {
  const int nb = div_up(g.n, TPB);
  uint4 *l = (uint4*)Lrec, *u = (uint4*)Urec;
#define REC_(PK, NS) k_ilu_records<PK, NS><<<nb, TPB, 0, st>>>(g, SB, LU, udinv, l, u)
  if (ns != 7 && ns != 19 && ns != 27) return cudaErrorInvalidValue;
  if (pk == K64) {
    if (ns == 27) REC_(K64, 27); else if (ns == 19) REC_(K64, 19); else REC_(K64, 7);
  } else if (pk == K32) {
    if (ns == 27) REC_(K32, 27); else if (ns == 19) REC_(K32, 19); else REC_(K32, 7);
  } else {
    if (ns == 27) REC_(KBF, 27); else if (ns == 19) REC_(KBF, 19); else REC_(KBF, 7);
  }
#undef REC_
  smg_count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_gs_records(Grid g, int ns, int SB, int pk, const double* A, const double* dinv, void* Grec,
                              cudaStream_t st) {
  const int nb = div_up(g.n, TPB);
  uint4* r = (uint4*)Grec;
#define REC_(PK, NS) k_gs_records<PK, NS><<<nb, TPB, 0, st>>>(g, SB, A, dinv, r)
  if (ns != 7 && ns != 19 && ns != 27) return cudaErrorInvalidValue;
  if (pk == K64) {
    if (ns == 27) REC_(K64, 27); else if (ns == 19) REC_(K64, 19); else REC_(K64, 7);
  } else if (pk == K32) {
    if (ns == 27) REC_(K32, 27); else if (ns == 19) REC_(K32, 19); else REC_(K32, 7);
  } else {
    if (ns == 27) REC_(KBF, 27); else if (ns == 19) REC_(KBF, 19); else REC_(KBF, 7);
  }
#undef REC_
  smg_count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_skew_copy(Grid g, int SB, int vb, bool to_skew, const void* src, void* dst, bool add,
                             cudaStream_t st) {
  const int nb = div_up(g.n, TPB);
  if (vb == 8) k_skew_copy<double><<<nb, TPB, 0, st>>>(g, SB, to_skew, (const double*)src, (double*)dst, add);
  else k_skew_copy<float><<<nb, TPB, 0, st>>>(g, SB, to_skew, (const float*)src, (float*)dst, add);
  smg_count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_permute(long long n, int ns, int bb, const int* perm, const double* in, double* out,
                           cudaStream_t st) {
  long long total = n * ns * bb;
  if (total <= 0) return cudaSuccess;
  k_permute<<<div_up(total, TPB), TPB, 0, st>>>(n, ns, bb, perm, in, out);
  smg_count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_d2f_array(const double* a, float* b, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_d2f<<<div_up(n, TPB), TPB, 0, st>>>(a, b, n);
  smg_count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_diag_inverse(Grid g, const Stencil& s, int B, const double* A, double* dinv, int* err,
                                cudaStream_t st) {
  k_diag_inverse<<<div_up(g.n, TPB), TPB, 0, st>>>(g, s, B, A, dinv, err);
  smg_count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_assemble_dense(Grid g, const Stencil& s, int B, const double* A, double* M, cudaStream_t st) {
  long long N = g.n * B;
  cudaError_t e = cudaMemsetAsync(M, 0, sizeof(double) * N * N, st);
  if (e != cudaSuccess) return e;
  k_assemble_dense<<<div_up(g.n, TPB), TPB, 0, st>>>(g, s, B, A, M);
  smg_count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_gauss_jordan(int n, double* M, double* Minv, double* colbuf, int* err, cudaStream_t st,
                                double* scratch, unsigned long long budget_ns) {
  if (scratch) {
    // one persistent cooperative launch (every CTA resident), at most
    // kGjMaxBlocks CTAs; the per-column launches below when it cannot run
    int dev = 0, nsm = 0, per = 0, coop = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_gj_persistent, TPB, 0);
    if (e != cudaSuccess) return e;
    if (coop && per > 0) {
      GjGrid A{n, M, Minv, scratch, (unsigned*)(scratch + 3 * kGjMaxBlocks), err, budget_ns};
      e = cudaMemsetAsync(A.bar, 0, 2 * sizeof(unsigned), st);
      if (e != cudaSuccess) return e;
      const int grid = std::min(nsm * per, kGjMaxBlocks);
      void* args[] = {&A};
      e = cudaLaunchCooperativeKernel((const void*)k_gj_persistent, grid, TPB, args, 0, st);
      smg_count_launch(1);
      if (e == cudaSuccess) return cudaSuccess;
      if (e != cudaErrorCooperativeLaunchTooLarge) return e;
      (void)cudaGetLastError();
    }
  }
  k_set_identity<<<div_up((long long)n * n, TPB), TPB, 0, st>>>(n, Minv);
  int nb = div_up((long long)n * 2 * n, TPB);
  for (int col = 0; col < n; ++col) {
    k_gj_pivot<<<1, 1024, 0, st>>>(n, col, M, Minv, colbuf, err);
    k_gj_elim<<<nb, TPB, 0, st>>>(n, col, M, Minv, colbuf, err);
  }
  smg_count_launch(1 + 2LL * n);
  return cudaGetLastError();
}

cudaError_t launch_dense_matvec(int n, const double* Minv, const double* x, double* y, cudaStream_t st) {
  k_dense_matvec<<<div_up((long long)n * 32, TPB), TPB, 0, st>>>(n, Minv, x, y);
  smg_count_launch(1);
  return cudaGetLastError();
}
