// Learned post-smoother (not in the paper): a three-layer 3x3x3 convolutional
// network applied on the finest level after the V-cycle, and its training.
//
// Network: conv(2->16) + ReLU, conv(16->16) + ReLU, conv(16->1).  Every
// convolution is an implicit GEMM on the tensor cores: BF16 operands, FP32
// accumulation (mma.sync m16n8k16).  Activations are stored channels-last,
// 16 BF16 channels per voxel (32 bytes), the 2-channel input padded with
// zeros; voxel index p = (i*ny + j)*nz + k as everywhere else.
//
// Parameters (FP32 master copy, 8241 values, PyTorch conv3d order):
//   W1[16][2][3][3][3] b1[16] W2[16][16][3][3][3] b2[16] W3[1][16][3][3][3] b3[1]
// with tap (a,b,c) multiplying the input at offset (a-1, b-1, c-1)
// (cross-correlation, zero padding).
#include "cnn.cuh"

namespace {

constexpr int TX = 2, TY = 4, TZ = 32;           // output brick of one CTA: 256 voxels
constexpr int HX = TX + 2, HY = TY + 2, HZ = TZ + 2;
constexpr int NTHR = 256;                         // 8 warps, 2 M-tiles (16 voxels) each
constexpr int CH = 16;

__device__ __forceinline__ unsigned pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Shared-memory rows of 16 BF16 channels (32 bytes) keep their two 16-byte
// halves swapped on every other group of four rows.  A warp's fragment load
// reads one 4-byte word from 8 consecutive rows; without the swap rows r and
// r+4 fall on the same bank (2-way conflict), with it the 8 rows cover all
// 32 banks.  smem_idx gives the element offset of channel c in row r.
__device__ __forceinline__ int smem_idx(int r, int c) { return r * CH + ((((c >> 3) ^ (r >> 2)) & 1) << 3) + (c & 7); }

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const __nv_bfloat16* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"((unsigned)__cvta_generic_to_shared(p)));
}
__device__ __forceinline__ void ldsm_x2(unsigned (&r)[4], const __nv_bfloat16* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];"
               : "=r"(r[0]), "=r"(r[1])
               : "r"((unsigned)__cvta_generic_to_shared(p)));
  r[2] = r[3] = 0u;
}

struct Tile {
  int x0, y0, z0;
};

__device__ __forceinline__ Tile tile_of(const CnnDims& d) {
  const int tz = (d.nz + TZ - 1) / TZ, ty = (d.ny + TY - 1) / TY;
  const int b = blockIdx.x;
  Tile t;
  t.z0 = (b % tz) * TZ;
  t.y0 = ((b / tz) % ty) * TY;
  t.x0 = (b / (tz * ty)) * TX;
  return t;
}

// Loads the input brick with a one-voxel halo (zero outside the grid).
__device__ __forceinline__ void load_brick(const CnnDims& d, const Tile& T, const __nv_bfloat16* __restrict__ in,
                                           __nv_bfloat16* s_in) {
  const int nvox = HX * HY * HZ;
  for (int q = threadIdx.x; q < nvox * 2; q += NTHR) {
    const int v = q >> 1, half = q & 1;
    const int hz = v % HZ, hy = (v / HZ) % HY, hx = v / (HZ * HY);
    const int x = T.x0 + hx - 1, y = T.y0 + hy - 1, z = T.z0 + hz - 1;
    uint4 val = make_uint4(0, 0, 0, 0);
    if ((unsigned)x < (unsigned)d.nx && (unsigned)y < (unsigned)d.ny && (unsigned)z < (unsigned)d.nz) {
      const long long p = ((long long)x * d.ny + y) * d.nz + z;
      val = reinterpret_cast<const uint4*>(in + p * CH)[half];
    }
    reinterpret_cast<uint4*>(s_in + (size_t)v * CH)[half ^ ((v >> 2) & 1)] = val;
  }
}

// ---------------------------------------------------------------------------
// Forward convolution (also the transposed convolution of the backward pass,
// with the flipped, channel-transposed weights).  NT = number of 8-wide
// output-channel tiles (2 for 16 outputs, 1 for the last layer).
// ---------------------------------------------------------------------------
// Halo-brick row of the input voxel at tap t (0..26) of output row m0 of an
// M tile (xl, yl, zhalf).
__device__ __forceinline__ int tap_row(int t, int xl, int yl, int zh) {
  const int dx = t / 9 - 1, dy = (t / 3) % 3 - 1, dz = t % 3 - 1;
  return ((xl + dx + 1) * HY + (yl + dy + 1)) * HZ + zh * 16 + dz + 1;
}

// IN2: the input has 2 channels (the first layer).  Its K dimension is then
// packed as 27 taps x 2 channels (padded to 64: four k-steps of 16) instead
// of 27 taps x 16 channels, a seventh of the MMA work; Wt is [4][co 16][k 16]
// with k = 2 * (tap - 8 * kstep) + ci.
template <int EPI, int NT, bool IN2>
__global__ void __launch_bounds__(NTHR) k_conv(CnnDims d, const __nv_bfloat16* __restrict__ in,
                                               const __nv_bfloat16* __restrict__ Wt,  // [27][co 16][ci 16]
                                               const float* __restrict__ bias,       // [16] or null
                                               const __nv_bfloat16* __restrict__ mask, void* out) {
  constexpr int WROWS = IN2 ? 4 * CH : 27 * CH;  // weight rows of 16 elements
  __shared__ __align__(16) __nv_bfloat16 s_in[HX * HY * HZ * CH];
  __shared__ __align__(16) __nv_bfloat16 s_w[WROWS * CH];
  const Tile T = tile_of(d);
  for (int q = threadIdx.x; q < WROWS * CH / 8; q += NTHR)
    reinterpret_cast<uint4*>(s_w)[q ^ (((q >> 3) & 1))] = reinterpret_cast<const uint4*>(Wt)[q];
  load_brick(d, T, in, s_in);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gid = lane >> 2, tig = lane & 3;
  // the warp's two M tiles: 16 voxels along z each (z half mt) of column
  // (xl, yl) of the brick
  const int yl = warp & 3, xl = warp >> 2;
  // ldmatrix addressing: lane l gives row (l & 7) of 8x8 matrix (l >> 3)
  const int lr = lane & 7, lm = lane >> 3;
  float acc[2][NT][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) acc[mt][nt][0] = acc[mt][nt][1] = acc[mt][nt][2] = acc[mt][nt][3] = 0.f;
  if (IN2) {
    // k-step kk: this thread's columns k = 2*tig + {0,1} are tap 8kk + tig,
    // columns k + 8 are tap 8kk + 4 + tig; channels 0 and 1 of each
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      unsigned b[4];
      ldsm_x4(b, s_w + smem_idx(kk * CH + (lm >> 1) * 8 + lr, (lm & 1) * 8));
      const int t0 = kk * 8 + tig, t1 = t0 + 4;
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        unsigned a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        if (t0 < 27) {
          const int h = tap_row(t0, xl, yl, mt);
          a0 = *reinterpret_cast<const unsigned*>(s_in + smem_idx(h + gid, 0));
          a1 = *reinterpret_cast<const unsigned*>(s_in + smem_idx(h + gid + 8, 0));
        }
        if (t1 < 27) {
          const int h = tap_row(t1, xl, yl, mt);
          a2 = *reinterpret_cast<const unsigned*>(s_in + smem_idx(h + gid, 0));
          a3 = *reinterpret_cast<const unsigned*>(s_in + smem_idx(h + gid + 8, 0));
        }
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) mma_bf16(acc[mt][nt], a0, a1, a2, a3, b[2 * nt], b[2 * nt + 1]);
      }
    }
  } else {
#pragma unroll 3
    for (int t = 0; t < 27; ++t) {
      // B: (n 0-7, k 0-7), (n 0-7, k 8-15), (n 8-15, k 0-7), (n 8-15, k 8-15)
      unsigned b[4];
      if (NT == 2) ldsm_x4(b, s_w + smem_idx(t * CH + (lm >> 1) * 8 + lr, (lm & 1) * 8));
      else ldsm_x2(b, s_w + smem_idx(t * CH + lr, (lm & 1) * 8));
      const int hb = tap_row(t, xl, yl, 0);
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        // A: (m 0-7, k 0-7), (m 8-15, k 0-7), (m 0-7, k 8-15), (m 8-15, k 8-15)
        unsigned a[4];
        ldsm_x4(a, s_in + smem_idx(hb + mt * 16 + lr + (lm & 1) * 8, (lm >> 1) * 8));
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) mma_bf16(acc[mt][nt], a[0], a[1], a[2], a[3], b[2 * nt], b[2 * nt + 1]);
      }
    }
  }
  for (int mt = 0; mt < 2; ++mt) {
    const int zh = mt;
    // epilogue: rows gid and gid+8 (voxels), columns tig*2, tig*2+1 (+8 nt)
    const int x = T.x0 + xl, y = T.y0 + yl;
#pragma unroll
    for (int hr = 0; hr < 2; ++hr) {
      const int z = T.z0 + zh * 16 + gid + hr * 8;
      if (x >= d.nx || y >= d.ny || z >= d.nz) continue;
      const long long p = ((long long)x * d.ny + y) * d.nz + z;
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int co = nt * 8 + tig * 2;
        float v0 = acc[mt][nt][hr * 2], v1 = acc[mt][nt][hr * 2 + 1];
        if (bias) {
          v0 += bias[co];
          v1 += bias[co + 1];
        }
        if (EPI == CNN_EPI_OUT0_F32) {
          if (nt == 0 && tig == 0) reinterpret_cast<float*>(out)[p] = v0;
        } else {
          if (EPI == CNN_EPI_RELU) {
            v0 = fmaxf(v0, 0.f);
            v1 = fmaxf(v1, 0.f);
          } else if (EPI == CNN_EPI_MASK) {
            const unsigned mk = *reinterpret_cast<const unsigned*>(mask + p * CH + co);
            if (!(__bfloat162float(__ushort_as_bfloat16(mk & 0xffff)) > 0.f)) v0 = 0.f;
            if (!(__bfloat162float(__ushort_as_bfloat16(mk >> 16)) > 0.f)) v1 = 0.f;
          }
          *reinterpret_cast<unsigned*>(reinterpret_cast<__nv_bfloat16*>(out) + p * CH + co) =
              pack2(__float2bfloat16(v0), __float2bfloat16(v1));
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Weight gradient of one layer over the CTA's brick, all 27 taps:
//   gW[t][ci][co] = sum_v in[v + d_t][ci] * g[v][co],  gb[co] = sum_v g[v][co]
// as GEMMs with M = ci, N = co and K = the brick's voxels; per-CTA partials
// are written to `part` ([blocks][27*256 + 16]) and summed in block order by
// k_reduce_grad.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NTHR) k_conv_wgrad(CnnDims d, const __nv_bfloat16* __restrict__ in,
                                                     const __nv_bfloat16* __restrict__ g, float* __restrict__ part) {
  __shared__ __align__(16) __nv_bfloat16 s_in[HX * HY * HZ * CH];
  __shared__ __align__(16) __nv_bfloat16 s_g[TX * TY * TZ * CH];
  const Tile T = tile_of(d);
  load_brick(d, T, in, s_in);
  for (int q = threadIdx.x; q < TX * TY * TZ * 2; q += NTHR) {
    const int v = q >> 1, half = q & 1;
    const int zz = v % TZ, yy = (v / TZ) % TY, xx = v / (TZ * TY);
    const int x = T.x0 + xx, y = T.y0 + yy, z = T.z0 + zz;
    uint4 val = make_uint4(0, 0, 0, 0);
    if (x < d.nx && y < d.ny && z < d.nz) {
      const long long p = ((long long)x * d.ny + y) * d.nz + z;
      val = reinterpret_cast<const uint4*>(g + p * CH)[half];
    }
    reinterpret_cast<uint4*>(s_g + (size_t)v * CH)[half ^ ((v >> 2) & 1)] = val;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gid = lane >> 2, tig = lane & 3;
  float* out = part + (size_t)blockIdx.x * (27 * CH * CH + CH);
  for (int t = warp; t < 27; t += NTHR / 32) {
    const int dx = t / 9 - 1, dy = (t / 3) % 3 - 1, dz = t % 3 - 1;
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    for (int ks = 0; ks < TX * TY * TZ / 16; ++ks) {
      // 16 voxels of this k-step: a run of 16 along z
      const int zh = ks & 1, yl = (ks >> 1) & 3, xl = ks >> 3;
      const int gbase = (xl * TY + yl) * TZ + zh * 16;
      const int hbase = ((xl + dx + 1) * HY + (yl + dy + 1)) * HZ + zh * 16 + dz + 1;
      const int k0 = tig * 2, k1 = tig * 2 + 1;
      // A[m = ci][k = voxel]
      const unsigned a0 = pack2(s_in[smem_idx(hbase + k0, gid)], s_in[smem_idx(hbase + k1, gid)]);
      const unsigned a1 = pack2(s_in[smem_idx(hbase + k0, gid + 8)], s_in[smem_idx(hbase + k1, gid + 8)]);
      const unsigned a2 = pack2(s_in[smem_idx(hbase + k0 + 8, gid)], s_in[smem_idx(hbase + k1 + 8, gid)]);
      const unsigned a3 = pack2(s_in[smem_idx(hbase + k0 + 8, gid + 8)], s_in[smem_idx(hbase + k1 + 8, gid + 8)]);
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        // B[k = voxel][n = co]
        const int co = nt * 8 + gid;
        const unsigned b0 = pack2(s_g[smem_idx(gbase + k0, co)], s_g[smem_idx(gbase + k1, co)]);
        const unsigned b1 = pack2(s_g[smem_idx(gbase + k0 + 8, co)], s_g[smem_idx(gbase + k1 + 8, co)]);
        mma_bf16(acc[nt], a0, a1, a2, a3, b0, b1);
      }
    }
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int hr = 0; hr < 2; ++hr) {
        const int ci = gid + hr * 8, co = nt * 8 + tig * 2;
        out[(t * CH + ci) * CH + co] = acc[nt][hr * 2];
        out[(t * CH + ci) * CH + co + 1] = acc[nt][hr * 2 + 1];
      }
  }
  // bias gradient: column sums of g over the brick
  if (threadIdx.x < CH) {
    float s = 0.f;
    for (int v = 0; v < TX * TY * TZ; ++v) s += __bfloat162float(s_g[smem_idx(v, threadIdx.x)]);
    out[27 * CH * CH + threadIdx.x] = s;
  }
}

// Sums the per-CTA partials in block order and adds them, in the master
// parameter layout, to grad (FP32, 8241 entries) for layer `layer`.
__global__ void k_reduce_grad(int nblocks, const float* __restrict__ part, int layer, float* __restrict__ grad) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;  // index into [27][16][16] + 16
  if (q >= 27 * CH * CH + CH) return;
  float s = 0.f;
  for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * (27 * CH * CH + CH) + q];
  const int cin = cnn_cin(layer), cout = cnn_cout(layer);
  const int woff = cnn_woff(layer), boff = woff + cout * cin * 27;
  if (q < 27 * CH * CH) {
    const int t = q / (CH * CH), ci = (q / CH) % CH, co = q % CH;
    if (ci < cin && co < cout) grad[woff + (co * cin + ci) * 27 + t] += s;
  } else {
    const int co = q - 27 * CH * CH;
    if (co < cout) grad[boff + co] += s;
  }
}

// Packs FP32 master parameters into the kernels' BF16 layouts:
//   fwd[l][t][co][ci] = W_l[co][ci][t]          (zero padded to 16 x 16)
//   bwd[l][t][ci][co] = W_l[co][ci][26 - t]     (flipped taps, channels swapped)
// and FP32 biases padded to 16.
__global__ void k_pack(const float* __restrict__ theta, __nv_bfloat16* __restrict__ fwd, __nv_bfloat16* __restrict__ bwd,
                       float* __restrict__ bias, __nv_bfloat16* __restrict__ fwd1) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < 4 * CH * CH) {
    // first layer, K packed as (tap, channel): fwd1[kk][co][k], tap = 8kk + k/2
    const int kk = q / (CH * CH), co = (q / CH) % CH, k = q % CH;
    const int tap = kk * 8 + k / 2, ci = k % 2;
    fwd1[q] = __float2bfloat16(tap < 27 ? theta[cnn_woff(0) + (co * cnn_cin(0) + ci) * 27 + tap] : 0.f);
  }
  if (q < 3 * CH) {
    const int l = q / CH, co = q % CH;
    bias[q] = co < cnn_cout(l) ? theta[cnn_woff(l) + cnn_cout(l) * cnn_cin(l) * 27 + co] : 0.f;
  }
  if (q >= 3 * 27 * CH * CH) return;
  const int l = q / (27 * CH * CH), r = q % (27 * CH * CH);
  const int t = r / (CH * CH), a = (r / CH) % CH, c = r % CH;  // fwd: a = co, c = ci
  const int cin = cnn_cin(l), cout = cnn_cout(l), off = cnn_woff(l);
  const float wf = (a < cout && c < cin) ? theta[off + (a * cin + c) * 27 + t] : 0.f;
  fwd[q] = __float2bfloat16(wf);
  // bwd entry [t][ci = a][co = c] of the transposed convolution
  const float wb = (c < cout && a < cin) ? theta[off + (c * cin + a) * 27 + (26 - t)] : 0.f;
  bwd[q] = __float2bfloat16(wb);
}

// act0[p] = (bf16(r[p] * inv_s), bf16(logk[p]), 0, ..., 0); inv_s read from
// device memory (the reciprocal RMS of r) when scale_dev != null.
__global__ void k_pack_input(long long n, const double* __restrict__ r, const double* __restrict__ logk,
                             const double* __restrict__ scale_dev, double inv_s_host, __nv_bfloat16* __restrict__ act0) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const double inv_s = scale_dev ? *scale_dev : inv_s_host;
  uint4 lo = make_uint4(pack2(__double2bfloat16(r[p] * inv_s), __double2bfloat16(logk[p])), 0, 0, 0);
  reinterpret_cast<uint4*>(act0 + p * CH)[0] = lo;
  reinterpret_cast<uint4*>(act0 + p * CH)[1] = make_uint4(0, 0, 0, 0);
}

// Training input: FP32 [2][n] sample planes -> act0.
__global__ void k_pack_input_f32(long long n, const float* __restrict__ in2, __nv_bfloat16* __restrict__ act0) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  uint4 lo = make_uint4(pack2(__float2bfloat16(in2[p]), __float2bfloat16(in2[n + p])), 0, 0, 0);
  reinterpret_cast<uint4*>(act0 + p * CH)[0] = lo;
  reinterpret_cast<uint4*>(act0 + p * CH)[1] = make_uint4(0, 0, 0, 0);
}

// loss += sum (y - t)^2 / n (one partial per block, summed in block order by
// the caller's reduction); g[p] = 2 (y - t) / n as channel 0 of a 16-channel
// BF16 volume (the other channels are kept zero).
__global__ void k_mse(long long n, const float* __restrict__ y, const float* __restrict__ tgt,
                      __nv_bfloat16* __restrict__ g16, float* __restrict__ loss_part) {
  __shared__ float sh[256];
  float s = 0.f;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    const float dlt = y[p] - tgt[p];
    s += dlt * dlt;
    const uint4 v = make_uint4(pack2(__float2bfloat16(2.f * dlt / (float)n), __float2bfloat16(0.f)), 0, 0, 0);
    reinterpret_cast<uint4*>(g16 + p * CH)[0] = v;
    reinterpret_cast<uint4*>(g16 + p * CH)[1] = make_uint4(0, 0, 0, 0);
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss_part[blockIdx.x] = sh[0] / (float)n;
}

__global__ void k_sum_in_order(int n, const float* __restrict__ part, float* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < n; ++i) s += part[i];
    *out += s;
  }
}

// Adam (Kingma & Ba) with bias correction on the FP32 master parameters;
// the gradient is multiplied by gscale (1 / batch size) first.
__global__ void k_adam(int n, float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ grad, int t, float lr, float b1, float b2, float eps, float gscale) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const float g = grad[q] * gscale;
  const float mm = b1 * m[q] + (1.f - b1) * g;
  const float vv = b2 * v[q] + (1.f - b2) * g * g;
  m[q] = mm;
  v[q] = vv;
  const float mh = mm / (1.f - powf(b1, (float)t));
  const float vh = vv / (1.f - powf(b2, (float)t));
  theta[q] -= lr * mh / (sqrtf(vh) + eps);
}

int conv_blocks(const CnnDims& d) {
  return ((d.nx + TX - 1) / TX) * ((d.ny + TY - 1) / TY) * ((d.nz + TZ - 1) / TZ);
}

}  // namespace

size_t cnn_partials_floats(const CnnDims& d) { return (size_t)conv_blocks(d) * (27 * CH * CH + CH); }

cudaError_t cnn_pack(const float* theta, CnnPacked& pk, cudaStream_t st) {
  k_pack<<<(3 * 27 * CH * CH + 255) / 256, 256, 0, st>>>(theta, pk.fwd, pk.bwd, pk.bias, pk.fwd1);
  smg_count_launch(1);
  return cudaGetLastError();
}

cudaError_t cnn_conv(const CnnDims& d, int epi, int ntiles, const __nv_bfloat16* in, const __nv_bfloat16* W,
                     const float* bias, const __nv_bfloat16* mask, void* out, cudaStream_t st) {
  const int nb = conv_blocks(d);
  if (epi == CNN_EPI_OUT0_F32)
    k_conv<CNN_EPI_OUT0_F32, 1, false><<<nb, NTHR, 0, st>>>(d, in, W, bias, mask, out);
  else if (epi == CNN_EPI_RELU && ntiles < 0)
    k_conv<CNN_EPI_RELU, 2, true><<<nb, NTHR, 0, st>>>(d, in, W, bias, mask, out);
  else if (epi == CNN_EPI_RELU)
    k_conv<CNN_EPI_RELU, 2, false><<<nb, NTHR, 0, st>>>(d, in, W, bias, mask, out);
  else
    k_conv<CNN_EPI_MASK, 2, false><<<nb, NTHR, 0, st>>>(d, in, W, bias, mask, out);
  smg_count_launch(1);
  return cudaGetLastError();
}

cudaError_t cnn_wgrad(const CnnDims& d, const __nv_bfloat16* in, const __nv_bfloat16* g, float* part, int layer,
                      float* grad, cudaStream_t st) {
  const int nb = conv_blocks(d);
  k_conv_wgrad<<<nb, NTHR, 0, st>>>(d, in, g, part);
  k_reduce_grad<<<(27 * CH * CH + CH + 255) / 256, 256, 0, st>>>(nb, part, layer, grad);
  smg_count_launch(2);
  return cudaGetLastError();
}

cudaError_t cnn_pack_input(long long n, const double* r, const double* logk, const double* inv_scale_dev,
                           double inv_s, __nv_bfloat16* act0, cudaStream_t st) {
  k_pack_input<<<(int)((n + 255) / 256), 256, 0, st>>>(n, r, logk, inv_scale_dev, inv_s, act0);
  smg_count_launch(1);
  return cudaGetLastError();
}

cudaError_t cnn_pack_input_f32(long long n, const float* in2, __nv_bfloat16* act0, cudaStream_t st) {
  k_pack_input_f32<<<(int)((n + 255) / 256), 256, 0, st>>>(n, in2, act0);
  smg_count_launch(1);
  return cudaGetLastError();
}

cudaError_t cnn_mse(long long n, const float* y, const float* tgt, __nv_bfloat16* g16, float* loss_part,
                    int nparts, float* loss, cudaStream_t st) {
  k_mse<<<nparts, 256, 0, st>>>(n, y, tgt, g16, loss_part);
  k_sum_in_order<<<1, 32, 0, st>>>(nparts, loss_part, loss);
  smg_count_launch(2);
  return cudaGetLastError();
}

cudaError_t cnn_adam(int n, float* theta, float* m, float* v, const float* grad, int t, float lr, float b1, float b2,
                     float eps, float gscale, cudaStream_t st) {
  k_adam<<<(n + 255) / 256, 256, 0, st>>>(n, theta, m, v, grad, t, lr, b1, b2, eps, gscale);
  smg_count_launch(1);
  return cudaGetLastError();
}
