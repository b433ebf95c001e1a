// C ABI of the learned post-smoother's network: forward, loss + gradient,
// Adam (all on the device, kernels in k_cnn.cu).
#include <algorithm>

#include "cnn.cuh"

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t cnn_workspace_bytes(const CnnDims& d) {
  const size_t n = (size_t)d.nx * d.ny * d.nz;
  size_t b = 0;
  b += 2 * align256(3 * 27 * 256 * sizeof(__nv_bfloat16));  // packed weights, forward and transposed
  b += align256(48 * sizeof(float));                         // biases
  b += align256(4 * 256 * sizeof(__nv_bfloat16));            // first layer, packed K
  b += 6 * align256(n * 16 * sizeof(__nv_bfloat16));         // a0, a1, a2, g1, g2, g3
  b += align256(n * sizeof(float));                          // y
  b += align256(cnn_partials_floats(d) * sizeof(float));     // weight-gradient partials
  b += align256(1024 * sizeof(float));                       // loss partials
  return b;
}

void cnn_carve(const CnnDims& d, void* base, CnnWork& w) {
  const size_t n = (size_t)d.nx * d.ny * d.nz;
  char* p = (char*)base;
  auto take = [&](size_t bytes) {
    char* q = p;
    p += align256(bytes);
    return (void*)q;
  };
  w.pk.fwd = (__nv_bfloat16*)take(3 * 27 * 256 * sizeof(__nv_bfloat16));
  w.pk.bwd = (__nv_bfloat16*)take(3 * 27 * 256 * sizeof(__nv_bfloat16));
  w.pk.bias = (float*)take(48 * sizeof(float));
  w.pk.fwd1 = (__nv_bfloat16*)take(4 * 256 * sizeof(__nv_bfloat16));
  w.a0 = (__nv_bfloat16*)take(n * 32);
  w.a1 = (__nv_bfloat16*)take(n * 32);
  w.a2 = (__nv_bfloat16*)take(n * 32);
  w.g1 = (__nv_bfloat16*)take(n * 32);
  w.g2 = (__nv_bfloat16*)take(n * 32);
  w.g3 = (__nv_bfloat16*)take(n * 32);
  w.y = (float*)take(n * sizeof(float));
  w.part = (float*)take(cnn_partials_floats(d) * sizeof(float));
  w.loss_part = (float*)take(1024 * sizeof(float));
}

cudaError_t cnn_forward_packed(const CnnDims& d, CnnWork& w, cudaStream_t st) {
  const size_t L = 27 * 256;
  cudaError_t e = cnn_conv(d, CNN_EPI_RELU, -1, w.a0, w.pk.fwd1, w.pk.bias, nullptr, w.a1, st);
  if (e == cudaSuccess) e = cnn_conv(d, CNN_EPI_RELU, 2, w.a1, w.pk.fwd + L, w.pk.bias + 16, nullptr, w.a2, st);
  if (e == cudaSuccess) e = cnn_conv(d, CNN_EPI_OUT0_F32, 1, w.a2, w.pk.fwd + 2 * L, w.pk.bias + 32, nullptr, w.y, st);
  return e;
}

cudaError_t cnn_backward(const CnnDims& d, CnnWork& w, float* grad, cudaStream_t st) {
  const size_t L = 27 * 256;
  // layer 3: z3 = conv(a2); dz3 = g3
  cudaError_t e = cnn_wgrad(d, w.a2, w.g3, w.part, 2, grad, st);
  if (e == cudaSuccess) e = cnn_conv(d, CNN_EPI_MASK, 2, w.g3, w.pk.bwd + 2 * L, nullptr, w.a2, w.g2, st);
  // layer 2: dz2 = conv3^T(dz3) * (a2 > 0)
  if (e == cudaSuccess) e = cnn_wgrad(d, w.a1, w.g2, w.part, 1, grad, st);
  if (e == cudaSuccess) e = cnn_conv(d, CNN_EPI_MASK, 2, w.g2, w.pk.bwd + L, nullptr, w.a1, w.g1, st);
  // layer 1: dz1 = conv2^T(dz2) * (a1 > 0)
  if (e == cudaSuccess) e = cnn_wgrad(d, w.a0, w.g1, w.part, 0, grad, st);
  return e;
}

static int check_dims(const int dims[3], CnnDims& d) {
  if (!dims) return SMG_EINVAL;
  for (int t = 0; t < 3; ++t)
    if (dims[t] < 1 || dims[t] > 4096) return SMG_EINVAL;
  d = CnnDims{dims[0], dims[1], dims[2]};
  return SMG_OK;
}

int cnn_check_dims(const int dims[3], CnnDims& d) { return check_dims(dims, d); }

// ---- post-smoother glue (FP64 vectors, scalars in device memory) ----------
namespace {
// out[0] = 1 / rms, out[1] = rms, with rms = sqrt(ss / n) (both 0 if ss == 0)
__global__ void k_inv_rms(const double* ss, double n, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const double rms = sqrt(*ss / n);
    out[0] = rms > 0.0 ? 1.0 / rms : 0.0;
    out[1] = rms;
  }
}
// delta = s * dinv * y
__global__ void k_scale_out(long long n, const float* __restrict__ y, const double* __restrict__ s,
                            const double* __restrict__ dinv, double* __restrict__ delta) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) delta[p] = s[0] * dinv[p] * (double)y[p];
}
// z += delta when the corrected residual is smaller (ww < rr), else keep z
__global__ void k_accept(long long n, double* __restrict__ z, const double* __restrict__ delta,
                         const double* __restrict__ ww, const double* __restrict__ rr) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n && *ww < *rr) z[p] += delta[p];
}
__global__ void k_sub(long long n, const double* __restrict__ a, const double* __restrict__ b,
                      double* __restrict__ c) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) c[p] = a[p] - b[p];
}
__global__ void k_sample_pack(long long n, const double* __restrict__ e1, const double* __restrict__ rp,
                              const double* __restrict__ logk, const double* __restrict__ inv_s,
                              const double* __restrict__ dinv, float* __restrict__ in2, float* __restrict__ target) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const double is = inv_s[0];
  in2[p] = (float)(rp[p] * is);
  in2[n + p] = (float)logk[p];
  target[p] = (float)(e1[p] * is / dinv[p]);
}
// q = t - in2[0..n)  (FP64)
__global__ void k_resid_q(long long n, const double* __restrict__ t, const float* __restrict__ in2,
                          double* __restrict__ q) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) q[p] = t[p] - (double)in2[p];
}
// loss += ss / n
__global__ void k_loss_add(const double* __restrict__ ss, double n, float* __restrict__ loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *loss += (float)(*ss / n);
}
// g3[p] = (bf16(2 dinv[p] t[p] / n), 0, ..., 0)
__global__ void k_grad_out(long long n, const double* __restrict__ t, const double* __restrict__ dinv,
                           __nv_bfloat16* __restrict__ g16) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const unsigned v = (unsigned)__bfloat16_as_ushort(__double2bfloat16(2.0 * dinv[p] * t[p] / (double)n));
  reinterpret_cast<uint4*>(g16 + p * 16)[0] = make_uint4(v, 0, 0, 0);
  reinterpret_cast<uint4*>(g16 + p * 16)[1] = make_uint4(0, 0, 0, 0);
}
// out = dinv * y (FP64)
__global__ void k_scale_in(long long n, const float* __restrict__ y, const double* __restrict__ dinv,
                           double* __restrict__ out) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) out[p] = dinv[p] * (double)y[p];
}
}  // namespace

cudaError_t cnn_resid_glue(int which, long long n, const double* a, const float* f, const double* dinv, double* out,
                           float* loss, __nv_bfloat16* g16, cudaStream_t st) {
  const int nb = (int)((n + 255) / 256);
  if (which == 0) k_resid_q<<<nb, 256, 0, st>>>(n, a, f, out);
  else if (which == 1) k_loss_add<<<1, 32, 0, st>>>(a, (double)n, loss);
  else if (which == 2) k_grad_out<<<nb, 256, 0, st>>>(n, a, dinv, g16);
  else k_scale_in<<<nb, 256, 0, st>>>(n, f, dinv, out);
  smg_count_launch(1);
  return cudaGetLastError();
}

cudaError_t cnn_sample_glue(int which, long long n, const double* e0, const double* z, double* e1, const double* rp,
                            const double* logk, const double* inv_s, const double* dinv, float* in2, float* target,
                            cudaStream_t st) {
  const int nb = (int)((n + 255) / 256);
  if (which == 0) k_sub<<<nb, 256, 0, st>>>(n, e0, z, e1);
  else k_sample_pack<<<nb, 256, 0, st>>>(n, e1, rp, logk, inv_s, dinv, in2, target);
  smg_count_launch(1);
  return cudaGetLastError();
}

cudaError_t cnn_post_glue(int which, long long n, const float* y, double* z, double* delta, const double* a,
                          const double* b, const double* dinv, double* out, cudaStream_t st) {
  const int nb = (int)((n + 255) / 256);
  if (which == 0) k_inv_rms<<<1, 32, 0, st>>>(a, (double)n, out);
  else if (which == 1) k_scale_out<<<nb, 256, 0, st>>>(n, y, a, dinv, delta);
  else k_accept<<<nb, 256, 0, st>>>(n, z, delta, a, b);
  smg_count_launch(1);
  return cudaGetLastError();
}

extern "C" int smg_cnn_param_count(void) { return kCnnParams; }

extern "C" int smg_cnn_workspace_bytes(const int dims[3], size_t* bytes) {
  CnnDims d;
  if (check_dims(dims, d) != SMG_OK || !bytes) return SMG_EINVAL;
  *bytes = cnn_workspace_bytes(d);
  return SMG_OK;
}

extern "C" int smg_cnn_forward(const int dims[3], const float* theta, const float* in2, float* out, void* ws,
                               size_t ws_bytes, void* stream) {
  CnnDims d;
  if (check_dims(dims, d) != SMG_OK || !theta || !in2 || !out || !ws) return SMG_EINVAL;
  if (ws_bytes < cnn_workspace_bytes(d)) return SMG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  CnnWork w;
  cnn_carve(d, ws, w);
  const long long n = (long long)d.nx * d.ny * d.nz;
  SMG_CUDA_TRY(cnn_pack(theta, w.pk, st));
  SMG_CUDA_TRY(cnn_pack_input_f32(n, in2, w.a0, st));
  SMG_CUDA_TRY(cnn_forward_packed(d, w, st));
  SMG_CUDA_TRY(cudaMemcpyAsync(out, w.y, n * sizeof(float), cudaMemcpyDeviceToDevice, st));
  SMG_CUDA_TRY(cudaStreamSynchronize(st));
  return SMG_OK;
}

extern "C" int smg_cnn_loss_grad(const int dims[3], const float* theta, const float* in2, const float* target,
                                 float* grad, float* loss, void* ws, size_t ws_bytes, void* stream) {
  CnnDims d;
  if (check_dims(dims, d) != SMG_OK || !theta || !in2 || !target || !grad || !loss || !ws) return SMG_EINVAL;
  if (ws_bytes < cnn_workspace_bytes(d)) return SMG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  CnnWork w;
  cnn_carve(d, ws, w);
  const long long n = (long long)d.nx * d.ny * d.nz;
  const size_t L = 27 * 256;
  SMG_CUDA_TRY(cnn_pack(theta, w.pk, st));
  SMG_CUDA_TRY(cnn_pack_input_f32(n, in2, w.a0, st));
  SMG_CUDA_TRY(cnn_forward_packed(d, w, st));
  const int nparts = (int)std::min<long long>(1024, (n + 255) / 256);
  SMG_CUDA_TRY(cnn_mse(n, w.y, target, w.g3, w.loss_part, nparts, loss, st));
  SMG_CUDA_TRY(cnn_backward(d, w, grad, st));
  return SMG_OK;
}

extern "C" int smg_cnn_adam(int n, float* theta, float* m, float* v, const float* grad, int step, float lr, float beta1,
                            float beta2, float eps, float grad_scale, void* stream) {
  if (n < 1 || !theta || !m || !v || !grad || step < 1) return SMG_EINVAL;
  SMG_CUDA_TRY(cnn_adam(n, theta, m, v, grad, step, lr, beta1, beta2, eps, grad_scale, (cudaStream_t)stream));
  return SMG_OK;
}
