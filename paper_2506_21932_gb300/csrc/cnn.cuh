// Learned post-smoother: shared constants and launchers (see k_cnn.cu).
#pragma once
#include "smg_internal.cuh"

// Layer shapes and offsets of the FP32 master parameter vector (8241 values).
__host__ __device__ constexpr int cnn_cin(int l) { return l == 0 ? 2 : 16; }
__host__ __device__ constexpr int cnn_cout(int l) { return l == 2 ? 1 : 16; }
__host__ __device__ constexpr int cnn_woff(int l) { return l == 0 ? 0 : (l == 1 ? 880 : 7808); }
constexpr int kCnnParams = 8241;

enum { CNN_EPI_RELU = 0, CNN_EPI_MASK = 1, CNN_EPI_OUT0_F32 = 2 };

struct CnnDims {
  int nx, ny, nz;
};

// BF16 weights in the kernels' layouts (per layer 27 x 16 x 16) and biases.
struct CnnPacked {
  __nv_bfloat16* fwd;   // [3][27][co][ci]
  __nv_bfloat16* bwd;   // [3][27][ci][co], taps flipped
  float* bias;          // [3][16]
  __nv_bfloat16* fwd1;  // first layer with K = (tap, channel): [4][co][16]
};

size_t cnn_partials_floats(const CnnDims& d);
cudaError_t cnn_pack(const float* theta, CnnPacked& pk, cudaStream_t st);
// ntiles: 2 (16 outputs), 1 (the last layer), or -1 for the first layer's
// packed form (2 input channels, W = CnnPacked::fwd1)
cudaError_t cnn_conv(const CnnDims& d, int epi, int ntiles, const __nv_bfloat16* in, const __nv_bfloat16* W,
                     const float* bias, const __nv_bfloat16* mask, void* out, cudaStream_t st);
cudaError_t cnn_wgrad(const CnnDims& d, const __nv_bfloat16* in, const __nv_bfloat16* g, float* part, int layer,
                      float* grad, cudaStream_t st);
cudaError_t cnn_pack_input(long long n, const double* r, const double* logk, const double* inv_scale_dev,
                           double inv_s, __nv_bfloat16* act0, cudaStream_t st);
cudaError_t cnn_pack_input_f32(long long n, const float* in2, __nv_bfloat16* act0, cudaStream_t st);
cudaError_t cnn_mse(long long n, const float* y, const float* tgt, __nv_bfloat16* g16, float* loss_part,
                    int nparts, float* loss, cudaStream_t st);
cudaError_t cnn_adam(int n, float* theta, float* m, float* v, const float* grad, int t, float lr, float b1, float b2,
                     float eps, float gscale, cudaStream_t st);

// Workspace of one volume: activations, gradients, per-CTA partials.
struct CnnWork {
  __nv_bfloat16 *a0, *a1, *a2, *g1, *g2, *g3;
  float* y;
  float* part;
  float* loss_part;
  CnnPacked pk;
};
size_t cnn_workspace_bytes(const CnnDims& d);
void cnn_carve(const CnnDims& d, void* base, CnnWork& w);
// y = f(act0) for the packed network (act0 already filled)
cudaError_t cnn_forward_packed(const CnnDims& d, CnnWork& w, cudaStream_t st);
// grad += d loss / d theta, from the output gradient in w.g3 (after a forward)
cudaError_t cnn_backward(const CnnDims& d, CnnWork& w, float* grad, cudaStream_t st);
int cnn_check_dims(const int dims[3], CnnDims& d);
// Residual-loss glue: which 0 -> out = a - f[0..n) (FP64); which 1 ->
// *loss += a[0] / n; which 2 -> g16 channel 0 = bf16(2 dinv a / n), others
// 0; which 3 -> out = dinv * f.
cudaError_t cnn_resid_glue(int which, long long n, const double* a, const float* f, const double* dinv, double* out,
                           float* loss, __nv_bfloat16* g16, cudaStream_t st);
// Post-smoother glue: which 0 -> out[0..1] = (1/rms, rms) of the sum of
// squares a[0] over n points; 1 -> delta = a[0] * dinv * y; 2 -> z += delta
// where a[0] < b[0].
cudaError_t cnn_post_glue(int which, long long n, const float* y, double* z, double* delta, const double* a,
                          const double* b, const double* dinv, double* out, cudaStream_t st);
// Training-pair glue: which 0 -> e1 = e0 - z; which 1 -> in2 = [rp * inv_s ;
// logk], target = e1 * inv_s / dinv (inv_s read from device memory).
cudaError_t cnn_sample_glue(int which, long long n, const double* e0, const double* z, double* e1, const double* rp,
                            const double* logk, const double* inv_s, const double* dinv, float* in2, float* target,
                            cudaStream_t st);
