// Krylov kernels: device scalar slots and launchers (all FP64).
#pragma once
#include "smg_internal.cuh"

// Slots of the device scalar array used by the Krylov loops.
enum {
  SC_RHO = 0, SC_PQ = 1, SC_RR = 2, SC_RZ = 3, SC_ALPHA = 4, SC_BETA = 5, SC_BB = 6, SC_WW = 7,
  SC_LS_RR = 8, SC_LS_INVS = 9, SC_LS_S = 10, SC_LS_WW = 11,  // learned post-smoother
  SC_H = 16,  // GMRES: Gram-Schmidt coefficients h[0..64)
  SC_H2 = 96, // GMRES: second Gram-Schmidt pass
  SC_COUNT = 192
};
#define RED_STRIDE 8

cudaError_t kry_rr_bb(long long n, const double* r, const double* b, double* sc, const RedWs& rw, cudaStream_t st);
cudaError_t kry_dot(long long n, const double* a, const double* b, double* sc, int slot, const RedWs& rw,
                    cudaStream_t st);
cudaError_t kry_pq_alpha(long long n, const double* p, const double* q, double* sc, int* err, const RedWs& rw,
                         cudaStream_t st);
cudaError_t kry_update_xr(long long n, double* x, const double* p, double* r, const double* q, double* rold,
                          double* sc, const RedWs& rw, cudaStream_t st);
cudaError_t kry_rz_beta(long long n, const double* r, const double* z, const double* rold, double* sc, int first,
                        const RedWs& rw, cudaStream_t st);
cudaError_t kry_update_p(long long n, double* p, const double* z, const double* sc, int use_beta, const RedWs& rw,
                         cudaStream_t st);
cudaError_t kry_multidot(long long n, int m, const double* V, long long ld, const double* w, double* out,
                         const RedWs& rw, cudaStream_t st);
cudaError_t kry_multiaxpy(long long n, int m, const double* V, long long ld, const double* h, double* w,
                          const RedWs& rw, cudaStream_t st);
cudaError_t kry_scale_rsqrt(long long n, const double* x, double* y, const double* sc, int slot, const RedWs& rw,
                            cudaStream_t st);
cudaError_t kry_combine(long long n, int m, const double* Z, long long ld, const double* y, double* x,
                        const RedWs& rw, cudaStream_t st);
cudaError_t vec_add(long long n, const void* src, void* dst, int dbl, const RedWs& rw, cudaStream_t st);
