// Sweep records and the skewed plane layout of the warp-pipelined
// triangular sweeps (sweep3.cuh).
//
// Records.  A sweep reads, per point, only the coefficients of its own
// triangle, packed with what else it needs into one record of whole 16-byte
// chunks:
//   ILU(0) lower solve:  [strictly-lower entries of L]
//   ILU(0) upper solve:  [strictly-upper entries of U][1/u_pp]
//   Gauss-Seidel:        [all entries, centre slot 0][1/a_pp]
// entries in lexicographic offset order, stored in the working precision;
// BF16 entries are divided by a row scale (FP32, the largest magnitude among
// the record's entries) that follows them; the inverse diagonal is stored in
// the vector type (FP64, or FP32 for FP32 / BF16 hierarchies).
//
// Skewed layout.  Lane J of a sweep warp treats point (j, k) = (J, s - SB*J)
// of its plane at step s, so the points of one step lie on a diagonal of the
// (j, k) plane.  The sweeps therefore keep their planes in rows
// r = (k + SB*j) mod nz:  every point of step s of a plane is in the same row,
// at column j, and a warp's 32 lanes read 32 consecutive slots.  Vectors:
// slot ((i*nz + r)*ny + j).  Records: chunk c of point (i, j, k) is the 16-byte
// unit ((i*nz + r)*CHUNKS + c)*ny + j, so one 128-bit load instruction of a
// warp reads 512 consecutive bytes.  The map is a bijection per column, for
// either sweep direction.
#pragma once

#include "shapes.cuh"
#include "smg_internal.cuh"

// KIND_REC: 0 lower solve, 1 upper solve, 2 Gauss-Seidel.
template <int PK, int NS, int KIND_REC>
struct SweepRec {
  using Val = typename Prec<PK>::val;
  using Vec = typename Prec<PK>::vec;
  static constexpr int EC = Shape<NS>::EC;
  static constexpr int NV = KIND_REC == 2 ? NS : EC;
  static constexpr int VB = NV * (int)sizeof(Val);
  static constexpr bool HAS_S = PK == KBF;
  static constexpr bool HAS_D = KIND_REC != 0;
  static constexpr int S_OFF = (VB + 3) / 4 * 4;  // FP32 row scale
  static constexpr int AFTER = HAS_S ? S_OFF + 4 : VB;
  static constexpr int D_OFF = (AFTER + (int)sizeof(Vec) - 1) / (int)sizeof(Vec) * (int)sizeof(Vec);
  static constexpr int RAW = HAS_D ? D_OFF + (int)sizeof(Vec) : AFTER;
  static constexpr int BYTES = (RAW + 15) / 16 * 16;
  static constexpr int CHUNKS = BYTES / 16;
  // record slot of stencil entry e
  __host__ __device__ static constexpr int slot(int e) { return KIND_REC == 1 ? e - EC - 1 : e; }
};

// Chunks of one record (0 when the mask has no records).
__host__ inline int sweep_rec_chunks(int pk, int ns, int kind_rec) {
#define R_(PK, NS) (kind_rec == 0 ? SweepRec<PK, NS, 0>::CHUNKS : kind_rec == 1 ? SweepRec<PK, NS, 1>::CHUNKS \
                                                                                : SweepRec<PK, NS, 2>::CHUNKS)
  if (ns != 7 && ns != 19 && ns != 27) return 0;
  if (pk == K64) return ns == 27 ? R_(K64, 27) : ns == 19 ? R_(K64, 19) : R_(K64, 7);
  if (pk == K32) return ns == 27 ? R_(K32, 27) : ns == 19 ? R_(K32, 19) : R_(K32, 7);
  return ns == 27 ? R_(KBF, 27) : ns == 19 ? R_(KBF, 19) : R_(KBF, 7);
#undef R_
}

// Row of point (j, k) in the skewed layout (j, k >= 0).
__host__ __device__ __forceinline__ int skew_row(int j, int k, int SB, int nz) { return (k + SB * j) % nz; }
__host__ __device__ __forceinline__ long long skew_slot(const Grid& g, int SB, int i, int j, int k) {
  return ((long long)i * g.nz + skew_row(j, k, SB, g.nz)) * g.ny + j;
}

// Records of every point in the skewed layout, from the FP64 ILU factors
// LU [n][ns] and 1/u_pp (Lrec, Urec), or from A [n][ns] and 1/a_pp (Grec),
// lowered to the working precision pk.  The mask must be the canonical one
// of ns; SB its in-plane skew.
cudaError_t launch_ilu_records(Grid g, int ns, int SB, int pk, const double* LU, const double* udinv, void* Lrec,
                               void* Urec, cudaStream_t st);
cudaError_t launch_gs_records(Grid g, int ns, int SB, int pk, const double* A, const double* dinv, void* Grec,
                              cudaStream_t st);

// Vector between the natural order and the skewed layout (vb = 8 for FP64
// vectors, 4 for FP32): to_skew copies nat -> skw; otherwise skw -> nat,
// added to nat when add != 0.
cudaError_t launch_skew_copy(Grid g, int SB, int vb, bool to_skew, const void* src, void* dst, bool add,
                             cudaStream_t st);
