// Split ILU(0) factor records read by the warp-pipelined triangular solves.
//
// The factorisation leaves L (unit lower) and U (upper, with the pivot u_pp)
// interleaved in one array of structures per point.  A lower solve reads only
// the strictly-lower entries and an upper solve only the strictly-upper ones
// plus 1/u_pp, so the sweeps get one record per point and triangle:
//
//   [NV entries in lexicographic offset order][1/u_pp (U, FP64 / FP32)]
//   [row scale, FP32 (BF16)][zero padding to a multiple of 16 bytes]
//
// with NV the number of strictly-lower (= strictly-upper) offsets of the
// canonical 7-, 19- or 27-point mask.  Records are 16-byte aligned, so a lane
// reads its point's record with 128-bit loads and a solve streams exactly the
// bytes of its own triangle.  BF16 values are the triangle's entries divided
// by the triangle's row scale (the largest magnitude among them), rounded to
// nearest even; the BF16 upper solve keeps 1/u_pp in the separate FP32
// inverse-diagonal array.
#pragma once

#include "shapes.cuh"
#include "smg_internal.cuh"

template <int PK, int NS, bool UPPER>
struct IluRec {
  using Val = typename Prec<PK>::val;
  static constexpr int NV = Shape<NS>::EC;
  static constexpr int VB = NV * (int)sizeof(Val);
  static constexpr bool HAS_D = UPPER && PK != KBF;
  static constexpr bool HAS_S = PK == KBF;
  static constexpr int D_OFF = VB;                 // a multiple of sizeof(Val)
  static constexpr int S_OFF = (VB + 3) / 4 * 4;   // FP32 row scale
  static constexpr int RAW = HAS_D ? D_OFF + (int)sizeof(Val) : (HAS_S ? S_OFF + 4 : VB);
  static constexpr int BYTES = (RAW + 15) / 16 * 16;
  static constexpr int CHUNKS = BYTES / 16;
};

// Bytes of one record (0 when the mask has no split records).
__host__ inline int ilu_rec_bytes(int pk, int ns, bool upper) {
#define R_(PK, NS) (upper ? IluRec<PK, NS, true>::BYTES : IluRec<PK, NS, false>::BYTES)
  if (ns != 7 && ns != 19 && ns != 27) return 0;
  if (pk == K64) return ns == 27 ? R_(K64, 27) : ns == 19 ? R_(K64, 19) : R_(K64, 7);
  if (pk == K32) return ns == 27 ? R_(K32, 27) : ns == 19 ? R_(K32, 19) : R_(K32, 7);
  return ns == 27 ? R_(KBF, 27) : ns == 19 ? R_(KBF, 19) : R_(KBF, 7);
#undef R_
}

// Writes both records of every point from the FP64 factors LU [n][ns] (unit
// L on the lower entries, U on the centre and upper ones) and 1/u_pp, in the
// working precision pk.  The mask must be the canonical one of ns.
cudaError_t launch_ilu_split(Grid g, int ns, int pk, const double* LU, const double* udinv, void* Lrec, void* Urec,
                             cudaStream_t st);
