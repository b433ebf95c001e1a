// Host-side symbolic analysis of the stencil Galerkin product (Sec. 4.3).
//
// A^C(I, I+dJ) = sum_{u,v} R(I,u) A^F(u,v) P(v, I+dJ) (Eq. 5).  With every
// operator given as a stencil pattern -- R as fine offsets from the fine
// anchor of I (R_from, Eq. 6), P as fine offsets from the fine anchor of
// I+dJ (P_to, Eq. 7), A^F as offsets of v from u (Ngb, Eq. 9) -- a chain
// (r, a, q) contributes to dJ exactly when
//     roff[r] + aoff[a] = 2*dJ + poff[q]          (stride-2 coarsening;
//                                                  dJ = aoff in a dimension
//                                                  that is not coarsened),
// i.e. when the fine neighbour u+aoff[a] lies in P_to of I+dJ (the
// intersection of Eq. 10).  The chain set depends only on the three
// patterns, so it is derived once and reused by every matrix with them.
#include <cstring>
#include <vector>

#include "chains.h"
#include "smg.h"

namespace smg_host {

int derive_chains(int dim, int nr, const int* roff, int na, const int* aoff, int np, const int* poff,
                  std::vector<Chain>& out) {
  const int stride[3] = {2, 2, 2};
  return derive_chains_strided(dim, stride, nr, roff, na, aoff, np, poff, out);
}

// The same with a coarsening stride of 2 or 1 per dimension: a dimension
// that is not coarsened (stride 1) maps fine offsets to coarse ones as is.
int derive_chains_strided(int dim, const int* stride, int nr, const int* roff, int na, const int* aoff, int np,
                          const int* poff, std::vector<Chain>& out) {
  out.clear();
  if (dim != 2 && dim != 3) return -1;
  for (int r = 0; r < nr; ++r)
    for (int a = 0; a < na; ++a)
      for (int q = 0; q < np; ++q) {
        int dj[3] = {0, 0, 0};
        bool ok = true;
        for (int t = 0; t < dim; ++t) {
          int d = roff[3 * r + t] + aoff[3 * a + t] - poff[3 * q + t];
          if (stride[t] == 1) {
            dj[t] = d;
            continue;
          }
          if (d & 1) { ok = false; break; }
          dj[t] = d / 2;
        }
        if (!ok) continue;
        for (int t = 0; t < dim; ++t)
          if (dj[t] < -1 || dj[t] > 1) return -1;
        int idx = 0;
        for (int t = 0; t < dim; ++t) idx = idx * 3 + (dj[t] + 1);
        out.push_back(Chain{r, a, q, idx});
      }
  return (int)out.size();
}

// 1-D full-weighting interpolation weight of fine offset d from the anchor.
static double w1(int d) { return d == 0 ? 1.0 : 0.5; }

// 1-D cell-centred interpolation weight of fine cell 2J + d from coarse cell J
// (3d64c): the fine centre is 1/4 of a coarse cell from J's centre for d in
// {0,1} and 3/4 from it for d in {-1,2}.
static double wc(int d) { return (d == 0 || d == 1) ? 0.75 : 0.25; }

// The fine offsets lo..hi in every dimension, lexicographic.
static void cube(int lo, int hi, std::vector<int>& out) {
  for (int a = lo; a <= hi; ++a)
    for (int b = lo; b <= hi; ++b)
      for (int c = lo; c <= hi; ++c) out.insert(out.end(), {a, b, c});
}

int build_rap_table(int transfer, int ns_f, const int (*off_f)[3], RapTable& T) {
  std::vector<int> rp, pp;  // R and P patterns: fine offsets from the anchor
  if (transfer == SMG_TRANSFER_FW27V) {
    cube(-1, 1, rp);  // anchor 2I+1
    pp = rp;
  } else if (transfer == SMG_TRANSFER_PC8C) {
    cube(0, 1, rp);  // anchor 2I
    pp = rp;
  } else if (transfer == SMG_TRANSFER_C64C) {
    cube(0, 1, rp);
    cube(-1, 2, pp);
  } else if (transfer == SMG_TRANSFER_C16C_XY) {
    // x and y as C64C, z not coarsened: every pattern has z offset 0
    for (int a = 0; a <= 1; ++a)
      for (int b = 0; b <= 1; ++b) rp.insert(rp.end(), {a, b, 0});
    for (int a = -1; a <= 2; ++a)
      for (int b = -1; b <= 2; ++b) pp.insert(pp.end(), {a, b, 0});
  } else {
    return -1;
  }
  std::vector<int> af(3 * ns_f);
  for (int e = 0; e < ns_f; ++e)
    for (int t = 0; t < 3; ++t) af[3 * e + t] = off_f[e][t];
  std::vector<Chain> ch;
  const int stride[3] = {2, 2, transfer == SMG_TRANSFER_C16C_XY ? 1 : 2};
  int n = derive_chains_strided(3, stride, (int)rp.size() / 3, rp.data(), ns_f, af.data(), (int)pp.size() / 3,
                                pp.data(), ch);
  if (n < 0) return -1;
  bool present[27] = {false};
  for (const Chain& c : ch) present[c.dj] = true;
  // coarse stencil: the reached offsets, lexicographic order
  T.ns_c = 0;
  int cidx[27];
  for (int o = 0; o < 27; ++o) {
    cidx[o] = -1;
    if (!present[o]) continue;
    cidx[o] = T.ns_c;
    T.off_c[T.ns_c][0] = o / 9 - 1;
    T.off_c[T.ns_c][1] = (o / 3) % 3 - 1;
    T.off_c[T.ns_c][2] = o % 3 - 1;
    ++T.ns_c;
  }
  T.start.assign(T.ns_c + 1, 0);
  T.entries.clear();
  T.weights.clear();
  for (int c = 0; c < T.ns_c; ++c) {
    T.start[c] = (int)T.entries.size();
    for (const Chain& x : ch) {
      if (cidx[x.dj] != c) continue;
      const int* ro = &rp[3 * x.r];
      const int* po = &pp[3 * x.q];
      double wr = 1.0, wp = 1.0;
      if (transfer == SMG_TRANSFER_FW27V) {
        wr = w1(ro[0]) * w1(ro[1]) * w1(ro[2]) / 8.0;
        wp = w1(po[0]) * w1(po[1]) * w1(po[2]);
      } else if (transfer == SMG_TRANSFER_C64C) {
        wp = wc(po[0]) * wc(po[1]) * wc(po[2]);
      } else if (transfer == SMG_TRANSFER_C16C_XY) {
        wp = wc(po[0]) * wc(po[1]);
      }
      RapEntry en;
      en.rx = ro[0]; en.ry = ro[1]; en.rz = ro[2];
      en.a = x.a;
      T.entries.push_back(en);
      T.weights.push_back(wr * wp);
    }
  }
  T.start[T.ns_c] = (int)T.entries.size();
  T.nchains = n;
  return n;
}

void build_ilu_updates(int ns, const int (*off)[3], int ec, std::vector<int>& kstart, std::vector<int>& pairs) {
  auto find = [&](int dx, int dy, int dz) {
    for (int e = 0; e < ns; ++e)
      if (off[e][0] == dx && off[e][1] == dy && off[e][2] == dz) return e;
    return -1;
  };
  kstart.assign(ec + 1, 0);
  pairs.clear();
  for (int ek = 0; ek < ec; ++ek) {
    kstart[ek] = (int)pairs.size() / 2;
    for (int ej = ek + 1; ej < ns; ++ej) {
      int eq = find(off[ej][0] - off[ek][0], off[ej][1] - off[ek][1], off[ej][2] - off[ek][2]);
      if (eq < 0) continue;
      pairs.push_back(ej);
      pairs.push_back(eq);
    }
  }
  kstart[ec] = (int)pairs.size() / 2;
}

void schedule_skews(int ns, const int (*off)[3], int* SA, int* SB) {
  int sb = 1;
  for (int e = 0; e < ns; ++e)
    if (off[e][0] == 0 && off[e][1] == -1) sb = off[e][2] + 1 > sb ? off[e][2] + 1 : sb;
  int sa = 1;
  for (int e = 0; e < ns; ++e)
    if (off[e][0] == -1) {
      int v = sb * off[e][1] + off[e][2] + 1;
      sa = v > sa ? v : sa;
    }
  *SA = sa;
  *SB = sb;
}

}  // namespace smg_host

extern "C" int smg_rap_chain_count(int transfer, int nstencil, const int* offsets, int* ncoarse) {
  if (nstencil < 1 || nstencil > 27 || !offsets) return -1;
  int off[27][3];
  for (int e = 0; e < nstencil; ++e)
    for (int t = 0; t < 3; ++t) off[e][t] = offsets[3 * e + t];
  smg_host::RapTable T;
  const int n = smg_host::build_rap_table(transfer, nstencil, off, T);
  if (n >= 0 && ncoarse) *ncoarse = T.ns_c;
  return n;
}

extern "C" int smg_derive_chains(int dim, int nr, const int* roff, int na, const int* aoff, int np, const int* poff,
                                 int max_chains, int* chains) {
  if (nr < 0 || na < 0 || np < 0 || (nr && !roff) || (na && !aoff) || (np && !poff)) return -1;
  std::vector<smg_host::Chain> ch;
  int n = smg_host::derive_chains(dim, nr, roff, na, aoff, np, poff, ch);
  if (n < 0) return -1;
  if (chains)
    for (int t = 0; t < n && t < max_chains; ++t) {
      chains[5 * t + 0] = ch[t].r;
      chains[5 * t + 1] = ch[t].a;
      chains[5 * t + 2] = ch[t].q;
      chains[5 * t + 3] = ch[t].dj;
      chains[5 * t + 4] = 0;
    }
  return n;
}
