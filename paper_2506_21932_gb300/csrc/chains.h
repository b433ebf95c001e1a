// Host-side symbolic analysis tables (no CUDA types).
#pragma once
#include <vector>

namespace smg_host {

struct Chain {
  int r, a, q, dj;  // R entry, A entry, P entry, coarse offset (lexicographic index)
};

// One term of a coarse coefficient: fine point u = anchor + (rx,ry,rz), its
// stencil entry a, times a constant weight R(I,u) * P(v,J).
struct RapEntry {
  int rx, ry, rz, a;
};

struct RapTable {
  int ns_c = 0;
  int off_c[27][3];
  int nchains = 0;
  std::vector<int> start;  // [ns_c + 1]
  std::vector<RapEntry> entries;
  std::vector<double> weights;
};

int derive_chains(int dim, int nr, const int* roff, int na, const int* aoff, int np, const int* poff,
                  std::vector<Chain>& out);
int derive_chains_strided(int dim, const int* stride, int nr, const int* roff, int na, const int* aoff, int np,
                          const int* poff, std::vector<Chain>& out);
int build_rap_table(int transfer, int ns_f, const int (*off_f)[3], RapTable& T);
void build_ilu_updates(int ns, const int (*off)[3], int ec, std::vector<int>& kstart, std::vector<int>& pairs);
void schedule_skews(int ns, const int (*off)[3], int* SA, int* SB);

}  // namespace smg_host
