// Canonical 7-, 19- and 27-point masks in lexicographic order (dx slowest)
// with the wavefront skews of their lexicographic sweeps: point (i, j, k)
// runs at t = SA*i + SB*j + k, the smallest skews that put every lower
// neighbour strictly earlier.  EC is the index of the centre entry.
#pragma once

template <int NS> struct Shape;
template <> struct Shape<27> {
  static constexpr int SA = 4, SB = 2, EC = 13;
  __host__ __device__ static constexpr int o(int e, int d) {
    return d == 0 ? e / 9 - 1 : (d == 1 ? (e / 3) % 3 - 1 : e % 3 - 1);
  }
};
template <> struct Shape<7> {
  static constexpr int SA = 1, SB = 1, EC = 3;
  __host__ __device__ static constexpr int o(int e, int d) {
    return d == 0 ? (e == 0 ? -1 : (e == 6 ? 1 : 0)) : d == 1 ? (e == 1 ? -1 : (e == 5 ? 1 : 0))
                                                               : (e == 2 ? -1 : (e == 4 ? 1 : 0));
  }
};
template <> struct Shape<19> {
  static constexpr int SA = 3, SB = 2, EC = 9;
  __host__ __device__ static constexpr int o(int e, int d) {
    constexpr int t[19][3] = {{-1, -1, 0}, {-1, 0, -1}, {-1, 0, 0}, {-1, 0, 1}, {-1, 1, 0}, {0, -1, -1}, {0, -1, 0},
                              {0, -1, 1},  {0, 0, -1},  {0, 0, 0},  {0, 0, 1},  {0, 1, -1}, {0, 1, 0},   {0, 1, 1},
                              {1, -1, 0},  {1, 0, -1},  {1, 0, 0},  {1, 0, 1},  {1, 1, 0}};
    return t[e][d];
  }
};
