// Host check of the flux kernels' segment mapping (seg_coords, flux_nseg,
// flux_seg_items in dev.cuh), compiled by tests/test_seg_coverage.py and run
// on the CPU.  For every direction, segment length and block shape below,
// the items of one launch must cover each face of each transverse line
// exactly once (lines: the interior plus one on each side; faces: n_d + 1),
// with 1 <= nf <= L, and along x every item before the remainders sweeps the
// same number of faces.  Prints "ok" and exits 0, else the first failure.
#include <cstdio>
#include <vector>

#include "dev.cuh"

using grmhd::DevBlock;

template <int d>
static bool check(const int n[3], int L) {
  DevBlock b{};
  for (int a = 0; a < 3; a++) b.n[a] = n[a];
  b.ng = 4;
  b.nseg[d] = grmhd::flux_nseg(n[d], L);
  const long long items = grmhd::flux_seg_items(n, d, L);
  const int t1 = (d + 1) % 3, t2 = (d + 2) % 3, nd = n[d] + 1;
  const int w1 = n[t1] + 2, w2 = n[t2] + 2;
  std::vector<int> cover((size_t)w1 * w2 * nd, 0);
  const long long full_items = (long long)(b.nseg[d] - 1) * (d == 0 ? (long long)(n[1] + 2) * (n[2] + 2) : 0);
  int first_nf = -1;
  for (long long loc = 0; loc < items; loc++) {
    int k, j, i, nf;
    grmhd::seg_coords<d>(b, (int)loc, k, j, i, nf);
    const int c[3] = {i - b.ng, j - b.ng, k - b.ng};
    const int f0 = c[d], a1 = c[t1] + 1, a2 = c[t2] + 1;
    if (nf < 1 || nf > L || f0 < 0 || f0 + nf > nd || a1 < 0 || a1 >= w1 || a2 < 0 || a2 >= w2) {
      std::printf("d=%d n=%d,%d,%d L=%d loc=%lld: f0=%d nf=%d lines %d %d\n", d, n[0], n[1], n[2], L, loc, f0, nf,
                  a1, a2);
      return false;
    }
    if (d == 0 && loc < full_items) {
      if (first_nf < 0) first_nf = nf;
      if (nf != first_nf) {
        std::printf("x: item %lld sweeps %d faces, item 0 %d (n=%d L=%d)\n", loc, nf, first_nf, n[0], L);
        return false;
      }
    }
    for (int f = f0; f < f0 + nf; f++) cover[((size_t)a2 * w1 + a1) * nd + f]++;
  }
  for (size_t q = 0; q < cover.size(); q++)
    if (cover[q] != 1) {
      std::printf("d=%d n=%d,%d,%d L=%d: face slot %zu covered %d times\n", d, n[0], n[1], n[2], L, q, cover[q]);
      return false;
    }
  return true;
}

int main() {
  const int shapes[][3] = {{1, 1, 1},   {2, 3, 5},    {7, 1, 4},    {8, 8, 8},    {16, 9, 3},  {21, 13, 10},
                           {30, 9, 17}, {33, 3, 1},   {31, 2, 6},   {64, 5, 4},   {96, 3, 2},  {104, 2, 3},
                           {128, 2, 2}, {129, 3, 2},  {255, 2, 1},  {3, 128, 2},  {2, 3, 128}};
  const int Ls[] = {1, 2, 3, 4, 8, 16};
  int cases = 0;
  for (const auto& n : shapes)
    for (int L : Ls) {
      if (!check<0>(n, L) || !check<1>(n, L) || !check<2>(n, L)) return 1;
      cases += 3;
    }
  std::printf("ok %d cases\n", cases);
  return 0;
}
