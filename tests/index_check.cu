// Host check of the kernels' index logic in dev.cuh, compiled by
// tests/test_index_logic.py and run on the CPU.
//  - Flux segments (seg_coords, flux_nseg, flux_seg_items): for every
//    direction, segment length and block shape below, the items of one launch
//    cover each face of each transverse line exactly once (lines: the
//    interior plus one on each side; faces: n_d + 1), with 1 <= nf <= L;
//    along x every item before the remainders sweeps the same number of
//    faces.  The cells a sweep reads (the five-cell stencils of the cells
//    next to its faces, as k_flux does) lie inside the ghosted block, and its
//    faces (fidx) inside the face array (nface).
//  - The face metric cache: the metric kernel's stores (fmc_index of each
//    face_coords item) are distinct slots inside fmc_count (for y and z the
//    item index itself), and a sweep's per-face index step (fmc_step) lands
//    on fmc_index of every face it visits.
//  - find_block: on prefix sums with empty blocks, item it belongs to the
//    block b returned, p[b] <= it < p[b + 1].
//  - The integer-pipe compares (lt0, gt0, eq0, gt_nn, below_thr,
//    finite_bits, and upw of the CT upwinding) against the IEEE comparisons
//    they replace, on special
//    values (+-0, subnormals, +-inf, NaNs of both signs) and random bit
//    patterns, within each one's stated domain.
// Prints "ok" and exits 0, else the first failure.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <vector>

#include "dev.cuh"

using grmhd::DevBlock;

// The metric cache kernel stores the face of work item `loc` (face_coords)
// at fmc_index: for y and z that is loc itself; for x (segments of length L,
// segment-major slots) every face must land on its own slot inside
// fmc_count.
template <int d>
static bool check_fmc(const int n[3], int L) {
  DevBlock b{};
  for (int a = 0; a < 3; a++) b.n[a] = n[a];
  b.ng = 4;
  b.nseg[0] = grmhd::flux_nseg(n[0], L);
  const long long cnt = grmhd::fmc_count(b, d);
  const long long faces = (long long)(n[0] + (d == 0 ? 1 : 2)) * (n[1] + (d == 1 ? 1 : 2)) * (n[2] + (d == 2 ? 1 : 2));
  std::vector<int> held((size_t)cnt, 0);
  for (long long loc = 0; loc < faces; loc++) {
    int k, j, i;
    grmhd::face_coords<d>(b, loc, k, j, i);
    const long long q = grmhd::fmc_index(b, d, k, j, i);
    if (q < 0 || q >= cnt || held[(size_t)q]++ || (d != 0 && q != loc)) {
      std::printf("fmc d=%d n=%d,%d,%d L=%d: item %lld -> slot %lld of %lld\n", d, n[0], n[1], n[2], L, loc, q, cnt);
      return false;
    }
  }
  return true;
}

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
    // k_flux reconstructs the cells next to its faces, c .. c + nf st along d
    // from the cell c below the first face, each from a five-cell stencil:
    // it reads c - 2 st .. c + (nf + 2) st (the face metric's four-point
    // stencils lie inside), and writes faces f .. f + (nf - 1) fst
    const int N[3] = {n[0] + 2 * b.ng, n[1] + 2 * b.ng, n[2] + 2 * b.ng};
    b.N[0] = N[0]; b.N[1] = N[1]; b.N[2] = N[2];
    const int cc[3] = {i, j, k};
    const int cd = cc[d] - 1;
    if (cd - 2 < 0 || cd + nf + 2 >= N[d] || cc[t1] < 0 || cc[t1] >= N[t1] || cc[t2] < 0 || cc[t2] >= N[t2]) {
      std::printf("d=%d n=%d,%d,%d L=%d loc=%lld: cells %d..%d of %d\n", d, n[0], n[1], n[2], L, loc, cd - 2,
                  cd + nf + 2, N[d]);
      return false;
    }
    const long long fl = grmhd::fidx(b, d, k, j, i);
    const long long fst = d == 0 ? 1 : (d == 1 ? (long long)N[0] : (long long)N[0] * N[1]);
    if (fl < 0 || fl + (nf - 1) * fst >= grmhd::nface(b, d)) {
      std::printf("d=%d n=%d,%d,%d L=%d loc=%lld: faces %lld..%lld of %lld\n", d, n[0], n[1], n[2], L, loc, fl,
                  fl + (nf - 1) * fst, grmhd::nface(b, d));
      return false;
    }
    // the face metric cache: the sweep steps its index by qst per face; every
    // face's index is fmc_index of that face and lies inside the cache
    {
      const long long q0 = grmhd::fmc_index(b, d, k, j, i), nq = grmhd::fmc_count(b, d);
      const long long qst = grmhd::fmc_step(b, d);
      for (int q = 0; q < nf; q++) {
        const int kk = k + (d == 2 ? q : 0), jj = j + (d == 1 ? q : 0), ii = i + (d == 0 ? q : 0);
        const long long want = grmhd::fmc_index(b, d, kk, jj, ii);
        if (want != q0 + q * qst || want < 0 || want >= nq) {
          std::printf("d=%d n=%d,%d,%d L=%d loc=%lld face %d: cache index %lld, stepped %lld of %lld\n", d, n[0],
                      n[1], n[2], L, loc, q, want, q0 + q * qst, nq);
          return false;
        }
      }
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

static bool check_find_block() {
  unsigned long long x = 12345;
  for (int trial = 0; trial < 200; trial++) {
    const int nb = 1 + trial % 37;
    std::vector<long long> pre((size_t)3 * (nb + 1), 0);
    for (int K = 0; K < 3; K++)
      for (int b = 0; b < nb; b++) {
        x = x * 6364136223846793005ull + 1442695040888963407ull;
        const long long sz = (x >> 33) % 4 == 0 ? 0 : (long long)((x >> 40) % 50);
        pre[(size_t)K * (nb + 1) + b + 1] = pre[(size_t)K * (nb + 1) + b] + sz;
      }
    grmhd::Work w{nullptr, pre.data(), nb};
    for (int K = 0; K < 3; K++) {
      const long long* p = pre.data() + (size_t)K * (nb + 1);
      for (long long it = 0; it < p[nb]; it++) {
        const int b = grmhd::find_block(w, K, it);
        if (b < 0 || b >= nb || !(p[b] <= it && it < p[b + 1])) {
          std::printf("find_block: trial %d K %d item %lld -> block %d\n", trial, K, it, b);
          return false;
        }
      }
    }
  }
  return true;
}

static double from_bits(unsigned long long u) {
  double x;
  std::memcpy(&x, &u, sizeof x);
  return x;
}

static bool check_compares() {
  std::vector<double> v = {0.0, -0.0, 1.0, -1.0, 0.5, -2.5, 1e-300, -1e-300,
                           std::numeric_limits<double>::denorm_min(), -std::numeric_limits<double>::denorm_min(),
                           from_bits(0x000FFFFFFFFFFFFFull), from_bits(0x800FFFFFFFFFFFFFull),
                           std::numeric_limits<double>::min(), -std::numeric_limits<double>::min(),
                           std::numeric_limits<double>::max(), -std::numeric_limits<double>::max(),
                           std::numeric_limits<double>::infinity(), -std::numeric_limits<double>::infinity(),
                           from_bits(0x7FF8000000000000ull), from_bits(0xFFF8000000000000ull),
                           from_bits(0x7FF0000000000001ull), from_bits(0xFFFFFFFFFFFFFFFFull), 1e-12, 1e-10};
  unsigned long long x = 987654321;
  for (int r = 0; r < 20000; r++) {
    x = x * 6364136223846793005ull + 1442695040888963407ull;
    v.push_back(from_bits(x));
  }
  for (double a : v) {
    if (grmhd::lt0(a) != (a < 0.0) || grmhd::gt0(a) != (a > 0.0) || grmhd::eq0(a) != (a == 0.0) ||
        grmhd::finite_bits(a) != (bool)std::isfinite(a)) {
      std::printf("sign tests differ at %a\n", a);
      return false;
    }
  }
  // gt_nn(x, y) == (x > y): neither NaN, at least one >= +0, not (+0, -0)
  auto in_domain = [](double a, double b) {
    if (std::isnan(a) || std::isnan(b)) return false;
    if (std::signbit(a) && std::signbit(b)) return false;
    if (a == 0.0 && b == 0.0 && !std::signbit(a) && std::signbit(b)) return false;
    return true;
  };
  long long pairs = 0;
  for (size_t i = 0; i < v.size(); i += (i < 64 ? 1 : 97))
    for (size_t j = 0; j < v.size(); j += (j < 64 ? 1 : 89)) {
      const double a = v[i], b = v[j];
      if (!in_domain(a, b)) continue;
      pairs++;
      if (grmhd::gt_nn(a, b) != (a > b)) {
        std::printf("gt_nn(%a, %a) differs\n", a, b);
        return false;
      }
    }
  // below_thr(P, x) == (x < rho_thr) for finite x, rho_thr > 0 or = 0
  for (double thr : {0.0, 1e-12, 1e-10, 1.0}) {
    grmhd::Par P{};
    P.rho_thr = thr;
    P.thr_pos = thr > 0.0;
    for (double a : v) {
      if (!std::isfinite(a)) continue;
      if (grmhd::below_thr(P, a) != (a < thr)) {
        std::printf("below_thr(%g, %a) differs\n", thr, a);
        return false;
      }
    }
  }
  // upw (CT upwinding) against the select form of FP64 compares
  for (double f : v) {
    const double a = 1.5, b = -0.25, c = 3.0, d = 0.75;
    const double ref = f > 0.0 ? a - b : (f < 0.0 ? c - d : 0.5 * ((a - b) + (c - d)));
    if (grmhd::upw(f, a, b, c, d) != ref) {
      std::printf("upw(%a) differs\n", f);
      return false;
    }
  }
  return pairs > 1000;
}

// Segment lengths that flux_seg_len picks on 152 SMs (x, y, z).
static bool check_seg_len() {
  struct Case { int n; int L[3]; } cases[] = {{128, {16, 16, 16}}, {104, {16, 16, 16}}, {96, {8, 8, 8}},
                                              {64, {2, 2, 2}}, {32, {1, 1, 1}}};
  for (const Case& c : cases) {
    const int n[1][3] = {{c.n, c.n, c.n}};
    for (int d = 0; d < 3; d++) {
      const int L = grmhd::flux_seg_len(n, 1, d, 152);
      if (L != c.L[d]) {
        std::printf("flux_seg_len(%d^3, d=%d) = %d, expected %d\n", c.n, d, L, c.L[d]);
        return false;
      }
    }
  }
  return true;
}

int main() {
  if (!check_find_block()) return 1;
  if (!check_seg_len()) return 1;
  if (!check_compares()) return 1;
  const int shapes[][3] = {{1, 1, 1},   {2, 3, 5},    {7, 1, 4},    {8, 8, 8},    {16, 9, 3},  {21, 13, 10},
                           {30, 9, 17}, {33, 3, 1},   {31, 2, 6},   {64, 5, 4},   {96, 3, 2},  {104, 2, 3},
                           {128, 2, 2}, {129, 3, 2},  {255, 2, 1},  {3, 128, 2},  {2, 3, 128}};
  const int Ls[] = {1, 2, 3, 4, 8, 16};
  int cases = 0;
  for (const auto& n : shapes) {
    if (!check_fmc<1>(n, 16) || !check_fmc<2>(n, 16)) return 1;
    for (int L : Ls) {
      if (!check_fmc<0>(n, L)) return 1;
      if (!check<0>(n, L) || !check<1>(n, L) || !check<2>(n, L)) return 1;
      cases += 3;
    }
  }
  std::printf("ok %d cases\n", cases);
  return 0;
}
