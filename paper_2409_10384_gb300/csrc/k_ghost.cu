// Ghost zones from same-level neighbours (no prolongation or restriction) and
// zero-gradient outflow, for the conserved variables and the face fields.
// Every source value is an interior value of some block, so one pass over all
// ghost entries, in any order, is free of races.
#include "dev.cuh"
#include "internal.h"

namespace grmhd {

// Region of index x along an axis with interior [g, g + n) (cells) or
// [g, g + n] (faces normal to the axis): -1 below, 0 inside, +1 above.
__device__ __forceinline__ int region(int x, int g, int n, bool normal_face) {
  if (x < g) return -1;
  if (normal_face ? x > g + n : x >= g + n) return 1;
  return 0;
}
// Source index along the axis for region r.  Neighbour block of the same
// size: shift by n.  Outflow: the block's own boundary cell or face.
__device__ __forceinline__ int src_index(int x, int r, int g, int n, bool normal_face, bool outflow) {
  if (r == 0) return x;
  if (!outflow) return r < 0 ? x + n : x - n;
  if (r < 0) return g;
  return normal_face ? g + n : g + n - 1;
}

// kind 0: cells (5 conserved components); kind 1 + d: face field d.
__global__ void __launch_bounds__(256) k_fill_ghosts(Work w, const int* __restrict__ nbr, int kind) {
  const int K = kind == 0 ? W_INIT : W_GFX + kind - 1;
  const long long* pre = w.pre + (long long)K * (w.nblocks + 1);
  const long long tot = pre[w.nblocks];
  const int d = kind - 1;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < tot; it += (long long)gridDim.x * blockDim.x) {
    const int bi = find_block(w, K, it);
    const DevBlock& b = w.blk[bi];
    long long loc = it - pre[bi];
    const int L0 = b.N[0] + (d == 0), L1 = b.N[1] + (d == 1);
    const int i = (int)(loc % L0);
    loc /= L0;
    const int j = (int)(loc % L1);
    const int k = (int)(loc / L1);
    const int g = b.ng;
    const int ri = region(i, g, b.n[0], d == 0), rj = region(j, g, b.n[1], d == 1), rk = region(k, g, b.n[2], d == 2);
    if ((ri | rj | rk) == 0) continue;
    const int s = nbr[(long long)b.id * 27 + (rk + 1) * 9 + (rj + 1) * 3 + (ri + 1)];
    if (s < -1) continue;
    const bool out = s == -1;
    const DevBlock& a = out ? b : w.blk[s - (b.id - bi)];   // w.blk may start at an offset of the list
    const int si = src_index(i, ri, g, b.n[0], d == 0, out), sj = src_index(j, rj, g, b.n[1], d == 1, out),
              sk = src_index(k, rk, g, b.n[2], d == 2, out);
    if (kind == 0) {
      const long long c = cidx(b, k, j, i), sc = cidx(a, sk, sj, si);
#pragma unroll
      for (int v = 0; v < 5; v++) b.cons[v * b.ncell + c] = a.cons[v * a.ncell + sc];
    } else {
      b.bf[d][fidx(b, d, k, j, i)] = a.bf[d][fidx(a, d, sk, sj, si)];
    }
  }
}

void launch_fill_ghosts(const Work& w, const int* nbr, int kind, cudaStream_t s, int grid) {
  k_fill_ghosts<<<grid, 256, 0, s>>>(w, nbr, kind);
}

}  // namespace grmhd
