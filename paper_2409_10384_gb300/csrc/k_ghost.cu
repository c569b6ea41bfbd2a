// Ghost zones from same-level neighbours (no prolongation or restriction) and
// zero-gradient outflow, for the conserved variables and the face fields.
// Three passes, x then y then z: pass a fills the ghost layers along axis a
// over the whole extent of the other two axes, copying from interior indices
// along a (of the block itself or a neighbour) at the same indices along the
// other axes, which earlier passes have already filled where they are
// ghosts.  Edges and corners thus come out right for any mix of neighbours,
// periodic wraps and outflow sides.  Within a pass every read is interior
// along a and every write a ghost along a, so a pass is free of races.
#include "dev.cuh"
#include "internal.h"

namespace grmhd {

// kind 0: cells (5 conserved components); kind 1 + d: face field d.  ax: the
// axis of this pass.  nbr [nblocks][6]: (-x, +x, -y, +y, -z, +z).
__global__ void __launch_bounds__(256) k_fill_ghosts(Work w, const int* __restrict__ nbr, int kind, int ax) {
  const int K = kind == 0 ? W_INIT : W_GFX + kind - 1;
  const long long* pre = w.pre + (long long)K * (w.nblocks + 1);
  const long long tot = pre[w.nblocks];
  const int d = kind - 1;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < tot; it += (long long)gridDim.x * blockDim.x) {
    const int bi = find_block(w, K, it);
    const DevBlock& b = w.blk[bi];
    long long loc = it - pre[bi];
    const int L0 = b.N[0] + (d == 0), L1 = b.N[1] + (d == 1);
    int x[3];
    x[0] = (int)(loc % L0);
    loc /= L0;
    x[1] = (int)(loc % L1);
    x[2] = (int)(loc / L1);
    const int g = b.ng, n = b.n[ax];
    const bool normal = d == ax;   // face array normal to this pass's axis
    const int v = x[ax];
    int r = 0;
    if (v < g) r = -1;
    else if (normal ? v > g + n : v >= g + n) r = 1;
    if (r == 0) continue;
    const int s = nbr[(long long)b.id * 6 + 2 * ax + (r > 0)];
    if (s < -1) continue;
    int y[3] = {x[0], x[1], x[2]};
    if (s == -1) {                       // zero-gradient outflow
      y[ax] = r < 0 ? g : (normal ? g + n : g + n - 1);
    } else if (s == b.id) {              // periodic wrap onto the block itself: modulo n
      y[ax] = g + (((v - g) % n) + n) % n;
    } else {                             // neighbour of the same size (n >= g)
      y[ax] = r < 0 ? v + n : v - n;
    }
    const DevBlock& a = s == -1 ? b : w.blk[s - (b.id - bi)];   // w.blk may start at an offset of the list
    if (kind == 0) {
      const long long c = cidx(b, x[2], x[1], x[0]), sc = cidx(a, y[2], y[1], y[0]);
#pragma unroll
      for (int q = 0; q < 5; q++) b.cons[q * b.ncell + c] = a.cons[q * a.ncell + sc];
    } else {
      b.bf[d][fidx(b, d, x[2], x[1], x[0])] = a.bf[d][fidx(a, d, y[2], y[1], y[0])];
    }
  }
}

void launch_fill_ghosts(const Work& w, const int* nbr, int kind, int ax, cudaStream_t s, int grid) {
  k_fill_ghosts<<<grid, 256, 0, s>>>(w, nbr, kind, ax);
}

}  // namespace grmhd
