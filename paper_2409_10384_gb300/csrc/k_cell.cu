// Cell-centred kernels: initial data, prim->cons, con2prim (Sec. 3.4) on
// independent cells and on the stencil region of every meshblock.
#include "dev.cuh"
#include "internal.h"

namespace grmhd {

// ---------------------------------------------------------------- init data
// face B~ = discrete curl of the edge potential, every face of the arrays
__global__ void k_init_faces(DevBlock b, const double* __restrict__ Ax, const double* __restrict__ Ay,
                             const double* __restrict__ Az) {
  const int N0 = b.N[0], N1 = b.N[1], N2 = b.N[2];
  const long long nx = (long long)N2 * N1 * (N0 + 1), ny = (long long)N2 * (N1 + 1) * N0,
                  nz = (long long)(N2 + 1) * N1 * N0;
  const long long tot = nx + ny + nz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    if (t < nx) {
      int i = t % (N0 + 1); long long r = t / (N0 + 1); int j = r % N1; int k = r / N1;
      b.bf[0][fidx(b, 0, k, j, i)] = (Az[eidx(b, 2, k, j + 1, i)] - Az[eidx(b, 2, k, j, i)]) * b.idx[1] -
                                     (Ay[eidx(b, 1, k + 1, j, i)] - Ay[eidx(b, 1, k, j, i)]) * b.idx[2];
    } else if (t < nx + ny) {
      long long u = t - nx;
      int i = u % N0; long long r = u / N0; int j = r % (N1 + 1); int k = r / (N1 + 1);
      b.bf[1][fidx(b, 1, k, j, i)] = (Ax[eidx(b, 0, k + 1, j, i)] - Ax[eidx(b, 0, k, j, i)]) * b.idx[2] -
                                     (Az[eidx(b, 2, k, j, i + 1)] - Az[eidx(b, 2, k, j, i)]) * b.idx[0];
    } else {
      long long u = t - nx - ny;
      int i = u % N0; long long r = u / N0; int j = r % N1; int k = r / N1;
      b.bf[2][fidx(b, 2, k, j, i)] = (Ay[eidx(b, 1, k, j, i + 1)] - Ay[eidx(b, 1, k, j, i)]) * b.idx[0] -
                                     (Ax[eidx(b, 0, k, j + 1, i)] - Ax[eidx(b, 0, k, j, i)]) * b.idx[1];
    }
  }
}

__device__ __forceinline__ void load_metric(const DevBlock& b, long long c, Metric& m) {
#pragma unroll
  for (int v = 0; v < 6; v++) m.g[v] = b.adm[(4 + v) * b.ncell + c];
  metric_setup(m);
}

__device__ __forceinline__ void cell_bcc(const DevBlock& b, int k, int j, int i, double* Bd) {
  Bd[0] = 0.5 * (b.bf[0][fidx(b, 0, k, j, i)] + b.bf[0][fidx(b, 0, k, j, i + 1)]);
  Bd[1] = 0.5 * (b.bf[1][fidx(b, 1, k, j, i)] + b.bf[1][fidx(b, 1, k, j + 1, i)]);
  Bd[2] = 0.5 * (b.bf[2][fidx(b, 2, k, j, i)] + b.bf[2][fidx(b, 2, k + 1, j, i)]);
}

// bcc and cons (Eq. 6) of blk.prim on every cell
__global__ void k_init_cells(DevBlock b, Par P) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < b.ncell; c += (long long)gridDim.x * blockDim.x) {
    int i = c % b.N[0]; long long r = c / b.N[0]; int j = r % b.N[1]; int k = r / b.N[1];
    double Bd[3];
    cell_bcc(b, k, j, i, Bd);
#pragma unroll
    for (int v = 0; v < 3; v++) b.bcc[v * b.ncell + c] = Bd[v];
    Metric m;
    load_metric(b, c, m);
    double pr[5], U[5];
#pragma unroll
    for (int v = 0; v < 5; v++) pr[v] = b.prim[v * b.ncell + c];
    prim2cons(P, pr, Bd, m, U);
#pragma unroll
    for (int v = 0; v < 5; v++) b.cons[v * b.ncell + c] = U[v];
  }
}

// ------------------------------------------------------------ flat cell arrays
__global__ void k_p2c_cells(Par P, long long n, const double* __restrict__ prim, const double* __restrict__ Bd,
                            const double* __restrict__ g, double* __restrict__ cons) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    Metric m;
#pragma unroll
    for (int v = 0; v < 6; v++) m.g[v] = g[v * n + c];
    metric_setup(m);
    double pr[5], B[3], U[5];
#pragma unroll
    for (int v = 0; v < 5; v++) pr[v] = prim[v * n + c];
#pragma unroll
    for (int v = 0; v < 3; v++) B[v] = Bd[v * n + c];
    prim2cons(P, pr, B, m, U);
#pragma unroll
    for (int v = 0; v < 5; v++) cons[v * n + c] = U[v];
  }
}

__global__ void __launch_bounds__(128) k_c2p_cells(Par P, long long n, double* __restrict__ cons,
                                                   const double* __restrict__ Bd, const double* __restrict__ g,
                                                   double* __restrict__ prim, unsigned char* __restrict__ flags,
                                                   int* __restrict__ iters_out, const float* __restrict__ guess,
                                                   unsigned long long* stats) {
  unsigned s_cells = 0, s_iters = 0, s_fail = 0, s_floor = 0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    Metric m;
#pragma unroll
    for (int v = 0; v < 6; v++) m.g[v] = g[v * n + c];
    metric_setup(m);
    double U[5], B[3], pr[5];
#pragma unroll
    for (int v = 0; v < 5; v++) U[v] = cons[v * n + c];
#pragma unroll
    for (int v = 0; v < 3; v++) B[v] = Bd[v * n + c];
    unsigned fl;
    int it;
    double lo = -1.0, hi = -1.0;
    if (guess) {
      lo = guess[2 * c];
      hi = guess[2 * c + 1];
    }
    con2prim(P, U, B, m, pr, fl, it, true, lo, hi);
#pragma unroll
    for (int v = 0; v < 5; v++) prim[v * n + c] = pr[v];
    if (fl & (FLOOR_BITS | F_FAIL)) {
#pragma unroll
      for (int v = 0; v < 5; v++) cons[v * n + c] = U[v];
    }
    flags[c] = (unsigned char)fl;
    if (iters_out) iters_out[c] = it;
    s_cells++;
    s_iters += it;
    s_fail += (fl & F_FAIL) ? 1u : 0u;
    s_floor += (fl & FLOOR_BITS) ? 1u : 0u;
  }
  warp_flush(&stats[0], s_cells);
  warp_flush(&stats[1], s_iters);
  warp_flush(&stats[2], s_fail);
  warp_flush(&stats[3], s_floor);
}

// ------------------------------------------------------ block stencil region
// con2prim of every cell within 3 of the interior, with bcc; the cell-centred
// E = -(alpha v - beta) x B~ on cells within 1 of the interior.
__global__ void __launch_bounds__(128) k_c2p_block(Work w, Par P, unsigned long long* stats) {
  const long long* pre = w.pre + (long long)W_C2P * (w.nblocks + 1);
  const long long tot = pre[w.nblocks];
  unsigned s_cells = 0, s_iters = 0, s_fail = 0, s_floor = 0;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < tot; it += (long long)gridDim.x * blockDim.x) {
    const int bi = find_block(w, W_C2P, it);
    const DevBlock& b = w.blk[bi];
    long long loc = it - pre[bi];
    const int R0 = b.n[0] + 6, R1 = b.n[1] + 6;
    int ii = loc % R0; long long r = loc / R0; int jj = r % R1; int kk = r / R1;
    const int i = ii + b.ng - 3, j = jj + b.ng - 3, k = kk + b.ng - 3;
    const long long c = cidx(b, k, j, i);
    const long long nc = b.ncell;
    double Bd[3];
    cell_bcc(b, k, j, i, Bd);
#pragma unroll
    for (int v = 0; v < 3; v++) b.bcc[v * nc + c] = Bd[v];
    Metric m;
    load_metric(b, c, m);
    double U[5], pr[5], iW;
#pragma unroll
    for (int v = 0; v < 5; v++) U[v] = b.cons[v * nc + c];
    unsigned fl;
    int itn;
    con2prim(P, U, Bd, m, pr, fl, itn, true, -1.0, -1.0, b.adm[c], &iW);
#pragma unroll
    for (int v = 0; v < 5; v++) b.prim[v * nc + c] = pr[v];
    if (fl & (FLOOR_BITS | F_FAIL)) {
#pragma unroll
      for (int v = 0; v < 5; v++) b.cons[v * nc + c] = U[v];
    }
    b.flags[c] = (unsigned char)fl;
    if (ii >= 2 && ii <= b.n[0] + 3 && jj >= 2 && jj <= b.n[1] + 3 && kk >= 2 && kk <= b.n[2] + 3) {
      const double alpha = b.adm[c];
      const double be0 = b.adm[nc + c], be1 = b.adm[2 * nc + c], be2 = b.adm[3 * nc + c];
      // alpha v^i - beta^i with 1/W from the recovery
      const double aiW = alpha * iW;
      double a0 = fma(aiW, pr[1], -be0), a1 = fma(aiW, pr[2], -be1), a2 = fma(aiW, pr[3], -be2);
      b.ecc[c] = -(a1 * Bd[2] - a2 * Bd[1]);
      b.ecc[nc + c] = -(a2 * Bd[0] - a0 * Bd[2]);
      b.ecc[2 * nc + c] = -(a0 * Bd[1] - a1 * Bd[0]);
    }
    s_cells++;
    s_iters += itn;
    s_fail += (fl & F_FAIL) ? 1u : 0u;
    s_floor += (fl & FLOOR_BITS) ? 1u : 0u;
  }
  warp_flush(&stats[0], s_cells);
  warp_flush(&stats[1], s_iters);
  warp_flush(&stats[2], s_fail);
  warp_flush(&stats[3], s_floor);
}

// The fast reciprocal against the correctly rounded division: out[i] = the
// relative difference of a * rcp_nr(x) from a / x, for a = 1 and a = x + 1.
__global__ void k_check_rcp(const double* __restrict__ x, long long n, double* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = x[i];
    const double r = rcp_nr(v), q = 1.0 / v;
    const double a = v + 1.0, qa = a / v, ra = a * r;
    out[2 * i] = fabs(r - q) / fabs(q);
    out[2 * i + 1] = qa != 0.0 ? fabs(ra - qa) / fabs(qa) : fabs(ra);
  }
}
void launch_check_rcp(const double* x, long long n, double* out, cudaStream_t s, int nsm) {
  long long nb = (n + 255) / 256;
  int grid = (int)(nb < (long long)nsm * 8 ? nb : (long long)nsm * 8);
  k_check_rcp<<<grid < 1 ? 1 : grid, 256, 0, s>>>(x, n, out);
}

// The FP32 enclosures of the FOFC decision (ival.cuh) against FP64 values:
// out[i] has bit 0 set when iv_d(x) misses x, bit 1 when ircp misses 1/|x|,
// bit 2 when irsqrt misses 1/sqrt(|x|), bit 3 when imul misses x y, bit 4
// when imulp misses x |y|, bit 5 when isq misses x^2, bit 6 when iadd / isub
// miss x + y / x - y (y = x[(i + 1) % n]).  Values whose FP32 image is not a
// normal float only check iv_d.  A NaN interval (what iv_d gives outside the
// FP32 range) claims nothing and decides nothing, so it counts as enclosing.
__global__ void k_check_iv(const double* __restrict__ x, long long n, unsigned char* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = x[i], u = x[(i + 1) % n];
    const Iv a = iv_d(v), b = iv_d(u);
    auto in = [](Iv r, double t) { return r.lo != r.lo || r.hi != r.hi || ((double)r.lo <= t && t <= (double)r.hi); };
    unsigned char f = 0;
    if (!in(a, v)) f |= 1;
    const double av = fabs(v), au = fabs(u);
    const bool nv = av >= 1.2e-38 && av < 3.0e38, nu = au >= 1.2e-38 && au < 3.0e38;
    if (nv) {
      const Iv aa = iv_d(av);
      if (!in(ircp(aa), 1.0 / av)) f |= 2;
      if (!in(irsqrt(aa), 1.0 / sqrt(av))) f |= 4;
      if (!in(isq(a), v * v)) f |= 32;
      if (nu) {
        if (!in(imul(a, b), v * u)) f |= 8;
        if (!in(imulp(a, iv_d(au)), v * au)) f |= 16;
        if (!in(iadd(a, b), v + u) || !in(isub(a, b), v - u)) f |= 64;
      }
    }
    out[i] = f;
  }
}
void launch_check_iv(const double* x, long long n, unsigned char* out, cudaStream_t s, int nsm) {
  long long nb = (n + 255) / 256;
  int grid = (int)(nb < (long long)nsm * 8 ? nb : (long long)nsm * 8);
  k_check_iv<<<grid < 1 ? 1 : grid, 256, 0, s>>>(x, n, out);
}

// ------------------------------------------------------------------ launchers
void launch_init_block(const DevBlock& b, const Par& P, const double* const A[3], cudaStream_t s, int nsm) {
  k_init_faces<<<nsm * 8, 256, 0, s>>>(b, A[0], A[1], A[2]);
  k_init_cells<<<nsm * 8, 256, 0, s>>>(b, P);
}
void launch_p2c_cells(const Par& P, long long n, const double* prim, const double* Bd, const double* g, double* cons,
                      cudaStream_t s, int nsm) {
  long long nb = (n + 255) / 256;
  int grid = (int)(nb < (long long)nsm * 16 ? nb : (long long)nsm * 16);
  if (grid < 1) grid = 1;
  k_p2c_cells<<<grid, 256, 0, s>>>(P, n, prim, Bd, g, cons);
}
void launch_c2p_cells(const Par& P, long long n, double* cons, const double* Bd, const double* g, double* prim,
                      unsigned char* flags, int* iters, const float* guess, unsigned long long* stats, cudaStream_t s,
                      int grid) {
  k_c2p_cells<<<grid, 128, 0, s>>>(P, n, cons, Bd, g, prim, flags, iters, guess, stats);
}
void launch_c2p_block(const Work& w, const Par& P, unsigned long long* stats, cudaStream_t s, int grid) {
  k_c2p_block<<<grid, 128, 0, s>>>(w, P, stats);
}

int occupancy_c2p(int* per_sm) {
  int a = 0, b = 0;
  cudaError_t e1 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_c2p_cells, 128, 0);
  cudaError_t e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_c2p_block, 128, 0);
  per_sm[0] = a;
  per_sm[1] = b;
  return (e1 == cudaSuccess && e2 == cudaSuccess) ? 0 : -1;
}

}  // namespace grmhd
