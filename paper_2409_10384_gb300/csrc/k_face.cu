// Face kernels: reconstruction (Sec. 3.2) and the LLF/HLLE flux of Eq. 8 with
// the ADM metric interpolated to the face, and the first-order flux
// correction of Sec. 3.3 with the relaxed DMP of Eq. 19.
#include "dev.cuh"
#include "flux_sweep.cuh"
#include "internal.h"

namespace grmhd {

// First-order (donor cell) flux through face (k,j,i) of direction d.
template <int d>
__device__ __forceinline__ void face_flux_donor(const DevBlock& b, const Par& P, int k, int j, int i, double* F) {
  constexpr int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  const long long nc = b.ncell;
  const long long c0 = cidx(b, k, j, i);
  const long long st = d == 0 ? 1 : (d == 1 ? (long long)b.N[0] : (long long)b.N[0] * b.N[1]);
  double L[7], R[7];
#pragma unroll
  for (int v = 0; v < 7; v++) {
    const double* a = v < 5 ? b.prim + v * nc : b.bcc + (v == 5 ? t1 : t2) * nc;
    L[v] = a[c0 - st];
    R[v] = a[c0];
  }
  FaceMetric fm;
  face_metric(b.adm, nc, c0 - st, st, fm);
  const double Bn = b.bf[d][fidx(b, d, k, j, i)];
  if (P.eos == 0) face_flux_states<d, 0>(P, L, R, Bn, fm, F);
  else face_flux_states<d, 1>(P, L, R, Bn, fm, F);
}

__device__ __forceinline__ bool interior(const DevBlock& b, int k, int j, int i) {
  return (unsigned)(i - b.ng) < (unsigned)b.n[0] && (unsigned)(j - b.ng) < (unsigned)b.n[1] &&
         (unsigned)(k - b.ng) < (unsigned)b.n[2];
}

// FOFC flag: U* = g0 U^n + g1 U + b dt (-div F) (no sources, no CT, B at the
// stage's bcc); flag when con2prim of U* fails or needs a floor, or (DMP)
// when D~* or tau~* leaves [min/M, M max] of the 27 cells around (stage input).
__global__ void __launch_bounds__(128) k_fofc_flag(Work w, Par P, double g0, double g1, double bdt,
                                                   unsigned long long* stats) {
  const long long* pre = w.pre + (long long)W_CELL * (w.nblocks + 1);
  const long long tot = pre[w.nblocks];
  unsigned s_flag = 0, s_dmp = 0;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < tot; it += (long long)gridDim.x * blockDim.x) {
    const int bi = find_block(w, W_CELL, it);
    const DevBlock& b = w.blk[bi];
    long long loc = it - pre[bi];
    int i = loc % b.n[0]; long long r = loc / b.n[0]; int j = r % b.n[1]; int k = r / b.n[1];
    i += b.ng; j += b.ng; k += b.ng;
    const long long nc = b.ncell, c = cidx(b, k, j, i);
    const long long fx0 = fidx(b, 0, k, j, i), fy0 = fidx(b, 1, k, j, i), fz0 = fidx(b, 2, k, j, i);
    const long long fx1 = fx0 + 1, fy1 = fidx(b, 1, k, j + 1, i), fz1 = fidx(b, 2, k + 1, j, i);
    const long long nx = nface(b, 0), ny = nface(b, 1), nz = nface(b, 2);
    double U[5];
#pragma unroll
    for (int v = 0; v < 5; v++) {
      double div = (b.flux[0][v * nx + fx1] - b.flux[0][v * nx + fx0]) * b.idx[0] +
                   (b.flux[1][v * ny + fy1] - b.flux[1][v * ny + fy0]) * b.idx[1] +
                   (b.flux[2][v * nz + fz1] - b.flux[2][v * nz + fz0]) * b.idx[2];
      double u = g1 * b.cons[v * nc + c];
      if (g0 != 0.0) u = fma(g0, b.cons0[v * nc + c], u);
      U[v] = fma(-bdt, div, u);
    }
    Metric m;
#pragma unroll
    for (int v = 0; v < 6; v++) m.g[v] = b.adm[(4 + v) * nc + c];
    metric_setup(m);
    double Bd[3] = {b.bcc[c], b.bcc[nc + c], b.bcc[2 * nc + c]};
    double pr[5];
    unsigned fl;
    int itn;
    con2prim(P, U, Bd, m, pr, fl, itn, false, -1.0, -1.0, b.adm[c]);
    bool flag = (fl & (FLOOR_BITS | F_FAIL)) != 0;
    if (!flag && P.dmp_M > 0.0) {
#pragma unroll
      for (int t = 0; t < 2; t++) {
        const int v = t == 0 ? 0 : 4;
        const double* a = b.cons + v * nc;
        double mn = a[c], mx = mn;
        for (int dk = -1; dk <= 1; dk++)
          for (int dj = -1; dj <= 1; dj++)
#pragma unroll
            for (int di = -1; di <= 1; di++) {
              double u = a[cidx(b, k + dk, j + dj, i + di)];
              mn = fmin(mn, u);
              mx = fmax(mx, u);
            }
        const double M = P.dmp_M;
        double lo = mn > 0.0 ? mn / M : mn * M;
        double hi = mx > 0.0 ? mx * M : mx / M;
        if (U[v] < lo || U[v] > hi) flag = true;
      }
      s_dmp += flag ? 1u : 0u;
    }
    b.fflag[c] = flag ? 1 : 0;
    unsigned char f0 = b.flags[c];
    b.flags[c] = flag ? (unsigned char)(f0 | F_FOFC) : (unsigned char)(f0 & ~F_FOFC);
    s_flag += flag ? 1u : 0u;
  }
  warp_flush(&stats[4], s_flag);
  warp_flush(&stats[5], s_dmp);
}

// First-order recompute of every face touching a flagged interior cell.
template <int d>
__global__ void __launch_bounds__(128) k_fofc_fix(Work w, Par P, unsigned long long* stats) {
  const long long* pre = w.pre + (long long)(W_FX + d) * (w.nblocks + 1);
  const long long tot = pre[w.nblocks];
  unsigned s_faces = 0;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < tot; it += (long long)gridDim.x * blockDim.x) {
    const int bi = find_block(w, W_FX + d, it);
    const DevBlock& b = w.blk[bi];
    int k, j, i;
    face_coords<d>(b, it - pre[bi], k, j, i);
    const int km = k - (d == 2), jm = j - (d == 1), im = i - (d == 0);
    bool fl = (interior(b, k, j, i) && b.fflag[cidx(b, k, j, i)]) ||
              (interior(b, km, jm, im) && b.fflag[cidx(b, km, jm, im)]);
    if (!fl) continue;
    double F[7];
    face_flux_donor<d>(b, P, k, j, i, F);
    const long long f = fidx(b, d, k, j, i), nf = nface(b, d);
    double* out = b.flux[d];
#pragma unroll
    for (int c = 0; c < 7; c++) out[c * nf + f] = F[c];
    s_faces++;
  }
  warp_flush(&stats[6], s_faces);
}

// The same recompute from the list of flagged interior cells that
// k_krp_finish_fofc keeps (kb.flist): each cell takes its lower face along
// each axis, and its upper face unless the cell above is a flagged interior
// cell (which takes that face as its lower one), so every face touching a
// flagged cell is recomputed once, with the values k_fofc_fix gives.
template <int d>
__device__ __forceinline__ void fix_face(const DevBlock& b, const Par& P, int k, int j, int i, unsigned& n) {
  double F[7];
  face_flux_donor<d>(b, P, k, j, i, F);
  const long long f = fidx(b, d, k, j, i), nf = nface(b, d);
  double* out = b.flux[d];
#pragma unroll
  for (int c = 0; c < 7; c++) out[c * nf + f] = F[c];
  n++;
}
__global__ void __launch_bounds__(128) k_fofc_fix_list(Work w, Par P, const unsigned long long* __restrict__ list,
                                                       long long cap, unsigned long long* stats) {
  const long long cnt = (long long)list[0];
  const long long n = cnt < cap ? cnt : cap;
  unsigned s_faces = 0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    int bi, k, j, i;
    fofc_cell(w, (long long)list[1 + q], bi, k, j, i);
    const DevBlock& b = w.blk[bi];
    fix_face<0>(b, P, k, j, i, s_faces);
    fix_face<1>(b, P, k, j, i, s_faces);
    fix_face<2>(b, P, k, j, i, s_faces);
    if (!(interior(b, k, j, i + 1) && b.fflag[cidx(b, k, j, i + 1)])) fix_face<0>(b, P, k, j, i + 1, s_faces);
    if (!(interior(b, k, j + 1, i) && b.fflag[cidx(b, k, j + 1, i)])) fix_face<1>(b, P, k, j + 1, i, s_faces);
    if (!(interior(b, k + 1, j, i) && b.fflag[cidx(b, k + 1, j, i)])) fix_face<2>(b, P, k + 1, j, i, s_faces);
  }
  warp_flush(&stats[6], s_faces);
}

// The metric of one RK step (Z4c is not evolved: the ADM variables are an
// input of the whole step): sqrt(gamma), 1/sqrt(gamma) and gamma^ij of every
// cell of the con2prim region (DevBlock.mc), the interpolated face metric of
// every face the flux sweeps visit (DevBlock.fmc) and the centred derivatives
// of the metric at the interior cells (DevBlock.dmc, Eq. 9).  The context's RK step
// runs it once, before its first stage; the stage-by-stage entry points run it
// in every mhd_c2p.
// One thread per face, x fastest (the four-point reads of the ADM variables
// coalesce).  y and z store at the item index itself; x at its segment-major
// slot, where neighbouring segments' faces (lanes of the same or the next
// warp) complete each sector.
template <int d>
__device__ __forceinline__ void face_metric_items(const Work& w) {
  const long long* pre = w.pre + (long long)(W_FX + d) * (w.nblocks + 1);
  const long long tot = pre[w.nblocks];
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < tot; it += (long long)gridDim.x * blockDim.x) {
    const int bi = find_block(w, W_FX + d, it);
    const DevBlock& b = w.blk[bi];
    const long long loc = it - pre[bi];
    int k, j, i;
    face_coords<d>(b, loc, k, j, i);
    const long long st = d == 0 ? 1 : (d == 1 ? (long long)b.N[0] : (long long)b.N[0] * b.N[1]);
    FaceMetric fm;
    face_metric(b.adm, b.ncell, cidx(b, k, j, i) - st, st, fm);
    fmc_store<d>(b.fmc[d], fmc_count(b, d), d == 0 ? fmc_index(b, 0, k, j, i) : loc, fm);
  }
}
__global__ void __launch_bounds__(256) k_metric_cache(Work w) {
  const long long* pre = w.pre + (long long)W_C2P * (w.nblocks + 1);
  const long long tot = pre[w.nblocks];
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < tot; it += (long long)gridDim.x * blockDim.x) {
    const int bi = find_block(w, W_C2P, it);
    const DevBlock& b = w.blk[bi];
    const long long loc = it - pre[bi];
    const int R0 = b.n[0] + 6, R1 = b.n[1] + 6;
    const int ii = loc % R0; const long long r = loc / R0; const int jj = r % R1; const int kk = r / R1;
    const long long nc = b.ncell, c = cidx(b, kk + b.ng - 3, jj + b.ng - 3, ii + b.ng - 3);
    Metric m;
#pragma unroll
    for (int v = 0; v < 6; v++) m.g[v] = b.adm[(4 + v) * nc + c];
    metric_setup(m);
    metric_store(b.mc, nc, c, m);
  }
  face_metric_items<0>(w);
  face_metric_items<1>(w);
  face_metric_items<2>(w);
  // derivatives of the metric at the interior cells (Eq. 9 sources)
  const long long* pc = w.pre + (long long)W_CELL * (w.nblocks + 1);
  const long long tc = pc[w.nblocks];
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < tc; it += (long long)gridDim.x * blockDim.x) {
    const int bi = find_block(w, W_CELL, it);
    const DevBlock& b = w.blk[bi];
    const long long loc = it - pc[bi];
    const int i = loc % b.n[0]; const long long r = loc / b.n[0]; const int j = r % b.n[1]; const int k = r / b.n[1];
    double D[DMC_N];
    adm_derivs(b, cidx(b, k + b.ng, j + b.ng, i + b.ng), D);
    const long long ni = (long long)b.n[0] * b.n[1] * b.n[2];
#pragma unroll
    for (int v = 0; v < DMC_N; v++) b.dmc[v * ni + loc] = D[v];
  }
}
void launch_metric_cache(const Work& w, cudaStream_t s, int grid) { k_metric_cache<<<grid, 256, 0, s>>>(w); }
int occ_metric_kernel() {
  int o = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_metric_cache, 256, 0);
  return o;
}

void launch_flux_dir(int d, const Work& w, const Par& P, cudaStream_t s, int grid, int threads) {
  launch_flux_dir_c<1>(d, w, P, s, grid, threads);
}
void launch_fofc_flag(const Work& w, const Par& P, double g0, double g1, double bdt, unsigned long long* stats,
                      cudaStream_t s, int grid) {
  k_fofc_flag<<<grid, 128, 0, s>>>(w, P, g0, g1, bdt, stats);
}
void launch_fofc_fix_list(const Work& w, const Par& P, const unsigned long long* list, long long cap,
                          unsigned long long* stats, cudaStream_t s, int grid) {
  k_fofc_fix_list<<<grid, 128, 0, s>>>(w, P, list, cap, stats);
}
void launch_fofc_fix(int d, const Work& w, const Par& P, unsigned long long* stats, cudaStream_t s, int grid) {
  if (d == 0) k_fofc_fix<0><<<grid, 128, 0, s>>>(w, P, stats);
  else if (d == 1) k_fofc_fix<1><<<grid, 128, 0, s>>>(w, P, stats);
  else k_fofc_fix<2><<<grid, 128, 0, s>>>(w, P, stats);
}
int occ_face_kernel(int kind, int threads) {
  int o = 0;
  if (kind == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_flux<0, 2, 0, 1>, threads, 0);
  else if (kind == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_flux<1, 2, 0, 1>, threads, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_flux<2, 2, 0, 1>, threads, 0);
  return o;
}
int occupancy_face(int* per_sm) {
  cudaError_t e = cudaSuccess;
  e = (cudaError_t)(e | cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[0], k_flux<0, 2, 0, 1>, 128, 0));
  e = (cudaError_t)(e | cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[1], k_flux<1, 2, 0, 1>, 128, 0));
  e = (cudaError_t)(e | cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[2], k_flux<2, 2, 0, 1>, 128, 0));
  e = (cudaError_t)(e | cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[3], k_fofc_flag, 128, 0));
  e = (cudaError_t)(e | cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[4], k_fofc_fix<0>, 128, 0));
  return e == cudaSuccess ? 0 : -1;
}

}  // namespace grmhd
