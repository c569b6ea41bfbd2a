// The flux sweep kernel (Sec. 3.2 reconstruction, Eq. 8 fluxes), shared by
// two translation units: k_face.cu instantiates it reading the per-step face
// metric cache (C = 1), k_face_inline.cu computing the face metric in the
// sweep (C = 0, for the allocation-free stage, which has no room for the
// cache).
#pragma once
#include "dev.cuh"

namespace grmhd {

// Fluxes of direction d, one thread per segment: the thread sweeps the cells
// along d, reconstructing each once (order R) and finishing one face per cell.
// C = 1: the face metric comes from the block's cache (fmc); C = 0: it is
// interpolated and inverted here.
template <int d, int R, int E, int C>
__global__ void __launch_bounds__(256) k_flux(Work w, Par P) {
  constexpr int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  const long long* pre = w.pre + (long long)(W_SX + d) * (w.nblocks + 1);
  const long long tot = pre[w.nblocks];
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < tot; it += (long long)gridDim.x * blockDim.x) {
    const int bi = find_block(w, W_SX + d, it);
    const DevBlock& b = w.blk[bi];
    int k, j, i, nf;
    seg_coords<d>(b, (int)(it - pre[bi]), k, j, i, nf);
    const long long nc = b.ncell;
    const long long st = d == 0 ? 1 : (d == 1 ? (long long)b.N[0] : (long long)b.N[0] * b.N[1]);
    const long long fst = d == 0 ? 1 : (d == 1 ? (long long)b.N[0] : (long long)b.N[0] * b.N[1]);
    const long long nfc = nface(b, d);
    const double* src[7] = {b.prim, b.prim + nc, b.prim + 2 * nc, b.prim + 3 * nc, b.prim + 4 * nc,
                            b.bcc + t1 * nc, b.bcc + t2 * nc};
    long long c = cidx(b, k, j, i) - st;   // cell m below the first face
    long long f = fidx(b, d, k, j, i);
    long long fq = C ? fmc_index(b, d, k, j, i) : 0;   // face metric cache index
    const long long nq = C ? fmc_count(b, d) : 0;
    const long long qst = C ? fmc_step(b, d) : 0;
    RecVar rv[7];
    double Ls[7];
#pragma unroll
    for (int v = 0; v < 7; v++) {
      const double* a = src[v] + c;
      rec_init<R>(rv[v], a[-2 * st], a[-st], a[0], a[st]);
      if constexpr (R != 2) {
        double lo;
        rec_step<R>(rv[v], a[2 * st], lo, Ls[v]);
      }
    }
    if constexpr (R == 2) {
      double x[7], nh[7], nl[7], dh[7], dl[7], lo[7];
#pragma unroll
      for (int v = 0; v < 7; v++) wz_parts(rv[v], src[v][c + 2 * st], x[v], nh[v], nl[v], dh[v], dl[v]);
      wz_finish<7>(x, nh, nl, dh, dl, Ls, lo);
    }
    for (int q = 0; q < nf; q++) {
      c += st;
      double Rs[7], Lnext[7];
      if constexpr (R == 2) {
        double x[7], nh[7], nl[7], dh[7], dl[7];
#pragma unroll
        for (int v = 0; v < 7; v++) wz_parts(rv[v], src[v][c + 2 * st], x[v], nh[v], nl[v], dh[v], dl[v]);
        wz_finish<7>(x, nh, nl, dh, dl, Lnext, Rs);
      } else {
#pragma unroll
        for (int v = 0; v < 7; v++) rec_step<R>(rv[v], src[v][c + 2 * st], Rs[v], Lnext[v]);
      }
      FaceMetric fm;
      if constexpr (C) fmc_load<d>(b.fmc[d], nq, fq, fm);
      else face_metric(b.adm, nc, c - st, st, fm);
      double F[7];
      face_flux_states<d, E>(P, Ls, Rs, b.bf[d][f], fm, F);
      double* out = b.flux[d];
#pragma unroll
      for (int v = 0; v < 7; v++) out[v * nfc + f] = F[v];
#pragma unroll
      for (int v = 0; v < 7; v++) Ls[v] = Lnext[v];
      f += fst;
      fq += qst;
    }
  }
}


template <int d, int E, int C>
void launch_flux_r(const Work& w, const Par& P, cudaStream_t s, int grid, int threads) {
  switch (P.recon) {
    case 4: k_flux<d, 4, E, C><<<grid, threads, 0, s>>>(w, P); break;
    case 3: k_flux<d, 3, E, C><<<grid, threads, 0, s>>>(w, P); break;
    case 2: k_flux<d, 2, E, C><<<grid, threads, 0, s>>>(w, P); break;
    case 1: k_flux<d, 1, E, C><<<grid, threads, 0, s>>>(w, P); break;
    default: k_flux<d, 0, E, C><<<grid, threads, 0, s>>>(w, P); break;
  }
}
template <int C>
void launch_flux_dir_c(int d, const Work& w, const Par& P, cudaStream_t s, int grid, int threads) {
  if (P.eos == 0) {
    if (d == 0) launch_flux_r<0, 0, C>(w, P, s, grid, threads);
    else if (d == 1) launch_flux_r<1, 0, C>(w, P, s, grid, threads);
    else launch_flux_r<2, 0, C>(w, P, s, grid, threads);
  } else {
    if (d == 0) launch_flux_r<0, 1, C>(w, P, s, grid, threads);
    else if (d == 1) launch_flux_r<1, 1, C>(w, P, s, grid, threads);
    else launch_flux_r<2, 1, C>(w, P, s, grid, threads);
  }
}

}  // namespace grmhd
