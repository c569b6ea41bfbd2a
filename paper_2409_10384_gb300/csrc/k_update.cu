// Upwind constrained transport (Sec. 3.2, Gardiner & Stone 2005) and the SSP-RK
// update of the conserved variables with the Eq. 9 sources and of the face B~.
#include "dev.cuh"
#include "internal.h"

namespace grmhd {

// Edge EMF of component cc at edge index (k,j,i) in the plane a = (cc+1)%3,
// b = (cc+2)%3: on a-faces E_cc = -F_a[5], on b-faces E_cc = +F_b[6].
template <int cc>
__device__ __forceinline__ double edge_emf(const DevBlock& b, int k, int j, int i) {
  constexpr int a = (cc + 1) % 3, bx = (cc + 2) % 3;
  int x[3] = {i, j, k};
  auto off = [&](int da, int db, int& kk, int& jj, int& ii) {
    int y[3] = {x[0], x[1], x[2]};
    y[a] += da;
    y[bx] += db;
    ii = y[0]; jj = y[1]; kk = y[2];
  };
  const double* Fa = b.flux[a];
  const double* Fb = b.flux[bx];
  const long long na = nface(b, a), nb = nface(b, bx);
  const double* E = b.ecc + cc * b.ncell;
  int kk, jj, ii;
  off(0, 0, kk, jj, ii);
  const long long fa0 = fidx(b, a, kk, jj, ii), fb0 = fidx(b, bx, kk, jj, ii), c00 = cidx(b, kk, jj, ii);
  off(0, -1, kk, jj, ii);
  const long long fa1 = fidx(b, a, kk, jj, ii), c01 = cidx(b, kk, jj, ii);
  off(-1, 0, kk, jj, ii);
  const long long fb1 = fidx(b, bx, kk, jj, ii), c10 = cidx(b, kk, jj, ii);
  off(-1, -1, kk, jj, ii);
  const long long c11 = cidx(b, kk, jj, ii);
  const double Eaf_B = -Fa[5 * na + fa0], Eaf_Bm = -Fa[5 * na + fa1];
  const double fDa_B = Fa[fa0], fDa_Bm = Fa[fa1];
  const double Ebf_A = Fb[6 * nb + fb0], Ebf_Am = Fb[6 * nb + fb1];
  const double fDb_A = Fb[fb0], fDb_Am = Fb[fb1];
  const double E_AB = E[c00], E_ABm = E[c01], E_AmB = E[c10], E_AmBm = E[c11];
  const double dEb_q = upw(fDa_B, E_AmB, Ebf_Am, E_AB, Ebf_A);
  const double dEb_tq = upw(fDa_Bm, Ebf_Am, E_AmBm, Ebf_A, E_ABm);
  const double dEa_q = upw(fDb_A, E_ABm, Eaf_Bm, E_AB, Eaf_B);
  const double dEa_tq = upw(fDb_Am, Eaf_Bm, E_AmBm, Eaf_B, E_AmB);
  return 0.25 * ((Eaf_B + Eaf_Bm) + (Ebf_A + Ebf_Am) + (dEb_tq - dEb_q) + (dEa_tq - dEa_q));
}

__global__ void __launch_bounds__(256) k_emf(Work w) {
  const long long* pre = w.pre + (long long)W_EDGE * (w.nblocks + 1);
  const long long tot = pre[w.nblocks];
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < tot; it += (long long)gridDim.x * blockDim.x) {
    const int bi = find_block(w, W_EDGE, it);
    const DevBlock& b = w.blk[bi];
    long long loc = it - pre[bi];
    const int L0 = b.n[0] + 1, L1 = b.n[1] + 1;
    int i = loc % L0; long long r = loc / L0; int j = r % L1; int k = r / L1;
    const bool xin = i < b.n[0], yin = j < b.n[1], zin = k < b.n[2];
    i += b.ng; j += b.ng; k += b.ng;
    if (xin) b.emf[0][eidx(b, 0, k, j, i)] = edge_emf<0>(b, k, j, i);
    if (yin) b.emf[1][eidx(b, 1, k, j, i)] = edge_emf<1>(b, k, j, i);
    if (zin) b.emf[2][eidx(b, 2, k, j, i)] = edge_emf<2>(b, k, j, i);
  }
}

// Sources of Eq. 9 at interior cell (k, j, i) (G[0] = 0 for D~).
__device__ __forceinline__ void sources(const DevBlock& b, const Par& P, int k, int j, int i, double* G) {
  const long long nc = b.ncell, c = cidx(b, k, j, i);
  const double* A = b.adm;
  Metric m;
  metric_cell(A, b.mc, nc, c, m);
  const double alpha = A[c];
  // centred derivatives of alpha, beta^i, gamma_ij: from the step's cache, or
  // taken here
  double D[DMC_N];
  if (b.dmc) {
    const long long ni = (long long)b.n[0] * b.n[1] * b.n[2];
    const long long q = ((long long)(k - b.ng) * b.n[1] + (j - b.ng)) * b.n[0] + (i - b.ng);
#pragma unroll
    for (int v = 0; v < DMC_N; v++) D[v] = b.dmc[v * ni + q];
  } else {
    adm_derivs(b, c, D);
  }
  double dal[3], dbe[3][3], dg[3][6];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    dal[a] = D[10 * a];
#pragma unroll
    for (int v = 0; v < 3; v++) dbe[a][v] = D[10 * a + 1 + v];
#pragma unroll
    for (int v = 0; v < 6; v++) dg[a][v] = D[10 * a + 4 + v];
  }
  const double* pr = b.prim;
  double rho = pr[c], p = pr[4 * nc + c];
  double w[3] = {pr[nc + c], pr[2 * nc + c], pr[3 * nc + c]};
  double wl[3];
  lower3(m.g, w, wl);
  const double iW = rsqrt(1.0 + dot3(w, wl));
  double B[3] = {b.bcc[c] * m.isdet, b.bcc[nc + c] * m.isdet, b.bcc[2 * nc + c] * m.isdet};
  double Bl[3];
  lower3(m.g, B, Bl);
  const double B2 = dot3(B, Bl), Bv = dot3(B, wl) * iW;   // B.v, with v_i = w_i / W
  const double b2 = fma(B2, iW * iW, Bv * Bv);
  const double rhoh = P.eos == 0 ? fma(P.gfac, p, rho) : eos_rhoh(P, rho, p);
  const double Ptot = fma(0.5, b2, p);
  // b^i = B^i/W + W (B.v) v^i = B^i/W + (B.v) w^i, and (rho h + b^2) W^2 v^i v^j
  // = (rho h + b^2) w^i w^j, with w^i = W v^i: no v^i or W needed
  const double bb[3] = {fma(Bv, w[0], B[0] * iW), fma(Bv, w[1], B[1] * iW), fma(Bv, w[2], B[2] * iW)};
  const double eh = rhoh + b2;
  // S^{ij} / sqrt(gamma); sqrt(gamma) rides in the coefficients of the contractions below
  double S[6];
  const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
  for (int q = 0; q < 6; q++)
    S[q] = fma(eh * w[ia[q]], w[ib[q]], fma(Ptot, m.gi[q], -bb[ia[q]] * bb[ib[q]]));
  const double* U = b.cons;
  double Sl[3] = {U[nc + c], U[2 * nc + c], U[3 * nc + c]};
  double Su[3];
  lower3(m.gi, Sl, Su);
  double E = U[4 * nc + c] + U[c];
  const double has = (0.5 * alpha) * m.sdet;   // alpha sqrt(gamma) / 2
  G[0] = 0.0;
  // S^{jk} d_i gamma_jk with the off-diagonal terms counted twice
#pragma unroll
  for (int a = 0; a < 3; a++) {
    double t = S[0] * dg[a][0] + S[3] * dg[a][3] + S[5] * dg[a][5] +
               2.0 * (S[1] * dg[a][1] + S[2] * dg[a][2] + S[4] * dg[a][4]);
    double s2 = dot3(Sl, dbe[a]);
    G[1 + a] = fma(has, t, fma(-E, dal[a], s2));
  }
  const double* K = A + 10 * nc + c;
  double kt = S[0] * K[0] + S[3] * K[3 * nc] + S[5] * K[5 * nc] + 2.0 * (S[1] * K[nc] + S[2] * K[2 * nc] + S[4] * K[4 * nc]);
  G[4] = fma(2.0 * has, kt, -dot3(Su, dal));
}

__global__ void __launch_bounds__(256) k_update_cells(Work w, Par P, double g0, double g1, double bdt, int first) {
  const long long* pre = w.pre + (long long)W_CELL * (w.nblocks + 1);
  const long long tot = pre[w.nblocks];
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < tot; it += (long long)gridDim.x * blockDim.x) {
    const int bi = find_block(w, W_CELL, it);
    const DevBlock& b = w.blk[bi];
    long long loc = it - pre[bi];
    int i = loc % b.n[0]; long long r = loc / b.n[0]; int j = r % b.n[1]; int k = r / b.n[1];
    i += b.ng; j += b.ng; k += b.ng;
    const long long nc = b.ncell, c = cidx(b, k, j, i);
    double G[5];
    sources(b, P, k, j, i, G);
    const long long fx0 = fidx(b, 0, k, j, i), fy0 = fidx(b, 1, k, j, i), fz0 = fidx(b, 2, k, j, i);
    const long long fx1 = fx0 + 1, fy1 = fidx(b, 1, k, j + 1, i), fz1 = fidx(b, 2, k + 1, j, i);
    const long long nx = nface(b, 0), ny = nface(b, 1), nz = nface(b, 2);
#pragma unroll
    for (int v = 0; v < 5; v++) {
      double div = (b.flux[0][v * nx + fx1] - b.flux[0][v * nx + fx0]) * b.idx[0] +
                   (b.flux[1][v * ny + fy1] - b.flux[1][v * ny + fy0]) * b.idx[1] +
                   (b.flux[2][v * nz + fz1] - b.flux[2][v * nz + fz0]) * b.idx[2];
      double u0 = b.cons[v * nc + c];
      double u = g1 * u0;
      if (first) b.cons0[v * nc + c] = u0;
      else u = fma(g0, b.cons0[v * nc + c], u);
      b.cons[v * nc + c] = fma(bdt, G[v] - div, u);
    }
  }
}

// face B~ <- g0 B^n + g1 B - b dt curl E on the faces bounding interior cells
__global__ void __launch_bounds__(256) k_update_faces(Work w, double g0, double g1, double bdt, int first) {
  const long long* pre = w.pre + (long long)W_FACE * (w.nblocks + 1);
  const long long tot = pre[w.nblocks];
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < tot; it += (long long)gridDim.x * blockDim.x) {
    const int bi = find_block(w, W_FACE, it);
    const DevBlock& b = w.blk[bi];
    long long loc = it - pre[bi];
    const long long nfx = (long long)(b.n[0] + 1) * b.n[1] * b.n[2], nfy = (long long)b.n[0] * (b.n[1] + 1) * b.n[2];
    int d, i, j, k;
    if (loc < nfx) {
      d = 0;
      i = loc % (b.n[0] + 1); long long r = loc / (b.n[0] + 1); j = r % b.n[1]; k = r / b.n[1];
    } else if (loc < nfx + nfy) {
      d = 1; loc -= nfx;
      i = loc % b.n[0]; long long r = loc / b.n[0]; j = r % (b.n[1] + 1); k = r / (b.n[1] + 1);
    } else {
      d = 2; loc -= nfx + nfy;
      i = loc % b.n[0]; long long r = loc / b.n[0]; j = r % b.n[1]; k = r / b.n[1];
    }
    i += b.ng; j += b.ng; k += b.ng;
    double curl;
    if (d == 0)
      curl = (b.emf[2][eidx(b, 2, k, j + 1, i)] - b.emf[2][eidx(b, 2, k, j, i)]) * b.idx[1] -
             (b.emf[1][eidx(b, 1, k + 1, j, i)] - b.emf[1][eidx(b, 1, k, j, i)]) * b.idx[2];
    else if (d == 1)
      curl = (b.emf[0][eidx(b, 0, k + 1, j, i)] - b.emf[0][eidx(b, 0, k, j, i)]) * b.idx[2] -
             (b.emf[2][eidx(b, 2, k, j, i + 1)] - b.emf[2][eidx(b, 2, k, j, i)]) * b.idx[0];
    else
      curl = (b.emf[1][eidx(b, 1, k, j, i + 1)] - b.emf[1][eidx(b, 1, k, j, i)]) * b.idx[0] -
             (b.emf[0][eidx(b, 0, k, j + 1, i)] - b.emf[0][eidx(b, 0, k, j, i)]) * b.idx[1];
    const long long f = fidx(b, d, k, j, i);
    double B0 = b.bf[d][f];
    double u = g1 * B0;
    if (first) b.bf0[d][f] = B0;
    else u = fma(g0, b.bf0[d][f], u);
    b.bf[d][f] = fma(-bdt, curl, u);
  }
}

void launch_emf(const Work& w, cudaStream_t s, int grid, int threads) { k_emf<<<grid, threads, 0, s>>>(w); }
void launch_update_cells(const Work& w, const Par& P, double g0, double g1, double bdt, int first, cudaStream_t s,
                         int grid, int threads) {
  k_update_cells<<<grid, threads, 0, s>>>(w, P, g0, g1, bdt, first);
}
void launch_update_faces(const Work& w, double g0, double g1, double bdt, int first, cudaStream_t s, int grid) {
  k_update_faces<<<grid, 256, 0, s>>>(w, g0, g1, bdt, first);
}
int occ_update_kernel(int kind, int threads) {
  int o = 0;
  if (kind == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_emf, threads, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_update_cells, threads, 0);
  return o;
}
int occupancy_update(int* per_sm) {
  cudaError_t e = cudaSuccess;
  e = (cudaError_t)(e | cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[0], k_emf, 128, 0));
  e = (cudaError_t)(e | cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[1], k_update_cells, 128, 0));
  e = (cudaError_t)(e | cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[2], k_update_faces, 256, 0));
  return e == cudaSuccess ? 0 : -1;
}


// ------------------------------------------------------ baryon-mass ledger
// Block-wide sum of one double per thread (blockDim a multiple of 32, <= 1024).
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += sh[k];
  return t;
}

// One CTA per block: the outward D~ flux through the block's interior
// boundary, integrated over the face areas, folded into the balance:
//   la += wF * lf - dtb * Phi,   lf = 0.
__global__ void __launch_bounds__(256) k_ledger_stage(Work w, double wF, double dtb) {
  __shared__ double sh[32];
  const DevBlock& b = w.blk[blockIdx.x];
  if (!b.la) return;
  const int g = b.ng, n0 = b.n[0], n1 = b.n[1], n2 = b.n[2];
  const long long m0 = (long long)n1 * n2, m1 = (long long)n0 * n2, m2 = (long long)n0 * n1;
  const double A0 = b.dx[1] * b.dx[2], A1 = b.dx[0] * b.dx[2], A2 = b.dx[0] * b.dx[1];
  double phi = 0.0;
  for (long long q = threadIdx.x; q < 2 * (m0 + m1 + m2); q += blockDim.x) {
    long long r = q;
    int d = 0;
    if (r >= 2 * m0) { r -= 2 * m0; d = 1; if (r >= 2 * m1) { r -= 2 * m1; d = 2; } }
    const long long m = d == 0 ? m0 : (d == 1 ? m1 : m2);
    const bool hi = r >= m;
    if (hi) r -= m;
    int i, j, k;
    if (d == 0) { j = g + (int)(r % n1); k = g + (int)(r / n1); i = g + (hi ? n0 : 0); }
    else if (d == 1) { i = g + (int)(r % n0); k = g + (int)(r / n0); j = g + (hi ? n1 : 0); }
    else { i = g + (int)(r % n0); j = g + (int)(r / n0); k = g + (hi ? n2 : 0); }
    const double F = b.flux[d][fidx(b, d, k, j, i)];   // component 0: D~
    const double A = d == 0 ? A0 : (d == 1 ? A1 : A2);
    phi += (hi ? F : -F) * A;
  }
  phi = block_sum(phi, sh);
  if (threadIdx.x == 0) {
    *b.la += wF * *b.lf - dtb * phi;
    *b.lf = 0.0;
  }
}

__global__ void __launch_bounds__(256) k_block_mass(Work w, double* out) {
  __shared__ double sh[32];
  const DevBlock& b = w.blk[blockIdx.x];
  const int g = b.ng, n0 = b.n[0], n1 = b.n[1];
  const long long tot = (long long)n0 * n1 * b.n[2];
  double s = 0.0;
  for (long long q = threadIdx.x; q < tot; q += blockDim.x) {
    const int i = g + (int)(q % n0);
    const long long r = q / n0;
    const int j = g + (int)(r % n1), k = g + (int)(r / n1);
    s += b.cons[cidx(b, k, j, i)];
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[b.id] = s * b.dV;
}

void launch_ledger_stage(const Work& w, double wF, double dtb, cudaStream_t s) {
  k_ledger_stage<<<w.nblocks, 256, 0, s>>>(w, wF, dtb);
}
void launch_block_mass(const Work& w, double* out, cudaStream_t s) {
  k_block_mass<<<w.nblocks, 256, 0, s>>>(w, out);
}

}  // namespace grmhd
