// con2prim as three kernels (Sec. 3.4): a uniform prep (floors, KRP variables,
// bracket), a root solve in which every lane refills itself from a global
// work queue as soon as its Illinois iteration converges, and a uniform
// finish (recovery, floors, write-back).  One thread per cell would leave most
// lanes of a warp idle while the slowest cell iterates, and idle lanes still
// occupy the narrow FP64 pipe; with refill the lanes stay busy until the
// queue runs dry.  When the prep polishes an FP32 root (c2p_guess 2) a cell
// left for the solve is a rare fallback: the finish kernels then solve it in
// place (solve_cell) and the solve kernel is not launched.
#include "dev.cuh"
#include "internal.h"

namespace grmhd {


__device__ __forceinline__ void kw_store(const KrpBuf& kb, long long i, const KrpCell& k) {
  const long long n = kb.n;
  double* w = kb.w;
  w[KW_QH * n + i] = k.s.qh; w[KW_R2 * n + i] = k.s.r2; w[KW_B2 * n + i] = k.s.b2;
  w[KW_RB2 * n + i] = k.s.rb2; w[KW_RP2 * n + i] = k.s.rperp2;
  w[KW_D * n + i] = k.D; w[KW_RB * n + i] = k.rb;
  w[KW_RU0 * n + i] = k.ru[0]; w[KW_RU1 * n + i] = k.ru[1]; w[KW_RU2 * n + i] = k.ru[2];
  w[KW_BU0 * n + i] = k.bu[0]; w[KW_BU1 * n + i] = k.bu[1]; w[KW_BU2 * n + i] = k.bu[2];
}
__device__ __forceinline__ void kw_load(const KrpBuf& kb, const Par& P, long long i, KrpCell& k) {
  const long long n = kb.n;
  const double* w = kb.w;
  k.s.qh = w[KW_QH * n + i]; k.s.r2 = w[KW_R2 * n + i]; k.s.b2 = w[KW_B2 * n + i];
  k.s.rb2 = w[KW_RB2 * n + i]; k.s.rperp2 = w[KW_RP2 * n + i];
  k.s.gam = P.gam; k.s.eps_min = P.eps_atm; k.s.vmax2 = P.vmax2;
  k.D = w[KW_D * n + i]; k.rb = w[KW_RB * n + i];
  k.s.D = k.D;
  k.ru[0] = w[KW_RU0 * n + i]; k.ru[1] = w[KW_RU1 * n + i]; k.ru[2] = w[KW_RU2 * n + i];
  k.bu[0] = w[KW_BU0 * n + i]; k.bu[1] = w[KW_BU1 * n + i]; k.bu[2] = w[KW_BU2 * n + i];
}

// prep of one cell: KRP variables and status.  mode 0: the plain bracket
// [0, mu+]; mode 1: status 4 (the seed kernel's network guess and FP32 search
// come later); mode 2: the FP32 secant search from [0, mu+] and the FP64
// polish here (krp_polish), the root when it is taken, else a bracket.
// feat (optional): the network's features of the cell.  guess > 0 (mode 0):
// the cell's previous root; the FP64 bracket starts as guess (1 -+
// WARM_DELTA), verified by the signs at both ends (krp_bracket).
// fofc: the FOFC estimate, which only needs to know whether con2prim of U*
// fails or a floor fires (Sec. 3.3).  A floor on the conserved state decides
// that before the solve, so such a cell gets status 5 (flagged, no bracket,
// no solve, no recovery); with P.dec32 fofc_decide_iv settles most of the
// other cells from enclosures of its FP64 KRP variables (status 5 or 7,
// counted in ndec) before any FP64 evaluation of f.  nf32 / nfb count the
// FP32 evaluations and the cells whose polish was not taken (mode 2).
__device__ __forceinline__ unsigned char prep_cell(const Par& P, const KrpBuf& kb, long long i, const double* U,
                                          const double* Bd, const Metric& m, int mode, unsigned& nf32,
                                          unsigned& nfb, float* feat = nullptr, double alpha = 1.0,
                                          double guess = 0.0, bool fofc = false, unsigned* ndec = nullptr) {
  KrpCell k;
  unsigned fl;
  const long long n = kb.n;
  unsigned char st = 2;
  int its = 0;
  bool solved = false;   // a bracket and root were formed (statuses 0-2 from the solver)
  double a = 0.0, b = 1.0, Ga = -1.0, Gb = 1.0, mu = 0.0;
  if (krp_prep(P, U, Bd, m, k, fl, alpha)) {
    if (feat) krp_features(k.s, feat + i * MLP_FSTRIDE);
    if (fofc && (fl & (F_DFLOOR | F_SIGMA | F_TAU))) {
      st = 5;
    } else {
      if (fofc && P.dec32) {
        KSI ki;
        ksi_of(k.s, k.D, ki);
        const int d = fofc_decide_iv(ki, P, nf32);
        if (d >= 0) {
          if (ndec) (*ndec)++;
          kb.st[i] = d ? 5 : 7;
          return kb.st[i];
        }
      }
      if (mode == 1) {
        st = 4;
      } else {
        int r;
        if (mode == 2) {
          const KSf sf = ks_f32(k.s);
          const float m32 = krp_secant32(sf, 0.0f, f32_mu_plus(sf), 8, nf32);
          const float isl = krp_islope32(sf, m32, nf32);
          bool fb;
          r = krp_polish(k.s, P, f64_of(m32), f64_of(isl), a, b, Ga, Gb, mu, its, fb);
          nfb += fb ? 1u : 0u;
        } else {
          const bool warm = guess > 0.0 && guess <= 1.0;
          const double glo = warm ? guess * (1.0 - WARM_DELTA) : -1.0;
          const double ghi = warm ? fmin(guess * (1.0 + WARM_DELTA), 1.0) : -1.0;
          r = krp_bracket(k.s, P, glo, ghi, a, b, Ga, Gb, mu, its);
        }
        st = (unsigned char)(r == 0 ? 0 : (r == 1 ? 1 : 2));
        solved = true;
      }
    }
  } else if (feat) {
    for (int f = 0; f < MLP_FSTRIDE; f++) feat[i * MLP_FSTRIDE + f] = 0.0f;
  }
  if (solved) {
    kb.w[KW_A * n + i] = a; kb.w[KW_B * n + i] = b;
    kb.w[KW_GA * n + i] = Ga; kb.w[KW_GB * n + i] = Gb;
    kb.w[KW_MU * n + i] = mu;
  }
  kw_store(kb, i, k);
  kb.w[KW_SDET * n + i] = m.sdet;
  kb.w[KW_ISDET * n + i] = m.isdet;
  kb.st[i] = st;
  kb.fl[i] = (unsigned char)fl;
  kb.it[i] = its;
  return st;
}

__device__ __forceinline__ void load_metric6(const double* g6, long long stride, long long c, Metric& m) {
#pragma unroll
  for (int v = 0; v < 6; v++) m.g[v] = g6[v * stride + c];
  metric_setup(m);
}

// The root solve of one status-0 cell in its own thread: the iteration of
// k_krp_solve (Illinois with the end-point nudge from the prep's bracket,
// its evaluations counted on from the prep's, capped at maxit in all)
// without the lane refill.  The finish kernels use it when the prep polishes
// the FP32 root (c2p_guess 2): a status-0 cell is then a rare fallback, and
// the separate solve launch, which would find no work in most calls, is left
// out.  Returns the status (1 root, 3 iteration cap); root and it as the
// solve kernel writes them.
__device__ __forceinline__ unsigned char solve_cell(const KS& s, const Par& P, double a, double Ga, double b,
                                                    double Gb, int& it, double& root) {
  double Fa = Ga, Fb = Gb;
  int side = 0;
  while (true) {
    bool fin = !gt_nn(b - a, P.tol * b), cap = false, exact = false;
    if (!fin) {
      if (it >= P.maxit) {
        cap = fin = true;
      } else {
        it++;
        double c = (a * Fb - b * Fa) * rcp_nr(Fb - Fa);   // Fb > 0 > Fa
        const double eta = 0.25 * P.tol * b;
        c += side == -1 ? eta : (side == 1 ? -eta : 0.0);
        if (!(gt_nn(c, a) && gt_nn(b, c))) c = 0.5 * (a + b);
        const double G = kev_G(s, P, c);
        if (lt0(G)) {
          a = c; Ga = G; Fa = G;
          if (side == -1) Fb *= 0.5;
          side = -1;
        } else if (gt0(G)) {
          b = c; Gb = G; Fb = G;
          if (side == 1) Fa *= 0.5;
          side = 1;
        } else {
          exact = fin = true;
          root = c;
        }
        if (!fin) fin = !gt_nn(b - a, P.tol * b);
      }
    }
    if (fin) {
      if (!exact && !cap) root = a - Ga * (b - a) * rcp_nr(Gb - Ga);   // Gb > 0 > Ga
      return cap ? 3 : 1;
    }
  }
}

// ------------------------------------------------------------------ root solve
// Illinois regula falsi with the end-point nudge (as in `illinois`) and lane
// refill.  Reads the
// bracket of every status-0 cell, writes mu, iterations and status 1 or 3.
__global__ void __launch_bounds__(256) k_krp_solve(Par P, KrpBuf kb) {
  if (*(volatile unsigned long long*)&kb.ctr[1] == 0ull) return;   // no cell has status 0
  const unsigned lane = threadIdx.x & 31;
  const long long n = kb.n;
  long long idx = -1;
  bool done = false;
  KS s;
  s.gam = P.gam; s.eps_min = P.eps_atm; s.vmax2 = P.vmax2;
  s.qh = s.r2 = s.b2 = s.rb2 = s.rperp2 = 0.0;
  s.D = 1.0;
  double a = 0.0, b = 1.0, Ga = -1.0, Gb = 1.0, Fa = -1.0, Fb = 1.0;
  int side = 0, it = 0;
  while (true) {
    const bool need = idx < 0 && !done;
    const unsigned m = __ballot_sync(0xffffffffu, need);
    if (m) {
      const int leader = __ffs(m) - 1;
      unsigned long long base = 0;
      if ((int)lane == leader) base = atomicAdd(kb.ctr, (unsigned long long)__popc(m));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (need) {
        const long long my = (long long)(base + __popc(m & ((1u << lane) - 1u)));
        if (my >= n) {
          done = true;
        } else if (kb.st[my] == 0) {
          idx = my;
          const double* w = kb.w;
          s.qh = w[KW_QH * n + my]; s.r2 = w[KW_R2 * n + my]; s.b2 = w[KW_B2 * n + my];
          s.rb2 = w[KW_RB2 * n + my]; s.rperp2 = w[KW_RP2 * n + my];
          s.D = w[KW_D * n + my];
          a = w[KW_A * n + my]; b = w[KW_B * n + my];
          Ga = w[KW_GA * n + my]; Gb = w[KW_GB * n + my];
          Fa = Ga; Fb = Gb;
          side = 0;
          it = kb.it[my];
        }
      }
    }
    const bool act = idx >= 0;
    if (__ballot_sync(0xffffffffu, act || !done) == 0) break;
    if (!act) continue;
    bool fin = !gt_nn(b - a, P.tol * b), cap = false, exact = false;
    double root = 0.0;
    if (!fin) {
      if (it >= P.maxit) {
        cap = fin = true;
      } else {
        it++;
        double c = (a * Fb - b * Fa) * rcp_nr(Fb - Fa);   // Fb > 0 > Fa
        const double eta = 0.25 * P.tol * b;
        c += side == -1 ? eta : (side == 1 ? -eta : 0.0);
        if (!(gt_nn(c, a) && gt_nn(b, c))) c = 0.5 * (a + b);
        const double G = kev_G(s, P, c);
        if (lt0(G)) {
          a = c; Ga = G; Fa = G;
          if (side == -1) Fb *= 0.5;
          side = -1;
        } else if (gt0(G)) {
          b = c; Gb = G; Fb = G;
          if (side == 1) Fa *= 0.5;
          side = 1;
        } else {
          exact = fin = true;
          root = c;
        }
        if (!fin) fin = !gt_nn(b - a, P.tol * b);
      }
    }
    if (fin) {
      if (!exact && !cap) root = a - Ga * (b - a) * rcp_nr(Gb - Ga);   // Gb > 0 > Ga
      kb.w[KW_MU * n + idx] = root;
      kb.it[idx] = it;
      kb.st[idx] = cap ? 3 : 1;
      idx = -1;
    }
  }
}

// -------------------------------------------------------- block stage con2prim
__global__ void __launch_bounds__(256) k_krp_prep_block(Work w, Par P, KrpBuf kb, int mode, float* feat,
                                                         unsigned long long* stats) {
  const long long* pre = w.pre + (long long)W_C2P * (w.nblocks + 1);
  const long long tot = pre[w.nblocks];
  if (blockIdx.x == 0 && threadIdx.x == 0) *kb.ctr = 0ull;
  unsigned s_f32 = 0, s_fb = 0;
  bool any0 = false;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < tot; it += (long long)gridDim.x * blockDim.x) {
    const int bi = find_block(w, W_C2P, it);
    const DevBlock& b = w.blk[bi];
    long long loc = it - pre[bi];
    const int R0 = b.n[0] + 6, R1 = b.n[1] + 6;
    int ii = loc % R0; long long r = loc / R0; int jj = r % R1; int kk = r / R1;
    const int i = ii + b.ng - 3, j = jj + b.ng - 3, k = kk + b.ng - 3;
    const long long c = cidx(b, k, j, i), nc = b.ncell;
    double Bd[3];
    Bd[0] = 0.5 * (b.bf[0][fidx(b, 0, k, j, i)] + b.bf[0][fidx(b, 0, k, j, i + 1)]);
    Bd[1] = 0.5 * (b.bf[1][fidx(b, 1, k, j, i)] + b.bf[1][fidx(b, 1, k, j + 1, i)]);
    Bd[2] = 0.5 * (b.bf[2][fidx(b, 2, k, j, i)] + b.bf[2][fidx(b, 2, k + 1, j, i)]);
#pragma unroll
    for (int v = 0; v < 3; v++) b.bcc[v * nc + c] = Bd[v];
    Metric m;
    metric_cell(b.adm, b.mc, nc, c, m);   // the step's metric cache (k_metric_cache)
    double U[5];
#pragma unroll
    for (int v = 0; v < 5; v++) U[v] = b.cons[v * nc + c];
    any0 |= prep_cell(P, kb, it, U, Bd, m, mode, s_f32, s_fb, feat, b.adm[c], b.mu ? b.mu[c] : 0.0) == 0;
  }
  warp_mark_solve(kb, any0);
  if (mode == 2) {
    warp_flush(&stats[7], s_fb);
    warp_flush(&stats[8], s_f32);
  }
}

// inl: status-0 cells are solved here (solve_cell), no solve launch before
__global__ void __launch_bounds__(256) k_krp_finish_block(Work w, Par P, KrpBuf kb, unsigned long long* stats,
                                                           bool inl) {
  const long long* pre = w.pre + (long long)W_C2P * (w.nblocks + 1);
  const long long tot = pre[w.nblocks];
  const long long n = kb.n;
  unsigned s_cells = 0, s_fail = 0, s_floor = 0, s_it = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) kb.ctr[1] = 0ull;   // the solve has run
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < tot; it += (long long)gridDim.x * blockDim.x) {
    const int bi = find_block(w, W_C2P, it);
    const DevBlock& b = w.blk[bi];
    long long loc = it - pre[bi];
    const int R0 = b.n[0] + 6, R1 = b.n[1] + 6;
    int ii = loc % R0; long long r = loc / R0; int jj = r % R1; int kk = r / R1;
    const int i = ii + b.ng - 3, j = jj + b.ng - 3, k = kk + b.ng - 3;
    const long long c = cidx(b, k, j, i), nc = b.ncell;
    KrpCell kc;
    kw_load(kb, P, it, kc);
    unsigned fl = kb.fl[it];
    unsigned char st = kb.st[it];
    double pr[5], iW;
    double root = kb.w[KW_MU * n + it];
    int its = kb.it[it];
    if (inl && st == 0)
      st = solve_cell(kc.s, P, kb.w[KW_A * n + it], kb.w[KW_GA * n + it], kb.w[KW_B * n + it],
                      kb.w[KW_GB * n + it], its, root);
    krp_finish(P, kc, root, st == 1, fl, pr, &iW);
    if (b.mu) b.mu[c] = (st == 1 && !(fl & F_FAIL)) ? root : 0.0;
#pragma unroll
    for (int v = 0; v < 5; v++) b.prim[v * nc + c] = pr[v];
    const double Bd[3] = {b.bcc[c], b.bcc[nc + c], b.bcc[2 * nc + c]};
    if (fl & (FLOOR_BITS | F_FAIL)) {   // only here is the metric needed
      Metric m;
#pragma unroll
      for (int v = 0; v < 6; v++) m.g[v] = b.adm[(4 + v) * nc + c];
      m.sdet = kb.w[KW_SDET * n + it];
      m.isdet = kb.w[KW_ISDET * n + it];
      double U[5];
      prim2cons(P, pr, Bd, m, U);
      const double D0 = b.cons[c];
#pragma unroll
      for (int v = 0; v < 5; v++) b.cons[v * nc + c] = U[v];
      const bool inner = ii >= 3 && ii < b.n[0] + 3 && jj >= 3 && jj < b.n[1] + 3 && kk >= 3 && kk < b.n[2] + 3;
      if (b.lf && inner && U[0] != D0) atomicAdd(b.lf, (U[0] - D0) * b.dV);
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
    s_it += (unsigned)its;
    s_fail += (fl & F_FAIL) ? 1u : 0u;
    s_floor += (fl & FLOOR_BITS) ? 1u : 0u;
  }
  warp_flush(&stats[0], s_cells);
  warp_flush(&stats[1], s_it);
  warp_flush(&stats[2], s_fail);
  warp_flush(&stats[3], s_floor);
}

// ------------------------------------------------------------------ FOFC U*

// The FOFC estimate's prep: U* = g1 U + g0 U^n - bdt div F in FP64, then
// prep_cell (fofc), which decides most cells from FP32 enclosures of their KRP
// variables.  U* and the KRP variables stay FP64: computing them as enclosures
// too (one FP32 interval kernel, no FP64) was measured slower, 0.25 against
// 0.20 ms at 96^3, latency-bound on the ~56 scattered loads per cell.
__global__ void __launch_bounds__(256) k_krp_prep_fofc(Work w, Par P, double g0, double g1, double bdt, KrpBuf kb,
                                                        int mode, float* feat, unsigned long long* stats) {
  const long long tot = w.pre[(long long)W_CELL * (w.nblocks + 1) + w.nblocks];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *kb.ctr = 0ull;
    if (kb.flist) kb.flist[0] = 0ull;   // the finish lists this stage's flagged cells
  }
  const long long n = kb.n;
  unsigned s_f32 = 0, s_fb = 0, s_dec = 0;
  bool any0 = false;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < tot; it += (long long)gridDim.x * blockDim.x) {
    int bi, k, j, i;
    fofc_cell(w, it, bi, k, j, i);
    const DevBlock& b = w.blk[bi];
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
    metric_cell(b.adm, b.mc, nc, c, m);
    const double Bd[3] = {b.bcc[c], b.bcc[nc + c], b.bcc[2 * nc + c]};
    any0 |= prep_cell(P, kb, it, U, Bd, m, mode, s_f32, s_fb, feat, b.adm[c], b.mu ? b.mu[c] : 0.0, true,
                      &s_dec) == 0;
    if (P.dmp_M > 0.0) {   // the DMP test of the finish reads U*
      kb.w[KW_USD * n + it] = U[0];
      kb.w[KW_UST * n + it] = U[4];
    }
  }
  warp_mark_solve(kb, any0);
  if (mode == 2) warp_flush(&stats[7], s_fb);
  warp_flush(&stats[8], s_f32);
  warp_flush(&stats[9], s_dec);
}

// inl: status-0 cells are solved here (solve_cell), no solve launch before
__global__ void __launch_bounds__(256) k_krp_finish_fofc(Work w, Par P, KrpBuf kb, unsigned long long* stats,
                                                          bool inl) {
  const long long tot = w.pre[(long long)W_CELL * (w.nblocks + 1) + w.nblocks];
  const long long n = kb.n;
  unsigned s_flag = 0, s_dmp = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) kb.ctr[1] = 0ull;   // the solve has run
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < tot; it += (long long)gridDim.x * blockDim.x) {
    int bi, k, j, i;
    fofc_cell(w, it, bi, k, j, i);
    const DevBlock& b = w.blk[bi];
    const long long nc = b.ncell, c = cidx(b, k, j, i);
    const unsigned char st = kb.st[it];
    bool flag = st != 7;   // 5: flagged, 7: not flagged, both without a recovery
    if (st != 5 && st != 7) {
      unsigned fl = kb.fl[it];
      KrpCell kc;
      kw_load(kb, P, it, kc);
      double pr[5];
      double root = kb.w[KW_MU * n + it];
      unsigned char s2 = st;
      if (inl && st == 0) {
        int its = kb.it[it];
        s2 = solve_cell(kc.s, P, kb.w[KW_A * n + it], kb.w[KW_GA * n + it], kb.w[KW_B * n + it],
                        kb.w[KW_GB * n + it], its, root);
      }
      krp_finish(P, kc, root, s2 == 1, fl, pr);
      flag = (fl & (FLOOR_BITS | F_FAIL)) != 0;
    }
    if (!flag && P.dmp_M > 0.0) {
      const double Us[2] = {kb.w[KW_USD * n + it], kb.w[KW_UST * n + it]};
#pragma unroll
      for (int t = 0; t < 2; t++) {
        const double* a = b.cons + (t == 0 ? 0 : 4) * nc;
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
        if (Us[t] < lo || Us[t] > hi) flag = true;
      }
      s_dmp += flag ? 1u : 0u;
    }
    b.fflag[c] = flag ? 1 : 0;
    if (flag && kb.flist) {   // rare: one atomic per flagged cell
      const unsigned long long pos = atomicAdd(kb.flist, 1ull);
      if ((long long)pos < kb.fcap) kb.flist[1 + pos] = (unsigned long long)it;
    }
    unsigned char f0 = b.flags[c];
    b.flags[c] = flag ? (unsigned char)(f0 | F_FOFC) : (unsigned char)(f0 & ~F_FOFC);
    s_flag += flag ? 1u : 0u;
  }
  warp_flush(&stats[4], s_flag);
  warp_flush(&stats[5], s_dmp);
}

// ------------------------------------------------------- independent cells
// fonly: flags only (the FOFC estimate's question), a template parameter so
// that the full con2prim keeps its registers
template <bool fonly>
__global__ void __launch_bounds__(128) k_krp_prep_cells(Par P, KrpBuf kb, const double* __restrict__ cons,
                                                        const double* __restrict__ Bd, const double* __restrict__ g,
                                                        int mode, float* __restrict__ feat,
                                                        unsigned long long* stats) {
  const long long n = kb.n;
  if (blockIdx.x == 0 && threadIdx.x == 0) *kb.ctr = 0ull;
  unsigned s_f32 = 0, s_fb = 0, s_dec = 0;
  bool any0 = false;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    Metric m;
    load_metric6(g, n, c, m);
    double U[5], B[3];
#pragma unroll
    for (int v = 0; v < 5; v++) U[v] = cons[v * n + c];
#pragma unroll
    for (int v = 0; v < 3; v++) B[v] = Bd[v * n + c];
    if (fonly && P.dec32) {   // the question in FP32 enclosures of U first
      Iv Ui[5];
#pragma unroll
      for (int v = 0; v < 5; v++) Ui[v] = iv_d(U[v]);
      KSI ki;
      int d = krp_prep_iv(P, Ui, B, m, 1.0, ki);
      if (d == 0) d = fofc_decide_iv(ki, P, s_f32);
      if (d >= 0) {
        kb.st[c] = d ? 5 : 7;
        s_dec++;
        continue;
      }
    }
    any0 |= prep_cell(P, kb, c, U, B, m, mode, s_f32, s_fb, feat, 1.0, 0.0, fonly, &s_dec) == 0;
  }
  warp_mark_solve(kb, any0);
  if (mode == 2) warp_flush(&stats[7], s_fb);
  warp_flush(&stats[8], s_f32);
  warp_flush(&stats[9], s_dec);
}

__global__ void __launch_bounds__(128) k_krp_finish_cells(Par P, KrpBuf kb, double* __restrict__ cons,
                                                          const double* __restrict__ Bd, const double* __restrict__ g,
                                                          double* __restrict__ prim, unsigned char* __restrict__ flags,
                                                          int* __restrict__ iters_out, unsigned long long* stats) {
  const long long n = kb.n;
  unsigned s_cells = 0, s_fail = 0, s_floor = 0, s_it = 0, s_flag = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) kb.ctr[1] = 0ull;   // the solve has run
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const unsigned char st = kb.st[c];
    if (!prim) {   // flags only: 1 where con2prim fails or a floor fires
      bool flag = st != 7;
      int its = 0;
      if (st != 5 && st != 7) {
        KrpCell kc;
        kw_load(kb, P, c, kc);
        unsigned fl = kb.fl[c];
        double pr[5];
        krp_finish(P, kc, kb.w[KW_MU * n + c], st == 1, fl, pr);
        flag = (fl & (FLOOR_BITS | F_FAIL)) != 0;
        its = kb.it[c];
      }
      flags[c] = flag ? 1 : 0;
      if (iters_out) iters_out[c] = its;
      s_cells++;
      s_it += (unsigned)its;
      s_flag += flag ? 1u : 0u;
      continue;
    }
    KrpCell kc;
    kw_load(kb, P, c, kc);
    unsigned fl = kb.fl[c];
    double pr[5];
    krp_finish(P, kc, kb.w[KW_MU * n + c], st == 1, fl, pr);
#pragma unroll
    for (int v = 0; v < 5; v++) prim[v * n + c] = pr[v];
    if (fl & (FLOOR_BITS | F_FAIL)) {
      Metric m;
#pragma unroll
      for (int v = 0; v < 6; v++) m.g[v] = g[v * n + c];
      m.sdet = kb.w[KW_SDET * n + c];
      m.isdet = kb.w[KW_ISDET * n + c];
      const double B[3] = {Bd[c], Bd[n + c], Bd[2 * n + c]};
      double U[5];
      prim2cons(P, pr, B, m, U);
#pragma unroll
      for (int v = 0; v < 5; v++) cons[v * n + c] = U[v];
    }
    flags[c] = (unsigned char)fl;
    if (iters_out) iters_out[c] = kb.it[c];
    s_cells++;
    s_it += (unsigned)kb.it[c];
    s_fail += (fl & F_FAIL) ? 1u : 0u;
    s_floor += (fl & FLOOR_BITS) ? 1u : 0u;
  }
  warp_flush(&stats[0], s_cells);
  warp_flush(&stats[1], s_it);
  warp_flush(&stats[2], s_fail);
  warp_flush(&stats[3], s_floor);
  warp_flush(&stats[4], s_flag);
}

// ------------------------------------------------------------------ launchers
size_t krp_bytes(long long n) {
  return (size_t)n * (sizeof(double) * KW_N + sizeof(int) + 2) + 1024;
}
// The counters sit at the start of the buffer, so every view of it (the
// stage input's and the FOFC estimate's, of different n) shares them; their
// uses follow one another in stream order (prep, solve, finish).
KrpBuf krp_view(void* base, long long n) {
  KrpBuf kb;
  char* p = (char*)base;
  kb.n = n;
  kb.ctr = (unsigned long long*)p;
  p += 256;
  kb.w = (double*)p;
  p += sizeof(double) * KW_N * n;
  kb.it = (int*)p;
  p += sizeof(int) * n;
  kb.st = (unsigned char*)p;
  p += n;
  kb.fl = (unsigned char*)p;
  return kb;
}

void launch_krp_prep_block(const Work& w, const Par& P, const KrpBuf& kb, unsigned long long* stats, cudaStream_t s,
                           int grid, int threads, int mode, float* feat) {
  k_krp_prep_block<<<grid, threads, 0, s>>>(w, P, kb, mode, feat, stats);
}
void launch_krp_solve(const Par& P, const KrpBuf& kb, cudaStream_t s, int grid) {
  k_krp_solve<<<grid, 256, 0, s>>>(P, kb);
}
void launch_krp_finish_block(const Work& w, const Par& P, const KrpBuf& kb, unsigned long long* stats,
                             cudaStream_t s, int grid, int threads, bool inl) {
  k_krp_finish_block<<<grid, threads, 0, s>>>(w, P, kb, stats, inl);
}
void launch_krp_prep_fofc(const Work& w, const Par& P, double g0, double g1, double bdt, const KrpBuf& kb,
                          unsigned long long* stats, cudaStream_t s, int grid, int threads, int mode, float* feat) {
  k_krp_prep_fofc<<<grid, threads, 0, s>>>(w, P, g0, g1, bdt, kb, mode, feat, stats);
}
void launch_krp_finish_fofc(const Work& w, const Par& P, const KrpBuf& kb, unsigned long long* stats,
                            cudaStream_t s, int grid, int threads, bool inl) {
  k_krp_finish_fofc<<<grid, threads, 0, s>>>(w, P, kb, stats, inl);
}
void launch_krp_prep_cells(const Par& P, const KrpBuf& kb, const double* cons, const double* Bd, const double* g,
                           int mode, float* feat, unsigned long long* stats, cudaStream_t s, int grid, bool fonly) {
  if (fonly) k_krp_prep_cells<true><<<grid, 128, 0, s>>>(P, kb, cons, Bd, g, mode, feat, stats);
  else k_krp_prep_cells<false><<<grid, 128, 0, s>>>(P, kb, cons, Bd, g, mode, feat, stats);
}
void launch_krp_finish_cells(const Par& P, const KrpBuf& kb, double* cons, const double* Bd, const double* g,
                             double* prim, unsigned char* flags, int* iters, unsigned long long* stats, cudaStream_t s,
                             int grid) {
  k_krp_finish_cells<<<grid, 128, 0, s>>>(P, kb, cons, Bd, g, prim, flags, iters, stats);
}
int occ_krp_kernel(int kind, int threads) {
  int o = 0;
  if (kind == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_krp_prep_block, threads, 0);
  else if (kind == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_krp_finish_block, threads, 0);
  else if (kind == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_krp_prep_fofc, threads, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_krp_finish_fofc, threads, 0);
  return o;
}
int occupancy_krp(int* per_sm) {
  cudaError_t e = cudaSuccess;
  e = (cudaError_t)(e | cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[0], k_krp_prep_block, 128, 0));
  e = (cudaError_t)(e | cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[1], k_krp_solve, 256, 0));
  e = (cudaError_t)(e | cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[2], k_krp_finish_block, 128, 0));
  e = (cudaError_t)(e | cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[3], k_krp_prep_fofc, 128, 0));
  e = (cudaError_t)(e | cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[4], k_krp_finish_fofc, 128, 0));
  e = (cudaError_t)(e | cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[5], k_krp_prep_cells<false>, 128, 0));
  e = (cudaError_t)(e | cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[6], k_krp_finish_cells, 128, 0));
  e = (cudaError_t)(e | cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[7], k_krp_prep_cells<true>, 128, 0));
  return e == cudaSuccess ? 0 : -1;
}

}  // namespace grmhd
