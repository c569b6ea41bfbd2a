// C-ABI of libgrmhd: context, block lists, scratch, launch sequencing and the
// CUDA-graph step.  Declarations and argument conventions: include/grmhd.h.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "grmhd.h"
#include "internal.h"

using namespace grmhd;

// tunable kernels
enum TKind { T_C2P_PREP = 0, T_C2P_FIN, T_FX, T_FY, T_FZ, T_FOFC_PREP, T_FOFC_FIN, T_EMF, T_UPD, T_N };

struct mhd_ctx {
  mhd_params hp;
  Par P;
  int dev = 0, nsm = 1;
  int occ_c2p[2] = {1, 1}, occ_face[5] = {1, 1, 1, 1, 1}, occ_upd[3] = {1, 1, 1};
  int occ_krp[8] = {1, 1, 1, 1, 1, 1, 1, 1};   // [7]: the flags-only cell prep
  int occ_seed = 1;   // the learned seed kernel
  int occ_metric = 1;         // metric cache kernel
  // side streams and events of the forked flux sweeps (y, z)
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_join[2] = {nullptr, nullptr};
  cudaEvent_t state_ready = nullptr;   // mhd_step_overlap: the stages wait for it after the metric kernel
  unsigned long long* fofc_list = nullptr;   // the FOFC estimate's flagged cells ([0] count)
  long long fofc_cap = 0;
  // three-phase con2prim scratch: of the block list, and of independent cells
  char* krp = nullptr;
  long long krp_n = 0;
  char* cells_buf = nullptr;
  size_t cells_bytes = 0;
  // learned con2prim guess (network state)
  float* mlp = nullptr;             // [4 * MLP_NPARAM]: params, Adam m, Adam v, gradient
  __nv_bfloat16* mlp_wb = nullptr;  // [MLP_NBF] bf16 operand copies
  float* mlp_loss = nullptr;        // device scalar
  double* mlp_acc = nullptr;        // [12] normalisation sums
  MlpNorm nm;
  double mlp_delta = 0.0;           // bracket half-width in log(mu)
  int mlp_t = 0;                    // Adam step
  bool mlp_ready = false;
  // current block list
  std::vector<mhd_block> key;
  std::vector<DevBlock> hblk;
  std::vector<long long> hpre;
  DevBlock* dblk = nullptr;
  long long* dpre = nullptr;
  char* scratch = nullptr;
  size_t scratch_bytes = 0;
  long long list_version = 0;
  int grid[W_NKIND] = {0};
  int g_kprep = 1, g_kfin = 1, g_fprep = 1, g_ffin = 1;
  // launch configuration (CTA size, waves of resident CTAs) per tunable kernel
  struct Cfg {
    int threads = 128, waves = 1;
  } cfg[T_N];
  int occ_t[T_N][3] = {{0}};   // occupancy at 64, 128, 256 threads
  long long* dpre_blk = nullptr;  // per-block work tables [nb][W_NKIND][2] (per-block launches)
  // baryon-mass ledger [nb][2] (lf, la) and per-block mass sums [nb]
  bool ledger_on = false;
  double* dledger = nullptr;
  double* dmass = nullptr;
  // neighbour table of the last ghost fill (grow-only)
  int* dnbr = nullptr;
  size_t dnbr_n = 0;
  // Grid of the refill root solve over n cells: one resident wave, capped by
  // the cells (a lane per cell).  Fewer CTAs for a small list (a few cells
  // per lane) measured slower: the 32^3 block's solve took 108 instead of 84
  // us, its SMs FP64-bound while a third of them held work.
  int solve_grid(long long n) const {
    const long long full = (long long)nsm * (occ_krp[1] > 0 ? occ_krp[1] : 1);
    return (int)std::max(1LL, std::min(full, (n + 255) / 256));
  }
  // counters
  unsigned long long* dstats = nullptr;
  long long launches = 0;
  // rhs/update ordering
  long long rhs_list = -1;
  int rhs_stage = -1;
  // graph cache
  cudaGraphExec_t gexec = nullptr;
  long long g_list = -1, g_par = -1;
  bool g_metric = true;   // the captured step includes the metric kernel
  double g_dt = 0.0;
  long long metric_list = -1;   // block list whose ADM arrays the metric cache holds
  cudaStream_t g_stream = nullptr;
  long long par_version = 0;
  int g_launches = 0;
  // per-kernel CUDA-event timing of non-captured launches
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  struct Rec { int kind; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  double prof_ms[MHD_NKERNEL] = {0};
  long long prof_n[MHD_NKERNEL] = {0};
};

namespace grmhd {
// Parameters -> kernel constants; validates every field.  allow_guess: the
// learned and FP32-search con2prims (1, 2) and the warm start (3) are
// accepted (the allocation-free path takes 0 only).
int fill_par(const mhd_params* p, Par& P, bool allow_guess) {
  if (!p) return MHD_EINVAL;
  if (!(p->gamma > 1.0) || !(p->rho_atm > 0.0) || !(p->T_atm > 0.0) || !(p->f_thr >= 0.0) || !(p->c2p_tol > 0.0) ||
      !(p->W_max > 1.0) || p->recon < 0 || p->recon > 4 || p->rsolver < 0 || p->rsolver > 1 ||
      (p->rk_order != 2 && p->rk_order != 3) || p->c2p_maxit < 1 || p->c2p_guess < 0 ||
      p->c2p_guess > (allow_guess ? 3 : 0) || (p->dmp_M > 0.0 && p->dmp_M < 1.0) || p->eos < 0 || p->eos > 1 ||
      p->fixed_metric < 0 || p->fixed_metric > 1)
    return MHD_EINVAL;
  std::memset(&P, 0, sizeof(P));
  P.eos = p->eos;
  if (p->eos == 1) {
    // hybrid EOS: pieces, K_i and eps_c constants a_i by continuity at the
    // dividing densities; the FP32 root searches assume the ideal gas
    const int np = p->eos_pieces;
    if (np < 1 || np > 4 || !(p->eos_K0 > 0.0) || !(p->eos_gamma_th > 1.0) || p->c2p_guess == 1 ||
        p->c2p_guess == 2)
      return MHD_EINVAL;
    for (int i = 0; i < np; i++)
      if (!(p->eos_gamma[i] > 1.0)) return MHD_EINVAL;
    for (int i = 0; i + 1 < np; i++)
      if (!(p->eos_rho[i] > 0.0) || (i > 0 && !(p->eos_rho[i] > p->eos_rho[i - 1]))) return MHD_EINVAL;
    P.npc = np;
    P.Kpc[0] = p->eos_K0;
    P.apc[0] = 0.0;
    for (int i = 0; i < 4; i++) P.Gpc[i] = p->eos_gamma[i < np ? i : np - 1];
    for (int i = 0; i < 3; i++) P.rpc[i] = i + 1 < np ? p->eos_rho[i] : 0.0;
    for (int i = 1; i < 4; i++) {
      if (i >= np) {
        P.Kpc[i] = P.Kpc[i - 1];
        P.apc[i] = P.apc[i - 1];
        continue;
      }
      const double rb = p->eos_rho[i - 1], G0 = P.Gpc[i - 1], G1 = P.Gpc[i];
      P.Kpc[i] = P.Kpc[i - 1] * std::pow(rb, G0 - G1);
      P.apc[i] = P.apc[i - 1] + P.Kpc[i - 1] * std::pow(rb, G0 - 1.0) / (G0 - 1.0) -
                 P.Kpc[i] * std::pow(rb, G1 - 1.0) / (G1 - 1.0);
    }
    P.Gth = p->eos_gamma_th;
  } else {
    P.Gth = p->gamma;
  }
  P.gth1 = P.Gth - 1.0;
  P.gam = p->gamma;
  P.gm1 = p->gamma - 1.0;
  P.gfac = p->gamma / (p->gamma - 1.0);
  P.rho_atm = p->rho_atm;
  P.T_atm = p->T_atm;
  P.rho_thr = p->f_thr * p->rho_atm;
  P.eps_atm = p->T_atm / P.gth1;
  if (p->eos == 1) {
    // the cold triple at rho_atm, as eos_cold computes it on the device
    int i = 0;
    for (int j = 0; j < 3; j++) i += (j < P.npc - 1 && p->rho_atm >= P.rpc[j]) ? 1 : 0;
    const double x = P.Kpc[i] * std::pow(p->rho_atm, P.Gpc[i] - 1.0);
    P.Pc_atm = x * p->rho_atm;
    P.epsc_atm = P.apc[i] + x / (P.Gpc[i] - 1.0);
    P.G_atm = P.Gpc[i];
  }
  P.eps_atm_rho = P.epsc_atm + P.eps_atm;
  P.P_atm = P.Pc_atm + p->rho_atm * p->T_atm;
  P.sigma_max = p->sigma_max;
  P.dmp_M = p->dmp_M;
  P.tol = p->c2p_tol;
  P.vmax2 = 1.0 - 1.0 / (p->W_max * p->W_max);
  P.alpha_exc = p->alpha_exc;
  P.exc_on = p->alpha_exc > 0.0 ? 1 : 0;
  P.sigma_on = p->sigma_max > 0.0 ? 1 : 0;
  P.thr_pos = P.rho_thr > 0.0 ? 1 : 0;
  // the FP32 decision of the FOFC flags: ideal gas, thresholds inside the FP32 range
  P.dec32 = (p->eos == 0 && P.eps_atm >= 1e-30 && P.eps_atm <= 1e30 &&
             (!P.thr_pos || (P.rho_thr >= 1e-30 && P.rho_thr <= 1e30)))
                ? 1
                : 0;
  P.recon = p->recon;
  P.rsolver = p->rsolver;
  P.fofc = p->fofc ? 1 : 0;
  P.rk_order = p->rk_order;
  P.maxit = p->c2p_maxit;
  P.guess = p->c2p_guess;
  return MHD_OK;
}

}  // namespace grmhd

namespace {

int set_par(mhd_ctx* c, const mhd_params* p) {
  Par P;
  const int r = fill_par(p, P, true);
  if (r) return r;
  c->hp = *p;
  c->P = P;
  c->par_version++;
  return MHD_OK;
}

inline int cuda_ok(cudaError_t e) { return e == cudaSuccess ? MHD_OK : MHD_ECUDA; }

long long ncell_of(const mhd_block& b) {
  return (long long)(b.n[0] + 2 * b.ng) * (b.n[1] + 2 * b.ng) * (b.n[2] + 2 * b.ng);
}

int check_block(const mhd_block& b) {
  if (b.n[0] < 1 || b.n[1] < 1 || b.n[2] < 1 || b.ng < 4) return MHD_EINVAL;
  if (!b.cons || !b.cons0 || !b.prim || !b.bcc || !b.adm || !b.flags) return MHD_EINVAL;
  for (int d = 0; d < 3; d++)
    if (!b.bf[d] || !b.bf0[d] || !(b.dx[d] > 0.0)) return MHD_EINVAL;
  return MHD_OK;
}

void destroy_graph(mhd_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  c->g_list = -1;
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Upload a new block list (descriptors, work prefix sums) and size scratch.
int prepare(mhd_ctx* c, const mhd_block* blocks, int nb) {
  if (!blocks || nb < 1) return MHD_EINVAL;
  if ((int)c->key.size() == nb && std::memcmp(c->key.data(), blocks, sizeof(mhd_block) * nb) == 0) return MHD_OK;
  for (int i = 0; i < nb; i++) {
    int r = check_block(blocks[i]);
    if (r) return r;
  }
  destroy_graph(c);
  cudaDeviceSynchronize();
  std::vector<int> nn(3 * (size_t)nb);
  for (int i = 0; i < nb; i++)
    for (int d = 0; d < 3; d++) nn[3 * (size_t)i + d] = blocks[i].n[d];
  int seg[3];
  for (int d = 0; d < 3; d++) seg[d] = flux_seg_len((const int (*)[3])nn.data(), nb, d, c->nsm);
  std::vector<DevBlock> hb(nb);
  std::vector<long long> pre((size_t)W_NKIND * (nb + 1), 0);
  size_t need = 0;
  for (int i = 0; i < nb; i++) {
    const mhd_block& s = blocks[i];
    DevBlock& b = hb[i];
    std::memset(&b, 0, sizeof(b));
    for (int d = 0; d < 3; d++) {
      b.n[d] = s.n[d];
      b.N[d] = s.n[d] + 2 * s.ng;
      b.dx[d] = s.dx[d];
      b.idx[d] = 1.0 / s.dx[d];
      b.bf[d] = s.bf[d];
      b.bf0[d] = s.bf0[d];
    }
    b.ng = s.ng;
    for (int d = 0; d < 3; d++) b.nseg[d] = flux_nseg(s.n[d], seg[d]);
    b.ncell = ncell_of(s);
    b.cons = s.cons; b.cons0 = s.cons0; b.prim = s.prim; b.bcc = s.bcc; b.adm = s.adm; b.flags = s.flags;
    const long long N0 = b.N[0], N1 = b.N[1], N2 = b.N[2];
    const long long nf[3] = {N2 * N1 * (N0 + 1), N2 * (N1 + 1) * N0, (N2 + 1) * N1 * N0};
    const long long ne[3] = {(N2 + 1) * (N1 + 1) * N0, (N2 + 1) * N1 * (N0 + 1), N2 * (N1 + 1) * (N0 + 1)};
    need += al256(sizeof(double) * 7 * (nf[0] + nf[1] + nf[2]));
    need += al256(sizeof(double) * (ne[0] + ne[1] + ne[2]));
    need += al256(sizeof(double) * 3 * b.ncell);
    need += al256((size_t)b.ncell);
    need += al256(sizeof(double) * 8 * (size_t)b.ncell);
    for (int d = 0; d < 3; d++) need += al256(sizeof(double) * FMC_N * (size_t)fmc_count(b, d));
    need += al256(sizeof(double) * DMC_N * (size_t)s.n[0] * s.n[1] * s.n[2]);
    if (c->P.guess == 3) need += al256(sizeof(double) * (size_t)b.ncell);
    const long long n0 = s.n[0], n1 = s.n[1], n2 = s.n[2];
    long long items[W_NKIND];
    items[W_C2P] = (n0 + 6) * (n1 + 6) * (n2 + 6);
    items[W_FX] = (n0 + 1) * (n1 + 2) * (n2 + 2);
    items[W_FY] = (n0 + 2) * (n1 + 1) * (n2 + 2);
    items[W_FZ] = (n0 + 2) * (n1 + 2) * (n2 + 1);
    items[W_CELL] = n0 * n1 * n2;
    items[W_EDGE] = (n0 + 1) * (n1 + 1) * (n2 + 1);
    items[W_FACE] = (n0 + 1) * n1 * n2 + n0 * (n1 + 1) * n2 + n0 * n1 * (n2 + 1);
    items[W_INIT] = b.ncell;
    for (int d = 0; d < 3; d++) items[W_SX + d] = flux_seg_items(s.n, d, seg[d]);
    for (int d = 0; d < 3; d++) items[W_GFX + d] = nf[d];   // every entry of face array d
    for (int k = 0; k < W_NKIND; k++) pre[(size_t)k * (nb + 1) + i + 1] = pre[(size_t)k * (nb + 1) + i] + items[k];
  }
  const long long nkrp = std::max(pre[(size_t)W_C2P * (nb + 1) + nb], pre[(size_t)W_CELL * (nb + 1) + nb]);
  const size_t krp_off = need;
  need += al256(krp_bytes(nkrp));
  const long long ncell_all = pre[(size_t)W_CELL * (nb + 1) + nb];
  const size_t list_off = need;
  need += al256(sizeof(unsigned long long) * (size_t)(ncell_all + 1));
  const size_t mass_off = need;
  need += al256(sizeof(double) * (size_t)nb);
  const size_t led_off = need;
  if (c->ledger_on) need += al256(sizeof(double) * 2 * (size_t)nb);
  if (need > c->scratch_bytes) {
    if (c->scratch) cudaFree(c->scratch);
    c->scratch = nullptr;
    c->scratch_bytes = 0;
    if (cudaMalloc(&c->scratch, need) != cudaSuccess) return MHD_ENOMEM;
    c->scratch_bytes = need;
  }
  char* p = c->scratch;
  for (int i = 0; i < nb; i++) {
    DevBlock& b = hb[i];
    const long long N0 = b.N[0], N1 = b.N[1], N2 = b.N[2];
    const long long nf[3] = {N2 * N1 * (N0 + 1), N2 * (N1 + 1) * N0, (N2 + 1) * N1 * N0};
    const long long ne[3] = {(N2 + 1) * (N1 + 1) * N0, (N2 + 1) * N1 * (N0 + 1), N2 * (N1 + 1) * (N0 + 1)};
    double* f = (double*)p;
    b.flux[0] = f;
    b.flux[1] = f + 7 * nf[0];
    b.flux[2] = f + 7 * (nf[0] + nf[1]);
    p += al256(sizeof(double) * 7 * (nf[0] + nf[1] + nf[2]));
    double* e = (double*)p;
    b.emf[0] = e;
    b.emf[1] = e + ne[0];
    b.emf[2] = e + ne[0] + ne[1];
    p += al256(sizeof(double) * (ne[0] + ne[1] + ne[2]));
    b.ecc = (double*)p;
    p += al256(sizeof(double) * 3 * b.ncell);
    b.fflag = (unsigned char*)p;
    p += al256((size_t)b.ncell);
    b.mc = (double*)p;
    p += al256(sizeof(double) * 8 * (size_t)b.ncell);
    for (int d = 0; d < 3; d++) {
      b.fmc[d] = (double*)p;
      p += al256(sizeof(double) * FMC_N * (size_t)fmc_count(b, d));
    }
    b.dmc = (double*)p;
    p += al256(sizeof(double) * DMC_N * (size_t)b.n[0] * b.n[1] * b.n[2]);
    b.mu = nullptr;
    if (c->P.guess == 3) {
      b.mu = (double*)p;
      if (cudaMemset(b.mu, 0, sizeof(double) * (size_t)b.ncell) != cudaSuccess) return MHD_ECUDA;
      p += al256(sizeof(double) * (size_t)b.ncell);
    }
  }
  c->krp = c->scratch + krp_off;
  c->fofc_list = (unsigned long long*)(c->scratch + list_off);
  c->fofc_cap = ncell_all;
  c->krp_n = nkrp;
  c->dmass = (double*)(c->scratch + mass_off);
  c->dledger = c->ledger_on ? (double*)(c->scratch + led_off) : nullptr;
  if (c->dledger && cudaMemset(c->dledger, 0, sizeof(double) * 2 * (size_t)nb) != cudaSuccess) return MHD_ECUDA;
  for (int i = 0; i < nb; i++) {
    DevBlock& b = hb[i];
    b.id = i;
    b.dV = b.dx[0] * b.dx[1] * b.dx[2];
    b.lf = c->dledger ? c->dledger + 2 * (size_t)i : nullptr;
    b.la = c->dledger ? c->dledger + 2 * (size_t)i + 1 : nullptr;
  }
  if (c->dblk) cudaFree(c->dblk);
  if (c->dpre) cudaFree(c->dpre);
  if (c->dpre_blk) cudaFree(c->dpre_blk);
  c->dblk = nullptr;
  c->dpre = nullptr;
  c->dpre_blk = nullptr;
  {
    std::vector<long long> pb((size_t)nb * W_NKIND * 2, 0);
    for (int i = 0; i < nb; i++)
      for (int k = 0; k < W_NKIND; k++)
        pb[((size_t)i * W_NKIND + k) * 2 + 1] = pre[(size_t)k * (nb + 1) + i + 1] - pre[(size_t)k * (nb + 1) + i];
    // Work::pre for one block is indexed [kind * 2 + {0,1}]
    if (cudaMalloc(&c->dpre_blk, sizeof(long long) * pb.size()) != cudaSuccess) return MHD_ENOMEM;
    if (cudaMemcpy(c->dpre_blk, pb.data(), sizeof(long long) * pb.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return MHD_ECUDA;
  }
  if (cudaMalloc(&c->dblk, sizeof(DevBlock) * nb) != cudaSuccess) return MHD_ENOMEM;
  if (cudaMalloc(&c->dpre, sizeof(long long) * pre.size()) != cudaSuccess) return MHD_ENOMEM;
  if (cudaMemcpy(c->dblk, hb.data(), sizeof(DevBlock) * nb, cudaMemcpyHostToDevice) != cudaSuccess) return MHD_ECUDA;
  if (cudaMemcpy(c->dpre, pre.data(), sizeof(long long) * pre.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return MHD_ECUDA;
  c->hblk = hb;
  c->hpre = pre;
  c->key.assign(blocks, blocks + nb);
  c->list_version++;
  c->rhs_list = -1;
  // grid sizes: one wave of resident CTAs, capped by the work
  auto grid_of = [&](int kind, int threads, int occ) {
    long long tot = pre[(size_t)kind * (nb + 1) + nb];
    long long g = (tot + threads - 1) / threads;
    long long cap = (long long)c->nsm * (occ > 0 ? occ : 1);
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
  };
  c->grid[W_C2P] = grid_of(W_C2P, 128, c->occ_c2p[1]);
  c->grid[W_FX] = grid_of(W_FX, 128, c->occ_face[0]);
  c->grid[W_FY] = grid_of(W_FY, 128, c->occ_face[1]);
  c->grid[W_FZ] = grid_of(W_FZ, 128, c->occ_face[2]);
  c->grid[W_CELL] = grid_of(W_CELL, 128, c->occ_face[3]);
  c->grid[W_EDGE] = grid_of(W_EDGE, 128, c->occ_upd[0]);
  c->grid[W_FACE] = grid_of(W_FACE, 256, c->occ_upd[2]);
  c->grid[W_INIT] = grid_of(W_CELL, 128, c->occ_upd[1]);
  c->g_kprep = grid_of(W_C2P, 128, c->occ_krp[0]);
  c->g_kfin = grid_of(W_C2P, 128, c->occ_krp[2]);
  c->g_fprep = grid_of(W_CELL, 128, c->occ_krp[3]);
  c->g_ffin = grid_of(W_CELL, 128, c->occ_krp[4]);
  return MHD_OK;
}

cudaEvent_t get_event(mhd_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
  return st != cudaStreamCaptureStatusNone;
}

// Launch one kernel, bracketed by CUDA events on its stream when profiling.
template <class F>
void timed(mhd_ctx* c, int kind, cudaStream_t s, F&& launch) {
  const bool on = c->prof && !capturing(s);
  cudaEvent_t a = nullptr, b = nullptr;
  if (on) {
    a = get_event(c);
    b = get_event(c);
    cudaEventRecord(a, s);
  }
  launch();
  c->launches += 1;
  if (on) {
    cudaEventRecord(b, s);
    c->recs.push_back({kind, a, b});
  }
}

int tidx(int threads) { return threads == 64 ? 0 : (threads == 128 ? 1 : 2); }

// grid of a tunable kernel over `items` work items with its configuration
int tgrid(const mhd_ctx* c, int k, long long items) {
  const int th = c->cfg[k].threads;
  long long g = (items + th - 1) / th;
  long long cap = (long long)c->nsm * std::max(c->occ_t[k][tidx(th)], 1) * c->cfg[k].waves;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

Work work_of(const mhd_ctx* c) {
  Work w;
  w.blk = c->dblk;
  w.pre = c->dpre;
  w.nblocks = (int)c->key.size();
  return w;
}

// One launch sequence over the work `w` with `items[W_NKIND]` items per kind
// (all blocks of the list, or one block for per-block launches).
// The prep's con2prim start for c2p_guess g: 1 (learned) leaves status 4 for
// the seed kernel, 2 runs the FP32 search and FP64 polish in the prep, 0 and
// 3 take the FP64 bracket (3 from the previous root where there is one).
int prep_mode(int g) { return g == 1 || g == 2 ? g : 0; }
// With the prep's polish (c2p_guess 2) a status-0 cell is a rare fallback:
// the finish kernels solve such cells themselves and the refill solve
// launch, which would find no work in most calls, is left out.
bool inline_solve(int g) { return prep_mode(g) == 2; }
// Between the prep and the FP64 root solve of the learned con2prim (c2p_guess
// 1): the seed kernel, which runs the network on features it forms from the
// prep's KRP variables, the FP32 search and the FP64 polish, and turns
// status-4 cells into roots or FP64 brackets.
void c2p_seed(mhd_ctx* c, const KrpBuf& kb, long long n, cudaStream_t s) {
  if (c->P.guess != 1) return;
  const long long g = std::max(1LL, std::min((n + 127) / 128, (long long)c->nsm * std::max(c->occ_seed, 1)));
  timed(c, MHD_K_MLP, s, [&] {
    launch_krp_seed(c->P, kb, (float)c->mlp_delta, c->mlp_wb, c->mlp, c->nm, c->dstats, s, (int)g);
  });
}

// refresh: first compute the metric cache of the step (cells and faces)
int enqueue_c2p(mhd_ctx* c, cudaStream_t s, const Work& w, const long long* items, bool refresh) {
  if (c->P.guess == 1 && !c->mlp_ready) return MHD_ENOMLP;
  if (refresh) {
    const long long tot = items[W_C2P] + items[W_FX] + items[W_FY] + items[W_FZ] + items[W_CELL];
    const long long g = std::max(1LL, std::min((tot + 255) / 256, (long long)c->nsm * std::max(c->occ_metric, 1)));
    timed(c, MHD_K_METRIC, s, [&] { launch_metric_cache(w, s, (int)g); });
    c->metric_list = c->list_version;
    if (c->state_ready && cudaStreamWaitEvent(s, c->state_ready, 0) != cudaSuccess) return MHD_ECUDA;
  }
  KrpBuf kb = krp_view(c->krp, items[W_C2P]);
  const mhd_ctx::Cfg& cp = c->cfg[T_C2P_PREP];
  const mhd_ctx::Cfg& cf = c->cfg[T_C2P_FIN];
  timed(c, MHD_K_C2P, s, [&] {
    launch_krp_prep_block(w, c->P, kb, c->dstats, s, tgrid(c, T_C2P_PREP, items[W_C2P]), cp.threads,
                          prep_mode(c->P.guess), nullptr);
  });
  c2p_seed(c, kb, items[W_C2P], s);
  const bool inl = inline_solve(c->P.guess);
  if (!inl) timed(c, MHD_K_SOLVE, s, [&] { launch_krp_solve(c->P, kb, s, c->solve_grid(items[W_C2P])); });
  timed(c, MHD_K_C2P, s, [&] {
    launch_krp_finish_block(w, c->P, kb, c->dstats, s, tgrid(c, T_C2P_FIN, items[W_C2P]), cf.threads, inl);
  });
  return cuda_ok(cudaGetLastError());
}

// emf: launch the edge EMFs here (the stage entry points); the whole step
// launches them in enqueue_update instead, beside the cell update.
int enqueue_rhs(mhd_ctx* c, double dt, int stage, cudaStream_t s, const Work& w, const long long* items,
                bool emf = true) {
  double g0, g1, be;
  rk_weights(c->P.rk_order, stage, g0, g1, be);
  // The three sweeps read the stage's primitives and write their own flux
  // arrays: y and z run on two side streams forked from s and joined back, so
  // that one sweep's last wave overlaps the next one's first.  With the
  // per-kernel profile on they run one after another on s, so that each
  // launch's event time is its own.
  const bool fork = !c->prof;
  cudaStream_t fs[3] = {s, fork ? c->side[0] : s, fork ? c->side[1] : s};
  if (fork) {
    if (cudaEventRecord(c->ev_fork, s) != cudaSuccess) return MHD_ECUDA;
    for (int d = 1; d < 3; d++)
      if (cudaStreamWaitEvent(fs[d], c->ev_fork, 0) != cudaSuccess) return MHD_ECUDA;
  }
  for (int d = 0; d < 3; d++)
    timed(c, MHD_K_FLUX_X + d, fs[d], [&] {
      launch_flux_dir(d, w, c->P, fs[d], tgrid(c, T_FX + d, items[W_SX + d]), c->cfg[T_FX + d].threads);
    });
  if (fork)
    for (int d = 1; d < 3; d++) {
      if (cudaEventRecord(c->ev_join[d - 1], fs[d]) != cudaSuccess) return MHD_ECUDA;
      if (cudaStreamWaitEvent(s, c->ev_join[d - 1], 0) != cudaSuccess) return MHD_ECUDA;
    }
  if (c->P.fofc) {
    if (c->P.guess == 1 && !c->mlp_ready) return MHD_ENOMLP;
    KrpBuf kb = krp_view(c->krp, items[W_CELL]);
    kb.flist = c->fofc_list;
    kb.fcap = c->fofc_cap;
    timed(c, MHD_K_FOFC_FLAG, s, [&] {
      launch_krp_prep_fofc(w, c->P, g0, g1, be * dt, kb, c->dstats, s, tgrid(c, T_FOFC_PREP, items[W_CELL]),
                           c->cfg[T_FOFC_PREP].threads, prep_mode(c->P.guess), nullptr);
    });
    c2p_seed(c, kb, items[W_CELL], s);
    const bool inl = inline_solve(c->P.guess);
    if (!inl) timed(c, MHD_K_SOLVE, s, [&] { launch_krp_solve(c->P, kb, s, c->solve_grid(items[W_CELL])); });
    timed(c, MHD_K_FOFC_FLAG, s, [&] {
      launch_krp_finish_fofc(w, c->P, kb, c->dstats, s, tgrid(c, T_FOFC_FIN, items[W_CELL]),
                             c->cfg[T_FOFC_FIN].threads, inl);
    });
    // the faces of the listed flagged cells (one launch; the list is short)
    const long long g = std::min<long long>((items[W_CELL] + 127) / 128, (long long)c->nsm * std::max(c->occ_face[4], 1));
    timed(c, MHD_K_FOFC_FIX, s, [&] {
      launch_fofc_fix_list(w, c->P, kb.flist, kb.fcap, c->dstats, s, (int)std::max(1LL, g));
    });
  }
  if (c->ledger_on) {
    // weight of this stage's L(U) in U^{n+1}; the floor mass of stage 0 enters U^n itself
    const double b3[3] = {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0}, b2[2] = {0.5, 0.5};
    const double bs = c->P.rk_order == 3 ? b3[stage] : b2[stage];
    timed(c, MHD_K_LEDGER, s, [&] { launch_ledger_stage(w, stage == 0 ? 1.0 : bs, dt * bs, s); });
  }
  if (emf)
    timed(c, MHD_K_EMF, s, [&] {
      launch_emf(w, s, tgrid(c, T_EMF, items[W_EDGE]), c->cfg[T_EMF].threads);
    });
  c->rhs_list = c->list_version;
  c->rhs_stage = stage;
  return cuda_ok(cudaGetLastError());
}

// emf: launch the edge EMFs first on the face update's stream (the whole
// step; the stage entry points have them from enqueue_rhs).
int enqueue_update(mhd_ctx* c, double dt, int stage, cudaStream_t s, const Work& w, const long long* items,
                   bool emf = false) {
  double g0, g1, be;
  rk_weights(c->P.rk_order, stage, g0, g1, be);
  const int first = stage == 0 ? 1 : 0;
  // U and the face B~ are updated from different inputs (fluxes and sources;
  // edge EMFs) into different arrays: the face update, and the EMFs it reads
  // when they are launched here, run on a side stream beside the cell update
  // (the EMF kernel waits on its scattered loads, the cell update on the FP64
  // pipe); sequentially with the per-kernel profile on.
  const bool fork = !c->prof;
  cudaStream_t sf = fork ? c->side[0] : s;
  if (fork) {
    if (cudaEventRecord(c->ev_fork, s) != cudaSuccess) return MHD_ECUDA;
    if (cudaStreamWaitEvent(sf, c->ev_fork, 0) != cudaSuccess) return MHD_ECUDA;
  }
  timed(c, MHD_K_UPDATE, s, [&] {
    launch_update_cells(w, c->P, g0, g1, be * dt, first, s, tgrid(c, T_UPD, items[W_CELL]), c->cfg[T_UPD].threads);
  });
  if (emf)
    timed(c, MHD_K_EMF, sf, [&] {
      launch_emf(w, sf, tgrid(c, T_EMF, items[W_EDGE]), c->cfg[T_EMF].threads);
    });
  long long gfa = std::min<long long>((items[W_FACE] + 255) / 256, (long long)c->nsm * std::max(c->occ_upd[2], 1));
  timed(c, MHD_K_FACEB, sf, [&] { launch_update_faces(w, g0, g1, be * dt, first, sf, (int)std::max(1LL, gfa)); });
  if (fork) {
    if (cudaEventRecord(c->ev_join[0], sf) != cudaSuccess) return MHD_ECUDA;
    if (cudaStreamWaitEvent(s, c->ev_join[0], 0) != cudaSuccess) return MHD_ECUDA;
  }
  return cuda_ok(cudaGetLastError());
}

// totals over the block list
void list_items(const mhd_ctx* c, long long* items) {
  const size_t nb = c->key.size();
  for (int k = 0; k < W_NKIND; k++) items[k] = c->hpre[(size_t)k * (nb + 1) + nb];
}
// one block of the list
void block_items(const mhd_ctx* c, int b, long long* items) {
  const size_t nb = c->key.size();
  for (int k = 0; k < W_NKIND; k++) items[k] = c->hpre[(size_t)k * (nb + 1) + b + 1] - c->hpre[(size_t)k * (nb + 1) + b];
}
Work block_work(const mhd_ctx* c, int b) {
  Work w;
  w.blk = c->dblk + b;
  w.pre = c->dpre_blk + (size_t)b * W_NKIND * 2;
  w.nblocks = 1;
  return w;
}

int enqueue_c2p(mhd_ctx* c, cudaStream_t s, bool refresh) {
  long long it[W_NKIND];
  list_items(c, it);
  return enqueue_c2p(c, s, work_of(c), it, refresh);
}
int enqueue_rhs(mhd_ctx* c, double dt, int stage, cudaStream_t s, bool emf = true) {
  long long it[W_NKIND];
  list_items(c, it);
  return enqueue_rhs(c, dt, stage, s, work_of(c), it, emf);
}
int enqueue_update(mhd_ctx* c, double dt, int stage, cudaStream_t s, bool emf = false) {
  long long it[W_NKIND];
  list_items(c, it);
  return enqueue_update(c, dt, stage, s, work_of(c), it, emf);
}

// every block on its own: one launch sequence per block and stage
int enqueue_step_per_block(mhd_ctx* c, double dt, cudaStream_t s, bool metric) {
  for (int st = 0; st < c->P.rk_order; st++)
    for (int b = 0; b < (int)c->key.size(); b++) {
      long long it[W_NKIND];
      block_items(c, b, it);
      Work w = block_work(c, b);
      int r = enqueue_c2p(c, s, w, it, st == 0 && metric);
      if (!r) r = enqueue_rhs(c, dt, st, s, w, it, false);
      if (!r) r = enqueue_update(c, dt, st, s, w, it, true);
      if (r) return r;
    }
  return MHD_OK;
}

// The metric is an input of the whole step: its cache is computed once,
// before the first stage, unless the spacetime is fixed (mhd_params.
// fixed_metric) and the cache already holds this block list's metric.
bool metric_needed(const mhd_ctx* c) { return !(c->hp.fixed_metric && c->metric_list == c->list_version); }
int enqueue_step(mhd_ctx* c, double dt, cudaStream_t s, bool metric) {
  // without the metric kernel the caller's state event is waited for here
  if (!metric && c->state_ready && cudaStreamWaitEvent(s, c->state_ready, 0) != cudaSuccess) return MHD_ECUDA;
  for (int st = 0; st < c->P.rk_order; st++) {
    int r = enqueue_c2p(c, s, st == 0 && metric);
    if (!r) r = enqueue_rhs(c, dt, st, s, false);
    if (!r) r = enqueue_update(c, dt, st, s, true);
    if (r) return r;
  }
  return MHD_OK;
}

// Counters added by one call (mhd_c2p, mhd_c2p_cells with a stats out-argument):
// the device counters before and after its launches, both read after a
// stream synchronisation.
int stats_host(mhd_ctx* c, cudaStream_t s, unsigned long long* h) {
  if (cudaMemcpyAsync(h, c->dstats, sizeof(unsigned long long) * MHD_NSTATS, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return MHD_ECUDA;
  return cuda_ok(cudaStreamSynchronize(s));
}
void stats_diff(const unsigned long long* a, const unsigned long long* b, mhd_stats* out) {
  long long* o = &out->cells;
  for (int k = 0; k < MHD_NSTATS; k++) o[k] = (long long)(b[k] - a[k]);
}
static_assert(sizeof(mhd_stats) == MHD_NSTATS * sizeof(long long), "mhd_stats is MHD_NSTATS counters");

}  // namespace

extern "C" {

int mhd_init(const mhd_params* p, mhd_ctx** out) {
  if (!out || !p) return MHD_EINVAL;
  *out = nullptr;
  mhd_ctx* c = new mhd_ctx();
  int r = set_par(c, p);
  if (r) { delete c; return r; }
  if (cudaGetDevice(&c->dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->dev) != cudaSuccess) {
    delete c;
    return MHD_ECUDA;
  }
  if (occupancy_c2p(c->occ_c2p) || occupancy_face(c->occ_face) || occupancy_update(c->occ_upd) ||
      occupancy_krp(c->occ_krp) || mlp_setup_attrs()) {
    delete c;
    return MHD_ECUDA;
  }
  c->occ_metric = occ_metric_kernel();
  c->occ_seed = occ_seed_kernel();
  for (int ti = 0; ti < 3; ti++) {
    const int th = 64 << ti;
    c->occ_t[T_C2P_PREP][ti] = occ_krp_kernel(0, th);
    c->occ_t[T_C2P_FIN][ti] = occ_krp_kernel(1, th);
    c->occ_t[T_FOFC_PREP][ti] = occ_krp_kernel(2, th);
    c->occ_t[T_FOFC_FIN][ti] = occ_krp_kernel(3, th);
    for (int d = 0; d < 3; d++) c->occ_t[T_FX + d][ti] = occ_face_kernel(d, th);
    c->occ_t[T_EMF][ti] = occ_update_kernel(0, th);
    c->occ_t[T_UPD][ti] = occ_update_kernel(1, th);
  }
  auto release = [](mhd_ctx* x) {
    for (int q = 0; q < 2; q++) {
      if (x->side[q]) cudaStreamDestroy(x->side[q]);
      if (x->ev_join[q]) cudaEventDestroy(x->ev_join[q]);
    }
    if (x->ev_fork) cudaEventDestroy(x->ev_fork);
    if (x->dstats) cudaFree(x->dstats);
    delete x;
  };
  bool ok = true;
  for (int q = 0; q < 2; q++) ok = ok && cudaStreamCreateWithFlags(&c->side[q], cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  for (int q = 0; q < 2; q++) ok = ok && cudaEventCreateWithFlags(&c->ev_join[q], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    release(c);
    return MHD_ECUDA;
  }
  if (cudaMalloc(&c->dstats, sizeof(unsigned long long) * MHD_NSTATS) != cudaSuccess) {
    c->dstats = nullptr;
    release(c);
    return MHD_ENOMEM;
  }
  if (cudaMemset(c->dstats, 0, sizeof(unsigned long long) * MHD_NSTATS) != cudaSuccess) {
    release(c);
    return MHD_ECUDA;
  }
  *out = c;
  return MHD_OK;
}

int mhd_set_params(mhd_ctx* c, const mhd_params* p) {
  if (!c) return MHD_EINVAL;
  const int old_guess = c->P.guess;
  int r = set_par(c, p);
  if (!r) destroy_graph(c);
  if (!r && old_guess != c->P.guess) {
    cudaDeviceSynchronize();
    c->key.clear();   // the next call re-plans the scratch (guess buffers)
  }
  return r;
}

int mhd_ledger(mhd_ctx* c, int enable) {
  if (!c) return MHD_EINVAL;
  if (c->ledger_on != (enable != 0)) {
    cudaDeviceSynchronize();
    c->ledger_on = enable != 0;
    c->key.clear();
    destroy_graph(c);
  }
  return MHD_OK;
}

int mhd_ledger_read(mhd_ctx* c, double* out, int reset, void* stream) {
  if (!c || !out) return MHD_EINVAL;
  if (!c->ledger_on || !c->dledger || c->key.empty()) return MHD_ESTATE;
  const size_t nb = c->key.size();
  std::vector<double> h(2 * nb);
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(h.data(), c->dledger, sizeof(double) * 2 * nb, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return MHD_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MHD_ECUDA;
  for (size_t i = 0; i < nb; i++) out[i] = h[2 * i + 1];
  if (reset && cudaMemsetAsync(c->dledger, 0, sizeof(double) * 2 * nb, s) != cudaSuccess) return MHD_ECUDA;
  return MHD_OK;
}

int mhd_fill_ghosts(mhd_ctx* c, const mhd_block* blocks, int nb, const int* nbr, void* stream) {
  if (!c || !nbr) return MHD_EINVAL;
  int r = prepare(c, blocks, nb);
  if (r) return r;
  for (int i = 0; i < nb; i++)
    for (int q = 0; q < 6; q++) {
      const int v = nbr[(size_t)i * 6 + q];
      if (v < -2 || v >= nb) return MHD_EINVAL;
      if (v >= 0 && (blocks[v].ng != blocks[i].ng || blocks[v].n[0] != blocks[i].n[0] ||
                     blocks[v].n[1] != blocks[i].n[1] || blocks[v].n[2] != blocks[i].n[2]))
        return MHD_EINVAL;
      // another block supplies whole ghost layers only if it is at least ng
      // wide along the axis (the block itself wraps modulo n)
      if (v >= 0 && v != i && blocks[i].n[q / 2] < blocks[i].ng) return MHD_EINVAL;
    }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)nb * 6;
  if (n > c->dnbr_n) {
    if (cudaStreamSynchronize(s) != cudaSuccess) return MHD_ECUDA;
    if (c->dnbr) cudaFree(c->dnbr);
    c->dnbr = nullptr;
    c->dnbr_n = 0;
    if (cudaMalloc(&c->dnbr, sizeof(int) * n) != cudaSuccess) return MHD_ENOMEM;
    c->dnbr_n = n;
  }
  if (cudaMemcpyAsync(c->dnbr, nbr, sizeof(int) * n, cudaMemcpyHostToDevice, s) != cudaSuccess) return MHD_ECUDA;
  long long it[W_NKIND];
  list_items(c, it);
  Work w = work_of(c);
  for (int ax = 0; ax < 3; ax++)
    for (int kind = 0; kind < 4; kind++) {
      const long long items = kind == 0 ? it[W_INIT] : it[W_GFX + kind - 1];
      const long long g = std::max(1LL, std::min((items + 255) / 256, (long long)c->nsm * 8));
      launch_fill_ghosts(w, c->dnbr, kind, ax, s, (int)g);
      c->launches += 1;
    }
  return cuda_ok(cudaGetLastError());
}

int mhd_block_mass(mhd_ctx* c, const mhd_block* blocks, int nb, double* out, void* stream) {
  if (!c || !out) return MHD_EINVAL;
  int r = prepare(c, blocks, nb);
  if (r) return r;
  cudaStream_t s = (cudaStream_t)stream;
  launch_block_mass(work_of(c), c->dmass, s);
  c->launches += 1;
  if (cudaMemcpyAsync(out, c->dmass, sizeof(double) * nb, cudaMemcpyDeviceToHost, s) != cudaSuccess) return MHD_ECUDA;
  return cuda_ok(cudaStreamSynchronize(s));
}

void mhd_finalize(mhd_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  destroy_graph(c);
  if (c->scratch) cudaFree(c->scratch);
  if (c->dblk) cudaFree(c->dblk);
  if (c->dpre) cudaFree(c->dpre);
  if (c->dpre_blk) cudaFree(c->dpre_blk);
  if (c->dstats) cudaFree(c->dstats);
  if (c->dnbr) cudaFree(c->dnbr);
  if (c->cells_buf) cudaFree(c->cells_buf);
  if (c->mlp) cudaFree(c->mlp);
  if (c->mlp_wb) cudaFree(c->mlp_wb);
  if (c->mlp_loss) cudaFree(c->mlp_loss);
  if (c->mlp_acc) cudaFree(c->mlp_acc);
  for (auto& r : c->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  for (int q = 0; q < 2; q++) {
    if (c->side[q]) cudaStreamDestroy(c->side[q]);
    if (c->ev_join[q]) cudaEventDestroy(c->ev_join[q]);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  delete c;
}

const char* mhd_strerror(int code) {
  switch (code) {
    case MHD_OK: return "ok";
    case MHD_EINVAL: return "invalid argument";
    case MHD_ECUDA: return "CUDA runtime error";
    case MHD_ENOMEM: return "device allocation failed";
    case MHD_ESTATE: return "call out of order";
    case MHD_ENOMLP: return "learned guess requested but no network loaded";
    case MHD_ETOOBIG: return "block exceeds the 16 MiB static scratch of mhd_stage_noalloc";
    default: return "unknown error";
  }
}

int mhd_init_block(mhd_ctx* c, mhd_block* blk, const double* const A[3], void* stream) {
  if (!c || !blk || !A || !A[0] || !A[1] || !A[2]) return MHD_EINVAL;
  int r = check_block(*blk);
  if (r) return r;
  DevBlock b;
  std::memset(&b, 0, sizeof(b));
  for (int d = 0; d < 3; d++) {
    b.n[d] = blk->n[d];
    b.N[d] = blk->n[d] + 2 * blk->ng;
    b.dx[d] = blk->dx[d];
    b.idx[d] = 1.0 / blk->dx[d];
    b.bf[d] = blk->bf[d];
  }
  b.ng = blk->ng;
  b.ncell = ncell_of(*blk);
  b.cons = blk->cons; b.prim = blk->prim; b.bcc = blk->bcc; b.adm = blk->adm;
  launch_init_block(b, c->P, A, (cudaStream_t)stream, c->nsm);
  c->launches += 2;
  return cuda_ok(cudaGetLastError());
}

int mhd_prim2cons(mhd_ctx* c, long n, const double* prim, const double* Bd, const double* g, double* cons,
                  void* stream) {
  if (!c || n < 0 || (n > 0 && (!prim || !Bd || !g || !cons))) return MHD_EINVAL;
  if (n == 0) return MHD_OK;
  launch_p2c_cells(c->P, n, prim, Bd, g, cons, (cudaStream_t)stream, c->nsm);
  c->launches += 1;
  return cuda_ok(cudaGetLastError());
}

}  // extern "C"

namespace {

// Grow-only buffer for independent-cell con2prim: KRP scratch, features, log(mu) guesses.
int cells_scratch(mhd_ctx* c, long n, cudaStream_t s, KrpBuf* kb, float** feat, float** logmu) {
  const size_t kbytes = al256(krp_bytes(n)), fbytes = al256(sizeof(float) * MLP_FSTRIDE * (size_t)n),
               lbytes = al256(sizeof(float) * (size_t)n);
  const size_t need = kbytes + fbytes + lbytes;
  if (need > c->cells_bytes) {
    cudaStreamSynchronize(s);
    if (c->cells_buf) cudaFree(c->cells_buf);
    c->cells_buf = nullptr;
    c->cells_bytes = 0;
    if (cudaMalloc(&c->cells_buf, need) != cudaSuccess) return MHD_ENOMEM;
    c->cells_bytes = need;
  }
  *kb = krp_view(c->cells_buf, n);
  *feat = (float*)(c->cells_buf + kbytes);
  *logmu = (float*)(c->cells_buf + kbytes + fbytes);
  return MHD_OK;
}

int cells_grid(const mhd_ctx* c, long n, int occ) {
  long long nb = (n + 127) / 128, cap = (long long)c->nsm * std::max(occ, 1);
  return (int)std::max(1LL, std::min(nb, cap));
}

}  // namespace

namespace {
int c2p_cells_enqueue(mhd_ctx* c, long n, double* cons, const double* Bd, const double* g, double* prim,
                      unsigned char* flags, int* iters, cudaStream_t s);
}

extern "C" {

int mhd_c2p_cells(mhd_ctx* c, long n, double* cons, const double* Bd, const double* g, double* prim,
                  unsigned char* flags, int* iters, void* stream, mhd_stats* stats) {
  if (!c || n < 0 || (n > 0 && (!cons || !Bd || !g || !flags))) return MHD_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long h0[MHD_NSTATS], h1[MHD_NSTATS];
  int r = stats ? stats_host(c, s, h0) : MHD_OK;
  if (!r && n > 0) r = c2p_cells_enqueue(c, n, cons, Bd, g, prim, flags, iters, s);
  if (!r && stats) r = stats_host(c, s, h1);
  if (!r && stats) stats_diff(h0, h1, stats);
  return r;
}

}  // extern "C"

namespace {
int c2p_cells_enqueue(mhd_ctx* c, long n, double* cons, const double* Bd, const double* g, double* prim,
                      unsigned char* flags, int* iters, cudaStream_t s) {
  // 0 plain, 1 learned + FP32 search + FP64 polish, 2 FP32 search from the
  // plain bracket + FP64 polish; independent cells have no previous root, so 3
  // solves as 0
  const int mode = c->P.guess == 3 ? 0 : c->P.guess;
  if (mode == 1 && !c->mlp_ready) return MHD_ENOMLP;
  KrpBuf kb;
  float *feat, *logmu;
  int r = cells_scratch(c, n, s, &kb, &feat, &logmu);
  if (r) return r;
  timed(c, MHD_K_C2P, s, [&] {
    launch_krp_prep_cells(c->P, kb, cons, Bd, g, mode, nullptr, c->dstats, s,
                          cells_grid(c, n, c->occ_krp[prim ? 5 : 7]), prim == nullptr);
  });
  c2p_seed(c, kb, n, s);
  timed(c, MHD_K_SOLVE, s, [&] { launch_krp_solve(c->P, kb, s, c->solve_grid(n)); });
  timed(c, MHD_K_C2P, s, [&] {
    launch_krp_finish_cells(c->P, kb, cons, Bd, g, prim, flags, iters, c->dstats, s, cells_grid(c, n, c->occ_krp[6]));
  });
  return cuda_ok(cudaGetLastError());
}
}  // namespace

extern "C" {

// ------------------------------------------------------------ learned guess
int mhd_mlp_init(mhd_ctx* c, unsigned long long seed) {
  if (!c) return MHD_EINVAL;
  if (!c->mlp) {
    if (cudaMalloc(&c->mlp, sizeof(float) * 4 * MLP_NPARAM) != cudaSuccess) return MHD_ENOMEM;
    if (cudaMalloc(&c->mlp_wb, sizeof(__nv_bfloat16) * MLP_NBF) != cudaSuccess) return MHD_ENOMEM;
    if (cudaMalloc(&c->mlp_loss, sizeof(float)) != cudaSuccess) return MHD_ENOMEM;
    if (cudaMalloc(&c->mlp_acc, sizeof(double) * 12) != cudaSuccess) return MHD_ENOMEM;
  }
  // Glorot-uniform weights from a splitmix64 stream, zero biases
  std::vector<float> h(4 * MLP_NPARAM, 0.0f);
  unsigned long long x = seed ? seed : 0x9E3779B97F4A7C15ull;
  auto uni = [&]() {
    x += 0x9E3779B97F4A7C15ull;
    unsigned long long z = x;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
  };
  const double l1 = std::sqrt(6.0 / (MLP_NIN + MLP_NH)), l2 = std::sqrt(6.0 / (2 * MLP_NH)),
               l3 = std::sqrt(6.0 / (MLP_NH + 1));
  for (int i = 0; i < MLP_NH * MLP_NIN; i++) h[MLP_W1 + i] = (float)(l1 * uni());
  for (int i = 0; i < MLP_NH * MLP_NH; i++) h[MLP_W2 + i] = (float)(l2 * uni());
  for (int i = 0; i < MLP_NH; i++) h[MLP_W3 + i] = (float)(l3 * uni());
  if (cudaMemcpy(c->mlp, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess) return MHD_ECUDA;
  launch_mlp_pack(c->mlp, c->mlp_wb, nullptr);
  for (int f = 0; f < MLP_NIN; f++) {
    c->nm.fmean[f] = 0.0f;
    c->nm.finv[f] = 1.0f;
  }
  c->nm.ymean = 0.0f;
  c->nm.ystd = 1.0f;
  c->mlp_delta = 0.0;
  c->mlp_t = 0;
  c->mlp_ready = false;
  return cuda_ok(cudaDeviceSynchronize());
}

int mhd_mlp_dataset(mhd_ctx* c, long n, const double* cons, const double* Bd, const double* g, float* feat,
                    float* logmu, void* stream) {
  if (!c || n <= 0 || !cons || !Bd || !g || !feat || !logmu) return MHD_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  KrpBuf kb;
  float *f2, *l2;
  int r = cells_scratch(c, n, s, &kb, &f2, &l2);
  if (r) return r;
  Par P = c->P;
  launch_krp_prep_cells(P, kb, cons, Bd, g, 0, feat, c->dstats, s, cells_grid(c, n, c->occ_krp[5]));
  launch_krp_solve(P, kb, s, c->solve_grid(n));
  launch_mlp_logmu(kb, logmu, s, c->nsm);
  c->launches += 3;
  return cuda_ok(cudaGetLastError());
}

int mhd_mlp_train(mhd_ctx* c, const float* feat, const float* logmu, long n, int epochs, int batch, float lr,
                  unsigned long long seed, float* loss_out, void* stream) {
  if (!c || !c->mlp || !feat || !logmu || n < 64 || epochs < 1 || batch < 32 || !(lr > 0.0f)) return MHD_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  // normalisation of the features and the target
  if (cudaMemsetAsync(c->mlp_acc, 0, sizeof(double) * 12, s) != cudaSuccess) return MHD_ECUDA;
  launch_mlp_stats(feat, logmu, n, c->mlp_acc, s, c->nsm);
  double acc[12];
  if (cudaMemcpyAsync(acc, c->mlp_acc, sizeof(acc), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MHD_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MHD_ECUDA;
  for (int f = 0; f < MLP_NIN; f++) {
    double m = acc[f] / n, v = acc[6 + f] / n - m * m;
    c->nm.fmean[f] = (float)m;
    c->nm.finv[f] = (float)(1.0 / std::sqrt(std::max(v, 1e-12)));
  }
  {
    double m = acc[5] / n, v = acc[11] / n - m * m;
    c->nm.ymean = (float)m;
    c->nm.ystd = (float)std::sqrt(std::max(v, 1e-12));
  }
  float* w = c->mlp;
  float* mm = c->mlp + MLP_NPARAM;
  float* vv = c->mlp + 2 * MLP_NPARAM;
  float* gr = c->mlp + 3 * MLP_NPARAM;
  if (cudaMemsetAsync(mm, 0, sizeof(float) * 3 * MLP_NPARAM, s) != cudaSuccess) return MHD_ECUDA;
  c->mlp_t = 0;
  unsigned long long x = seed ? seed : 12345ull;
  auto rnd = [&]() {
    x ^= x << 13; x ^= x >> 7; x ^= x << 17;
    return x;
  };
  auto gcd = [](unsigned long long a, unsigned long long b) {
    while (b) { unsigned long long t = a % b; a = b; b = t; }
    return a;
  };
  const long steps_per_epoch = (n + batch - 1) / batch;
  const long total = steps_per_epoch * epochs;
  for (int ep = 0; ep < epochs; ep++) {
    unsigned long long pa = 1 + rnd() % (unsigned long long)(n - 1);
    while (gcd(pa, (unsigned long long)n) != 1) pa = 1 + rnd() % (unsigned long long)(n - 1);
    unsigned long long pb = rnd() % (unsigned long long)n;
    if (ep == epochs - 1 && cudaMemsetAsync(c->mlp_loss, 0, sizeof(float), s) != cudaSuccess) return MHD_ECUDA;
    for (long st = 0; st < steps_per_epoch; st++) {
      const long off = st * batch;
      const int b = (int)std::min<long>(batch, n - off);
      launch_mlp_train_step(feat, logmu, n, (long long)pa, (long long)pb, off, b, c->nm, c->mlp_wb, w, gr,
                            c->mlp_loss, s);
      c->mlp_t++;
      const double frac = (double)c->mlp_t / (double)total;
      const float lr_t = (float)(lr * 0.5 * (1.0 + std::cos(3.141592653589793 * frac)));
      launch_mlp_adam(w, mm, vv, gr, lr_t, c->mlp_t, c->mlp_wb, s);
      c->launches += 3;
    }
  }
  float L = 0.0f;
  if (cudaMemcpyAsync(&L, c->mlp_loss, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MHD_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MHD_ECUDA;
  if (loss_out) *loss_out = L / (float)n;
  c->mlp_delta = 0.0;
  c->mlp_ready = false;
  return cuda_ok(cudaGetLastError());
}

int mhd_mlp_infer(mhd_ctx* c, const float* feat, long n, float* logmu_out, void* stream) {
  if (!c || !c->mlp || !feat || !logmu_out || n < 0) return MHD_EINVAL;
  if (n == 0) return MHD_OK;
  launch_mlp_infer(feat, n, c->nm, c->mlp_wb, c->mlp, logmu_out, (cudaStream_t)stream, c->nsm);
  c->launches += 1;
  return cuda_ok(cudaGetLastError());
}

int mhd_mlp_calibrate(mhd_ctx* c, const float* feat, const float* logmu, long n, double quantile, double* delta_out,
                      void* stream) {
  if (!c || !c->mlp || !feat || !logmu || n < 1 || !(quantile > 0.0 && quantile <= 1.0)) return MHD_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  KrpBuf kb;
  float *f2, *pred;
  int r = cells_scratch(c, n, s, &kb, &f2, &pred);
  if (r) return r;
  launch_mlp_infer(feat, n, c->nm, c->mlp_wb, c->mlp, pred, s, c->nsm);
  c->launches += 1;
  std::vector<float> hp(n), ht(n);
  if (cudaMemcpyAsync(hp.data(), pred, sizeof(float) * n, cudaMemcpyDeviceToHost, s) != cudaSuccess) return MHD_ECUDA;
  if (cudaMemcpyAsync(ht.data(), logmu, sizeof(float) * n, cudaMemcpyDefault, s) != cudaSuccess) return MHD_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MHD_ECUDA;
  std::vector<double> e(n);
  for (long i = 0; i < n; i++) e[i] = std::fabs((double)hp[i] - (double)ht[i]);
  long k = std::min<long>(n - 1, (long)std::ceil(quantile * n) - 1);
  if (k < 0) k = 0;
  std::nth_element(e.begin(), e.begin() + k, e.end());
  c->mlp_delta = std::max(e[k], 1e-6);
  c->mlp_ready = true;
  if (delta_out) *delta_out = c->mlp_delta;
  return MHD_OK;
}

int mhd_mlp_grad(mhd_ctx* c, const float* feat, const float* logmu, long n, float* grad_out, float* loss_out,
                 void* stream) {
  if (!c || !c->mlp || !feat || !logmu || n < 1 || n > (1L << 30) || !grad_out) return MHD_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  float* gr = c->mlp + 3 * MLP_NPARAM;
  if (cudaMemsetAsync(gr, 0, sizeof(float) * MLP_NPARAM, s) != cudaSuccess) return MHD_ECUDA;
  if (cudaMemsetAsync(c->mlp_loss, 0, sizeof(float), s) != cudaSuccess) return MHD_ECUDA;
  launch_mlp_train_step(feat, logmu, n, 1, 0, 0, (int)n, c->nm, c->mlp_wb, c->mlp, gr, c->mlp_loss, s);
  c->launches += 1;
  if (cudaMemcpyAsync(grad_out, gr, sizeof(float) * MLP_NPARAM, cudaMemcpyDefault, s) != cudaSuccess)
    return MHD_ECUDA;
  float L = 0.0f;
  if (cudaMemcpyAsync(&L, c->mlp_loss, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MHD_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MHD_ECUDA;
  if (cudaMemsetAsync(gr, 0, sizeof(float) * MLP_NPARAM, s) != cudaSuccess) return MHD_ECUDA;
  if (loss_out) *loss_out = L / (float)n;
  return cuda_ok(cudaStreamSynchronize(s));
}

int mhd_mlp_get(mhd_ctx* c, float* state) {
  if (!c || !c->mlp || !state) return MHD_EINVAL;
  if (cudaMemcpy(state, c->mlp, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess) return MHD_ECUDA;
  float* t = state + MLP_NPARAM;
  for (int f = 0; f < MLP_NIN; f++) {
    t[f] = c->nm.fmean[f];
    t[MLP_NIN + f] = c->nm.finv[f];
  }
  t[2 * MLP_NIN] = c->nm.ymean;
  t[2 * MLP_NIN + 1] = c->nm.ystd;
  t[2 * MLP_NIN + 2] = (float)c->mlp_delta;
  return MHD_OK;
}

int mhd_mlp_set(mhd_ctx* c, const float* state) {
  if (!c || !state) return MHD_EINVAL;
  if (!c->mlp) {
    int r = mhd_mlp_init(c, 1);
    if (r) return r;
  }
  if (cudaMemcpy(c->mlp, state, sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice) != cudaSuccess) return MHD_ECUDA;
  launch_mlp_pack(c->mlp, c->mlp_wb, nullptr);
  const float* t = state + MLP_NPARAM;
  for (int f = 0; f < MLP_NIN; f++) {
    c->nm.fmean[f] = t[f];
    c->nm.finv[f] = t[MLP_NIN + f];
  }
  c->nm.ymean = t[2 * MLP_NIN];
  c->nm.ystd = t[2 * MLP_NIN + 1];
  c->mlp_delta = t[2 * MLP_NIN + 2];
  c->mlp_ready = c->mlp_delta > 0.0;
  return cuda_ok(cudaDeviceSynchronize());
}

int mhd_mlp_save(mhd_ctx* c, void* blob, long bytes, long* size) {
  if (size) *size = MHD_MLP_BLOB_BYTES;
  if (!c || !c->mlp || !blob || bytes < (long)MHD_MLP_BLOB_BYTES) return MHD_EINVAL;
  std::vector<float> st(MHD_MLP_NSTATE);
  int r = mhd_mlp_get(c, st.data());
  if (r) return r;
  unsigned char* o = (unsigned char*)blob;
  for (int i = 0; i < MLP_NPARAM; i++) {
    const unsigned short h = __bfloat16_as_ushort(__float2bfloat16_rn(st[i]));
    o[2 * i] = (unsigned char)(h & 0xff);
    o[2 * i + 1] = (unsigned char)(h >> 8);
  }
  std::memcpy(o + 2 * MLP_NPARAM, st.data() + MLP_NPARAM, sizeof(float) * (MHD_MLP_NSTATE - MLP_NPARAM));
  return MHD_OK;
}

int mhd_mlp_load(mhd_ctx* c, const void* bf16_weights, long bytes) {
  if (!c || !bf16_weights || bytes != (long)MHD_MLP_BLOB_BYTES) return MHD_EINVAL;
  const unsigned char* in = (const unsigned char*)bf16_weights;
  std::vector<float> st(MHD_MLP_NSTATE);
  for (int i = 0; i < MLP_NPARAM; i++) {
    const unsigned short h = (unsigned short)(in[2 * i] | (in[2 * i + 1] << 8));
    st[i] = __bfloat162float(__ushort_as_bfloat16(h));
  }
  std::memcpy(st.data() + MLP_NPARAM, in + 2 * MLP_NPARAM, sizeof(float) * (MHD_MLP_NSTATE - MLP_NPARAM));
  return mhd_mlp_set(c, st.data());
}

int mhd_c2p(mhd_ctx* c, const mhd_block* blocks, int nb, void* stream, mhd_stats* stats) {
  if (!c) return MHD_EINVAL;
  int r = prepare(c, blocks, nb);
  if (r) return r;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long h0[MHD_NSTATS], h1[MHD_NSTATS];
  if (stats && (r = stats_host(c, s, h0))) return r;
  r = enqueue_c2p(c, s, true);
  if (!r && stats) r = stats_host(c, s, h1);
  if (!r && stats) stats_diff(h0, h1, stats);
  return r;
}

int mhd_rhs(mhd_ctx* c, const mhd_block* blocks, int nb, double dt, int stage, void* stream) {
  if (!c || !(dt > 0.0) || stage < 0 || stage >= c->P.rk_order) return MHD_EINVAL;
  int r = prepare(c, blocks, nb);
  if (r) return r;
  return enqueue_rhs(c, dt, stage, (cudaStream_t)stream);
}

int mhd_rk_update(mhd_ctx* c, const mhd_block* blocks, int nb, double dt, int stage, void* stream) {
  if (!c || !(dt > 0.0) || stage < 0 || stage >= c->P.rk_order) return MHD_EINVAL;
  int r = prepare(c, blocks, nb);
  if (r) return r;
  if (c->rhs_list != c->list_version || c->rhs_stage != stage) return MHD_ESTATE;
  r = enqueue_update(c, dt, stage, (cudaStream_t)stream);
  c->rhs_list = -1;
  return r;
}

int mhd_step(mhd_ctx* c, const mhd_block* blocks, int nb, double dt, int graph, void* stream) {
  if (!c || !(dt > 0.0)) return MHD_EINVAL;
  int r = prepare(c, blocks, nb);
  if (r) return r;
  cudaStream_t s = (cudaStream_t)stream;
  const bool metric = metric_needed(c);
  if (graph == 2) return enqueue_step_per_block(c, dt, s, metric);
  if (!graph) return enqueue_step(c, dt, s, metric);
  if (!s) return MHD_EINVAL;  // the legacy default stream cannot be captured
  if (!(c->gexec && c->g_list == c->list_version && c->g_par == c->par_version && c->g_dt == dt && c->g_stream == s &&
        c->g_metric == metric)) {
    destroy_graph(c);
    long long before = c->launches;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return MHD_ECUDA;
    int er = enqueue_step(c, dt, s, metric);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(s, &g);
    if (er || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return er ? er : MHD_ECUDA;
    }
    ce = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) { c->gexec = nullptr; return MHD_ECUDA; }
    c->g_launches = (int)(c->launches - before);
    c->launches = before;
    c->g_list = c->list_version;
    c->g_par = c->par_version;
    c->g_dt = dt;
    c->g_stream = s;
    c->g_metric = metric;
  }
  c->launches += c->g_launches;
  return cuda_ok(cudaGraphLaunch(c->gexec, s));
}

int mhd_check_rcp(const double* x, long n, double* rel_out, void* stream) {
  if (n < 0 || (n > 0 && (!x || !rel_out))) return MHD_EINVAL;
  if (n == 0) return MHD_OK;
  int dev = 0, nsm = 1;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MHD_ECUDA;
  if (cudaPeekAtLastError() != cudaSuccess) return MHD_ECUDA;
  launch_check_rcp(x, n, rel_out, (cudaStream_t)stream, nsm);
  return cuda_ok(cudaPeekAtLastError());
}

int mhd_check_enclosures(const double* x, long n, unsigned char* miss_out, void* stream) {
  if (n < 0 || (n > 0 && (!x || !miss_out))) return MHD_EINVAL;
  if (n == 0) return MHD_OK;
  int dev = 0, nsm = 1;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MHD_ECUDA;
  if (cudaPeekAtLastError() != cudaSuccess) return MHD_ECUDA;
  launch_check_iv(x, n, miss_out, (cudaStream_t)stream, nsm);
  return cuda_ok(cudaPeekAtLastError());
}

int mhd_step_overlap(mhd_ctx* c, const mhd_block* blocks, int nb, double dt, void* stream, void* state_ready) {
  if (!c || !(dt > 0.0)) return MHD_EINVAL;
  int r = prepare(c, blocks, nb);
  if (r) return r;
  c->state_ready = (cudaEvent_t)state_ready;
  r = enqueue_step(c, dt, (cudaStream_t)stream, metric_needed(c));
  c->state_ready = nullptr;
  return r;
}

int mhd_graph_step(mhd_ctx* c, const mhd_block* blocks, int nb, double dt, void* stream) {
  return mhd_step(c, blocks, nb, dt, 1, stream);
}

int mhd_read_stats(mhd_ctx* c, mhd_stats* out, void* stream) {
  if (!c || !out) return MHD_EINVAL;
  unsigned long long h[MHD_NSTATS];
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(h, c->dstats, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MHD_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MHD_ECUDA;
  long long* o = &out->cells;
  for (int k = 0; k < MHD_NSTATS; k++) o[k] = (long long)h[k];
  return MHD_OK;
}

int mhd_reset_stats(mhd_ctx* c, void* stream) {
  if (!c) return MHD_EINVAL;
  return cuda_ok(cudaMemsetAsync(c->dstats, 0, sizeof(unsigned long long) * MHD_NSTATS, (cudaStream_t)stream));
}

int mhd_scratch_copy(mhd_ctx* c, int b, int which, double* dst, long count, long* size, void* stream) {
  if (!c || b < 0 || b >= (int)c->hblk.size() || which < 0 || which > 5) return MHD_EINVAL;
  const DevBlock& d = c->hblk[b];
  const long long N0 = d.N[0], N1 = d.N[1], N2 = d.N[2];
  const long long nf[3] = {N2 * N1 * (N0 + 1), N2 * (N1 + 1) * N0, (N2 + 1) * N1 * N0};
  const long long ne[3] = {(N2 + 1) * (N1 + 1) * N0, (N2 + 1) * N1 * (N0 + 1), N2 * (N1 + 1) * (N0 + 1)};
  const double* src = which < 3 ? d.flux[which] : d.emf[which - 3];
  long n = (long)(which < 3 ? 7 * nf[which] : ne[which - 3]);
  if (size) *size = n;
  if (count == 0) return MHD_OK;
  if (!dst || count != n) return MHD_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDefault, s) != cudaSuccess) return MHD_ECUDA;
  return cuda_ok(cudaStreamSynchronize(s));
}

long long mhd_kernel_launches(const mhd_ctx* c) { return c ? c->launches : 0; }

int mhd_autotune(mhd_ctx* c, const mhd_block* blocks, int nb, double dt, void* stream, int* cfg_out) {
  if (!c || !(dt > 0.0)) return MHD_EINVAL;
  int r = prepare(c, blocks, nb);
  if (r) return r;
  cudaStream_t s = (cudaStream_t)stream;
  const bool prof = c->prof;
  c->prof = false;
  // valid inputs for every kernel: con2prim and the right-hand side of stage 0
  r = enqueue_c2p(c, s, true);
  if (!r) r = enqueue_rhs(c, dt, 0, s);
  if (r) { c->prof = prof; return r; }
  long long it[W_NKIND];
  list_items(c, it);
  Work w = work_of(c);
  double g0, g1, be;
  rk_weights(c->P.rk_order, 0, g0, g1, be);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // kernel kinds in an order that keeps the scratch valid: a prep phase is
  // followed by its root solve before the finish phase is timed; the update is
  // timed with weights (g0, g1, b dt) = (0, 1, 0), which leaves U unchanged.
  const int order[T_N] = {T_C2P_PREP, T_C2P_FIN, T_FX, T_FY, T_FZ, T_FOFC_PREP, T_FOFC_FIN, T_EMF, T_UPD};
  for (int oi = 0; oi < T_N; oi++) {
    const int k = order[oi];
    if ((k == T_FOFC_PREP || k == T_FOFC_FIN) && !c->P.fofc) continue;
    const bool fofc_k = k == T_FOFC_PREP || k == T_FOFC_FIN;
    KrpBuf kb = krp_view(c->krp, fofc_k ? it[W_CELL] : it[W_C2P]);
    auto launch = [&]() {
      const int th = c->cfg[k].threads;
      switch (k) {
        case T_C2P_PREP:
          launch_krp_prep_block(w, c->P, kb, c->dstats, s, tgrid(c, k, it[W_C2P]), th, prep_mode(c->P.guess),
                                nullptr);
          break;
        case T_C2P_FIN: launch_krp_finish_block(w, c->P, kb, c->dstats, s, tgrid(c, k, it[W_C2P]), th); break;
        case T_FX: case T_FY: case T_FZ:
          launch_flux_dir(k - T_FX, w, c->P, s, tgrid(c, k, it[W_SX + k - T_FX]), th);
          break;
        case T_FOFC_PREP:
          launch_krp_prep_fofc(w, c->P, g0, g1, be * dt, kb, c->dstats, s, tgrid(c, k, it[W_CELL]), th,
                               prep_mode(c->P.guess), nullptr);
          break;
        case T_FOFC_FIN: launch_krp_finish_fofc(w, c->P, kb, c->dstats, s, tgrid(c, k, it[W_CELL]), th); break;
        case T_EMF: launch_emf(w, s, tgrid(c, k, it[W_EDGE]), th); break;
        default: launch_update_cells(w, c->P, 0.0, 1.0, 0.0, 0, s, tgrid(c, k, it[W_CELL]), th); break;
      }
    };
    mhd_ctx::Cfg best = c->cfg[k];
    float best_ms = 1e30f;
    for (int th = 64; th <= 256; th *= 2)
      for (int wv = 1; wv <= 4; wv *= 2) {
        c->cfg[k].threads = th;
        c->cfg[k].waves = wv;
        launch();
        cudaEventRecord(e0, s);
        for (int rep = 0; rep < 3; rep++) launch();
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); return MHD_ECUDA; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) { best_ms = ms; best = c->cfg[k]; }
      }
    c->cfg[k] = best;
    if (k == T_C2P_PREP || k == T_FOFC_PREP) {
      launch();
      c2p_seed(c, kb, fofc_k ? it[W_CELL] : it[W_C2P], s);
      launch_krp_solve(c->P, kb, s, c->solve_grid(fofc_k ? it[W_CELL] : it[W_C2P]));
    }
    if (cfg_out) {
      cfg_out[2 * k] = best.threads;
      cfg_out[2 * k + 1] = best.waves;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->prof = prof;
  c->rhs_list = -1;
  destroy_graph(c);
  return cuda_ok(cudaStreamSynchronize(s));
}

int mhd_set_launch(mhd_ctx* c, int kind, int threads, int waves) {
  if (!c || kind < 0 || kind >= T_N || (threads != 64 && threads != 128 && threads != 256) || waves < 1 || waves > 64)
    return MHD_EINVAL;
  c->cfg[kind].threads = threads;
  c->cfg[kind].waves = waves;
  destroy_graph(c);
  return MHD_OK;
}

int mhd_get_launch(const mhd_ctx* c, int kind, int* threads, int* waves) {
  if (!c || kind < 0 || kind >= T_N || !threads || !waves) return MHD_EINVAL;
  *threads = c->cfg[kind].threads;
  *waves = c->cfg[kind].waves;
  return MHD_OK;
}

int mhd_profile(mhd_ctx* c, int enable) {
  if (!c) return MHD_EINVAL;
  c->prof = enable != 0;
  return MHD_OK;
}

int mhd_profile_read(mhd_ctx* c, double* ms, long long* count) {
  if (!c || !ms || !count) return MHD_EINVAL;
  for (auto& r : c->recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) return MHD_ECUDA;
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return MHD_ECUDA;
    c->prof_ms[r.kind] += t;
    c->prof_n[r.kind] += 1;
    c->ev_pool.push_back(r.a);
    c->ev_pool.push_back(r.b);
  }
  c->recs.clear();
  for (int k = 0; k < MHD_NKERNEL; k++) {
    ms[k] = c->prof_ms[k];
    count[k] = c->prof_n[k];
    c->prof_ms[k] = 0.0;
    c->prof_n[k] = 0;
  }
  return MHD_OK;
}

const char* mhd_kernel_name(int kind) {
  static const char* names[MHD_NKERNEL] = {"c2p", "flux_x", "flux_y", "flux_z", "fofc_flag", "fofc_fix", "emf",
                                           "update", "faceb", "c2p_solve", "mlp", "ledger", "metric"};
  return (kind >= 0 && kind < MHD_NKERNEL) ? names[kind] : "unknown";
}

}  // extern "C"
