// Allocation-free variant of one RK stage for a single meshblock.
//
// Some callers cannot let a library allocate device memory: a host code that
// has handed its whole GPU memory budget to its own pool allocator, or one
// that cannot afford the device-wide synchronisation a cudaFree implies in the
// middle of a time step, or one that has nowhere to keep a library context.
// mhd_stage_noalloc serves them: it gives the results of mhd_c2p + mhd_rhs +
// mhd_rk_update (the same fluxes, CT and update kernels; its con2prim and
// FOFC estimate are the one-thread-per-cell kernels k_c2p_block and
// k_fofc_flag, which need no solve scratch, in place of the three-phase
// ones), and its scratch (fluxes, EMFs, cell-centred E, FOFC flags, the block
// descriptor and the work table) lives in the file-scope array below, so no
// call allocates or frees anything.
//
// The array is MHD_NOALLOC_SCRATCH_BYTES (16 MiB) per device and stays
// resident on every GPU that loads the library until the process exits.
// Every call shares it and it keeps the last call's contents; calls whose
// kernels overlap on the GPU (different streams, or the same stream from
// several host threads without ordering) race on it.
#include <cstring>
#include <mutex>

#include "grmhd.h"
#include "internal.h"

using namespace grmhd;

namespace {

constexpr size_t kBytes = MHD_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_scratch[kBytes];

constexpr int kMaxDev = 64;
std::mutex g_mu;
unsigned char* g_base[kMaxDev] = {nullptr};  // device address of g_scratch per device
int g_nsm[kMaxDev] = {0};

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Header of the array: descriptor, work prefix table, counters.
constexpr size_t kOffBlk = 0;
constexpr size_t kOffPre = 512;
constexpr size_t kOffStats = 1024;
constexpr size_t kOffData = 2048;

// Writes the descriptor and the work table into the static array and clears
// the counters (the only scratch that must start at zero).
struct PreTable {
  long long v[W_NKIND * 2];
};
__global__ void k_noalloc_setup(DevBlock b, PreTable t, DevBlock* dblk, long long* dpre, unsigned long long* st) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *dblk = b;
    for (int k = 0; k < W_NKIND * 2; k++) dpre[k] = t.v[k];
    for (int k = 0; k < MHD_NSTATS; k++) st[k] = 0ull;
  }
}

int to_par(const mhd_params* p, Par& P) { return fill_par(p, P, false); }

// Per-device set-up on the first call with that device current: look up the
// device address of the static array (host code cannot use its name as one).
int device_base(unsigned char** base, int* nsm) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return MHD_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_base[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
    if (e != cudaSuccess || !ptr) return MHD_ECUDA;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return MHD_ECUDA;
    g_base[dev] = (unsigned char*)ptr;
    g_nsm[dev] = n;
  }
  *base = g_base[dev];
  *nsm = g_nsm[dev];
  return MHD_OK;
}

}  // namespace

extern "C" int mhd_stage_noalloc(const mhd_params* p, const mhd_block* blk, double dt, int stage, void* stream) {
  Par P;
  int r = to_par(p, P);
  if (r) return r;
  if (!blk || !(dt > 0.0) || stage < 0 || stage >= P.rk_order) return MHD_EINVAL;
  const mhd_block& s = *blk;
  if (s.n[0] < 1 || s.n[1] < 1 || s.n[2] < 1 || s.ng < 4 || !s.cons || !s.cons0 || !s.prim || !s.bcc || !s.adm ||
      !s.flags)
    return MHD_EINVAL;
  for (int d = 0; d < 3; d++)
    if (!s.bf[d] || !s.bf0[d] || !(s.dx[d] > 0.0)) return MHD_EINVAL;
  // scratch this block needs, laid out after the header
  const long long N0 = s.n[0] + 2 * s.ng, N1 = s.n[1] + 2 * s.ng, N2 = s.n[2] + 2 * s.ng;
  const long long ncell = N0 * N1 * N2;
  const long long nf[3] = {N2 * N1 * (N0 + 1), N2 * (N1 + 1) * N0, (N2 + 1) * N1 * N0};
  const long long ne[3] = {(N2 + 1) * (N1 + 1) * N0, (N2 + 1) * N1 * (N0 + 1), N2 * (N1 + 1) * (N0 + 1)};
  const size_t b_flux = al256(sizeof(double) * 7 * (nf[0] + nf[1] + nf[2]));
  const size_t b_emf = al256(sizeof(double) * (ne[0] + ne[1] + ne[2]));
  const size_t b_ecc = al256(sizeof(double) * 3 * ncell);
  const size_t b_flag = al256((size_t)ncell);
  if (kOffData + b_flux + b_emf + b_ecc + b_flag > kBytes) return MHD_ETOOBIG;

  unsigned char* base = nullptr;
  int nsm = 1;
  r = device_base(&base, &nsm);
  if (r) return r;

  DevBlock b;
  std::memset(&b, 0, sizeof(b));
  for (int d = 0; d < 3; d++) {
    b.n[d] = s.n[d];
    b.dx[d] = s.dx[d];
    b.idx[d] = 1.0 / s.dx[d];
    b.bf[d] = s.bf[d];
    b.bf0[d] = s.bf0[d];
  }
  b.N[0] = (int)N0; b.N[1] = (int)N1; b.N[2] = (int)N2;
  b.ng = s.ng;
  int seg[3];
  for (int d = 0; d < 3; d++) {
    seg[d] = flux_seg_len((const int (*)[3])s.n, 1, d, nsm);
    b.nseg[d] = flux_nseg(s.n[d], seg[d]);
  }
  b.ncell = ncell;
  b.cons = s.cons; b.cons0 = s.cons0; b.prim = s.prim; b.bcc = s.bcc; b.adm = s.adm; b.flags = s.flags;
  unsigned char* q = base + kOffData;
  double* f = (double*)q;
  b.flux[0] = f;
  b.flux[1] = f + 7 * nf[0];
  b.flux[2] = f + 7 * (nf[0] + nf[1]);
  q += b_flux;
  double* e = (double*)q;
  b.emf[0] = e;
  b.emf[1] = e + ne[0];
  b.emf[2] = e + ne[0] + ne[1];
  q += b_emf;
  b.ecc = (double*)q;
  q += b_ecc;
  b.fflag = q;

  const long long n0 = s.n[0], n1 = s.n[1], n2 = s.n[2];
  long long items[W_NKIND];
  items[W_C2P] = (n0 + 6) * (n1 + 6) * (n2 + 6);
  items[W_FX] = (n0 + 1) * (n1 + 2) * (n2 + 2);
  items[W_FY] = (n0 + 2) * (n1 + 1) * (n2 + 2);
  items[W_FZ] = (n0 + 2) * (n1 + 2) * (n2 + 1);
  items[W_CELL] = n0 * n1 * n2;
  items[W_EDGE] = (n0 + 1) * (n1 + 1) * (n2 + 1);
  items[W_FACE] = (n0 + 1) * n1 * n2 + n0 * (n1 + 1) * n2 + n0 * n1 * (n2 + 1);
  items[W_INIT] = ncell;
  for (int d = 0; d < 3; d++) items[W_SX + d] = flux_seg_items(s.n, d, seg[d]);
  for (int d = 0; d < 3; d++) items[W_GFX + d] = nf[d];
  PreTable t;
  for (int k = 0; k < W_NKIND; k++) {
    t.v[2 * k] = 0;
    t.v[2 * k + 1] = items[k];
  }
  DevBlock* dblk = (DevBlock*)(base + kOffBlk);
  long long* dpre = (long long*)(base + kOffPre);
  unsigned long long* dstats = (unsigned long long*)(base + kOffStats);
  static_assert(sizeof(DevBlock) <= kOffPre - kOffBlk, "descriptor slot");
  static_assert(sizeof(PreTable) <= kOffStats - kOffPre, "work table slot");

  // A launch error left pending by the caller's earlier work is reported
  // (and left pending) before anything is launched, so that every error seen
  // after a launch below belongs to this call.
  if (cudaPeekAtLastError() != cudaSuccess) return MHD_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  auto launched = [] { return cudaPeekAtLastError() == cudaSuccess; };
  k_noalloc_setup<<<1, 32, 0, st>>>(b, t, dblk, dpre, dstats);
  if (!launched()) return MHD_ECUDA;
  Work w;
  w.blk = dblk;
  w.pre = dpre;
  w.nblocks = 1;
  auto grid = [&](int kind, int threads) {
    long long g = (items[kind] + threads - 1) / threads;
    long long cap = (long long)nsm * 2;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
  };
  double g0, g1, be;
  rk_weights(P.rk_order, stage, g0, g1, be);
  launch_c2p_block(w, P, dstats, st, grid(W_C2P, 128));
  if (!launched()) return MHD_ECUDA;
  for (int d = 0; d < 3; d++) {
    launch_flux_dir_inline(d, w, P, st, grid(W_SX + d, 128));
    if (!launched()) return MHD_ECUDA;
  }
  if (P.fofc) {
    launch_fofc_flag(w, P, g0, g1, be * dt, dstats, st, grid(W_CELL, 128));
    if (!launched()) return MHD_ECUDA;
    for (int d = 0; d < 3; d++) {
      launch_fofc_fix(d, w, P, dstats, st, grid(W_FX + d, 128));
      if (!launched()) return MHD_ECUDA;
    }
  }
  launch_emf(w, st, grid(W_EDGE, 128));
  if (!launched()) return MHD_ECUDA;
  launch_update_cells(w, P, g0, g1, be * dt, stage == 0 ? 1 : 0, st, grid(W_CELL, 128));
  if (!launched()) return MHD_ECUDA;
  launch_update_faces(w, g0, g1, be * dt, stage == 0 ? 1 : 0, st, grid(W_FACE, 256));
  return launched() ? MHD_OK : MHD_ECUDA;
}
