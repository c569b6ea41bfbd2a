// Device-side data structures and physics functions of libgrmhd (sm_103a).
//
// GB300 has a narrow FP64 pipe (about 2 DFMA per clock per SM; a double
// divide costs ~6 DFMA slots, a square root ~10) next to a wide FP32/INT
// pipe, so the per-cell arithmetic below is arranged to issue as few FP64
// divides and square roots as possible: reciprocals are shared, 1/W comes from
// rsqrt, and the con2prim master function of Kastaun et al. (2021) is written
// with a single division.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ival.cuh"

namespace grmhd {

enum : unsigned {
  F_FAIL = 1u, F_DFLOOR = 2u, F_SIGMA = 4u, F_TAU = 8u, F_RHO = 16u, F_TEMP = 32u, F_VMAX = 64u, F_FOFC = 128u
};
constexpr unsigned FLOOR_BITS = F_DFLOOR | F_SIGMA | F_TAU | F_RHO | F_TEMP | F_VMAX;

// Parameters with derived constants, passed by value to every kernel.
struct Par {
  double gam, gm1, gfac;        // Gamma, Gamma-1, Gamma/(Gamma-1) (ideal gas)
  double rho_atm, T_atm, rho_thr;
  double eps_atm;               // T_atm/(G_th - 1): eps of the T floor without the cold part
  double eps_atm_rho;           // the atmosphere's eps (hybrid: eps_c(rho_atm) + eps_atm)
  double P_atm;                 // the atmosphere's pressure (hybrid: P_c(rho_atm) + rho_atm T_atm)
  double sigma_max, dmp_M, tol, vmax2;
  double alpha_exc;             // excision lapse (<= 0: off)
  // hybrid EOS (eos = 1): pieces npc, dividing densities, K_i, G_i, eps_c
  // constants a_i, thermal index, and the cold triple at rho_atm
  double rpc[3], Kpc[4], Gpc[4], apc[4];
  double Gth, gth1;             // G_th and G_th - 1 (ideal gas: Gamma, Gamma - 1)
  double Pc_atm, epsc_atm, G_atm;
  int recon, rsolver, fofc, rk_order, maxit, guess, eos, npc;
  int exc_on, sigma_on;         // alpha_exc > 0, sigma_max > 0
  int thr_pos;                  // rho_thr > 0
  int dec32;                    // the FOFC flags may come from FP32 enclosures
                                // (fofc_decide_iv): ideal gas, eps_atm and rho_thr
                                // (when > 0) within [1e-30, 1e30]
};

// One meshblock as seen by the kernels: caller arrays plus context scratch.
struct DevBlock {
  int n[3], ng, N[3];
  int nseg[3];       // flux-sweep segments per transverse line of direction d
  long long ncell;
  double dx[3], idx[3];
  double *cons, *cons0, *prim, *bcc;
  double *bf[3], *bf0[3];
  const double* adm;
  unsigned char* flags;
  double* flux[3];   // [7][face array of direction d]
  double* emf[3];    // edge arrays E_x, E_y, E_z
  double* ecc;       // [3][ncell] cell-centred E = -alpha (vhat x B~)
  unsigned char* fflag;  // [ncell] FOFC flag of the current stage
  // baryon-mass ledger (null when off): interior D~ dV added by the floors
  // of the last con2prim (lf) and the running RK-weighted balance (la)
  double *lf, *la;
  double dV;         // cell volume dx dy dz
  int id;            // index of the block in its list
  double* mu;        // [ncell] con2prim root of the last stage-input con2prim
                     // (c2p_guess 3; 0: none), else null
  double* mc;        // [8][ncell] metric of the con2prim region: sqrt(gamma),
                     // 1/sqrt(gamma), gamma^ij; written by k_metric_cache,
                     // read by con2prim, the FOFC estimate and the update
                     // (null: each computes its own)
  double* dmc;       // [DMC_N][n0 n1 n2] centred derivatives of the ADM
                     // variables at the interior cells (Eq. 9 sources),
                     // written by k_metric_cache (null: the update takes them)
  double* fmc[3];    // face metric of the faces the sweeps of direction d
                     // visit ([FMC_N][fmc_count], fmc_index order); written
                     // by k_metric_cache, read by k_flux (null: computed in
                     // the sweep)
};
// Derivative cache: per axis a, the centred differences (q[+1] - q[-1]) / (2
// dx_a) of alpha, beta^1..3 and gamma_ij at slots a * 10 + (0 .. 9).
constexpr int DMC_N = 30;
// Face metric cache: alpha, beta^1..3, gamma_ij (6), sqrt(gamma),
// 1/sqrt(gamma) and gamma^{dd} of a face of direction d.
constexpr int FMC_N = 13;
// Face index (k,j,i) of item `loc` of direction d: along d the interior faces,
// transversally one extra layer each side (the CT stencil needs them).
template <int d>
__host__ __device__ __forceinline__ void face_coords(const DevBlock& b, long long loc, int& k, int& j, int& i) {
  const int L0 = b.n[0] + (d == 0 ? 1 : 2), L1 = b.n[1] + (d == 1 ? 1 : 2);
  int a0 = loc % L0; long long r = loc / L0; int a1 = r % L1; int a2 = r / L1;
  i = a0 + b.ng - (d == 0 ? 0 : 1);
  j = a1 + b.ng - (d == 1 ? 0 : 1);
  k = a2 + b.ng - (d == 2 ? 0 : 1);
}
// The face metric cache of direction d (DevBlock.fmc[d], [FMC_N][fmc_count]).
// y and z: in face_coords order (x fastest), as the lanes of a y or z sweep
// take neighbouring lines.  x: the lanes of an x sweep take neighbouring
// segments of a line, so the face at position q of the segment of sweep item
// `item` (seg_coords<0>) sits at q * nitems + item: every step of the sweep
// reads consecutive slots.  Segments hold fmc_lx faces but the remainder of
// each line fewer; its unused slots stay unwritten and unread.
__host__ __device__ inline int fmc_lx(const DevBlock& b) {
  const int ns = b.nseg[0], nd = b.n[0] + 1;
  return (nd + ns - 1) / ns;
}
__host__ __device__ inline long long fmc_xitems(const DevBlock& b) {
  return (long long)b.nseg[0] * (b.n[1] + 2) * (b.n[2] + 2);
}
__host__ __device__ inline long long fmc_count(const DevBlock& b, int d) {
  if (d == 0) return fmc_lx(b) * fmc_xitems(b);
  return (long long)(b.n[0] + 2) * (b.n[1] + (d == 1 ? 1 : 2)) * (b.n[2] + (d == 2 ? 1 : 2));
}
// index step between consecutive faces of a sweep of direction d
__host__ __device__ inline long long fmc_step(const DevBlock& b, int d) {
  return d == 0 ? fmc_xitems(b) : (d == 1 ? (long long)(b.n[0] + 2) : (long long)(b.n[0] + 2) * (b.n[1] + 2));
}
// index of face (k,j,i) of direction d in its cache
__host__ __device__ inline long long fmc_index(const DevBlock& b, int d, int k, int j, int i) {
  if (d == 0) {
    const int f = i - b.ng, lx = fmc_lx(b), full = b.nseg[0] - 1;
    const long long lines = (long long)(b.n[1] + 2) * (b.n[2] + 2);
    const long long r = (long long)(k - b.ng + 1) * (b.n[1] + 2) + (j - b.ng + 1);
    const int s = f / lx;   // <= full: the remainder holds fewer than lx faces
    const long long item = s < full ? r * full + s : full * lines + r;
    return (long long)(f - s * lx) * fmc_xitems(b) + item;
  }
  const int L0 = b.n[0] + 2, L1 = b.n[1] + (d == 1 ? 1 : 2);
  const int a0 = i - b.ng + 1, a1 = j - b.ng + (d == 1 ? 0 : 1), a2 = k - b.ng + (d == 2 ? 0 : 1);
  return ((long long)a2 * L1 + a1) * L0 + a0;
}
// Relative half-width of the bracket around a previous root (c2p_guess 3).
constexpr double WARM_DELTA = 1e-3;

// Work lists: item ranges of every block for one kernel kind.
enum WorkKind { W_C2P = 0, W_FX, W_FY, W_FZ, W_CELL, W_EDGE, W_FACE, W_INIT, W_SX, W_SY, W_SZ, W_GFX, W_GFY, W_GFZ,
                W_NKIND };

// Flux sweeps: the n_d + 1 faces of direction d on one transverse line (one
// extra line on each side, for the CT stencil) are split into ns = ceil((n_d +
// 1)/L) segments of at most L faces (near-equal along y and z; along x equal
// plus one remainder, see seg_coords); one thread sweeps one segment.  L is FLUX_SEG
// (FLUX_SEG_X along x) unless the block list is too small to give every SM
// two waves of sweeps at that length; then it halves (down to 1) until it
// does (flux_seg_len).  The x sweep's lanes read neighbouring segments of one
// line.  Each segment reconstructs one cell more than it has faces; on the
// 128^3 star x segments of 16 faces ran the x sweep 2.5% faster than 8 or
// 12, and y / z segments of 24 ran 2.6% slower than 16 (fewer waves, a
// longer idle tail).
constexpr int FLUX_SEG = 16;
constexpr int FLUX_SEG_X = 16;
// segments per line for an interior of n cells (n + 1 faces)
__host__ __device__ inline int flux_nseg(int n, int L) { return (n + L) / L; }
__host__ __device__ inline long long flux_seg_items(const int* n, int d, int L) {
  long long t = 1;
  for (int a = 0; a < 3; a++) t *= a == d ? (long long)flux_nseg(n[a], L) : (long long)(n[a] + 2);
  return t;
}
// Segment length of direction d for a list of nb blocks with interiors n[b][3]
// on a GPU of nsm SMs: the largest L <= FLUX_SEG (FLUX_SEG_X for d = 0)
// reached by halving, with at least 2 nsm 256 segments, else 1.
inline int flux_seg_len(const int (*n)[3], int nb, int d, int nsm) {
  const long long target = 2LL * nsm * 256;
  int L = d == 0 ? FLUX_SEG_X : FLUX_SEG;
  while (L > 1) {
    long long segs = 0;
    for (int b = 0; b < nb; b++) segs += flux_seg_items(n[b], d, L);
    if (segs >= target) break;
    L /= 2;
  }
  return L;
}

// Segment of the transverse line of item `loc`: (k,j,i) is the cell on the
// upper side of the segment's first face, nf its number of faces.
// y and z: the lanes of a warp take neighbouring lines (x fastest) at the same
// segment index, so they sweep equal lengths; the segments are near-equal.
// x: the lanes take neighbouring segments of a line, so every line gets ns - 1
// segments of Lx = ceil(nd / ns) faces (items [0, (ns - 1) lines)) and one
// remainder of nd - (ns - 1) Lx >= 1 faces (the items after them); a warp
// then never mixes lengths, except where the two ranges meet.
template <int d>
__host__ __device__ __forceinline__ void seg_coords(const DevBlock& b, int loc, int& k, int& j, int& i, int& nf) {
  const int ns = b.nseg[d], nd = b.n[d] + 1;
  int a0, a1, f0;
  if (d == 0) {
    const int lines = (b.n[1] + 2) * (b.n[2] + 2), full = ns - 1, Lx = (nd + ns - 1) / ns;
    int r;
    if (loc < full * lines) {
      const int s = loc % full;
      r = loc / full; f0 = s * Lx; nf = Lx;
    } else {
      r = loc - full * lines; f0 = full * Lx; nf = nd - f0;
    }
    a0 = r % (b.n[1] + 2); a1 = r / (b.n[1] + 2);
  } else {
    int s;
    a0 = loc % (b.n[0] + 2); int r = loc / (b.n[0] + 2);
    if (d == 1) { a1 = r % (b.n[2] + 2); s = r / (b.n[2] + 2); }
    else { a1 = r % (b.n[1] + 2); s = r / (b.n[1] + 2); }
    f0 = (int)((long long)s * nd / ns);
    nf = (int)((long long)(s + 1) * nd / ns) - f0;
  }
  const int g = b.ng;
  if (d == 0) { i = g + f0; j = g - 1 + a0; k = g - 1 + a1; }
  else if (d == 1) { j = g + f0; i = g - 1 + a0; k = g - 1 + a1; }
  else { k = g + f0; i = g - 1 + a0; j = g - 1 + a1; }
}

// Slots of the per-cell con2prim scratch (SoA, [KW_N][n]).
enum {
  KW_QH = 0, KW_R2, KW_B2, KW_RB2, KW_RP2, KW_D, KW_RB, KW_RU0, KW_RU1, KW_RU2, KW_BU0, KW_BU1, KW_BU2,
  KW_A, KW_B, KW_GA, KW_GB, KW_MU, KW_SDET, KW_ISDET, KW_USD, KW_UST, KW_N
};
// solve status: 0 solve needed, 1 root known, 2 no bracket / bad input,
// 3 iteration cap, 4 bracket to be built from the learned guess, 5 FOFC
// estimate flagged without a recovery (a floor on U* before the solve, or the
// FP32 decision, fofc_decide_iv), 7 FOFC estimate not flagged by the FP32
// decision (no solve, no recovery)

// Learned-guess network 5 -> 64 -> 64 -> 1: fp32 parameter offsets, bf16
// operand copies (W1 padded to [64][16], W2 [64][64], w3 padded to [8][64]).
constexpr int MLP_NIN = 5, MLP_NH = 64, MLP_FSTRIDE = 8;
constexpr int MLP_W1 = 0, MLP_B1 = MLP_W1 + MLP_NH * MLP_NIN, MLP_W2 = MLP_B1 + MLP_NH,
              MLP_B2 = MLP_W2 + MLP_NH * MLP_NH, MLP_W3 = MLP_B2 + MLP_NH, MLP_B3 = MLP_W3 + MLP_NH,
              MLP_NPARAM = MLP_B3 + 1;
constexpr int MLP_BF_W1 = 0, MLP_BF_W2 = MLP_NH * 16, MLP_BF_W3 = MLP_BF_W2 + MLP_NH * MLP_NH,
              MLP_NBF = MLP_BF_W3 + 8 * MLP_NH;
struct MlpNorm {
  float fmean[MLP_NIN], finv[MLP_NIN];  // feature mean and 1/std
  float ymean, ystd;                    // target (log mu) mean and std
};

// Per-cell scratch of the three-phase con2prim (k_krp.cu).
struct KrpBuf {
  double* w;                 // [KW_N][n] KRP variables, bracket, root
  int* it;                   // [n] iterations
  unsigned char* st;         // [n] solve status
  unsigned char* fl;         // [n] flags of the prep phase
  unsigned long long* ctr;   // [0] work-queue head of the root solve; [1] nonzero
                             // when a cell may have status 0 (set by the kernels
                             // that give status 0, cleared by the finish after the
                             // solve: the solve returns at once on 0)
  long long n;
  unsigned long long* flist = nullptr;   // FOFC estimate: [0] count, then the W_CELL
                                         // items of the flagged cells (null: none kept)
  long long fcap = 0;                    // entries flist can hold
};

struct Work {
  const DevBlock* blk;          // device array [nblocks]
  const long long* pre;         // device [W_NKIND][nblocks+1] item prefix sums
  int nblocks;
};

// ---------------------------------------------------------------- indexing
__host__ __device__ __forceinline__ long long cidx(const DevBlock& b, int k, int j, int i) {
  return ((long long)k * b.N[1] + j) * b.N[0] + i;
}
__host__ __device__ __forceinline__ long long fidx(const DevBlock& b, int d, int k, int j, int i) {
  if (d == 0) return ((long long)k * b.N[1] + j) * (b.N[0] + 1) + i;
  if (d == 1) return ((long long)k * (b.N[1] + 1) + j) * b.N[0] + i;
  return ((long long)k * b.N[1] + j) * b.N[0] + i;
}
__host__ __device__ __forceinline__ long long nface(const DevBlock& b, int d) {
  if (d == 0) return (long long)b.N[2] * b.N[1] * (b.N[0] + 1);
  if (d == 1) return (long long)b.N[2] * (b.N[1] + 1) * b.N[0];
  return (long long)(b.N[2] + 1) * b.N[1] * b.N[0];
}
__device__ __forceinline__ long long eidx(const DevBlock& b, int c, int k, int j, int i) {
  if (c == 0) return ((long long)k * (b.N[1] + 1) + j) * b.N[0] + i;
  if (c == 1) return ((long long)k * b.N[1] + j) * (b.N[0] + 1) + i;
  return ((long long)k * (b.N[1] + 1) + j) * (b.N[0] + 1) + i;
}

// block owning global item `it` of kind K (binary search of the prefix sums)
__host__ __device__ __forceinline__ int find_block(const Work& w, int K, long long it) {
  const long long* p = w.pre + (long long)K * (w.nblocks + 1);
  int lo = 0, hi = w.nblocks;  // p[lo] <= it < p[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (p[mid] <= it) lo = mid; else hi = mid;
  }
  return lo;
}

// ------------------------------------------------------------- metric (Eq. 5)
// Compares on the integer pipe.  An FP64 compare takes a slot of the narrow
// FP64 pipe; from the bit patterns the answers are the same:
//  lt0 / gt0 / eq0: x < 0, x > 0, x == 0 with IEEE semantics (false on NaN,
//    +0 and -0 equal to 0);
//  gt_nn(x, y): x > y for operands that are not NaN, at least one of them
//    >= +0, and not the pair (+0, -0) - the signed order of the bit patterns.
// They are host functions too, so that tests/index_check.cu can compare them
// with the IEEE comparisons on the CPU; only the bit reinterpretation differs.
__host__ __device__ __forceinline__ long long dbits(double x) {
#ifdef __CUDA_ARCH__
  return __double_as_longlong(x);
#else
  long long u;
  __builtin_memcpy(&u, &x, sizeof u);
  return u;
#endif
}
__host__ __device__ __forceinline__ bool lt0(double x) {
  const unsigned long long u = (unsigned long long)dbits(x);
  return (u >> 63) && ((u & 0x7FFFFFFFFFFFFFFFull) - 1ull < 0x7FF0000000000000ull);
}
__host__ __device__ __forceinline__ bool gt0(double x) {
  const unsigned long long u = (unsigned long long)dbits(x);
  return !(u >> 63) && (u - 1ull < 0x7FF0000000000000ull);
}
__host__ __device__ __forceinline__ bool eq0(double x) { return (dbits(x) << 1) == 0; }
__host__ __device__ __forceinline__ bool gt_nn(double x, double y) { return dbits(x) > dbits(y); }
// x < rho_thr for a finite x: with rho_thr > 0 the bit order decides exactly
// (-0 included); with rho_thr = 0 it is the sign test
__host__ __device__ __forceinline__ bool below_thr(const Par& P, double x) {
  return P.thr_pos ? gt_nn(P.rho_thr, x) : lt0(x);
}
// CT upwinding (k_emf) by the sign of the face mass flux fD: (a - b) for
// fD > 0, (c - d) for fD < 0, their average for fD = 0 (or NaN).  The sign test
// reads the bit pattern on the integer pipe, the operands of the chosen
// difference are selected there too, and one FP64 subtraction forms it: the
// same values as comparing fD with 0 in FP64.  The average (fD = 0, rare) is a
// call of its own, so that the compiler branches to it instead of forming
// both differences in every lane.
static __host__ __device__ __noinline__ double upw_avg(double a, double b, double c, double d) {
  return 0.5 * ((a - b) + (c - d));
}
__host__ __device__ __forceinline__ double upw(double fD, double a, double b, double c, double d) {
  const unsigned long long u = (unsigned long long)dbits(fD);
  const unsigned long long mag = u & 0x7FFFFFFFFFFFFFFFull;
  if (mag - 1ull < 0x7FF0000000000000ull) {   // fD != 0, not NaN
    const bool neg = (u >> 63) != 0;
    return (neg ? c : a) - (neg ? d : b);
  }
  return upw_avg(a, b, c, d);
}
// min / max of two doubles that are not NaN, on the integer pipe: the key
// u ^ ((u >> 63) & 0x7FF..F) of the bit pattern u orders doubles as numbers
// (-0 below +0), and an FP64 min or max would take a slot of the FP64 pipe.
__host__ __device__ __forceinline__ long long okey(double x) {
  const long long u = dbits(x);
  return u ^ ((u >> 63) & 0x7FFFFFFFFFFFFFFFll);
}
__host__ __device__ __forceinline__ double imin(double a, double b) { return okey(b) < okey(a) ? b : a; }
__host__ __device__ __forceinline__ double imax(double a, double b) { return okey(b) > okey(a) ? b : a; }
// finite (not inf, not NaN): the exponent field is not all ones
__host__ __device__ __forceinline__ bool finite_bits(double x) {
#ifdef __CUDA_ARCH__
  return (__double2hiint(x) & 0x7FF00000) != 0x7FF00000;
#else
  return ((int)(dbits(x) >> 32) & 0x7FF00000) != 0x7FF00000;
#endif
}

// Reciprocal for the hot divisions: the hardware's approximate FP64
// reciprocal (rcp.approx.ftz.f64) refined by two Newton-Raphson steps for
// 1/x (r <- r + r (1 - x r); each step squares the relative error), then
// a / x = a * r.  Within ~1 ulp of the correctly rounded quotient, where a
// correctly rounded division costs about twice the FP64 issue slots.  For
// normal x only (the approximation flushes subnormals): callers use it on
// denominators bounded away from zero.
__device__ __forceinline__ double rcp_nr(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

struct Metric {
  double g[6], gi[6], sdet, isdet;
};
__device__ __forceinline__ void metric_setup(Metric& m) {
  const double* g = m.g;
  double c0 = g[3] * g[5] - g[4] * g[4];
  double c1 = g[2] * g[4] - g[1] * g[5];
  double c2 = g[1] * g[4] - g[2] * g[3];
  double det = g[0] * c0 + g[1] * c1 + g[2] * c2;
  double isd = rsqrt(det);
  double idet = isd * isd;
  m.isdet = isd;
  m.sdet = det * isd;
  m.gi[0] = c0 * idet;
  m.gi[1] = c1 * idet;
  m.gi[2] = c2 * idet;
  m.gi[3] = (g[0] * g[5] - g[2] * g[2]) * idet;
  m.gi[4] = (g[1] * g[2] - g[0] * g[4]) * idet;
  m.gi[5] = (g[0] * g[3] - g[1] * g[1]) * idet;
}
// The stage's metric cache (DevBlock.mc) at cell c: store after metric_setup,
// or load g from the ADM array and the rest from the cache.
__device__ __forceinline__ void metric_store(double* mc, long long nc, long long c, const Metric& m) {
  mc[c] = m.sdet;
  mc[nc + c] = m.isdet;
#pragma unroll
  for (int v = 0; v < 6; v++) mc[(2 + v) * nc + c] = m.gi[v];
}
__device__ __forceinline__ void metric_cell(const double* adm, const double* mc, long long nc, long long c,
                                            Metric& m) {
#pragma unroll
  for (int v = 0; v < 6; v++) m.g[v] = adm[(4 + v) * nc + c];
  if (mc) {
    m.sdet = mc[c];
    m.isdet = mc[nc + c];
#pragma unroll
    for (int v = 0; v < 6; v++) m.gi[v] = mc[(2 + v) * nc + c];
  } else {
    metric_setup(m);
  }
}
__device__ __forceinline__ void lower3(const double* g, const double* u, double* l) {
  l[0] = g[0] * u[0] + g[1] * u[1] + g[2] * u[2];
  l[1] = g[1] * u[0] + g[3] * u[1] + g[4] * u[2];
  l[2] = g[2] * u[0] + g[4] * u[1] + g[5] * u[2];
}
__device__ __forceinline__ double dot3(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// ------------------------------------------------------- EOS (Sec. 3.4)
// Hybrid EOS: cold part at rho, P_c = K_i rho^G_i and eps_c = a_i +
// K_i rho^(G_i-1)/(G_i-1) on the piece that holds rho (one pow).  The piece
// constants come from the parameters (host side, by continuity).
__device__ __forceinline__ void eos_cold(const Par& P, double rho, double& Pc, double& epsc, double& Gi) {
  int i = 0;
#pragma unroll
  for (int j = 0; j < 3; j++) i += (j < P.npc - 1 && rho >= P.rpc[j]) ? 1 : 0;
  const double K = i == 0 ? P.Kpc[0] : (i == 1 ? P.Kpc[1] : (i == 2 ? P.Kpc[2] : P.Kpc[3]));
  const double a = i == 0 ? P.apc[0] : (i == 1 ? P.apc[1] : (i == 2 ? P.apc[2] : P.apc[3]));
  Gi = i == 0 ? P.Gpc[0] : (i == 1 ? P.Gpc[1] : (i == 2 ? P.Gpc[2] : P.Gpc[3]));
  const double x = K * pow(rho, Gi - 1.0);   // K rho^(G_i - 1)
  Pc = x * rho;
  epsc = a + x / (Gi - 1.0);
}
// rho h = rho + rho eps + P and rho h c_s^2 = G_i P_c + G_th P_th of the hybrid
// EOS from rho, P and the cold triple at rho
__device__ __forceinline__ void eos_hyb_rhoh_chi(const Par& P, double rho, double p, double Pc, double epsc, double Gi,
                                                 double& rhoh, double& chi) {
  const double Pth = p - Pc;
  rhoh = rho + fma(rho, epsc, Pth / P.gth1) + p;
  chi = fma(Gi, Pc, P.Gth * Pth);
}
// rho h at (rho, P), either EOS
__device__ __forceinline__ double eos_rhoh(const Par& P, double rho, double p) {
  if (P.eos == 0) return fma(P.gfac, p, rho);
  double Pc, epsc, Gi, rhoh, chi;
  eos_cold(P, rho, Pc, epsc, Gi);
  eos_hyb_rhoh_chi(P, rho, p, Pc, epsc, Gi, rhoh, chi);
  return rhoh;
}

// ----------------------------------------------------- prim -> cons (Eq. 6)
// prim = rho, w^i = W v^i, P;  Bd = densitised B~;  out = D~, S~_i, tau~.
__device__ __forceinline__ void prim2cons(const Par& P, const double* prim, const double* Bd, const Metric& m,
                                          double* out) {
  double B[3] = {Bd[0] * m.isdet, Bd[1] * m.isdet, Bd[2] * m.isdet};
  double w[3] = {prim[1], prim[2], prim[3]};
  double wl[3], Bl[3];
  lower3(m.g, w, wl);
  lower3(m.g, B, Bl);
  double W2 = 1.0 + dot3(w, wl);
  double iW = rsqrt(W2);
  double W = W2 * iW;
  double vl[3] = {wl[0] * iW, wl[1] * iW, wl[2] * iW};
  double B2 = dot3(B, Bl);
  double Bv = dot3(B, vl);
  double rho = prim[0], p = prim[4];
  double rhoh = P.eos == 0 ? rho + P.gfac * p : eos_rhoh(P, rho, p);
  double e = rhoh * W2;
  double D = rho * W;
  double eB = e + B2;
  out[0] = m.sdet * D;
  out[1] = m.sdet * (eB * vl[0] - Bv * Bl[0]);
  out[2] = m.sdet * (eB * vl[1] - Bv * Bl[1]);
  out[3] = m.sdet * (eB * vl[2] - Bv * Bl[2]);
  out[4] = m.sdet * ((e - D) + B2 - p - 0.5 * (Bv * Bv + B2 * iW * iW));
}

// --------------------------------------------------------- con2prim (Sec. 3.4)
// Kastaun, Kalinani & Ciolfi (2021) variables per unit D.
struct KS {
  double qh;      // q - b^2/2
  double r2, b2, rb2, rperp2, gam, eps_min, vmax2;
  double D;       // undensitised D (the hybrid EOS needs rho = D/W)
};
struct KEval {
  double x, rbar2, W, eps, eps_raw, G;
  double eps_min, rho, P, Pc;   // hybrid EOS: eps floor at rho, rho = D/W, P, cold P_c
  bool vcap;
};
// The KRP master function f(mu) = mu - 1/(nu + mu rbar^2) with
// nu = (1 + Gamma eps)/W, i.e. f = mu - W/(1 + Gamma eps + mu rbar^2 W).  For
// an ideal gas with only the lower eps clamp, nu_A = (1+a)(1+eps)/W >= nu_B =
// (1+a)(1 + qbar - mu rbar^2), so nu = max(nu_A, nu_B) = nu_A.  (Stored in the
// field G.)  f is nearly linear near the root (mu -> mu-hat contracts), which
// keeps regula falsi fast; a division-free multiple of it is not.
__device__ __forceinline__ void kev(const KS& s, double mu, KEval& e) {
  // x = 1/d, rbar^2 and W from one rsqrt (the d, N, E, y of kev_g below)
  const double d = fma(mu, s.b2, 1.0);
  const double N = fma(mu * (d + 1.0), s.rb2, s.r2);
  const double mu2 = mu * mu, d2 = d * d;
  double W, x, id2, vh2;
  e.vcap = gt_nn(mu2 * N, s.vmax2 * d2);
  if (e.vcap) {
    x = 1.0 / d;
    id2 = x * x;
    vh2 = s.vmax2;
    W = rsqrt(1.0 - s.vmax2);
  } else if (eq0(N)) {   // r = 0: at rest, W = 1 exactly (x multiplies r only)
    x = id2 = vh2 = 0.0;
    W = 1.0;
  } else {
    const double E = fma(-mu2, N, d2);
    const double y = rsqrt(E * d2);
    W = d2 * y;
    id2 = (y * y) * E;
    x = d * id2;
    vh2 = (mu2 * N) * id2;
  }
  const double rbar2 = N * id2;
  const double qbar = fma(-0.5 * mu2 * s.rperp2, id2, s.qh);
  double wm1 = vh2 * W * W * rcp_nr(1.0 + W);  // W - 1 without cancellation (1 + W >= 2)
  e.eps_raw = fma(W, qbar - mu * rbar2, wm1);
  e.eps = gt_nn(s.eps_min, e.eps_raw) ? s.eps_min : e.eps_raw;
  e.x = x;
  e.rbar2 = rbar2;
  e.W = W;
  e.G = mu - W * rcp_nr(fma(mu * rbar2, W, fma(s.gam, e.eps, 1.0)));   // denominator >= 1
}
// f(mu) alone, with one division where kev takes two; for the bracket and
// the root iteration (the recovery at the root uses kev).  With
// d = 1 + mu b^2, N = r^2 + mu (d + 1) (r.b)^2 and E = d^2 - mu^2 N,
//   rbar^2 = N / d^2,  1 - v^2 = E / d^2,
// so y = 1/sqrt(E d^2) gives W = d^2 y and 1/d^2 = y^2 E.  Multiplying by
// 1 + W clears the other two denominators:
//   (1 + W) eps_raw = (1 + W) W (qbar - mu rbar^2) + v^2 W^2,
//   f = mu - W (1 + W) / [(1 + W)(1 + mu rbar^2 W) + Gamma (1 + W) eps].
// Under the velocity cap (mu^2 N > vmax^2 d^2) W is the capped value and
// 1/d^2 takes a division; at r = 0 (N = 0) the state is at rest and W = 1
// exactly, as 1/sqrt(1 - v^2) gives it.  The same function as kev up to
// rounding.
__device__ __forceinline__ double kev_g(const KS& s, double mu) {
  const double d = fma(mu, s.b2, 1.0);
  const double N = fma(mu * (d + 1.0), s.rb2, s.r2);
  const double mu2 = mu * mu, d2 = d * d;
  double W, id2, v2;
  if (gt_nn(mu2 * N, s.vmax2 * d2)) {
    const double x = 1.0 / d;
    id2 = x * x;
    v2 = s.vmax2;
    W = rsqrt(1.0 - s.vmax2);
  } else if (eq0(N)) {   // r = 0 (then r_perp = 0 too): at rest, W = 1 exactly
    id2 = v2 = 0.0;
    W = 1.0;
  } else {
    const double E = fma(-mu2, N, d2);
    const double y = rsqrt(E * d2);
    W = d2 * y;
    id2 = (y * y) * E;
    v2 = (mu2 * N) * id2;
  }
  const double rbar2 = N * id2;
  const double A = fma(-fma(0.5 * mu2, s.rperp2, mu * N), id2, s.qh);   // qbar - mu rbar^2
  const double P1 = 1.0 + W;
  const double T = fma(P1 * W, A, v2 * (W * W));                          // (1 + W) eps_raw
  const double Te = gt_nn(s.eps_min * P1, T) ? s.eps_min * P1 : T;
  const double Z = fma(P1, fma(mu * rbar2, W, 1.0), s.gam * Te);   // >= 1
  return mu - (W * P1) * rcp_nr(Z);
}
// The master function with the hybrid EOS, in the general form of Kastaun
// et al. (2021): rho = D/W, eps clamped below at eps_c(rho) + T_atm/(G_th-1),
// P = P(rho, eps), a = P/(rho (1 + eps)), nu = max(nu_A, nu_B) with
// nu_A = (1 + a)(1 + eps)/W and nu_B = (1 + a)(1 + qbar - mu rbar^2), and
// f = mu - 1/(nu + mu rbar^2).  (With the ideal gas nu_A >= nu_B, which kev
// uses; here nu_B can win where eps is clamped.)
__device__ __forceinline__ void kev_hyb(const KS& s, const Par& P, double mu, KEval& e) {
  const double x = 1.0 / fma(mu, s.b2, 1.0);
  const double mux = mu * x;
  const double rbar2 = x * fma(s.r2, x, mu * (1.0 + x) * s.rb2);
  const double qbar = fma(-0.5 * mux * mux, s.rperp2, s.qh);
  const double v2 = mu * mu * rbar2;
  e.vcap = v2 > s.vmax2;
  const double vh2 = e.vcap ? s.vmax2 : v2;
  const double W = rsqrt(1.0 - vh2);
  const double rho = s.D / W;
  double Pc, epsc, Gi;
  eos_cold(P, rho, Pc, epsc, Gi);
  const double A = qbar - mu * rbar2;
  e.eps_min = epsc + P.eps_atm;
  e.eps_raw = fma(W, A, vh2 * W * W / (1.0 + W));
  e.eps = e.eps_raw < e.eps_min ? e.eps_min : e.eps_raw;
  const double Ph = fma(P.gth1 * rho, e.eps - epsc, Pc);
  const double a1 = 1.0 + Ph / (rho * (1.0 + e.eps));
  const double nu = fmax(a1 * (1.0 + e.eps) / W, a1 * (1.0 + A));
  e.x = x;
  e.rbar2 = rbar2;
  e.W = W;
  e.rho = rho;
  e.P = Ph;
  e.Pc = Pc;
  e.G = mu - 1.0 / fma(mu, rbar2, nu);
}
// f(mu) for either EOS
__device__ __forceinline__ double kev_G(const KS& s, const Par& P, double mu) {
  if (P.eos == 0) return kev_g(s, mu);
  KEval e;
  kev_hyb(s, P, mu, e);
  return e.G;
}
// f(0): at mu = 0, v = 0, W = 1 and eps = qbar = q_h; the ideal gas gives
// -1/(1 + Gamma eps(0)).
__device__ __forceinline__ double f_zero(const KS& s, const Par& P) {
  if (P.eos != 0) return kev_G(s, P, 0.0);
  double e0 = gt_nn(s.eps_min, s.qh) ? s.eps_min : s.qh;
  return -rcp_nr(fma(s.gam, e0, 1.0));   // >= 1
}

// Upper bracket end.  rbar^2(mu) = r_perp^2 x^2 + r_par^2 >= r_par^2 for every
// mu, so 1/sqrt(1 + r_par^2) bounds the root of f_a(mu) = mu sqrt(1 +
// rbar^2(mu)) - 1 (h_min = 1), and with it the master function's root, from
// above.  Three fixed-point steps mu <- 1/sqrt(1 + rbar^2(mu)) tighten it;
// they move it by less than r_perp^2/(1 + r_par^2), so a cell with
// r_perp^2 <= 1e-3 (1 + r_par^2) (nearly static or field-aligned flow, most of
// a star) keeps the bound itself: on the 128^3 star that left the evaluations
// per cell unchanged and saved 1.7% of the RK3 step, while relativistic cells
// keep the tighter bracket.
__device__ __forceinline__ double mu_plus(const KS& s) {
  const double rpar2 = gt0(s.b2) ? s.rb2 / s.b2 : s.r2;
  double mu = rsqrt(1.0 + rpar2);
  if (gt_nn(s.r2 - rpar2, 1e-3 * (1.0 + rpar2))) {
#pragma unroll
    for (int it = 0; it < 3; it++) {
      // 1/sqrt(1 + rbar^2) = d / sqrt(d^2 + N) with d, N as in kev_g
      const double d = fma(mu, s.b2, 1.0);
      const double N = fma(mu * (d + 1.0), s.rb2, s.r2);
      mu = d * rsqrt(fma(d, d, N));
    }
  }
  return mu;
}

// Five features of the KRP variables for the learned guess (FP32):
// log q_h with q_h = q - b^2/2 >= 0 (the energy per D without the magnetic
// b^2/2, which dominates q in magnetised cells), log(1 + r^2/(1+q_h)^2),
// log(1 + b^2), the r-b alignment (r.b)^2/(r^2 b^2), log(1 + (r.b)^2/(1+q_h)^2).
// Written with stride MLP_FSTRIDE.
__device__ __forceinline__ void krp_features(const KS& s, float* f) {
  const float qh = (float)s.qh;
  const float r2 = (float)s.r2, b2 = (float)s.b2, rb2 = (float)s.rb2;
  const float iq = 1.0f / ((1.0f + qh) * (1.0f + qh));
  f[0] = __logf(fmaxf(qh, 1e-30f));
  f[1] = log1pf(r2 * iq);
  f[2] = log1pf(b2);
  const float rb = r2 * b2;
  f[3] = rb > 0.0f ? fminf(rb2 / rb, 1.0f) : 0.0f;
  f[4] = log1pf(rb2 * iq);
  f[5] = f[6] = f[7] = 0.0f;
}

// Illinois regula falsi with bisection safeguard on [a,b], f(a) < 0 <= f(b);
// every point is nudged by tol b/4 away from the end replaced last, so the
// bracket closes one step after the iterate converges; stops when b - a <=
// tol b, then one regula-falsi step with the true end values.  Returns false
// when the iteration cap is reached.
__device__ __forceinline__ bool illinois(const KS& s, const Par& P, double a, double Ga, double b, double Gb,
                                         double tol, int maxit, double& root, int& iters) {
  iters = 0;
  if (eq0(Gb)) { root = b; return true; }
  double Fa = Ga, Fb = Gb;
  int side = 0;
  while (gt_nn(b - a, tol * b)) {
    if (iters >= maxit) return false;
    iters++;
    double c = (a * Fb - b * Fa) * rcp_nr(Fb - Fa);   // Fb > 0 > Fa
    // nudge away from the end replaced last: once the iterate is within eta of
    // the root the next point lands past it and closes the bracket
    const double eta = 0.25 * tol * b;
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
      root = c;
      return true;
    }
  }
  root = a - Ga * (b - a) * rcp_nr(Gb - Ga);   // Gb > 0 > Ga
  return true;
}

// Everything the root solve and the recovery need of one cell.
struct KrpCell {
  KS s;
  double D, rb, ru[3], bu[3];
};

// Phase 1: undensitise, apply the floors on the conserved state (Sec. 3.3) and
// form the KRP variables.  Returns false (F_FAIL set) on non-finite input.
// alpha: the cell's lapse, for the excision floor (1 where none applies).
__device__ __forceinline__ bool krp_prep(const Par& P, const double* U, const double* Bd, const Metric& m,
                                         KrpCell& k, unsigned& flags, double alpha = 1.0) {
  flags = 0;
  const double isd = m.isdet;
  double D = U[0] * isd, tau = U[4] * isd;
  double Sl[3] = {U[1] * isd, U[2] * isd, U[3] * isd};
  double B[3] = {Bd[0] * isd, Bd[1] * isd, Bd[2] * isd};
  double Bl[3];
  lower3(m.g, B, Bl);
  double B2 = dot3(B, Bl);
  bool fin = finite_bits(D) && finite_bits(tau) && finite_bits(Sl[0]) && finite_bits(Sl[1]) &&
             finite_bits(Sl[2]) && finite_bits(B2) && gt0(m.sdet);
  if (!fin) {
    flags |= F_FAIL;
    return false;
  }
  // inside the excision region (Sec. 4.7) every cell takes the D-floor reset
  if (below_thr(P, D) || (P.exc_on && alpha < P.alpha_exc)) {
    D = P.rho_atm;
    Sl[0] = Sl[1] = Sl[2] = 0.0;
    tau = fma(D, P.eps_atm_rho, 0.5 * B2);
    flags |= F_DFLOOR;
  }
  if (P.sigma_on && B2 > P.sigma_max * D) {
    D = B2 / P.sigma_max;
    flags |= F_SIGMA;
  }
  double tau_atm = fma(D, P.eps_atm, 0.5 * B2);
  if (tau < tau_atm) {
    tau = tau_atm;
    flags |= F_TAU;
  }
  KS& s = k.s;
  const double isD = rsqrt(D);
  const double iD = isD * isD;
  double rl[3] = {Sl[0] * iD, Sl[1] * iD, Sl[2] * iD};
  lower3(m.gi, rl, k.ru);
  k.bu[0] = B[0] * isD; k.bu[1] = B[1] * isD; k.bu[2] = B[2] * isD;
  s.b2 = B2 * iD;
  s.r2 = dot3(rl, k.ru);
  k.rb = dot3(rl, k.bu);
  s.rb2 = k.rb * k.rb;
  double rp = s.r2 * s.b2 - s.rb2;
  s.rperp2 = gt0(rp) ? rp : 0.0;
  s.qh = fma(tau, iD, -0.5 * s.b2);
  s.gam = P.gam;
  s.eps_min = P.eps_atm;
  s.vmax2 = P.vmax2;
  s.D = D;
  k.D = D;
  return true;
}

// Phase 2a: a bracket [a,b] with f(a) < 0 <= f(b), with f(0) < 0 from
// f_zero.  `iters` counts the evaluations of f it made.  A learned guess [glo, ghi] is used when given and verified by the
// signs at both ends; otherwise [0, mu+] (or [mu+, 1] when G(mu+) < 0).
// Returns 0: solve needed; 1: root found (in mu); 2: no bracket (failure).
__device__ __forceinline__ int krp_bracket(const KS& s, const Par& P, double glo, double ghi, double& a, double& b,
                                           double& Ga, double& Gb, double& mu, int& iters) {
  a = 0.0; Ga = f_zero(s, P); b = 1.0; Gb = 0.0;
  iters = 0;
  bool have = false;
  if (glo >= 0.0 && ghi > glo) {
    const double Gl = kev_G(s, P, glo), Gh = kev_G(s, P, ghi);
    if (lt0(Gl) && (eq0(Gh) || gt0(Gh))) {
      a = glo; Ga = Gl; b = ghi; Gb = Gh; have = true;
    } else if (eq0(Gl) || gt0(Gl)) {
      b = glo; Gb = Gl; have = true;
    } else {
      a = ghi; Ga = Gh;
    }
    iters += 2;
  }
  if (!have) {
    double mp = mu_plus(s);
    if (mp <= a) mp = 1.0;
    iters++;
    b = mp; Gb = kev_G(s, P, mp);
    if (lt0(Gb)) {
      a = mp; Ga = Gb;
      b = 1.0;
      iters++;
      Gb = kev_G(s, P, b);
    }
  }
  if (!(lt0(Ga) && (eq0(Gb) || gt0(Gb)))) return 2;
  if (eq0(Gb)) { mu = b; return 1; }
  return 0;
}

// ------------------------------------------- FP32 start for the KRP root
// The FP32 pipe issues about 64 times the FP64 one on this part, so a root
// estimate in FP32 is nearly free next to one FP64 evaluation of f.  These are
// the master function and the upper bracket end in FP32 (ideal gas), the
// secant search, and the slope estimate that the FP64 polish uses.
struct KSf {
  float qh, r2, b2, rb2, rp2, gam, emin, vmax2;
};
// Conversions between double and float on the integer pipe (a conversion
// instruction takes an FP64 issue slot on this part).  f32_tz: toward zero,
// which is all the search's start needs; beyond the float range inf (NaN
// stays NaN), below 2^-126 a signed zero.  f64_of: exact for a normal float
// and zero, the conversion instruction for the rest.
__device__ __forceinline__ float f32_tz(double x) {
  const unsigned h = (unsigned)__double2hiint(x), l = (unsigned)__double2loint(x);
  const unsigned sg = h & 0x80000000u;
  const int e = (int)((h >> 20) & 0x7FFu);
  if (e >= 897 && e <= 1150) return __uint_as_float(sg | ((unsigned)(e - 896) << 23) | ((h & 0xFFFFFu) << 3) | (l >> 29));
  if (e < 897) return __uint_as_float(sg);
  const bool nan = e == 0x7FF && ((h & 0xFFFFFu) | l) != 0u;
  return __uint_as_float(sg | 0x7F800000u | (nan ? 0x400000u : 0u));
}
__device__ __forceinline__ double f64_of(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  if (e != 0u && e != 0xFFu)
    return __hiloint2double((int)((u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3)), (int)(u << 29));
  return (double)f;
}
__device__ __forceinline__ KSf ks_f32(const KS& s) {
  KSf f;
  f.qh = f32_tz(s.qh); f.r2 = f32_tz(s.r2); f.b2 = f32_tz(s.b2); f.rb2 = f32_tz(s.rb2); f.rp2 = f32_tz(s.rperp2);
  f.gam = f32_tz(s.gam); f.emin = fmaxf(f32_tz(s.eps_min), 1e-37f); f.vmax2 = f32_tz(s.vmax2);
  return f;
}
__device__ __forceinline__ float f32_master(const KSf& s, float mu) {
  const float x = 1.0f / fmaf(mu, s.b2, 1.0f);
  const float mux = mu * x;
  const float rbar2 = x * fmaf(s.r2, x, mu * (1.0f + x) * s.rb2);
  const float qbar = s.qh - 0.5f * mux * mux * s.rp2;
  const float v2 = fminf(mu * mu * rbar2, s.vmax2);
  const float W = rsqrtf(1.0f - v2);
  const float wm1 = v2 * W * W / (1.0f + W);
  const float eps = fmaxf(fmaf(W, qbar - mu * rbar2, wm1), s.emin);
  return mu - W / fmaf(mu * rbar2, W, fmaf(s.gam, eps, 1.0f));
}
__device__ __forceinline__ float f32_mu_plus(const KSf& s) {
  const float rpar2 = s.b2 > 0.0f ? s.rb2 / s.b2 : s.r2;
  float mu = rsqrtf(1.0f + rpar2);
  for (int it = 0; it < 3; it++) {
    const float x = 1.0f / fmaf(mu, s.b2, 1.0f);
    mu = rsqrtf(1.0f + x * fmaf(s.r2, x, mu * (1.0f + x) * s.rb2));
  }
  return mu;
}
// FP32 secant steps from the pair (x0, x1), at most nsteps, stopping once a
// step moves mu by less than 2^-21 mu; nf counts the FP32 evaluations of f.
__device__ __forceinline__ float krp_secant32(const KSf& sf, float x0, float x1, int nsteps, unsigned& nf) {
  float f0 = f32_master(sf, x0), f1 = f32_master(sf, x1);
  nf += 2;
  for (int it = 0; it < nsteps; it++) {
    const float den = f1 - f0;
    if (den == 0.0f || !(f1 == f1)) break;
    float x2 = x1 - f1 * (x1 - x0) / den;
    if (!(x2 > 0.0f && x2 <= 1.0f)) x2 = 0.5f * (x1 + (f1 < 0.0f ? 1.0f : 0.0f));
    const bool conv = fabsf(x2 - x1) <= 4.76837158e-7f * x1;   // 2^-21
    x0 = x1; f0 = f1;
    x1 = x2;
    if (conv) break;
    f1 = f32_master(sf, x2);
    nf++;
  }
  return x1;
}
// FP32 estimate of 1/f'(mu): the central difference over mu (1 -+ 2^-8).
__device__ __forceinline__ float krp_islope32(const KSf& sf, float mu, unsigned& nf) {
  const float h = 0.00390625f * mu;
  nf += 2;
  return (2.0f * h) / (f32_master(sf, mu + h) - f32_master(sf, mu - h));
}

// FP64 root of f from the FP32 estimate m0 and isl ~ 1/f'(m0): a Newton step
// with the FP32 slope, m1 = m0 - f(m0) isl, then the FP64 secant through
// (m0, f(m0)) and (m1, f(m1)), m2 = m1 - f(m1) (m1 - m0)/(f(m1) - f(m0)).
// The secant's error is about |f''/(2 f')| |m0 - mu*| |m1 - mu*|, so m2 is
// taken as the root (returns 1, root in mu) when both steps contracted:
// |m1 - m0| <= 2^-16 m0 and |m2 - m1| <= 2^-30 m2.  Otherwise the two
// evaluations give the bracket for the FP64 solve (returns 0): [m_lo, m_hi]
// when f changes sign between them, [m_hi, 1] when both are negative (f(1) >=
// 0 for a physical state: one more evaluation), [0, m_lo] when both are
// positive (f(0) < 0 from f_zero); a non-finite value falls back to the plain
// bracket.  Returns 2 when there is no bracket, as krp_bracket does.  its
// counts the FP64 evaluations of f; fb is set when the root was not taken.
__device__ __forceinline__ int krp_polish(const KS& s, const Par& P, double m0, double isl, double& a, double& b,
                                          double& Ga, double& Gb, double& mu, int& its, bool& fb) {
  fb = false;
  if (!(m0 > 1e-300 && m0 <= 1.0)) m0 = 0.5;
  const double G0 = kev_g(s, m0);
  its = 1;
  if (eq0(G0)) { mu = m0; return 1; }
  double m1 = fma(-G0, isl, m0);
  if (!(m1 > 0.0)) m1 = 0.5 * m0;
  if (!(m1 <= 1.0)) m1 = 1.0;
  const double G1 = kev_g(s, m1);
  its = 2;
  if (eq0(G1)) { mu = m1; return 1; }
  const double dm = m1 - m0, dG = G1 - G0;
  const bool fin = finite_bits(G0) && finite_bits(G1);
  if (fin && !eq0(dG)) {
    const double q = gt_nn(fabs(dG), 1e-280) ? dm * rcp_nr(dG) : dm / dG;
    const double m2 = fma(-G1, q, m1);
    if (!gt_nn(fabs(dm), 1.52587890625e-5 * m0) && !gt_nn(fabs(m2 - m1), 9.313225746154785e-10 * m2) &&
        gt0(m2) && !gt_nn(m2, 1.0)) {
      mu = m2;
      return 1;
    }
  }
  fb = true;
  if (!fin) {
    int e = 0;
    const int r = krp_bracket(s, P, -1.0, -1.0, a, b, Ga, Gb, mu, e);
    its += e;
    return r;
  }
  const bool o = m0 <= m1;
  const double lo = o ? m0 : m1, hi = o ? m1 : m0, Glo = o ? G0 : G1, Ghi = o ? G1 : G0;
  if (lt0(Glo) && !lt0(Ghi)) {
    a = lo; Ga = Glo; b = hi; Gb = Ghi;
  } else if (lt0(Ghi)) {
    a = hi; Ga = Ghi; b = 1.0;
    Gb = kev_g(s, 1.0);
    its++;
  } else {
    a = 0.0; Ga = f_zero(s, P); b = lo; Gb = Glo;
  }
  if (!(lt0(Ga) && (eq0(Gb) || gt0(Gb)))) return 2;
  if (eq0(Gb)) { mu = b; return 1; }
  return 0;
}

// ------------------------------------------- FOFC flags from FP32 enclosures
// The FOFC estimate asks of con2prim(U*) only whether it fails or a floor on
// the conserved state or the primitives fires (Sec. 3.3).  Away from every
// threshold FP32 interval arithmetic (ival.cuh) answers that: every quantity
// is an enclosure of its exact value for every state in the enclosure of the
// inputs, so a threshold test that holds for a whole enclosure holds for the
// exact value, and with a gap of at least one FP32 unit it holds for the FP64
// path's value too (FP64 rounding is 2^-29 of that).

// KRP variables per unit D (krp_prep) as enclosures, and D.
struct KSI {
  Iv qh, r2, b2, rb2, rp2, D;
};

// The floors on the conserved state (excision, D, magnetisation, tau) and the
// KRP variables of krp_prep, from an enclosure U of the densitised conserved
// state.  Returns 1 when a floor on the conserved state fires for the whole
// enclosure (the FOFC estimate flags the cell), 0 when none fires (k holds the
// KRP variables), -1 when an enclosure straddles a threshold.
__device__ __forceinline__ int krp_prep_iv(const Par& P, const Iv* U, const double* Bd, const Metric& m, double alpha,
                                           KSI& k) {
  if (P.exc_on && alpha < P.alpha_exc) return 1;
  const Iv isd = iv_d(m.isdet);
  const Iv D = imul(U[0], isd), tau = imul(U[4], isd);
  Iv Sl[3], B[3], Bl[3], g[6], gi[6];
#pragma unroll
  for (int v = 0; v < 3; v++) {
    Sl[v] = imul(U[1 + v], isd);
    B[v] = imul(iv_d(Bd[v]), isd);
  }
#pragma unroll
  for (int v = 0; v < 6; v++) {
    g[v] = iv_d(m.g[v]);
    gi[v] = iv_d(m.gi[v]);
  }
  ilower3(g, B, Bl);
  const Iv B2 = imax(idot3(B, Bl), iv_pt(0.0f));   // B^2 >= 0 (gamma positive definite)
  if (P.thr_pos) {
    const Iv t = iv_d(P.rho_thr);
    if (ilt(D, t)) return 1;
    if (!igt(D, t)) return -1;
  } else {
    if (D.hi < 0.0f) return 1;
    if (!(D.lo > 0.0f)) return -1;
  }
  if (P.sigma_on) {
    const Iv sD = imul(iv_d(P.sigma_max), D);
    if (igt(B2, sD)) return 1;
    if (!ilt(B2, sD)) return -1;
  }
  const Iv ta = iadd(imul(D, iv_d(P.eps_atm)), iscale(B2, 0.5f));
  if (ilt(tau, ta)) return 1;
  if (!igt(tau, ta)) return -1;
  const Iv iD = idiv(iv_pt(1.0f), D), isD = irsqrt(D);
  Iv rl[3], ru[3], bu[3];
#pragma unroll
  for (int v = 0; v < 3; v++) {
    rl[v] = imul(Sl[v], iD);
    bu[v] = imul(B[v], isD);
  }
  ilower3(gi, rl, ru);
  k.b2 = imul(B2, iD);
  k.r2 = imax(idot3(rl, ru), iv_pt(0.0f));   // r^2 >= 0
  k.rb2 = isq(idot3(rl, bu));
  k.rp2 = imax(isub(imul(k.r2, k.b2), k.rb2), iv_pt(0.0f));   // r_perp^2 = max(r^2 b^2 - (r.b)^2, 0)
  k.qh = isub(imul(tau, iD), iscale(k.b2, 0.5f));
  k.D = D;
  return 0;
}

// The KRP variables of an FP64 krp_prep as enclosures (each exact value in its
// FP32 interval).
__device__ __forceinline__ void ksi_of(const KS& s, double D, KSI& k) {
  k.qh = iv_d(s.qh); k.r2 = iv_d(s.r2); k.b2 = iv_d(s.b2); k.rb2 = iv_d(s.rb2); k.rp2 = iv_d(s.rperp2);
  k.D = iv_d(D);
}

// Enclosures of f (the ideal-gas master function), v^2 (without the cap), W
// and eps_raw at mu (an enclosure itself), for every state in k.
struct RecIv {
  Iv f, v2, W, eps_raw;
};
__device__ __forceinline__ void rec_iv(const KSI& k, Iv gam, Iv emin, Iv vmax2, Iv mu, RecIv& e) {
  const Iv one = iv_pt(1.0f);
  const Iv x = idiv(one, iadd(imul(mu, k.b2), one));
  const Iv mux = imul(mu, x);
  const Iv rbar2 = imul(x, iadd(imul(k.r2, x), imul(imul(mu, iadd(one, x)), k.rb2)));
  const Iv qp = iscale(imul(isq(mux), k.rp2), 0.5f);
  const Iv murb = imul(mu, rbar2);
  const Iv v2 = imul(mu, murb);
  const Iv vh2 = imin(v2, vmax2);
  const Iv W = irsqrt(isub(one, vh2));
  const Iv wm1 = idiv(imul(vh2, isq(W)), iadd(one, W));   // W - 1
  const Iv eps_raw = iadd(imul(W, isub(isub(k.qh, qp), murb)), wm1);
  const Iv Z = iadd(imul(murb, W), iadd(imul(gam, imax(eps_raw, emin)), one));
  e.f = isub(mu, idiv(W, Z));
  e.v2 = v2;
  e.W = W;
  e.eps_raw = eps_raw;
}

// The FOFC question for KRP enclosures k (ideal gas): 1 flagged for sure, 0 not
// flagged for sure, -1 undecided (the FP64 path decides).  The FP32 secant
// search from [0, mu+] on the enclosures' midpoints gives m; lo, hi = m (1 -+ h)
// certify the root when the enclosure of f is below 0 at lo and above 0 at hi
// (h = 2^-18, 2^-14, 2^-10 in turn).  At hi = 1 no test is needed: f(1) >= 0 for
// every eps >= eps_min > 0 (Z >= 1 + vh^2 W + Gamma eps >= W, as W - 1 = vh^2
// W^2/(1 + W) <= vh^2 W); cold cells, whose root is 1 - Gamma eps + ..., need
// this.  Then v^2, rho = D/W and eps_raw are enclosed over mu in [lo, hi] and
// compared with the velocity cap, the density floor and the T floor (with the
// ideal gas p < rho T_atm is eps < T_atm/(Gamma - 1) = eps_atm).  nf counts the
// FP32 evaluations of f.
__device__ __forceinline__ int fofc_decide_iv(const KSI& k, const Par& P, unsigned& nf) {
  const Iv gam = iv_d(P.gam), emin = iv_d(P.eps_atm), vmax2 = iv_d(P.vmax2);
  KSf sf;
  sf.qh = 0.5f * (k.qh.lo + k.qh.hi);
  sf.r2 = 0.5f * (k.r2.lo + k.r2.hi);
  sf.b2 = 0.5f * (k.b2.lo + k.b2.hi);
  sf.rb2 = 0.5f * (k.rb2.lo + k.rb2.hi);
  sf.rp2 = 0.5f * (k.rp2.lo + k.rp2.hi);
  sf.gam = gam.lo;
  sf.emin = fmaxf(emin.lo, 1e-37f);
  sf.vmax2 = vmax2.lo;
  const float m = krp_secant32(sf, 0.0f, f32_mu_plus(sf), 8, nf);
  if (!(m > 1e-30f && m <= 1.0f)) return -1;
  float lo = 0.0f, hi = 0.0f, h = 3.81469727e-6f;   // 2^-18
  bool ok = false;
  for (int t = 0; t < 3 && !ok; t++, h *= 16.0f) {
    lo = m * (1.0f - h);
    hi = fminf(m * (1.0f + h), 1.0f);
    RecIv a;
    rec_iv(k, gam, emin, vmax2, iv_pt(lo), a);
    nf++;
    ok = a.f.hi < 0.0f;
    if (ok && hi < 1.0f) {
      RecIv b;
      rec_iv(k, gam, emin, vmax2, iv_pt(hi), b);
      nf++;
      ok = b.f.lo > 0.0f;
    }
  }
  if (!ok) return -1;
  RecIv q;
  rec_iv(k, gam, emin, vmax2, Iv{lo, hi}, q);
  if (igt(q.v2, vmax2)) return 1;     // the velocity cap
  if (!ilt(q.v2, vmax2)) return -1;
  bool low_rho = false;               // the density floor (rho_thr = 0: rho = D/W > 0 never floors)
  if (P.thr_pos) {
    const Iv rho = idiv(k.D, q.W), t = iv_d(P.rho_thr);
    if (ilt(rho, t)) low_rho = true;
    else if (!igt(rho, t)) return -1;
  }
  if (ilt(q.eps_raw, emin)) return 1;   // the T floor
  if (!igt(q.eps_raw, emin)) return low_rho ? 1 : -1;
  return low_rho ? 1 : 0;
}

// Phase 3: primitives at the root mu (Sec. 3.4 recovery) and the floors on
// the primitives (Sec. 3.3).  On failure the static atmosphere.  iWo
// (optional): 1/W of the written velocity, W (1 - v^2) of the recovery (the
// capped v^2 under the velocity cap), 1 where the velocity is set to 0.
__device__ __forceinline__ void krp_finish(const Par& P, const KrpCell& k, double mu, bool ok, unsigned& flags,
                                           double* prim, double* iWo = nullptr) {
  double rho = P.rho_atm, p = P.P_atm, w0 = 0.0, w1 = 0.0, w2 = 0.0, iWr = 1.0;
  if (!ok || !isfinite(mu)) {
    flags |= F_FAIL;
  } else {
    const KS& s = k.s;
    KEval e;
    if (P.eos == 0) {
      kev(s, mu, e);
      if (gt_nn(s.eps_min, e.eps_raw)) flags |= F_TEMP;
      double iW = e.W * (1.0 - (e.vcap ? s.vmax2 : mu * mu * e.rbar2));
      rho = k.D * iW;
      p = P.gm1 * rho * e.eps;
      iWr = iW;
    } else {
      kev_hyb(s, P, mu, e);
      if (e.eps_raw < e.eps_min) flags |= F_TEMP;
      rho = e.rho;
      p = e.P;
      if (iWo) iWr = e.W * (1.0 - (e.vcap ? s.vmax2 : mu * mu * e.rbar2));
    }
    if (e.vcap) flags |= F_VMAX;
    double vs = 1.0;
    if (e.vcap) vs = sqrt(s.vmax2 / (mu * mu * e.rbar2));
    double f = e.W * vs * mu * e.x;
    double mrb = mu * k.rb;
    w0 = f * fma(mrb, k.bu[0], k.ru[0]);
    w1 = f * fma(mrb, k.bu[1], k.ru[1]);
    w2 = f * fma(mrb, k.bu[2], k.ru[2]);
    if (below_thr(P, rho)) {
      rho = P.rho_atm; p = P.P_atm; w0 = w1 = w2 = 0.0; iWr = 1.0;
      flags |= F_RHO;
    } else {
      // T floor: P >= P_c(rho) + rho T_atm (the cold part at this rho is
      // e.Pc for the hybrid EOS, 0 for the ideal gas)
      const double pf = P.eos == 0 ? rho * P.T_atm : fma(rho, P.T_atm, e.Pc);
      if (p < pf) {
        p = pf;
        flags |= F_TEMP;
      }
    }
  }
  if (flags & F_FAIL) {
    rho = P.rho_atm; p = P.P_atm; w0 = w1 = w2 = 0.0; iWr = 1.0;
  }
  prim[0] = rho; prim[1] = w0; prim[2] = w1; prim[3] = w2; prim[4] = p;
  if (iWo) *iWo = iWr;
}

// The con2prim of one cell in one thread.  U: densitised conserved state
// (overwritten with the floored state when write_cons and a floor fired); Bd:
// cell-centred B~; m: metric with inverse.  glo/ghi: optional bracket guess
// (glo < 0: none); alpha: the lapse, for the excision floor.
__device__ __forceinline__ void con2prim(const Par& P, double* U, const double* Bd, const Metric& m, double* prim,
                                         unsigned& flags, int& iters, bool write_cons, double glo = -1.0,
                                         double ghi = -1.0, double alpha = 1.0, double* iWo = nullptr) {
  KrpCell k;
  iters = 0;
  bool ok = krp_prep(P, U, Bd, m, k, flags, alpha);
  double mu = 0.0;
  if (ok) {
    double a, b, Ga, Gb;
    int st = krp_bracket(k.s, P, glo, ghi, a, b, Ga, Gb, mu, iters);
    if (st == 2) ok = false;
    else if (st == 0) {
      int it = 0;
      ok = illinois(k.s, P, a, Ga, b, Gb, P.tol, P.maxit, mu, it);
      iters += it;
    }
  }
  krp_finish(P, k, mu, ok, flags, prim, iWo);
  if (write_cons && (flags & (FLOOR_BITS | F_FAIL))) prim2cons(P, prim, Bd, m, U);
}

// -------------------------------------------------- reconstruction (Sec. 3.2)
// The flux kernels sweep a line of cells along the face normal, so every cell
// is reconstructed once and yields both of its face values: "hi" at x_{m+1/2}
// (the left state of that face) and "lo" at x_{m-1/2} (the right state of the
// face below).  With differences delta_k = x_{k+1} - x_k carried along the
// sweep, each three-cell window is evaluated once and serves as stencil 0 of
// the cell to its right, stencil 1 of its centre cell and stencil 2 of the
// cell to its left.
//
// Smoothness of the window (x_{c-1}, x_c, x_{c+1}) from dl = x_c - x_{c-1} and
// dr = x_{c+1} - x_c, in the three one-sided forms of WENO5 (Jiang & Shu):
// 13/12 (x0 - 2x1 + x2)^2 + 1/4 u^2 with u = x0 - 4x1 + 3x2 (b0), x0 - x2 (b1)
// or 3x0 - 4x1 + x2 (b2).  Returned scaled by 4 and with the WENO-Z epsilon
// added, e_k = 4 (b_k + eps) = 13/3 t^2 + eps4 + u_k^2 with t = dr - dl and
// u_0 = 3 dr - dl, u_1 = dl + dr, u_2 = dr - 3 dl: the WENO-Z weights are
// homogeneous of degree 0 in (b_k + eps, |b_0 - b_2|), so the common factor
// changes only rounding, and eps rides in the shared term's FMA.
constexpr double WZ_EPS4 = 4e-40;   // 4 eps, eps = 1e-40
__device__ __forceinline__ void wz_window(double dl, double dr, double& e0, double& e1, double& e2) {
  const double t = dr - dl;
  const double kt2 = fma((13.0 / 3.0) * t, t, WZ_EPS4);
  const double u0 = fma(3.0, dr, -dl), u1 = dl + dr, u2 = fma(-3.0, dl, dr);
  e0 = fma(u0, u0, kt2);
  e1 = fma(u1, u1, kt2);
  e2 = fma(u2, u2, kt2);
}

// Sliding state of one reconstructed variable at cell m of a sweep.
struct RecVar {
  double x1, x2;          // x_m, x_{m+1}
  double d0, d1, d2;      // delta_{m-2}, delta_{m-1}, delta_m
  double e0p, e0c, e1c;   // e0 of window m-1, e0 and e1 of window m (wz_window)
  double xm2, xm1;        // PPM: x_{m-2}, x_{m-1}
  double aL, dm;          // PPM: value at the face m-1/2; PPM4: limited slope of cell m
};

// PPM4 (Colella & Woodward 1984): monotonised average slope of the middle value.
__device__ __forceinline__ double cw_slope(double am, double a0, double ap) {
  const double dl = a0 - am, dr = ap - a0;
  if (!(dl * dr > 0.0)) return 0.0;
  const double dc = 0.5 * (ap - am);
  const double m = fmin(fabs(dc), fmin(2.0 * fabs(dl), 2.0 * fabs(dr)));
  return dc < 0.0 ? -m : m;
}
// PPMX (Colella & Sekora 2008): limited second difference and face value.
__device__ __forceinline__ double cs_d2lim(double d, double d1, double d2) {
  const double C = 1.25;
  if (d > 0.0 && d1 > 0.0 && d2 > 0.0) return fmin(d, fmin(C * d1, C * d2));
  if (d < 0.0 && d1 < 0.0 && d2 < 0.0) return fmax(d, fmax(C * d1, C * d2));
  return 0.0;
}
__device__ __forceinline__ double cs_face(double am, double a0, double ap, double app) {
  double f = 7.0 / 12.0 * (a0 + ap) - 1.0 / 12.0 * (am + app);
  if ((f - a0) * (ap - f) < 0.0) {
    const double d = 3.0 * (a0 - 2.0 * f + ap);
    f = 0.5 * (a0 + ap) - cs_d2lim(d, am - 2.0 * a0 + ap, a0 - 2.0 * ap + app) / 6.0;
  }
  return f;
}
// Limited parabola of cell j from its face values aL, aR and a_{j-2..j+2}.
__device__ __forceinline__ void ppm4_limit(double aj, double& aL, double& aR) {
  if (!((aR - aj) * (aj - aL) > 0.0)) {
    aL = aj;
    aR = aj;
  } else {
    const double da = aR - aL, a6 = 6.0 * (aj - 0.5 * (aL + aR));
    if (da * a6 > da * da) aL = 3.0 * aj - 2.0 * aR;
    else if (-(da * da) > da * a6) aR = 3.0 * aj - 2.0 * aL;
  }
}
__device__ __forceinline__ void ppmx_limit(double am2, double am1, double aj, double ap1, double ap2, double& aL,
                                           double& aR) {
  const double C = 1.25;
  if (!((aR - aj) * (aj - aL) > 0.0) || !((am1 - aj) * (aj - ap1) > 0.0)) {
    const double d = 6.0 * (aL + aR) - 12.0 * aj;
    const double dc = am1 - 2.0 * aj + ap1, dl = am2 - 2.0 * am1 + aj, dr = aj - 2.0 * ap1 + ap2;
    double lim = 0.0;
    if (d > 0.0 && dc > 0.0 && dl > 0.0 && dr > 0.0) lim = fmin(d, fmin(C * dc, fmin(C * dl, C * dr)));
    if (d < 0.0 && dc < 0.0 && dl < 0.0 && dr < 0.0) lim = fmax(d, fmax(C * dc, fmax(C * dl, C * dr)));
    if (d == 0.0) {
      aL = aj;
      aR = aj;
    } else {
      const double r = lim / d;
      aL = aj + (aL - aj) * r;
      aR = aj + (aR - aj) * r;
    }
  } else {
    const double dL = aL - aj, dR = aR - aj;
    if (fabs(dR) >= 2.0 * fabs(dL)) aR = aj - 2.0 * dL;
    if (fabs(dL) >= 2.0 * fabs(dR)) aL = aj - 2.0 * dR;
  }
}

// R = 0 donor cell, 1 PLM with the van Leer limiter, 2 WENO-Z, 3 PPM4, 4 PPMX.
// Start at cell m from x_{m-2} .. x_{m+1}.
template <int R>
__device__ __forceinline__ void rec_init(RecVar& s, double xm2, double xm1, double x0, double xp1) {
  s.x1 = x0;
  s.x2 = xp1;
  if (R >= 3) {
    s.xm2 = xm2;
    s.xm1 = xm1;
    if (R == 3) {
      const double dmm = cw_slope(xm2, xm1, x0);
      s.dm = cw_slope(xm1, x0, xp1);
      s.aL = xm1 + 0.5 * (x0 - xm1) - (s.dm - dmm) / 6.0;
    } else {
      s.aL = cs_face(xm2, xm1, x0, xp1);
    }
    return;
  }
  s.d0 = xm1 - xm2;
  s.d1 = x0 - xm1;
  s.d2 = xp1 - x0;
  if (R == 2) {
    double u, v;
    wz_window(s.d0, s.d1, s.e0p, u, v);
    wz_window(s.d1, s.d2, s.e0c, s.e1c, v);
  }
}

// Face values of cell m given x_{m+2}; advances the state to cell m+1.
// R = 0, 1, 3, 4; WENO-Z (R = 2) goes through wz_parts and wz_finish.
template <int R>
__device__ __forceinline__ void rec_step(RecVar& s, double xn, double& lo, double& hi) {
  if (R >= 3) {
    double aR, aL = s.aL;
    if (R == 3) {
      const double dmn = cw_slope(s.x1, s.x2, xn);
      aR = s.x1 + 0.5 * (s.x2 - s.x1) - (dmn - s.dm) / 6.0;
      s.dm = dmn;
      s.aL = aR;
      ppm4_limit(s.x1, aL, aR);
    } else {
      aR = cs_face(s.xm1, s.x1, s.x2, xn);
      s.aL = aR;
      ppmx_limit(s.xm2, s.xm1, s.x1, s.x2, xn, aL, aR);
    }
    lo = aL;
    hi = aR;
    s.xm2 = s.xm1;
    s.xm1 = s.x1;
    s.x1 = s.x2;
    s.x2 = xn;
    return;
  }
  static_assert(R != 2, "WENO-Z: wz_parts / wz_finish");
  const double dn = xn - s.x2;  // delta_{m+1}
  if (R == 1) {
    const double dl = s.d1, dr = s.d2;
    const double pr = dl * dr;
    const double h = pr > 0.0 ? pr / (dl + dr) : 0.0;   // half the van Leer slope
    hi = s.x1 + h;
    lo = s.x1 - h;
  } else {
    hi = lo = s.x1;
  }
  s.x1 = s.x2;
  s.x2 = xn;
  s.d0 = s.d1;
  s.d1 = s.d2;
  s.d2 = dn;
}

// WENO-Z (Borges et al. 2008, p = 1, linear weights (1, 6, 3)/10:
// omega_k ~ d_k (1 + tau5/(b_k + eps)), multiplied through by the product of
// the three (b_k + eps) so that they need no division) of cell m given
// x_{m+2}, without the final division: x_m, the two numerators and
// denominators of hi = x + n_hi / (6 den_hi), lo = x + n_lo / (6 den_lo);
// advances the state to cell m+1.
__device__ __forceinline__ void wz_parts(RecVar& s, double xn, double& x, double& n_hi, double& n_lo, double& d_hi,
                                         double& d_lo) {
  const double dn = xn - s.x2;
  double e0n, e1n, e2n;
  wz_window(s.d2, dn, e0n, e1n, e2n);
  const double e0 = s.e0p, e1 = s.e1c, e2 = e2n;   // 4 (b_k + eps)
  const double tau = fabs(e0 - e2);                 // 4 tau5
  // A_k = (e_k + tau) prod_{j != k} e_j = P + tau prod_{j != k} e_j, P = e0 e1 e2
  const double p12 = e1 * e2, p02 = e0 * e2, p01 = e0 * e1, P3 = p01 * e2;
  const double A0 = fma(tau, p12, P3);
  const double A1 = fma(tau, p02, P3);
  const double A2 = fma(tau, p01, P3);
  const double a1 = 6.0 * A1, a2h = 3.0 * A2, a0l = 3.0 * A0;
  // Explicit FMAs: left to the compiler, these sums would be contracted by
  // the use count of each product, which differs where the caller drops the
  // lower face value (the first cell of a sweep).  A face would then depend
  // in its last bit on where its segment starts.
  d_hi = fma(6.0, A1, fma(3.0, A2, A0));
  d_lo = fma(6.0, A1, fma(3.0, A0, A2));
  const double da = s.d0, db = s.d1, dc = s.d2, dd = dn;
  n_hi = fma(A0, fma(5.0, db, -2.0 * da), fma(a1, fma(2.0, dc, db), a2h * fma(4.0, dc, -dd)));
  n_lo = fma(A2, fma(-5.0, dc, 2.0 * dd), fma(-a1, fma(2.0, db, dc), a0l * fma(-4.0, db, da)));
  x = s.x1;
  s.e0p = s.e0c;
  s.e0c = e0n;
  s.e1c = e1n;
  s.x1 = s.x2;
  s.x2 = xn;
  s.d0 = s.d1;
  s.d1 = s.d2;
  s.d2 = dn;
}

// The face values of N variables from wz_parts with one division for all
// (Montgomery's simultaneous inversion): the products p_v = d_hi d_lo are
// scaled to [1, 2) by their binary exponents (integer operations), chained,
// inverted once and unchained; 1/(6 p_v) regains its exponent the same way.
// Products outside [2^-959, 2^977] (never for physical data: eps4 = 4e-40
// bounds them below by ~4e-235) take one division each.
template <int N>
__device__ __forceinline__ void wz_finish(const double* x, const double* n_hi, const double* n_lo,
                                          const double* d_hi, const double* d_lo, double* hi, double* lo) {
  double m[N];
  int e[N];
  bool ok = true;
#pragma unroll
  for (int v = 0; v < N; v++) {
    const double p = d_hi[v] * d_lo[v];
    const int h = __double2hiint(p);
    const int ex = (h >> 20) & 0x7FF;
    ok = ok && ex >= 64 && ex <= 2000;
    m[v] = __hiloint2double((h & 0x000FFFFF) | 0x3FF00000, __double2loint(p));
    e[v] = ex - 1023;
  }
  if (ok) {
    double c[N];
    c[0] = m[0];
#pragma unroll
    for (int v = 1; v < N; v++) c[v] = c[v - 1] * m[v];
    double inv = (1.0 / 6.0) * rcp_nr(c[N - 1]);   // c[N - 1] in [1, 2^N)
#pragma unroll
    for (int v = N - 1; v >= 0; v--) {
      double r;
      if (v > 0) {
        r = inv * c[v - 1];
        inv *= m[v];
      } else {
        r = inv;
      }
      r = __hiloint2double(__double2hiint(r) - (e[v] << 20), __double2loint(r));
      hi[v] = fma(n_hi[v], d_lo[v] * r, x[v]);
      lo[v] = fma(n_lo[v], d_hi[v] * r, x[v]);
    }
  } else {
#pragma unroll
    for (int v = 0; v < N; v++) {
      hi[v] = x[v] + n_hi[v] / (6.0 * d_hi[v]);
      lo[v] = x[v] + n_lo[v] / (6.0 * d_lo[v]);
    }
  }
}

// E = 0 ideal gas; E = 1 hybrid EOS, which also returns the cold triple
// (P_c, eps_c, G_i) at the floored density in cold[3] for face_side.
template <int E = 0>
__device__ __forceinline__ void face_floor(const Par& P, double* s, double* cold = nullptr) {
  if (below_thr(P, s[0])) {
    s[0] = P.rho_atm; s[1] = s[2] = s[3] = 0.0; s[4] = P.P_atm;
    if (E) { cold[0] = P.Pc_atm; cold[1] = P.epsc_atm; cold[2] = P.G_atm; }
  } else if (E) {
    eos_cold(P, s[0], cold[0], cold[1], cold[2]);
    const double pf = fma(s[0], P.T_atm, cold[0]);
    if (s[4] < pf) s[4] = pf;
  } else {
    // p < rho T_atm by the integer key, as an FP64 compare decides it for
    // p that is not NaN (a -0 pressure counts below +0)
    const double pf = s[0] * P.T_atm;
    if (okey(s[4]) < okey(pf)) s[4] = pf;
  }
}

// --------------------------------------------------------- face fluxes (Eq. 8)
// Face metric: alpha, beta, gamma with inverse and sqrt(gamma).
struct FaceMetric {
  Metric m;
  double alpha, beta[3];
};
// Conserved state and flux of one side of a face of direction d, in the
// linear form the Riemann combination takes (Eq. 8; avd = alpha v^d - beta^d,
// avh^t = alpha v^t - beta^t, wl_i = W v_i, Bl_i = B_i):
//   D~:     U = UD,               F = UD avd
//   S~_i:   U = a wl_i + b Bl_i,  F = c wl_i + e Bl_i (+ asP along i = d)
//   tau~:   U = Ut,               F = Ut avd + t
//   B~^t:   U = B~^t,             F = B~^t avd - B~^d avh^t  (t = t1, t2)
// plus the pieces of the fast magnetosonic speeds lambda = alpha (vq -/+ sq)
// / den - beta^d.  The combination then weighs these per-side coefficients
// instead of 14 assembled components.
struct Side {
  double wl[3], Bl[3], a, b, c, e, UD, Ut, t, asP, avd, avh1, avh2, Bt1, Bt2, vq, sq, den;
};
// st = rho, w^1..3 (= W v^i), P, B~^{t1}, B~^{t2}; Bn = B~^d.
//
// Speeds: with c_f^2 = c_s^2 + v_A^2 - c_s^2 v_A^2 = (Gamma P + b^2)/(rho h +
// b^2) (c_s^2 = Gamma P/(rho h), v_A^2 = b^2/(rho h + b^2)), the roots of the
// characteristic quadratic along d become
//   lambda = alpha [v^d Q -/+ sqrt(N X / W^2)] / (Dn - v^2 N) - beta^d,
//   N = Gamma P + b^2,  Dn = rho h + b^2,  Q = rho h - Gamma P,
//   X = gamma^{dd} (Dn - v^2 N) - (v^d)^2 Q,
// which needs one square root and (shared with the other side) one division.
// E = 1: the hybrid EOS, rho h and rho h c_s^2 from the cold triple in cold[3].
template <int d, int E = 0>
__device__ __forceinline__ void face_side(const Par& P, const double* st, double Bn, const FaceMetric& fm, Side& o,
                                          const double* cold = nullptr) {
  constexpr int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  const Metric& m = fm.m;
  double Bt[3];
  Bt[d] = Bn; Bt[t1] = st[5]; Bt[t2] = st[6];
  const double B[3] = {Bt[0] * m.isdet, Bt[1] * m.isdet, Bt[2] * m.isdet};
  const double w[3] = {st[1], st[2], st[3]};
  double wl[3], Bl[3];
  lower3(m.g, w, wl);
  lower3(m.g, B, Bl);
  const double W2 = fma(w[0], wl[0], fma(w[1], wl[1], fma(w[2], wl[2], 1.0)));
  const double iW = rsqrt(W2);
  const double iW2 = iW * iW;
  const double W = W2 * iW;
  const double Bw = dot3(B, wl);          // W (B.v)
  const double Bv = Bw * iW;
  const double B2 = dot3(B, Bl);
  const double b2 = fma(B2, iW2, Bv * Bv);
  const double rho = st[0], p = st[4];
  double rhoh, gp;   // rho h and rho h c_s^2 (ideal gas: Gamma P)
  if (E) {
    eos_hyb_rhoh_chi(P, rho, p, cold[0], cold[1], cold[2], rhoh, gp);
  } else {
    rhoh = fma(P.gfac, p, rho);
    gp = P.gam * p;
  }
  const double eB = fma(rhoh, W2, B2);     // rho h W^2 + B^2
  const double D = rho * W;
  const double sd = m.sdet, alpha = fm.alpha;
  const double aiW = alpha * iW;
  double avh[3];  // alpha vhat^i = alpha v^i - beta^i
#pragma unroll
  for (int a = 0; a < 3; a++) avh[a] = fma(aiW, w[a], -fm.beta[a]);
  const double Ptot = fma(0.5, b2, p);
  const double sdeBW = sd * (eB * iW);
  const double sdBv = sd * Bv;
  const double avd = avh[d];
  const double aBn = alpha * Bn;
  const double aBi = aBn * iW2;
  // S~_i = sd (eB/W w_i - (B.v) B_i); its flux S~_i avd - alpha B~^d b_i/W
  // with b_i/W = (Bw w_i + B_i)/W^2, plus alpha sd P_tot along d
#pragma unroll
  for (int a = 0; a < 3; a++) {
    o.wl[a] = wl[a];
    o.Bl[a] = Bl[a];
  }
  o.a = sdeBW;
  o.b = -sdBv;
  o.c = fma(sdeBW, avd, -aBi * Bw);
  o.e = -fma(sdBv, avd, aBi);
  o.asP = alpha * (sd * Ptot);
  o.UD = sd * D;
  o.Ut = sd * ((eB - D) - Ptot);
  const double vd = w[d] * iW;
  o.t = fma(o.asP, vd, -aBn * Bv);
  o.avd = avd;
  o.avh1 = avh[t1];
  o.avh2 = avh[t2];
  o.Bt1 = Bt[t1];
  o.Bt2 = Bt[t2];
  const double N = gp + b2;
  const double Q = rhoh - gp;
  const double den = fma(iW2 - 1.0, N, rhoh + b2);   // Dn - v^2 N, v^2 = 1 - 1/W^2
  const double X = fma(m.gi[d == 0 ? 0 : (d == 1 ? 3 : 5)], den, -(vd * vd) * Q);
  const double S = (N * iW2) * X;
  // sqrt(S) as S rsqrt(S): within ~1 ulp, in fewer FP64 issue slots than the
  // correctly rounded square root (S <= 0 or NaN: 0, as before)
  o.sq = gt0(S) ? S * rsqrt(S) : 0.0;
  o.vq = vd * Q;
  o.den = den;
}

// LLF (rs 0) or HLLE (rs 1) flux from the two sides of a face of direction d
// (Bn = B~^d), both as F = kFL F_L + kFR F_R + kdU (U_R - U_L): HLLE
// (lR, -lL, lL lR)/(lR - lL), or (1/2, 1/2, 0) where lR = lL; LLF (1/2, 1/2,
// -a/2).  The per-side linear forms (Side) fold kFL, kFR and kdU into one
// coefficient per side vector.
template <int d>
__device__ __forceinline__ void riemann(int rs, const FaceMetric& fm, double Bn, const Side& L, const Side& R,
                                        double* F) {
  const double r = fm.alpha * rcp_nr(L.den * R.den);   // den = rho h + b^2 - v^2 N > 0
  const double aL = r * R.den, aR = r * L.den;
  const double bd = fm.beta[d];
  const double lmL = fma(aL, L.vq - L.sq, -bd), lpL = fma(aL, L.vq + L.sq, -bd);
  const double lmR = fma(aR, R.vq - R.sq, -bd), lpR = fma(aR, R.vq + R.sq, -bd);
  double kFL = 0.5, kFR = 0.5, kdU = 0.0;
  if (rs == 1) {
    // min / max on the integer pipe: the speeds are finite for physical
    // states (a NaN state is caught by the con2prim of the next stage)
    const double lL = imin(imin(lmL, lmR), 0.0);
    const double lR = imax(imax(lpL, lpR), 0.0);
    const double dl = lR - lL;   // >= 0
    if (!eq0(dl)) {
      const double inv = gt_nn(dl, 1e-280) ? rcp_nr(dl) : 1.0 / dl;   // dl > 0 here
      kFL = lR * inv;
      kFR = -lL * inv;
      kdU = (lL * lR) * inv;
    }
  } else {
    // the largest |lambda| by the integer key (the speeds are finite)
    kdU = -0.5 * imax(imax(fabs(lmL), fabs(lpL)), imax(fabs(lmR), fabs(lpR)));
  }
  // kFL F_L - kdU U_L and kFR F_R + kdU U_R per side vector
  const double gL = fma(kFL, L.avd, -kdU), gR = fma(kFR, R.avd, kdU);
  const double pL = fma(kFL, L.c, -kdU * L.a), qL = fma(kFL, L.e, -kdU * L.b);
  const double pR = fma(kFR, R.c, kdU * R.a), qR = fma(kFR, R.e, kdU * R.b);
  F[0] = fma(L.UD, gL, R.UD * gR);
#pragma unroll
  for (int i = 0; i < 3; i++) F[1 + i] = fma(L.wl[i], pL, fma(L.Bl[i], qL, fma(R.wl[i], pR, R.Bl[i] * qR)));
  F[1 + d] += fma(kFL, L.asP, kFR * R.asP);
  F[4] = fma(L.Ut, gL, fma(R.Ut, gR, fma(kFL, L.t, kFR * R.t)));
  F[5] = fma(L.Bt1, gL, fma(R.Bt1, gR, -Bn * fma(kFL, L.avh1, kFR * R.avh1)));
  F[6] = fma(L.Bt2, gL, fma(R.Bt2, gR, -Bn * fma(kFL, L.avh2, kFR * R.avh2)));
}

// x / 16 on the integer pipe (the exponent field less 4) where the result is a
// normal double, else (0, tiny, inf, NaN) by the FP64 multiply: exact either
// way, so fma(9, s1, -s2) / 16 has the bits of fma(0.5625, s1, -0.0625 s2).
__device__ __forceinline__ double mul_2m4(double x) {
  const int h = __double2hiint(x);
  const int e = (h >> 20) & 0x7FF;
  if (e > 4 && e < 0x7FF) return __hiloint2double(h - (4 << 20), __double2loint(x));
  return 0.0625 * x;
}
// Interpolates the ADM variables to the face between the cells at a and a+st
// (4-point Lagrange, weights (-1, 9, 9, -1)/16) and prepares the metric.
__device__ __forceinline__ void face_metric(const double* adm, long long nc, long long a, long long st, FaceMetric& fm) {
  double mv[10];
#pragma unroll
  for (int v = 0; v < 10; v++) {
    const double* q = adm + v * nc + a;
    mv[v] = mul_2m4(fma(9.0, q[0] + q[st], -(q[-st] + q[2 * st])));   // (9 (q0 + q1) - (q-1 + q2)) / 16
  }
  fm.alpha = mv[0];
  fm.beta[0] = mv[1]; fm.beta[1] = mv[2]; fm.beta[2] = mv[3];
#pragma unroll
  for (int v = 0; v < 6; v++) fm.m.g[v] = mv[4 + v];
  metric_setup(fm.m);
}

// Centred derivatives of the ten ADM metric variables at cell c along each
// axis (the derivative cache's slots), second order (Eq. 9 sources).
__device__ __forceinline__ void adm_derivs(const DevBlock& b, long long c, double* D) {
  const double* A = b.adm;
  const long long nc = b.ncell;
  const long long st[3] = {1, (long long)b.N[0], (long long)b.N[0] * b.N[1]};
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const double h = 0.5 * b.idx[a];
#pragma unroll
    for (int v = 0; v < 10; v++) D[10 * a + v] = (A[v * nc + c + st[a]] - A[v * nc + c - st[a]]) * h;
  }
}

// The face metric cache of direction d at index q (count n): store / load.
template <int d>
__device__ __forceinline__ void fmc_store(double* fc, long long n, long long q, const FaceMetric& fm) {
  constexpr int gd = d == 0 ? 0 : (d == 1 ? 3 : 5);
  fc[q] = fm.alpha;
#pragma unroll
  for (int a = 0; a < 3; a++) fc[(1 + a) * n + q] = fm.beta[a];
#pragma unroll
  for (int v = 0; v < 6; v++) fc[(4 + v) * n + q] = fm.m.g[v];
  fc[10 * n + q] = fm.m.sdet;
  fc[11 * n + q] = fm.m.isdet;
  fc[12 * n + q] = fm.m.gi[gd];
}
// Only gamma^{dd} of the inverse is loaded: it is the one face_side reads.
template <int d>
__device__ __forceinline__ void fmc_load(const double* __restrict__ fc, long long n, long long q, FaceMetric& fm) {
  constexpr int gd = d == 0 ? 0 : (d == 1 ? 3 : 5);
  fm.alpha = fc[q];
#pragma unroll
  for (int a = 0; a < 3; a++) fm.beta[a] = fc[(1 + a) * n + q];
#pragma unroll
  for (int v = 0; v < 6; v++) fm.m.g[v] = fc[(4 + v) * n + q];
  fm.m.sdet = fc[10 * n + q];
  fm.m.isdet = fc[11 * n + q];
  fm.m.gi[gd] = fc[12 * n + q];
}

// Flux through one face from its reconstructed (unfloored) states.
template <int d, int E = 0>
__device__ __forceinline__ void face_flux_states(const Par& P, double* L, double* R, double Bn, const FaceMetric& fm,
                                                 double* F) {
  double cl[3], cr[3];
  face_floor<E>(P, L, cl);
  face_floor<E>(P, R, cr);
  Side sl, sr;
  face_side<d, E>(P, L, Bn, fm, sl, cl);
  face_side<d, E>(P, R, Bn, fm, sr, cr);
  riemann<d>(P.rsolver, fm, Bn, sl, sr, F);
}

// SSP-RK weights (g0, g1, beta) of a stage: U <- g0 U^n + g1 U + beta dt L(U)
__host__ __device__ inline void rk_weights(int order, int stage, double& g0, double& g1, double& be) {
  if (order == 2) {
    if (stage == 0) { g0 = 0.0; g1 = 1.0; be = 1.0; }
    else { g0 = 0.5; g1 = 0.5; be = 0.5; }
  } else {
    if (stage == 0) { g0 = 0.0; g1 = 1.0; be = 1.0; }
    else if (stage == 1) { g0 = 0.75; g1 = 0.25; be = 0.25; }
    else { g0 = 1.0 / 3.0; g1 = 2.0 / 3.0; be = 2.0 / 3.0; }
  }
}

// Warp-level sum of per-thread counters, one atomic per warp.  Call where the
// whole warp has converged (end of a kernel; blockDim a multiple of 32).
__device__ __forceinline__ void warp_flush(unsigned long long* ctr, unsigned v) {
  unsigned s = __reduce_add_sync(0xffffffffu, v);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(ctr, (unsigned long long)s);
}
// Interior cell (block bi, k, j, i) of item `it` of the interior-cell work
// list (W_CELL, x fastest).
__device__ __forceinline__ void fofc_cell(const Work& w, long long it, int& bi, int& k, int& j, int& i) {
  const long long* pre = w.pre + (long long)W_CELL * (w.nblocks + 1);
  bi = find_block(w, W_CELL, it);
  const DevBlock& b = w.blk[bi];
  long long loc = it - pre[bi];
  i = loc % b.n[0]; long long r = loc / b.n[0]; j = r % b.n[1]; k = r / b.n[1];
  i += b.ng; j += b.ng; k += b.ng;
}
// Marks the solve's work list as non-empty when any lane of the warp gave a
// cell status 0 (every lane of the warp calls it).
__device__ __forceinline__ void warp_mark_solve(const KrpBuf& kb, bool any0) {
  if (__any_sync(0xffffffffu, any0) && (threadIdx.x & 31) == 0) kb.ctr[1] = 1ull;
}

}  // namespace grmhd
