/*
 * libgrmhd — GB300 (sm_103a) Valencia GRMHD meshblock right-hand side and
 * update in a 3+1 metric, after arXiv:2409.10384 (AthenaK, Sec. 2-3).
 *
 * All state arrays are caller-owned DEVICE memory (e.g. torch tensors), FP64,
 * structure-of-arrays, ghost-inclusive, index [var][k][j][i] with i fastest:
 *   N_d = n_d + 2*ng,  cell (k,j,i) at offset (k*N2 + j)*N1 + i.
 * Face arrays hold the densitised field B~ = sqrt(gamma) B on the low face of
 * each index: x [N3][N2][N1+1], y [N3][N2+1][N1], z [N3+1][N2][N1].
 * Edge arrays (vector potential in mhd_init_block): A_x at (i, j-1/2, k-1/2)
 * [N3+1][N2+1][N1], A_y at (i-1/2, j, k-1/2) [N3+1][N2][N1+1], A_z at
 * (i-1/2, j-1/2, k) [N3][N2+1][N1+1].
 *
 * Errors: every entry point returns 0 on success or a negative MHD_E* code;
 * mhd_strerror() names it.  Per-cell con2prim failures are not errors: they
 * set flag bits and count in mhd_stats (the FOFC of Sec. 3.3 consumes them).
 * Calls are asynchronous on the given cudaStream_t (passed as void*; NULL =
 * legacy default stream) unless stated otherwise.  No call allocates device
 * memory except mhd_init (context), the first call that sees a new block list
 * (scratch sized for it) and mhd_mlp_train (training buffers).
 */
#ifndef GRMHD_H
#define GRMHD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mhd_ctx mhd_ctx; /* opaque; owns scratch only, never state */

/* Error codes. */
#define MHD_OK 0
#define MHD_EINVAL (-1)    /* bad argument (NULL pointer, size, parameter) */
#define MHD_ECUDA (-2)     /* a CUDA runtime call failed */
#define MHD_ENOMEM (-3)    /* scratch allocation failed */
#define MHD_ESTATE (-4)    /* call out of order (e.g. rk_update before rhs) */
#define MHD_ENOMLP (-5)    /* learned guess requested but no network loaded */
#define MHD_ETOOBIG (-6)   /* block too large for mhd_stage_noalloc's static scratch */

/* Per-cell flag bits written to mhd_block.flags (and mhd_c2p_cells). */
#define MHD_F_FAIL 1u      /* root solve failed: cell reset to atmosphere */
#define MHD_F_DFLOOR 2u    /* D < f_thr*rho_atm before the solve (Sec. 3.3) */
#define MHD_F_SIGMA 4u     /* B^2/D cap applied (Sec. 3.3) */
#define MHD_F_TAU 8u       /* tau < tau_atm(D,B) (Sec. 3.3) */
#define MHD_F_RHO 16u      /* rho < f_thr*rho_atm after the solve */
#define MHD_F_TEMP 32u     /* temperature floor T_atm */
#define MHD_F_VMAX 64u     /* Lorentz-factor cap W_max active */
#define MHD_F_FOFC 128u    /* FOFC recomputed this cell's faces (Sec. 3.3) */

/* Method parameters (Sec. 3.2-3.4).  Units G = c = 1, m_b = 1: T = P/rho. */
typedef struct {
  double gamma;     /* ideal-gas index, P = (gamma-1) rho eps (Sec. 3.4) */
  double rho_atm;   /* atmosphere density (Sec. 3.3) */
  double T_atm;     /* atmosphere temperature (Sec. 3.3) */
  double f_thr;     /* floor threshold factor: rho < f_thr*rho_atm (Sec. 3.3) */
  double sigma_max; /* cap on B^2/D; <= 0 disables (Sec. 3.3) */
  double dmp_M;     /* relaxed DMP factor M >= 1 (Eq. 19); <= 0 disables */
  double c2p_tol;   /* relative width of the final root bracket (1e-10) */
  double W_max;     /* Lorentz-factor cap of the root solve (1e3) */
  double alpha_exc; /* excision (Sec. 4.7): block con2prims floor every cell whose
                       lapse is below alpha_exc to the static atmosphere (reported
                       as F_DFLOOR); <= 0 disables */
  int recon;        /* 0 donor cell, 1 PLM (van Leer), 2 WENO-Z, 3 PPM4 (Colella &
                       Woodward 1984), 4 PPMX (Colella & Sekora 2008) (Sec. 3.2) */
  int rsolver;      /* 0 LLF, 1 HLLE (Sec. 3.2) */
  int fofc;         /* 1: first-order flux correction (Sec. 3.3) */
  int rk_order;     /* 2 or 3: SSP-RK (Sec. 3.2) */
  int c2p_maxit;    /* cap on root-solve iterations (64) */
  int c2p_guess;    /* root search of every con2prim (cells, stage input, FOFC U*):
                       0 FP64 Illinois on the plain bracket [0, mu+];
                       1 network guess of log(mu), FP32 secant steps, then the
                         FP64 polish: two FP64 evaluations of f (a Newton step
                         with the FP32 slope, then the FP64 secant), whose
                         result is the root when both steps contracted
                         (|m1 - m0| <= 2^-16 m0, |m2 - m1| <= 2^-30 m2), else
                         a bracket for the FP64 Illinois solve (needs a network:
                         MHD_ENOMLP otherwise);
                       2 as 1 but the FP32 steps start from [0, mu+];
                       3 block con2prims: FP64 bracket of relative half-width
                         1e-3 around the cell's root of the last stage-input
                         con2prim (verified by the signs at both ends, else
                         the plain bracket); the FOFC estimate starts from the
                         same root.  A new block list starts without roots.
                       Every mode finds the same root of f in FP64 (modes 1, 2
                       within the rounding of f; not bit-identical to 0). */
  int eos;          /* 0: ideal gas, P = (gamma-1) rho eps, T = P/rho.
                       1: hybrid piecewise polytrope (Sec. 3.4 names it as
                       PrimitiveSolver's second analytic EOS): a cold part
                       P_c = K_i rho^eos_gamma[i] on eos_pieces (1..4) pieces
                       split at the increasing densities eos_rho[0..pieces-2],
                       with K_0 = eos_K0, the other K_i from the continuity of
                       P_c and eps_c = a_i + K_i rho^(G_i-1)/(G_i-1) continuous
                       (a_0 = 0); plus a thermal ideal gas
                       P_th = (eos_gamma_th - 1) rho (eps - eps_c).  T = P_th/rho
                       (the floors: P >= P_c + rho T_atm).  gamma is unused;
                       c2p_guess 1 and 2 need eos = 0 (MHD_EINVAL otherwise). */
  int eos_pieces;   /* 1..4 (eos = 1) */
  double eos_K0;    /* K of the lowest-density piece (> 0) */
  double eos_gamma_th;  /* thermal index (> 1) */
  double eos_rho[3];    /* dividing densities, increasing, > 0 */
  double eos_gamma[4];  /* piece indices (> 1) */
  int fixed_metric;     /* 1: a fixed spacetime (the Cowling runs of Sec. 4.4: the
                           metric is not evolved): the caller keeps the ADM arrays
                           unchanged between mhd_step calls, so the step's metric
                           cache is computed once per block list and reused by
                           later steps (a new block list recomputes it; mhd_c2p
                           still recomputes it every call).  0: every mhd_step
                           recomputes it from the ADM arrays. */
} mhd_params;

/* One meshblock: views into caller-owned device arrays. */
typedef struct {
  int n[3];            /* interior cells (x, y, z); each >= 1 */
  int ng;              /* ghost cells per side; must be >= 4 */
  double dx[3];        /* cell widths */
  double* cons;        /* [5] D~, S~_1, S~_2, S~_3, tau~ (Eq. 6, densitised) */
  double* cons0;       /* [5] U^n of the RK step; written by stage 0 */
  double* prim;        /* [5] rho, w^i = W v^i, P; written by mhd_c2p */
  double* bf[3];       /* face B~ (layout above) */
  double* bf0[3];      /* face B~ at t^n; written by stage 0 */
  double* bcc;         /* [3] cell-centred B~ (face average); written by mhd_c2p */
  const double* adm;   /* [16] alpha, beta^1..3, gamma_11,12,13,22,23,33, K_11..K_33 (Eq. 5, 9) */
  unsigned char* flags;/* [N3][N2][N1] MHD_F_* bits */
} mhd_block;

/* Counters accumulated on the device since the last mhd_reset_stats. */
typedef struct {
  long long cells;      /* con2prim solves on stage inputs */
  long long iters;      /* FP64 evaluations of the master function in those
                           solves (bracket, polish and root iteration; the FOFC
                           estimate's solves are not counted) */
  long long fails;      /* failures (MHD_F_FAIL) */
  long long floors;     /* cells where a floor fired */
  long long fofc_cells; /* cells flagged by FOFC (incl. DMP) */
  long long dmp_cells;  /* cells flagged by the DMP test */
  long long fofc_faces; /* faces recomputed at first order */
  long long guess_fallbacks; /* c2p_guess 1, 2: cells whose FP64 polish was not
                                taken as the root (the FP64 solve then runs from
                                the bracket its two evaluations give) */
  long long fp32_evals; /* FP32 evaluations of the master function in the
                           searches of c2p_guess 1, 2 (the two starting points,
                           one per secant step, two for the slope) and in the
                           FP32 decisions of the FOFC estimate (every mode) */
  long long fofc_fp32;  /* FOFC estimate cells (and cells of a flags-only
                           mhd_c2p_cells) whose flag was decided from FP32
                           interval enclosures, without an FP64 evaluation of
                           the master function (ideal gas) */
} mhd_stats;
#define MHD_NSTATS 10

/* Create a context on the current device.  *out receives it.  Copies p. */
int mhd_init(const mhd_params* p, mhd_ctx** out);
/* Replace the parameters (validated as in mhd_init). */
int mhd_set_params(mhd_ctx* ctx, const mhd_params* p);
/* Free the context and all its scratch (synchronises the device). */
void mhd_finalize(mhd_ctx* ctx);
const char* mhd_strerror(int code);

/* Initial data: face B~ = discrete curl of the edge potential A (so div B~ = 0
 * to round-off, Sec. 4.3), bcc = face average, cons = Eq. 6 of blk->prim on
 * every cell.  A[c] are device arrays in the edge layout above. */
int mhd_init_block(mhd_ctx* ctx, mhd_block* blk, const double* const A[3], void* stream);

/* Eq. 6 on n independent cells: prim [5][n], Bd [3][n] (densitised),
 * g [6][n] (gamma_ij) -> cons [5][n].  Device pointers. */
int mhd_prim2cons(mhd_ctx* ctx, long n, const double* prim, const double* Bd, const double* g, double* cons,
                  void* stream);

/* con2prim (Sec. 3.4, Kastaun et al. 2021 bracketed root) with the atmosphere
 * floors of Sec. 3.3 on n independent cells.  cons [5][n] is overwritten where
 * a floor changed it; prim [5][n] and flags [n] are written; iters [n] (may be
 * NULL) receives the FP64 evaluations of the master function per cell.
 * Device pointers.  stats (host, may be NULL): the counters this call added
 * (cells, iters, fails, floors, guess_fallbacks, fp32_evals); a non-NULL stats
 * makes the call synchronise the stream (before and after its launches).
 * prim = NULL asks only the question of the FOFC estimate (Sec. 3.3): flags[c]
 * = 1 where con2prim of the cell fails or a floor fires, else 0; cons is not
 * written.  With the ideal gas most cells are then decided from FP32 interval
 * enclosures, which contain the exact values, without FP64 work (stats:
 * fofc_fp32; iters 0 for them); the others take the FP64 con2prim.  The
 * flagged cells are counted in fofc_cells (fails and floors are not). */
int mhd_c2p_cells(mhd_ctx* ctx, long n, double* cons, const double* Bd, const double* g, double* prim,
                  unsigned char* flags, int* iters, void* stream, mhd_stats* stats);

/* con2prim of every cell within 3 of the interior of each block (the stencil
 * region of WENO-Z), with bcc and the cell-centred EMF; floors write back to
 * cons.  This is step 1 of a stage.  It also keeps sqrt(gamma), 1/sqrt(gamma)
 * and gamma^ij of every cell in context scratch for steps 2-5 of the same
 * stage, so the ADM arrays must not change between mhd_c2p and mhd_rk_update
 * of one stage (the metric is an input of the whole stage; it first computes
 * the cell and face metric of the stage into context scratch, which the
 * fluxes, the FOFC estimate and the update read).  stats (host,
 * may be NULL): the counters this call added, as in mhd_c2p_cells (the call
 * then synchronises the stream). */
int mhd_c2p(mhd_ctx* ctx, const mhd_block* blocks, int nblocks, void* stream, mhd_stats* stats);

/* Steps 2-4 of stage `stage` (0-based) with time step dt: reconstruction and
 * Riemann fluxes (Eq. 8) on every face the update needs, FOFC (+DMP) and the
 * upwind-CT edge EMFs, all into context scratch.  Requires mhd_c2p. */
int mhd_rhs(mhd_ctx* ctx, const mhd_block* blocks, int nblocks, double dt, int stage, void* stream);

/* Step 5: U <- g0 U^n + g1 U + b dt (-div F + G) (Eq. 9 sources), face B~ <-
 * g0 B^n + g1 B - b dt curl E, with the SSP-RK weights of `stage`.  Stage 0
 * also stores U and face B~ as U^n.  Requires mhd_rhs on the same blocks. */
int mhd_rk_update(mhd_ctx* ctx, const mhd_block* blocks, int nblocks, double dt, int stage, void* stream);

/* A full RK step (rk_order stages of c2p, rhs, update).  The ADM variables are
 * an input of the whole step: their cell and face metric is computed once,
 * before the first stage, and every stage reads it.  Ghost zones are not
 * refreshed between stages (they keep their values).  graph = 0: each kernel
 * launched once per stage over all blocks; 1: the same launches captured once
 * into a CUDA graph per (block list, dt, parameters, stream) and replayed (the
 * stream must not be the legacy default stream); 2: one launch sequence per
 * block (a reference for the batched launches; same results). */
int mhd_step(mhd_ctx* ctx, const mhd_block* blocks, int nblocks, double dt, int graph, void* stream);
/* The captured full RK step: mhd_step with graph = 1 (one CUDA graph of all
 * rk_order stages per block list, dt, parameters and stream, replayed on
 * later calls; stream must not be the legacy default stream). */
int mhd_graph_step(mhd_ctx* ctx, const mhd_block* blocks, int nblocks, double dt, void* stream);
/* mhd_step with graph = 0 whose stages wait for the CUDA event state_ready
 * (a cudaEvent_t, recorded by the caller after its copies of the blocks'
 * state, cons and face B~; NULL: no wait).  The step first enqueues its
 * metric kernel, which reads only the ADM arrays, and then the wait: a caller
 * that copies the state in on another stream overlaps those copies with the
 * metric computation.  Not in the paper's hot path; its introduction (Sec. 1)
 * motivates overlapping transfers with computation.  Same results as
 * mhd_step.  Errors as mhd_step (MHD_ECUDA if the wait cannot be enqueued). */
int mhd_step_overlap(mhd_ctx* ctx, const mhd_block* blocks, int nblocks, double dt, void* stream,
                     void* state_ready);

/* Autotuner for a block list: times each tunable kernel (the two con2prim
 * phases, the three flux directions, the two FOFC-estimate phases, the EMF
 * and the cell update) at CTA sizes 64/128/256 and 1/2/4 waves of resident
 * CTAs on these blocks and keeps the fastest for later launches of this
 * context.  It runs con2prim (which applies the floors to cons, as the first
 * step of a stage does) and the right-hand side of stage 0; the state is
 * otherwise unchanged.  cfg_out (host, may be NULL): [MHD_NTUNE][2] CTA size
 * and waves.  Synchronises the stream. */
#define MHD_NTUNE 9
int mhd_autotune(mhd_ctx* ctx, const mhd_block* blocks, int nblocks, double dt, void* stream, int* cfg_out);

/* Pin the launch shape of one tunable kernel (kind in the order of
 * mhd_autotune's output, 0 .. MHD_NTUNE-1): threads per CTA (64, 128 or 256)
 * and waves (1 .. 64; the grid is at most waves x resident CTAs per SM x SMs).
 * The arithmetic of a cell or face does not depend on the launch shape.
 * MHD_EINVAL on a bad kind or shape; a cached CUDA graph is dropped. */
int mhd_set_launch(mhd_ctx* ctx, int kind, int threads, int waves);
/* Current launch shape of a tunable kernel. */
int mhd_get_launch(const mhd_ctx* ctx, int kind, int* threads, int* waves);

/* Self-check of the library's fast reciprocal (the paper has no counterpart).
 * The hot divisions (the master function of con2prim, its regula-falsi step,
 * the WENO-Z weights and the HLLE speeds) multiply by an approximate FP64
 * reciprocal refined by two Newton-Raphson steps, within ~1 ulp of the
 * correctly rounded quotient.  For n device values x (normal, nonzero),
 * rel_out[2i] and rel_out[2i+1] (device) receive the relative differences of
 * 1 * r(x) and (x + 1) * r(x) from the correctly rounded 1/x and (x + 1)/x. */
int mhd_check_rcp(const double* x, long n, double* rel_out, void* stream);

/* Self-check of the FP32 enclosures (interval arithmetic with outward
 * rounding) from which the FOFC estimate decides its flags (Sec. 3.3; the
 * paper has no counterpart).  For n device values x, miss_out[i] (device)
 * receives 0 when every enclosure of x and of y = x[(i + 1) % n] contains the
 * FP64 value it encloses: x itself, 1/|x|, 1/sqrt(|x|), x y, x |y|, x^2,
 * x + y and x - y; else a bit per miss (1, 2, 4, 8, 16, 32, 64 in that
 * order).  Values whose FP32 image is not a normal float check x only, and an
 * empty (NaN) enclosure, which decides nothing, counts as enclosing. */
int mhd_check_enclosures(const double* x, long n, unsigned char* miss_out, void* stream);

/* Copy the counters to *out (synchronises the stream) / zero them. */
int mhd_read_stats(mhd_ctx* ctx, mhd_stats* out, void* stream);
int mhd_reset_stats(mhd_ctx* ctx, void* stream);

/* Copy a scratch array of block b of the last block list into dst (device or
 * host memory, count elements; count must equal the array size, which
 * count == 0 queries into *size).  which = 0..2: face fluxes of direction
 * x, y, z ([7][face array]: D~, S~_1..3, tau~, then B~ of the transverse
 * directions (d+1)%3 and (d+2)%3); 3..5: edge EMFs E_x, E_y, E_z (edge layout
 * above).  Synchronises the stream. */
int mhd_scratch_copy(mhd_ctx* ctx, int b, int which, double* dst, long count, long* size, void* stream);

/* Kernel launches this context has issued so far (a graph replay counts the
 * kernels it contains). */
long long mhd_kernel_launches(const mhd_ctx* ctx);

/* Baryon-mass ledger (a diagnostic, off by default).  The paper reports
 * baryon-mass conservation to ~1e-11 through collapse (Sec. 4); with the
 * ledger on, every RK stage folds, per block, the interior D~ dV that the
 * stage's con2prim floors wrote (weight 1 in the first stage, where it becomes
 * part of U^n, else the stage weight b_s) and -dt b_s times the outward D~ flux
 * through the block's interior boundary (after FOFC), integrated over the face
 * areas, into a running balance.  b_s = (1/6, 1/6, 2/3) for SSP-RK3 and
 * (1/2, 1/2) for RK2: the weights with which each stage's L(U) enters
 * U^{n+1}.  Over full steps, mass(after) - mass(before) - balance is then the
 * round-off of the update alone.
 * mhd_ledger: switch on/off; the next call re-plans the scratch, and a new
 * block list starts from a zero balance.
 * mhd_ledger_read: host out[nblocks] = the balance of each block of the last
 * list since the last reset (reset != 0 zeroes it).  MHD_ESTATE when the
 * ledger is off or no list was run.  Synchronises the stream.
 * mhd_block_mass: host out[nblocks] = sum over interior cells of D~ dx dy dz.
 * Synchronises the stream. */
int mhd_ledger(mhd_ctx* ctx, int enable);
int mhd_ledger_read(mhd_ctx* ctx, double* out, int reset, void* stream);
int mhd_block_mass(mhd_ctx* ctx, const mhd_block* blocks, int nblocks, double* out, void* stream);

/* Ghost zones of the blocks of a list from same-level neighbours: copies, no
 * prolongation or restriction.  The paper's AMR driver fills them with
 * prolongation and restriction at level changes (Sec. 2); that part is not
 * here.  nbr: host int [nblocks][6], the neighbour across each side, in the
 * order -x, +x, -y, +y, -z, +z:
 *   >= 0  a block of the list (same n and ng, and at least ng cells along
 *         that axis; periodic wrap: the block across the domain, or the
 *         block itself, which wraps modulo n for any n);
 *   -1    zero-gradient outflow: copies of the block's own boundary layer;
 *   -2    leave these ghosts untouched.
 * The fill runs along x, then y, then z, each pass over the whole extent of
 * the other axes (ghosts included), so edges and corners combine the sides'
 * rules (e.g. outflow along x and periodic along y).  Fills cons and the
 * three face-field arrays (not cons0/bf0/prim: con2prim recomputes prim and
 * bcc on the ghost layers it needs).  MHD_EINVAL on a bad entry or a
 * neighbour of another size.  Asynchronous on the stream; nbr may be reused
 * after return. */
int mhd_fill_ghosts(mhd_ctx* ctx, const mhd_block* blocks, int nblocks, const int* nbr, void* stream);

/* Kernel kinds for per-kernel timing. */
#define MHD_K_C2P 0        /* con2prim of the stencil region (prep + finish) */
#define MHD_K_FLUX_X 1     /* reconstruction + Riemann flux, x faces */
#define MHD_K_FLUX_Y 2
#define MHD_K_FLUX_Z 3
#define MHD_K_FOFC_FLAG 4  /* FOFC estimate U*, its con2prim prep + finish, DMP */
#define MHD_K_FOFC_FIX 5   /* first-order recompute of flagged faces */
#define MHD_K_EMF 6        /* upwind CT edge EMFs */
#define MHD_K_UPDATE 7     /* RK update of U with the Eq. 9 sources */
#define MHD_K_FACEB 8      /* RK update of the face B~ */
#define MHD_K_SOLVE 9      /* con2prim root solves (stage input and U*) */
#define MHD_K_MLP 10       /* learned guess: network inference fused with the
                              FP32 search and the FP64 polish (c2p_guess 1;
                              c2p_guess 2 runs its search and polish in the
                              prep, under MHD_K_C2P) */
#define MHD_K_LEDGER 11    /* baryon-mass ledger (only with mhd_ledger on) */
#define MHD_K_METRIC 12    /* the step's metric: sqrt(gamma), gamma^ij of the con2prim
                              region and the interpolated face metric (Eq. 8) of
                              every swept face, once per RK step (mhd_step) or
                              per mhd_c2p */
#define MHD_NKERNEL 13

/* enable != 0: bracket every kernel launched outside stream capture by CUDA
 * events on its own stream.  mhd_profile_read waits for them and returns, per
 * kind, the summed milliseconds (ms[MHD_NKERNEL]) and launch counts
 * (count[MHD_NKERNEL]) since the previous read. */
int mhd_profile(mhd_ctx* ctx, int enable);
int mhd_profile_read(mhd_ctx* ctx, double* ms, long long* count);
const char* mhd_kernel_name(int kind);

/* Learned con2prim guess (not in the paper; an addition of this library).
 * A 5 -> 64 -> 64 -> 1 tanh network with BF16 operands and FP32
 * accumulation on the tensor cores predicts log(mu) of the Kastaun et al. root
 * from five features of the cell's KRP variables; with mhd_params.c2p_guess = 1
 * every con2prim starts FP32 secant steps at the guess (second point at
 * exp(delta) x guess) and polishes their result in FP64 (c2p_guess above):
 * the same root, with fewer FP32 steps than from the plain bracket.
 * Features: float [n][MHD_MLP_FSTRIDE] (5 used); targets: float log(mu) [n].
 * State (get/set): MHD_MLP_NPARAM fp32 parameters (W1 [64][5], b1, W2
 * [64][64], b2, w3, b3), then feature mean [5], feature 1/std [5], target
 * mean, target std, delta.  Device pointers unless stated. */
#define MHD_MLP_NPARAM 4609
#define MHD_MLP_NSTATE (4609 + 13)
#define MHD_MLP_FSTRIDE 8
/* Allocate the network state and draw Glorot-uniform weights (seed). */
int mhd_mlp_init(mhd_ctx* ctx, unsigned long long seed);
/* Plain con2prim of n cells -> features and log(mu) of the root (training data). */
int mhd_mlp_dataset(mhd_ctx* ctx, long n, const double* cons, const double* Bd, const double* g, float* feat,
                    float* logmu, void* stream);
/* Normalise, then Adam (cosine-decayed lr) over `epochs` passes of shuffled
 * mini-batches, forward and backward on the tensor cores.  *loss_out: mean
 * squared error (normalised units) of the last epoch.  Synchronises. */
int mhd_mlp_train(mhd_ctx* ctx, const float* feat, const float* logmu, long n, int epochs, int batch, float lr,
                  unsigned long long seed, float* loss_out, void* stream);
/* delta = the `quantile` of |predicted - true log(mu)| on the given samples;
 * enables the learned guess.  Synchronises. */
int mhd_mlp_calibrate(mhd_ctx* ctx, const float* feat, const float* logmu, long n, double quantile,
                      double* delta_out, void* stream);
/* Predicted log(mu) of n samples. */
int mhd_mlp_infer(mhd_ctx* ctx, const float* feat, long n, float* logmu_out, void* stream);
/* Gradient (grad_out[MHD_MLP_NPARAM], device or host) and loss of the mean
 * squared error over n samples in normalised units.  Synchronises. */
int mhd_mlp_grad(mhd_ctx* ctx, const float* feat, const float* logmu, long n, float* grad_out, float* loss_out,
                 void* stream);
/* Copy the state out / in (host arrays of MHD_MLP_NSTATE floats). */
int mhd_mlp_get(mhd_ctx* ctx, float* state);
int mhd_mlp_set(mhd_ctx* ctx, const float* state);
/* The trained network as a BF16 weight blob (host memory, little-endian):
 * MHD_MLP_NPARAM bf16 parameters in the order of mhd_mlp_get, then the 13
 * fp32 values that follow them there (feature mean, feature 1/std, target
 * mean and std, delta); MHD_MLP_BLOB_BYTES in all.  mhd_mlp_save writes it
 * (bytes must be at least MHD_MLP_BLOB_BYTES; size, may be NULL, receives the
 * length).  mhd_mlp_load reads one (bytes must equal MHD_MLP_BLOB_BYTES,
 * else MHD_EINVAL) into the context: the parameters become the fp32 master
 * weights and the tensor-core operands, and the guess is enabled when delta
 * > 0.  Inference runs on bf16 operands, so a loaded blob predicts what the
 * saved network predicted.  Synchronise the device. */
#define MHD_MLP_BLOB_BYTES (2 * 4609 + 4 * 13)
int mhd_mlp_save(mhd_ctx* ctx, void* blob, long bytes, long* size);
int mhd_mlp_load(mhd_ctx* ctx, const void* bf16_weights, long bytes);

/* Allocation-free stage (the paper has no counterpart: this serves callers).
 * Some callers cannot let a library allocate device memory: a host code that
 * gives its whole GPU memory budget to its own pool allocator, one that cannot
 * accept the device-wide synchronisation a cudaFree implies inside a time
 * step, or one with nowhere to keep a library context.  mhd_stage_noalloc runs
 * one RK stage (`stage`, 0-based, of p->rk_order) of ONE block -- con2prim,
 * fluxes, FOFC, CT EMFs and the update, with the results of mhd_c2p +
 * mhd_rhs + mhd_rk_update (the same flux, CT and update kernels; its
 * con2prim and FOFC estimate run one thread per cell, which needs no solve
 * scratch, where the context path uses its three-phase kernels) -- with no
 * context and without calling cudaMalloc, cudaFree or any allocating
 * routine.  Its scratch is a
 * file-scope device array of MHD_NOALLOC_SCRATCH_BYTES (16 MiB), held by
 * every GPU that loads the library until the process exits; a block whose
 * scratch does not fit (e.g. interior larger than 32^3 with 4 ghosts) is
 * rejected with MHD_ETOOBIG before any device work.  The caller still owns
 * every state array of `blk` (device memory).  The first call on a device,
 * with that device current, looks up the array's device address; make that
 * first call before any stream capture.  All calls share the array and it
 * keeps the last call's contents: calls whose kernels overlap on the GPU
 * race.  p->c2p_guess must be 0.  Counters are not reported.  A launch error
 * already pending from the caller's earlier work is returned as MHD_ECUDA
 * before any launch (and left pending); otherwise MHD_ECUDA reports a failed
 * launch of this call. */
#define MHD_NOALLOC_SCRATCH_BYTES (16u << 20)
int mhd_stage_noalloc(const mhd_params* p, const mhd_block* blk, double dt, int stage, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GRMHD_H */
