// Host-side launchers shared between the kernel translation units and the C-ABI.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include "dev.cuh"
#include "grmhd.h"

namespace grmhd {
// mhd_params -> kernel constants, with validation (api.cu); allow_guess: accept
// c2p_guess 1-3 (the allocation-free path takes 0 only)
int fill_par(const mhd_params* p, Par& P, bool allow_guess);
void launch_init_block(const DevBlock& b, const Par& P, const double* const A[3], cudaStream_t s, int nsm);
void launch_p2c_cells(const Par& P, long long n, const double* prim, const double* Bd, const double* g, double* cons,
                      cudaStream_t s, int nsm);
void launch_c2p_cells(const Par& P, long long n, double* cons, const double* Bd, const double* g, double* prim,
                      unsigned char* flags, int* iters, const float* guess, unsigned long long* stats, cudaStream_t s,
                      int grid);
void launch_c2p_block(const Work& w, const Par& P, unsigned long long* stats, cudaStream_t s, int grid);
// flux sweeps reading the face metric cache (context path) / computing the
// face metric in the sweep (allocation-free stage)
void launch_flux_dir(int d, const Work& w, const Par& P, cudaStream_t s, int grid, int threads = 128);
void launch_flux_dir_inline(int d, const Work& w, const Par& P, cudaStream_t s, int grid, int threads = 128);
// metric of a step: cell cache (mc) of the con2prim region, face cache (fmc)
void launch_metric_cache(const Work& w, cudaStream_t s, int grid);
int occ_metric_kernel();
// the fast reciprocal (rcp_nr) against the correctly rounded division
void launch_check_rcp(const double* x, long long n, double* out, cudaStream_t s, int nsm);
void launch_check_iv(const double* x, long long n, unsigned char* out, cudaStream_t s, int nsm);
void launch_fofc_flag(const Work& w, const Par& P, double g0, double g1, double bdt, unsigned long long* stats,
                      cudaStream_t s, int grid);
void launch_fofc_fix(int d, const Work& w, const Par& P, unsigned long long* stats, cudaStream_t s, int grid);
// the flagged cells' faces from the list k_krp_finish_fofc keeps (list[0]
// entries of at most cap)
void launch_fofc_fix_list(const Work& w, const Par& P, const unsigned long long* list, long long cap,
                          unsigned long long* stats, cudaStream_t s, int grid);
void launch_emf(const Work& w, cudaStream_t s, int grid, int threads = 128);
void launch_update_cells(const Work& w, const Par& P, double g0, double g1, double bdt, int first, cudaStream_t s,
                         int grid, int threads = 128);
// baryon-mass ledger: fold the floor mass of the last con2prim (weight wF)
// and -dtb x the outward boundary D~ flux of the stage into each block's
// balance; interior mass sum D~ dV of each block into out[id]
void launch_fill_ghosts(const Work& w, const int* nbr, int kind, int ax, cudaStream_t s, int grid);
void launch_ledger_stage(const Work& w, double wF, double dtb, cudaStream_t s);
void launch_block_mass(const Work& w, double* out, cudaStream_t s);
void launch_update_faces(const Work& w, double g0, double g1, double bdt, int first, cudaStream_t s, int grid);
size_t krp_bytes(long long n);
KrpBuf krp_view(void* base, long long n);
// mode: the prep's con2prim start (0 plain bracket, 1 status 4 for the seed
// kernel's network, 2 FP32 search and FP64 polish); stats: the context's
// counters (mode 2 adds its FP32 evaluations and polish fallbacks)
void launch_krp_prep_block(const Work& w, const Par& P, const KrpBuf& kb, unsigned long long* stats, cudaStream_t s,
                           int grid, int threads = 128, int mode = 0, float* feat = nullptr);
void launch_krp_solve(const Par& P, const KrpBuf& kb, cudaStream_t s, int grid);
// inl: the finish solves status-0 cells itself (no solve launch before it)
void launch_krp_finish_block(const Work& w, const Par& P, const KrpBuf& kb, unsigned long long* stats,
                             cudaStream_t s, int grid, int threads = 128, bool inl = false);
void launch_krp_prep_fofc(const Work& w, const Par& P, double g0, double g1, double bdt, const KrpBuf& kb,
                          unsigned long long* stats, cudaStream_t s, int grid, int threads = 128, int mode = 0,
                          float* feat = nullptr);
void launch_krp_finish_fofc(const Work& w, const Par& P, const KrpBuf& kb, unsigned long long* stats,
                            cudaStream_t s, int grid, int threads = 128, bool inl = false);
// fonly: flags only (the FOFC estimate's question, no recovery written; the
// finish then gets prim = null)
void launch_krp_prep_cells(const Par& P, const KrpBuf& kb, const double* cons, const double* Bd, const double* g,
                           int mode, float* feat, unsigned long long* stats, cudaStream_t s, int grid,
                           bool fonly = false);
void launch_krp_finish_cells(const Par& P, const KrpBuf& kb, double* cons, const double* Bd, const double* g,
                             double* prim, unsigned char* flags, int* iters, unsigned long long* stats, cudaStream_t s,
                             int grid);
// per_sm[8]: prep / solve / finish of the block, prep / finish of the FOFC
// estimate, prep / finish of independent cells, the flags-only cell prep
int occupancy_krp(int* per_sm);
int mlp_setup_attrs();
void launch_mlp_infer(const float* feat, long long n, const MlpNorm& nm, const __nv_bfloat16* wb, const float* w,
                      float* out, cudaStream_t s, int nsm);
void launch_mlp_train_step(const float* feat, const float* target, long long n, long long pa, long long pb,
                           long long off, int batch, const MlpNorm& nm, const __nv_bfloat16* wb, const float* w,
                           float* grad, float* loss, cudaStream_t s);
void launch_mlp_adam(float* w, float* m, float* v, float* grad, float lr, int t, __nv_bfloat16* wb, cudaStream_t s);
void launch_mlp_pack(const float* w, __nv_bfloat16* wb, cudaStream_t s);
void launch_mlp_logmu(const KrpBuf& kb, float* out, cudaStream_t s, int nsm);
void launch_mlp_stats(const float* feat, const float* target, long long n, double* acc, cudaStream_t s, int nsm);
// Network guess (inferred in the kernel; wb, w, nm: its operands), FP32
// search and FP64 polish of every status-4 cell
void launch_krp_seed(const Par& P, const KrpBuf& kb, float delta, const __nv_bfloat16* wb, const float* w,
                     const MlpNorm& nm, unsigned long long* stats, cudaStream_t s, int grid);
int occ_seed_kernel();
int occupancy_c2p(int* per_sm);
int occ_face_kernel(int kind, int threads);
int occ_krp_kernel(int kind, int threads);
int occ_update_kernel(int kind, int threads);
int occupancy_face(int* per_sm);
int occupancy_update(int* per_sm);
}  // namespace grmhd
