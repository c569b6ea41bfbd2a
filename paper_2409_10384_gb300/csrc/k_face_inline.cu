// The flux sweeps with the face metric computed in the sweep (no cache): the
// allocation-free stage's flux kernels (flux_sweep.cuh).
#include "flux_sweep.cuh"
#include "internal.h"

namespace grmhd {

void launch_flux_dir_inline(int d, const Work& w, const Par& P, cudaStream_t s, int grid, int threads) {
  launch_flux_dir_c<0>(d, w, P, s, grid, threads);
}

}  // namespace grmhd
