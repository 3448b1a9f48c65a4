// Instantiations of the generic cell kernel for d = 2 (all n, all precisions).
#include "dg_generic.cuh"

namespace dg {
cudaError_t launch_cell_d2(int n, int combo, KParams& p, const LaunchCfg& cfg, cudaStream_t s) {
  return launch_generic_dim<2>(n, combo, p, cfg, s);
}
}  // namespace dg
