// Instantiations of the generic cell kernel for d = 4 (all n, all precisions).
#include "dg_generic.cuh"

namespace dg {
cudaError_t launch_cell_d4(int n, int combo, KParams& p, const LaunchCfg& cfg, cudaStream_t s) {
  return launch_generic_dim<4>(n, combo, p, cfg, s);
}
}  // namespace dg
