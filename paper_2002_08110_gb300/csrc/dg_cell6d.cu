// Specialised 6D, n = 4 cell kernel (placeholder until the tuned kernel lands).
#include "dg_internal.h"

namespace dg {
cudaError_t launch_cell_6d4(int combo, KParams& p, const LaunchCfg& cfg, cudaStream_t s) {
  (void)combo; (void)p; (void)cfg; (void)s;
  return cudaErrorNotSupported;
}
}  // namespace dg
