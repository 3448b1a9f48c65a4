// Batched persistent execution (placeholder).
#include "dg_internal.h"

extern "C" {
dg_status dg_batch_create(int, const dg_handle*, dg_batch* out) { if (out) *out = nullptr; return DG_ERR_UNSUPPORTED; }
dg_status dg_batch_destroy(dg_batch) { return DG_OK; }
dg_status dg_batch_rk_step(dg_batch, double* const*, void* const*, void* const*, const double*, int, int, void*) { return DG_ERR_UNSUPPORTED; }
dg_status dg_batch_info(dg_batch, long long*, long long*) { return DG_ERR_UNSUPPORTED; }
}
