// Batched lattices (implemented in a later step; entry points reject for now).
#include "lbm.h"
#include "lbm_capi_internal.h"

extern "C" {
lbm_status lbm_tune(const lbm_params *, const uint8_t *, void *, size_t, void *, lbm_tuning *) {
    return lbm_fail(LBM_EUNSUPPORTED, "lbm_tune: not built yet");
}
lbm_status lbm_batch_plan(int32_t, lbm_params *, const lbm_tuning *) {
    return lbm_fail(LBM_EUNSUPPORTED, "batch: not built yet");
}
lbm_status lbm_batch_workspace_bytes(int32_t, const lbm_params *, size_t *) {
    return lbm_fail(LBM_EUNSUPPORTED, "batch: not built yet");
}
lbm_status lbm_batch_create(int32_t, const lbm_params *, const uint8_t *const *, void *, size_t, void *,
                            lbm_batch **) {
    return lbm_fail(LBM_EUNSUPPORTED, "batch: not built yet");
}
lbm_status lbm_batch_init(lbm_batch *, int32_t, const double *, const double *, const double *) {
    return lbm_fail(LBM_EUNSUPPORTED, "batch: not built yet");
}
lbm_status lbm_batch_step(lbm_batch *, int64_t, uint32_t) { return lbm_fail(LBM_EUNSUPPORTED, "batch"); }
lbm_status lbm_batch_sync(lbm_batch *) { return lbm_fail(LBM_EUNSUPPORTED, "batch"); }
lbm_status lbm_batch_read_moments(lbm_batch *, int32_t, double *, double *, double *) {
    return lbm_fail(LBM_EUNSUPPORTED, "batch");
}
lbm_status lbm_batch_read_populations(lbm_batch *, int32_t, void *, int32_t) {
    return lbm_fail(LBM_EUNSUPPORTED, "batch");
}
lbm_status lbm_batch_get_info(lbm_batch *, int64_t *, int32_t *, int64_t *) {
    return lbm_fail(LBM_EUNSUPPORTED, "batch");
}
void lbm_batch_destroy(lbm_batch *) {}
}
