// Combination-scheme plans (batched transform, gather): not built yet.
#include "gbh_internal.h"

struct gbh_plan { int unused; };

extern "C" {
int gbh_plan_create_scheme(int, int, int, gbh_plan **) { return GBH_EUNSUPPORTED; }
int gbh_plan_create(int, int, const int32_t *, int, gbh_plan **) { return GBH_EUNSUPPORTED; }
int gbh_plan_destroy(gbh_plan *) { return GBH_OK; }
int gbh_plan_num_grids(const gbh_plan *, int *) { return GBH_EUNSUPPORTED; }
int gbh_plan_grid_levels(const gbh_plan *, int, int32_t *) { return GBH_EUNSUPPORTED; }
int gbh_plan_coeffs(const gbh_plan *, double *) { return GBH_EUNSUPPORTED; }
int gbh_plan_sparse_points(const gbh_plan *, int64_t *) { return GBH_EUNSUPPORTED; }
int gbh_plan_total_points(const gbh_plan *, int64_t *) { return GBH_EUNSUPPORTED; }
int gbh_plan_bind(gbh_plan *, void *const *, void *) { return GBH_EUNSUPPORTED; }
int gbh_plan_execute(gbh_plan *, int, void *) { return GBH_EUNSUPPORTED; }
int gbh_plan_gather(gbh_plan *, double *, void *) { return GBH_EUNSUPPORTED; }
int gbh_plan_status(gbh_plan *, void *) { return GBH_EUNSUPPORTED; }
}
