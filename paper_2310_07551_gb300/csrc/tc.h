// Tensor-core (tcgen05) split-BF16 path: internal interface.
#pragma once

#include "ds_internal.h"

namespace ds {
namespace tc {

struct MixedPlan;

ds_status mixed_plan_create(const ds_grid *grid, const ds_phi_set *set, DevStatus *status,
                            MixedPlan **out);
void mixed_plan_destroy(MixedPlan *mp);
// Enqueue one EXPRK3DS_REAL step on the split-BF16 path; returns the number
// of kernel launches, or -1 on failure.
int enqueue_step_mixed(MixedPlan *mp, const ds_phi_set *set, const Model &model,
                       const Stencil *sten, double *U, cudaStream_t st, Prof *prof);
ds_status tucker_mixed(const ds_grid *grid, const double *X, double *Y, const double *const *L,
                       int transpose, cudaStream_t st);

}  // namespace tc
}  // namespace ds
