// Tensor-core (tcgen05) split-BF16 path.
#include "tc.h"

namespace ds {
namespace tc {

struct MixedPlan {
    int dummy;
};

ds_status mixed_plan_create(const ds_grid *, const ds_phi_set *, DevStatus *, MixedPlan **)
{
    return fail(DS_ERR_UNSUPPORTED, "split-BF16 path not built yet");
}
void mixed_plan_destroy(MixedPlan *mp) { delete mp; }
int enqueue_step_mixed(MixedPlan *, const ds_phi_set *, const Model &, const Stencil *, double *,
                       cudaStream_t)
{
    return -1;
}
ds_status tucker_mixed(const ds_grid *, const double *, double *, const double *const *, int,
                       cudaStream_t)
{
    return fail(DS_ERR_UNSUPPORTED, "split-BF16 path not built yet");
}

}  // namespace tc
}  // namespace ds
