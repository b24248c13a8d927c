// Tensor-core (tcgen05) split-BF16 path: internal interface.
#pragma once

#include <vector>

#include "ds_internal.h"

namespace ds {
namespace tc {

struct MixedPlan;

// compensated: dual-accumulator 128-column tiles (DS_PREC_BF16X6C); fx: the F
// group in fixed-head FP16 operands (DS_PREC_F16X10); fx_all: all three groups,
// with double-float increments and stage kernels (DS_PREC_F16X13)
ds_status mixed_plan_create(const ds_grid *grid, const ds_phi_set *set, DevStatus *status,
                            MixedPlan **out, bool compensated = false, bool fx = false, bool fx_all = false);
void mixed_plan_destroy(MixedPlan *mp);
// autotuner record of launch (group g, mode mu): chosen split, output tiles,
// candidate times in ms (0 = not tried); -1 on bad indices
int mixed_plan_tuning(const MixedPlan *mp, int g, int mu, int *ksplit, int64_t *tiles, int *tile_n, float *times);
// the stream-K candidates' times (ms; [0] 256-, [1] 128-column tiles; 0 = not tried)
int mixed_plan_streamk_times(const MixedPlan *mp, int g, int mu, float *times);
// tile order of the launch (mode-1 launches; 0 row tiles fastest, 1 column tiles fastest)
// and the tuner's time of each (ms; 0 = not tried)
int mixed_plan_tile_order(const MixedPlan *mp, int g, int mu, int *order, float *times);
int mixed_plan_set_tile_order(MixedPlan *mp, int g, int mu, int order);
int mixed_plan_fusion(const MixedPlan *mp, int g, int *fused, float *ms_fused, float *ms_separate);
int mixed_plan_set_fusion(MixedPlan *mp, int g, int fused);
int mixed_plan_set_tiles(MixedPlan *mp, int g, int mu, int tile_n, int ksplit);
// Enqueue one EXPRK3DS_REAL step on the split-BF16 path; returns the number
// of kernel launches, or -1 on failure.  calibrate (FX plans): measure every
// FX tensor before writing it instead of using the previous step's scales.
int enqueue_step_mixed(MixedPlan *mp, const ds_phi_set *set, const Model &model,
                       const Stencil *sten, double *U, cudaStream_t st, Prof *prof, bool calibrate = false);
// FX plans: the scale table's overflow flag (and clear it), -1 if none
int mixed_plan_fx_overflow(MixedPlan *mp, bool clear);
// F = K U + g(U) of one problem (the first kernel of its step; FX plans: FX
// planes with the scales already set for the step)
int enqueue_rhs_mixed(MixedPlan *mp, const Model &model, double *U, cudaStream_t st);
// Grouped launches for batches: the same mode product of every problem in
// one persistent launch (tables built for one set of state pointers).
struct MixedGroup;
// force_fused[g]: -1 = timed choice (or DS_TUNE_CACHE), 0 = separate stage
// kernel, 1 = fused epilogue for group g's last mode
ds_status mixed_group_create(const std::vector<MixedPlan *> &mps, const std::vector<double *> &U,
                             const std::vector<Model> &models, const int force_fused[3], MixedGroup **out);
void mixed_group_destroy(MixedGroup *G);
int mixed_group_enqueue(const MixedGroup *G, cudaStream_t st, Prof *prof);
// every problem's F planes in one launch; 0 (nothing launched) where some
// problem's grid has no tiled stencil kernel
int mixed_group_enqueue_rhs(const MixedGroup *G, cudaStream_t st);
// FX batches: the start-of-step rescale of every problem's scale table (one
// launch; 0 for other precisions).  Enqueue it before the F planes.
int mixed_group_enqueue_rescale(const MixedGroup *G, cudaStream_t st);
int mixed_group_fusion(const MixedGroup *G, int g, int *fused, float *ms_fused, float *ms_separate);
int mixed_group_tile_order(const MixedGroup *G, int g, int *order, float *times);
// FP32 CUDA-core path pointwise kernels (two components, N points each)
void launch_rhs_f32(const Stencil *sten, const Model &m, int64_t N, const double *U, float *F,
                    cudaStream_t st);
void launch_stage_f32(const Model &m, int64_t N, const double *U, const float *a, double w1,
                      const float *b, double w2, float *D, cudaStream_t st);
void launch_final_f32(int64_t N, double *U, const float *a, double w1, const float *b, double w2,
                      cudaStream_t st);
void launch_convert_f64_f32(int64_t n, const double *x, float *y, cudaStream_t st);
void launch_convert_f32_f64(int64_t n, const float *x, double *y, cudaStream_t st);
ds_status tucker_mixed(const ds_grid *grid, const double *X, double *Y, const double *const *L,
                       int transpose, cudaStream_t st, bool compensated = false);
ds_status tucker_fx(const ds_grid *grid, const double *X, double *Y, const double *const *L, int transpose,
                    cudaStream_t st);

}  // namespace tc
}  // namespace ds
