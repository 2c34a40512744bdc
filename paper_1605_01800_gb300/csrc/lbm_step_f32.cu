// FP32 instantiations of the fused step kernel (deviation or plain storage),
// for batches without lattices open in x; lbm_step_f32_open.cu instantiates
// the same shapes for batches with them.
#define LBM_STEP_F32_OPEN false
#define LBM_STEP_F32_NAME launch_step_f32_closed
#include "lbm_step_f32.inc"
