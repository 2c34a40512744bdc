// FP32 instantiations of the fused step kernel for batches that hold lattices
// open in x (x-slabs): the same shapes as lbm_step_f32.cu, with the general
// path's pulls reading the frame across the x edges of such lattices.
#define LBM_STEP_F32_OPEN true
#define LBM_STEP_F32_NAME launch_step_f32_open
#include "lbm_step_f32.inc"
