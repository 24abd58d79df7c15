// 2-D step and ghost-fill kernels with FP32 population storage.
#define MFC_DIM 2
#define MFC_ST float
#define MFC_STEP_FN launch_step_2d_f32
#define MFC_FILL_FN launch_fill_ghosts_2d_f32
#include "lbm_launch.cuh"
