// 2-D step and ghost-fill kernels with FP16 population storage.
#define MFC_DIM 2
#define MFC_ST __half
#define MFC_STEP_FN launch_step_2d_f16
#define MFC_FILL_FN launch_fill_ghosts_2d_f16
#include "lbm_launch.cuh"
