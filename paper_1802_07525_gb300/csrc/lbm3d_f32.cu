// 3-D step, batch-step and ghost-fill kernels with FP32 population storage.
#define MFC_DIM 3
#define MFC_ST float
#define MFC_STEP_FN launch_step_3d_f32
#define MFC_FILL_FN launch_fill_ghosts_3d_f32
#define MFC_BATCH_FN launch_batch_3d_f32
#define MFC_ARGS_FN step_args_3d_f32
#define MFC_OCC_FN batch_occupancy_3d_f32
#include "lbm_launch.cuh"
