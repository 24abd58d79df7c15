// 2-D step, batch-step and ghost-fill kernels with FP16 population storage.
#define MFC_DIM 2
#define MFC_ST __half
#define MFC_STEP_FN launch_step_2d_f16
#define MFC_FILL_FN launch_fill_ghosts_2d_f16
#define MFC_BATCH_FN launch_batch_2d_f16
#define MFC_ARGS_FN step_args_2d_f16
#define MFC_OCC_FN batch_occupancy_2d_f16
#include "lbm_launch.cuh"
