// 2-D step and ghost-fill kernels with FP64 population storage and FP64 arithmetic (the
// double-precision instantiation, a parity reference).
#define MFC_DIM 2
#define MFC_ST double
#define MFC_STEP_FN launch_step_2d_f64
#define MFC_FILL_FN launch_fill_ghosts_2d_f64
#include "lbm_launch.cuh"
