// 2-D step and ghost-fill kernels with D2Q9 transport (the equilibrium of Eq. 5), FP64
// population storage and FP64 arithmetic (the double-precision instantiation).
#define MFC_DIM 2
#define MFC_AQ 9
#define MFC_ST double
#define MFC_STEP_FN launch_step_2d9_f64
#define MFC_FILL_FN launch_fill_ghosts_2d9_f64
#include "lbm_launch.cuh"
