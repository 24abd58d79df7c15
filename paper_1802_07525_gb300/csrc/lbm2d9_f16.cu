// 2-D step and ghost-fill kernels with D2Q9 transport (the equilibrium of Eq. 5) and
// FP16 population storage.
#define MFC_DIM 2
#define MFC_AQ 9
#define MFC_ST __half
#define MFC_STEP_FN launch_step_2d9_f16
#define MFC_FILL_FN launch_fill_ghosts_2d9_f16
#include "lbm_launch.cuh"
