// Step kernels for float precision on the D2Q9 lattice.
#define LBM_REAL float
#define LBM_DIM 2
#define LBM_OPS_NAME get_ops_f32_2d
#include "lbm_inst.cuh"
