// Step kernels for float precision on the D3Q27 lattice.
#define LBM_REAL float
#define LBM_DIM 3
#define LBM_OPS_NAME get_ops_f32_3d
#include "lbm_inst.cuh"
