// Step kernels for double precision on the D3Q27 lattice.
#define LBM_REAL double
#define LBM_DIM 3
#define LBM_OPS_NAME get_ops_f64_3d
#include "lbm_inst.cuh"
