// Step kernels for double precision on the D2Q9 lattice.
#define LBM_REAL double
#define LBM_DIM 2
#define LBM_OPS_NAME get_ops_f64_2d
#include "lbm_inst.cuh"
