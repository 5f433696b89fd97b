// Adjoint kernels for double precision (D2Q9).
#define LBM_REAL double
#define LBM_ADJ_OPS_NAME get_adj_ops_f64
#include "lbm_adj_inst.cuh"
