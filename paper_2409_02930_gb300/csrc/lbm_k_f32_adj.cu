// Adjoint kernels for float precision (D2Q9).
#define LBM_REAL float
#define LBM_ADJ_OPS_NAME get_adj_ops_f32
#include "lbm_adj_inst.cuh"
