// Batched-form kernels for double precision (D2Q9).
#define LBM_REAL double
#define LBM_BATCH_OPS_NAME get_batch_ops_f64
#include "lbm_batch_inst.cuh"
