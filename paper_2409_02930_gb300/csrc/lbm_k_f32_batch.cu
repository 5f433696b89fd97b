// Batched-form kernels for float precision (D2Q9).
#define LBM_REAL float
#define LBM_BATCH_OPS_NAME get_batch_ops_f32
#include "lbm_batch_inst.cuh"
