// Placeholder for the tensor-core Gram path; replaced below.
#include "internal.cuh"
als_status launch_sweep_tc(als_ctx *c, const SweepArgs &a) {
    (void)c; (void)a;
    als_set_error("tensor-core Gram path not built");
    return ALS_ENOTSUP;
}
