// xy-plane block sweeps (Sec. 2 with full-plane blocks).
#include "plane.cuh"

int plane_setup(brs_ctx*) { return BRS_ERR_UNSUPPORTED; }
void plane_teardown(brs_ctx*) {}
int plane_sweep_launch(brs_ctx*, const void*, void*, const void*, cudaStream_t)
{
    return BRS_ERR_UNSUPPORTED;
}
