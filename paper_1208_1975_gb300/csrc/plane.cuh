// xy-plane block path (plane.cu): setup, teardown and one sweep launch.
#pragma once
#include "brs_internal.cuh"

int plane_setup(brs_ctx* c);
void plane_teardown(brs_ctx* c);
int plane_sweep_launch(brs_ctx* c, const void* uin, void* uout, const void* b, cudaStream_t s);
