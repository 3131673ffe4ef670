// Box-block path (box.cu): setup, teardown and one sweep launch.
#pragma once
#include "brs_internal.cuh"

int box_setup(brs_ctx* c);
void box_teardown(brs_ctx* c);
int box_sweep_launch(brs_ctx* c, const void* uin, void* uout, const void* b, cudaStream_t s);
