// Batched many-patch x-line path (batched.cu).
#pragma once
#include "brs_internal.cuh"

int batched_setup(brs_ctx* c, int npatch, const int* dims);
void batched_teardown(brs_ctx* c);
int batched_sweep(brs_ctx* c, void* u, const void* b, int nsweeps, cudaStream_t s);
void batched_describe(const brs_ctx* c, int* kc, int* warps, int* grid, int* nitems);
