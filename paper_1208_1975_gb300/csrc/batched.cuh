// Batched many-patch x-line path (batched.cu).
#pragma once
#include "brs_internal.cuh"

int batched_setup(brs_ctx* c, int npatch, const int* dims);
// Turns a batched context into a level: face-neighbour table (6 per patch, validated by
// the caller), boundary-cell chunks and the b_eff array.
int level_setup(brs_ctx* c, const int* nbr);
void batched_teardown(brs_ctx* c);
int batched_sweep(brs_ctx* c, void* u, const void* b, int nsweeps, cudaStream_t s);
int level_keep_ghosts(brs_ctx* c, int on);
void batched_describe(const brs_ctx* c, int* kc, int* warps, int* grid, int* nitems);
