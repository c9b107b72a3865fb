// Learned-rank network (mlp.cu): inference launcher used by the build.
#pragma once

#include "common.cuh"

// y[b] = network(X[b, 0:16]) for b < n (device pointers; FP32).
int mlp_forward(const float *d_params, const float *d_X, int n, float *d_y, cudaStream_t s);
