// Leaf diagonal blocks of the forward operator on the tensor cores with an
// Ozaki-type bf16 split (fw_tc.cu).
#pragma once

#include "fds_internal.cuh"

// Slices of the leaf level's FP64 diagonal blocks (d_blocks: one d x d
// complex block per leaf, d <= 128), kept in the level (oz_a, oz_rowexp).
int oz_leaf_prepare(Level &C, const MatRef *d_blocks, cudaStream_t s);
// y += D x over the leaves of level C: x, y leaf-order float pairs, leading
// dimension ld, nc columns.
int oz_leaf_apply(fds_handle *h, Level &C, const float4 *x, float4 *y, int64_t ld, int nc, cudaStream_t s);
// Reads and clears the timeout status of the leaf-block products (synchronises s).
int oz_status_take(cudaStream_t s, int *status);
// Arms (1) or clears (0) the injected stall of the next leaf-block product launch.
int oz_fault_arm(int on);
