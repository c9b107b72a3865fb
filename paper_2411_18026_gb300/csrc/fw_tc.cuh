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

// One block product y[ymap] (+)= op(A) x[xmap] of a plan (host description).
struct OzSpec {
    const cplx *a = nullptr;   // device: the stored block
    int lda = 1;
    int op = 0;                // 0: op(A) = A, stored m x k; 1: op(A) = A^H, stored k x m
    int m = 0, k = 0;          // complex rows and columns of op(A)
    int64_t x_row = 0, y_row = 0;
    const int *xmap = nullptr; // host: the k rows of x (relative to x_row); nullptr: contiguous
    const int *ymap = nullptr; // host: the m rows of y (relative to y_row); nullptr: contiguous
    bool set = false;          // y = product (y is not read)
};
// Cuts the blocks of specs into slices, one plan per 128-column K pass;
// the jobs of a pass must write disjoint rows of y.  Synchronises s.
int oz_plan_build(const std::vector<OzSpec> &specs, std::vector<OzPlan> &passes, cudaStream_t s);
// Runs the passes in order on float-pair vectors x (ld ldx) and y (ld ldy), nc columns.
int oz_plan_apply(fds_handle *h, const std::vector<OzPlan> &passes, const float4 *x, int64_t ldx, float4 *y,
                  int64_t ldy, int nc, cudaStream_t s);
// Reads and clears the timeout status of the general block products (synchronises s).
int ozj_status_take(cudaStream_t s, int *status);
// Arms (1) or clears (0) the injected stall of the next general block-product launch.
int ozj_fault_arm(int on);

