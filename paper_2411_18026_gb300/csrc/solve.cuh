// Solve sweep shared by the FP64 solve and the mixed-precision refinement loop.
#pragma once

#include "fds_internal.cuh"

constexpr int SOLVE_CHUNK = 256;   // right-hand sides per sweep

int fds_max_cells(const fds_handle *h);
// Grow the sweep workspace of precision C for ncmax columns.
template <class C>
int sweep_workspace(fds_handle *h, int ncmax);
// Leaf-order vector (D_L x nc, column-major) the sweep reads and overwrites.
template <class C>
C *sweep_leaf_vector(fds_handle *h);
// One sweep over nc columns of the leaf-order vector, in place.
template <class C>
int sweep_chunk(fds_handle *h, int nc, cudaStream_t s);
