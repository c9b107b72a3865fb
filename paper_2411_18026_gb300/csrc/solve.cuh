// Solve sweep shared by the FP64 solve and the mixed-precision refinement loop.
#pragma once

#include "fds_internal.cuh"

constexpr int SOLVE_CHUNK = 256;   // right-hand sides per sweep

int fds_max_cells(const fds_handle *h);
// Grow the sweep workspace of precision C for ncmax columns.
template <class C>
int sweep_workspace(fds_handle *h, int ncmax);
// Leaf-order vectors (D_L x nc, column-major): the sweep reads the right-hand
// sides from sweep_leaf_in and leaves the solution in sweep_leaf_out (the
// same buffer when the leaves are the top level).
template <class C>
C *sweep_leaf_in(fds_handle *h);
template <class C>
C *sweep_leaf_out(fds_handle *h);
// One sweep over nc columns.
template <class C>
int sweep_chunk(fds_handle *h, int nc, cudaStream_t s);
