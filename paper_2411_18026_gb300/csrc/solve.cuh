// Solve sweep shared by the FP64 solve and the mixed-precision refinement loop.
#pragma once

#include "fds_internal.cuh"

constexpr int SOLVE_CHUNK = 256;   // right-hand sides per sweep

// arithmetic of a level's sweep
enum { PREC_C128 = 0, PREC_C64 = 1, PREC_FF = 2 };
int level_prec(const fds_handle *h, int l);

int fds_max_cells(const fds_handle *h);
// Last level (from the top) of the sweep that runs in complex128: L for
// FDS_FP64; for FDS_MIXED min(L - 1, l0 + sweep_fp64_levels) (L when L = l0).
int sweep_split(const fds_handle *h);
// Grow the sweep workspace for ncmax columns.
int sweep_workspace(fds_handle *h, int ncmax);
// Leaf-order vectors (D_L x nc, column-major): the sweep reads the right-hand
// sides from sweep_leaf_in and leaves the solution in sweep_leaf_out (the
// same buffer when the leaves are the top level).
template <class C>
C *sweep_leaf_in(fds_handle *h);
template <class C>
C *sweep_leaf_out(fds_handle *h);
// One sweep over nc columns (levels above sweep_split in complex64).
int sweep_chunk(fds_handle *h, int nc, cudaStream_t s);
// sweep_chunk, or (use_graph, on a capturable stream) the replay of a CUDA
// graph of it captured on the first sweep of nc columns
int sweep_chunk_run(fds_handle *h, int nc, cudaStream_t s);
