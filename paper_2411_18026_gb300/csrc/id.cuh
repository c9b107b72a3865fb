// Batched CPQR interpolative decomposition (launcher used by the build).
#pragma once

#include "common.cuh"

int id_batched(int batch, int max_m, int max_n, const int *d_m, const int *d_n, const int64_t *d_off, cplx *d_Y,
               double tol, int *d_rank, int *d_perm, const int64_t *d_poff, cplx *d_T, const int64_t *d_toff,
               cudaStream_t s);
