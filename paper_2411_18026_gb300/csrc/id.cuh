// Batched CPQR interpolative decomposition (launcher used by the build).
#pragma once

#include "common.cuh"

// d_sel (nullable): matrix indices of the CTAs (a subset of the batch).
int id_batched(int batch, int max_m, int max_n, const int *d_m, const int *d_n, const int64_t *d_off, cplx *d_Y,
               double tol, int *d_rank, int *d_perm, const int64_t *d_poff, cplx *d_T, const int64_t *d_toff,
               cudaStream_t s, const int *d_sel = nullptr);
// Learned-rank ID (learned.cu): sparse-sign sketch with frac[b] * n[b] + extra
// rows, CPQR of the sketch, ID residual checked on all of Y (Y is read
// only).  fail[b] = 1 where the check failed (outputs of b then undefined).
int id_sketched(int batch, int max_m, const int *d_m, const int *d_n, const int64_t *d_off, const cplx *d_Y,
                const float *d_frac, int extra, double tol, int *d_rank, int *d_perm, const int64_t *d_poff,
                cplx *d_T, const int64_t *d_toff, int *d_fail, unsigned long long seed, cudaStream_t s);
// Geometry features of the learned-rank network for the 2 nb (cell,
// component) rows of one level (row 2b + c); see fds_features_get.
int level_features(int nb, const int *d_lo, const int *d_hi, const double *d_xy, int N, const double *d_R,
                   const int *d_n1, const int *d_n2, const int *d_nnd, int height, double kT, double kL, double tol,
                   float *d_feat, cudaStream_t s);
