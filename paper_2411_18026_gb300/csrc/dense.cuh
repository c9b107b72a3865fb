// Batched dense complex128 linear algebra on variable-size per-cell blocks:
// LU with partial pivoting, multi-RHS LU solve, and GEMM.  Used by the merge
// of Sec. 6.2 (A_i^{-1} U_i, S_i = V_i A_i^{-1} U_i, A~_i = S_i^{-1}), the top
// LU of Sec. 6.3 and the solve sweeps.  Matrices are column-major.
#pragma once

#include "common.cuh"

// Per-matrix descriptor of a batch (complex128 or complex64 elements).
template <class C>
struct MatRefT {
    C *p;          // base pointer
    int rows, cols, ld;
};
typedef MatRefT<cplx> MatRef;
typedef MatRefT<cplxf> MatRefF;
typedef MatRefT<float4> MatRefP;

// Row maps of one batch entry of a mapped GEMM (device pointers, nullable).
struct RowMaps {
    const int *b;   // B row k is read from row b[k] (0 <= b[k] < B.rows)
    const int *c;   // C row i is written to row c[i] (0 <= c[i] < cext)
    int cext;       // rows of the buffer C's map addresses
};

// Launch helpers (device pointers to descriptor arrays; all enqueue on stream).
// LU in place of square A[b] (rows == cols), pivots piv + poff[b], info[b].
int dense_lu(int batch, int max_n, const MatRef *d_A, int *d_piv, const int64_t *d_poff, int *d_info,
             cudaStream_t s);
// Solve A X = B in place of B for each b with the LU of dense_lu (B[b].rows
// must equal the order of A[b]).  max_rows / max_cols bound the sizes.
int dense_lu_solve(int batch, int max_rows, int max_cols, const MatRef *d_LU, const int *d_piv,
                   const int64_t *d_poff, const MatRef *d_B, cudaStream_t s);
// C = alpha * op(A) * op(B) + beta * C, op = N (0), or conjugate transpose (2).
int dense_gemm(int batch, int max_m, int max_n, const MatRef *d_A, int opA, const MatRef *d_B, int opB,
               const MatRef *d_C, cplx alpha, cplx beta, cudaStream_t s);
// Register-tiled GEMM (gemm.cu), op(B) = B; dense_gemm routes here when opB = 0.
int dense_gemm_rt(int batch, int max_m, int max_n, const MatRef *d_A, int opA, const MatRef *d_B, const MatRef *d_C,
                  cplx alpha, cplx beta, cudaStream_t s);
int dense_gemm_rt(int batch, int max_m, int max_n, const MatRefF *d_A, int opA, const MatRefF *d_B,
                  const MatRefF *d_C, cplxf alpha, cplxf beta, cudaStream_t s);
// Same with operands already split into float pairs (float4 = re_hi, im_hi,
// re_lo, im_lo per complex entry) and a float-pair result; C = op(A) B
// (+ C when accumulate).
int dense_gemm_ffp(int batch, int max_m, int max_n, const MatRefP *d_A, int opA, const MatRefP *d_B,
                   const MatRefP *d_C, int accumulate, cudaStream_t s);
// float-pair GEMM with alpha = +-1 (sign of alpha.x), beta = 0 or 1 (beta.x), opB = 0
int dense_gemm(int batch, int max_m, int max_n, const MatRefP *d_A, int opA, const MatRefP *d_B, int opB,
               const MatRefP *d_C, float4 alpha, float4 beta, cudaStream_t s);
// C = op(A) B[bmap] (+ C when accumulate), rows of C written through cmap
// (the interpolation matrices applied without their identity part).
int dense_gemm_map(int batch, int max_m, int max_n, const MatRef *d_A, int opA, const MatRef *d_B, const MatRef *d_C,
                   const RowMaps *d_maps, int accumulate, cudaStream_t s);
int dense_gemm_map(int batch, int max_m, int max_n, const MatRefF *d_A, int opA, const MatRefF *d_B,
                   const MatRefF *d_C, const RowMaps *d_maps, int accumulate, cudaStream_t s);
int dense_gemm_map(int batch, int max_m, int max_n, const MatRefP *d_A, int opA, const MatRefP *d_B,
                   const MatRefP *d_C, const RowMaps *d_maps, int accumulate, cudaStream_t s);
// complex64 GEMM on the tensor cores (tcgen05, bf16 pieces; gemm_tc.cu): real
// alpha, beta; opA 0 or 2; optional row maps.
int dense_gemm_tc(int batch, int max_m, int max_n, const MatRefF *d_A, int opA, const MatRefF *d_B,
                  const MatRefF *d_C, float alpha, float beta, const RowMaps *d_maps, cudaStream_t s);
// LU with partial pivoting of one n x n matrix A (leading dimension ld) in
// 32-column panels, the trailing updates as GEMMs (the top system); pivots in
// d_piv[0..n), d_info as for dense_lu.  Synchronises s.
int dense_lu_blocked(int n, cplx *A, int ld, int *d_piv, int *d_info, cudaStream_t s);
// Reads and clears the tensor-core timeout status (synchronises s).
int tc_status_take(cudaStream_t s, int *status);
// Arms (1) or clears (0) the injected stall of the next complex64 tensor-core GEMM launch.
int tc_fault_arm(int on);
// X[b] = A[b]^{-1} for complex64 blocks of order n <= GJ_MAX_N by Gauss-Jordan
// elimination with row pivoting in shared memory (one CTA per block; A is
// read, not changed); info[b] as for dense_lu.  FDS_ERR_ARG for max_n > GJ_MAX_N.
constexpr int GJ_MAX_N = 160;
int dense_inverse_gj(int batch, int max_n, const MatRefF *d_A, const MatRefF *d_X, int *d_info, cudaStream_t s);
// complex64 versions (mixed-precision merge and sweep)
int dense_lu(int batch, int max_n, const MatRefF *d_A, int *d_piv, const int64_t *d_poff, int *d_info,
             cudaStream_t s);
int dense_lu_solve(int batch, int max_rows, int max_cols, const MatRefF *d_LU, const int *d_piv,
                   const int64_t *d_poff, const MatRefF *d_B, cudaStream_t s);
int dense_gemm(int batch, int max_m, int max_n, const MatRefF *d_A, int opA, const MatRefF *d_B, int opB,
               const MatRefF *d_C, cplxf alpha, cplxf beta, cudaStream_t s);
