// Structured application of a level's interpolation matrices (vapply.cu).
#pragma once

#include "fds_internal.cuh"

// out (R_l x nc) = V_l x (D_l x nc);  Tb: the level's T blocks in precision T.
template <class T>
int apply_V(fds_handle *h, const Level &C, const T *Tb, const T *x, int64_t ldx, T *out, int64_t ldo, int nc,
            cudaStream_t s);
// Descriptor workspace of every structured application (allocated up front,
// so that a sweep captured into a CUDA graph allocates nothing).
int vapply_workspace(fds_handle *h);
// The skeleton rows of the structured V alone: dir 0 out[k rows] = x[skeleton],
// dir 1 y[skeleton] = t[k rows] (the T parts then run elsewhere).
template <class T>
int vskel_apply(const Level &C, int dir, const T *src, int64_t lds, T *dst, int64_t ldd, int nc, cudaStream_t s);
// y (D_l x nc) = V_l^H t (R_l x nc).
template <class T>
int apply_VH(fds_handle *h, const Level &C, const T *Tb, const T *t, int64_t ldt, T *y, int64_t ldy, int nc,
             cudaStream_t s);
