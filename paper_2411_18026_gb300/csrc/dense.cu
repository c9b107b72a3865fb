// Batched complex128 LU / LU-solve / GEMM kernels (one CTA per matrix or
// per output tile).  FP64 throughout.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "dense.cuh"
#include "fds_internal.cuh"

namespace {

constexpr int LU_THREADS = 256;

template <class C>
__device__ __forceinline__ bool finite_c(C a) { return isfinite(a.x) && isfinite(a.y); }

// Right-looking unblocked LU with partial pivoting (largest |a_ik|, ties to the
// lowest row), one CTA per matrix, the matrix in global memory.
template <class C>
__global__ void __launch_bounds__(LU_THREADS) k_lu(const MatRefT<C> *__restrict__ mats, int *__restrict__ piv,
                                                   const int64_t *__restrict__ poff, int *__restrict__ info) {
    const MatRefT<C> M = mats[blockIdx.x];
    const int n = M.rows, ld = M.ld;
    C *A = M.p;
    int *pv = piv + poff[blockIdx.x];
    __shared__ double s_val[LU_THREADS];
    __shared__ int s_idx[LU_THREADS];
    __shared__ int s_piv;
    __shared__ int s_bad;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        // pivot search in column k
        double best = -1.0;
        int bi = n;
        for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
            double v = cabs2(A[i + (long)k * ld]);
            if (v > best) { best = v; bi = i; }
        }
        s_val[threadIdx.x] = best;
        s_idx[threadIdx.x] = bi;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) {
                double v2 = s_val[threadIdx.x + o];
                int i2 = s_idx[threadIdx.x + o];
                if (v2 > s_val[threadIdx.x] || (v2 == s_val[threadIdx.x] && i2 < s_idx[threadIdx.x])) {
                    s_val[threadIdx.x] = v2;
                    s_idx[threadIdx.x] = i2;
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            int p = s_idx[0];
            if (p >= n) p = k;
            s_piv = p;
            pv[k] = p;
            const C d = A[p + (long)k * ld];
            if (!(s_val[0] > 0.0) || !finite_c(d)) {
                if (!s_bad) s_bad = k + 1;
            }
        }
        __syncthreads();
        const int p = s_piv;
        if (p != k) {
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                const C t = A[k + (long)j * ld];
                A[k + (long)j * ld] = A[p + (long)j * ld];
                A[p + (long)j * ld] = t;
            }
        }
        __syncthreads();
        const C d = A[k + (long)k * ld];
        const C dinv = (cabs2(d) > 0) ? cinv(d) : czero<C>();
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[i + (long)k * ld] = cmul(A[i + (long)k * ld], dinv);
        __syncthreads();
        // trailing update A[k+1:, k+1:] -= l u^T
        const int m = n - k - 1;
        const long tot = (long)m * m;
        for (long e = threadIdx.x; e < tot; e += blockDim.x) {
            const int i = k + 1 + (int)(e % m), j = k + 1 + (int)(e / m);
            cfms(A[i + (long)j * ld], A[i + (long)k * ld], A[k + (long)j * ld]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) info[blockIdx.x] = s_bad;
}

// Blocked LU of one large matrix (the top system): panel kernel on columns
// k0 .. k0+nb-1 (pivot search in the panel column over rows k.., row swap
// across all n columns, scaling, update of the panel's remaining columns),
// then the block row U12 = L11^{-1} A12 (one thread per column) and the
// trailing update A22 -= L21 U12 as a register-tiled GEMM over many CTAs.
template <class C>
__global__ void __launch_bounds__(LU_THREADS) k_lu_panel(C *A, int n, int ld, int k0, int nb, int *pv,
                                                         int *info) {
    __shared__ double s_val[LU_THREADS];
    __shared__ int s_idx[LU_THREADS];
    __shared__ int s_piv;
    for (int k = k0; k < k0 + nb; ++k) {
        double best = -1.0;
        int bi = n;
        for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
            const double v = cabs2(A[i + (long)k * ld]);
            if (v > best) { best = v; bi = i; }
        }
        s_val[threadIdx.x] = best;
        s_idx[threadIdx.x] = bi;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) {
                const double v2 = s_val[threadIdx.x + o];
                const int i2 = s_idx[threadIdx.x + o];
                if (v2 > s_val[threadIdx.x] || (v2 == s_val[threadIdx.x] && i2 < s_idx[threadIdx.x])) {
                    s_val[threadIdx.x] = v2;
                    s_idx[threadIdx.x] = i2;
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            int p = s_idx[0];
            if (p >= n) p = k;
            s_piv = p;
            pv[k] = p;
            const C d = A[p + (long)k * ld];
            if ((!(s_val[0] > 0.0) || !finite_c(d)) && *info == 0) *info = k + 1;
        }
        __syncthreads();
        const int p = s_piv;
        if (p != k) {
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                const C t = A[k + (long)j * ld];
                A[k + (long)j * ld] = A[p + (long)j * ld];
                A[p + (long)j * ld] = t;
            }
        }
        __syncthreads();
        const C d = A[k + (long)k * ld];
        const C dinv = (cabs2(d) > 0) ? cinv(d) : czero<C>();
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[i + (long)k * ld] = cmul(A[i + (long)k * ld], dinv);
        __syncthreads();
        const int m = n - k - 1, w = k0 + nb - k - 1;   // rows below, panel columns right of k
        for (long e = threadIdx.x; e < (long)m * w; e += blockDim.x) {
            const int i = k + 1 + (int)(e % m), j = k + 1 + (int)(e / m);
            cfms(A[i + (long)j * ld], A[i + (long)k * ld], A[k + (long)j * ld]);
        }
        __syncthreads();
    }
}

template <class C>
__global__ void k_trsm_l11(C *A, int n, int ld, int k0, int nb) {
    const int j = k0 + nb + blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    for (int i = k0 + 1; i < k0 + nb; ++i) {
        C acc = A[i + (long)j * ld];
        for (int t = k0; t < i; ++t) cfms(acc, A[i + (long)t * ld], A[t + (long)j * ld]);
        A[i + (long)j * ld] = acc;
    }
}

// Multi-RHS LU solve: CTA per (matrix, tile of RT right-hand sides).  The RHS
// tile lives in shared memory during the row swaps, the unit-lower forward
// substitution and the upper back substitution.
constexpr int SOLVE_THREADS = 256;

template <class C>
__global__ void __launch_bounds__(SOLVE_THREADS) k_lu_solve(const MatRefT<C> *__restrict__ LUs,
                                                            const int *__restrict__ piv,
                                                            const int64_t *__restrict__ poff,
                                                            const MatRefT<C> *__restrict__ Bs, int rt) {
    extern __shared__ __align__(16) unsigned char sh_raw[];
    C *sh = reinterpret_cast<C *>(sh_raw);
    const MatRefT<C> L = LUs[blockIdx.y];
    const MatRefT<C> B = Bs[blockIdx.y];
    const int n = L.rows;
    const int c0 = blockIdx.x * rt;
    if (c0 >= B.cols || n == 0) return;
    const int nc = min(rt, B.cols - c0);
    const int *pv = piv + poff[blockIdx.y];
    // load tile: sh[i + c * n]
    for (long e = threadIdx.x; e < (long)n * nc; e += blockDim.x) {
        const int i = (int)(e % n), c = (int)(e / n);
        sh[e] = B.p[i + (long)(c0 + c) * B.ld];
    }
    __syncthreads();
    if (threadIdx.x < nc) {
        const int c = threadIdx.x;
        for (int k = 0; k < n; ++k) {
            const int p = pv[k];
            if (p != k) {
                C t = sh[k + c * n];
                sh[k + c * n] = sh[p + c * n];
                sh[p + c * n] = t;
            }
        }
    }
    __syncthreads();
    // forward: x_i -= L_ij x_j (j < i), column sweep
    for (int j = 0; j < n - 1; ++j) {
        const int m = n - j - 1;
        for (long e = threadIdx.x; e < (long)m * nc; e += blockDim.x) {
            const int i = j + 1 + (int)(e % m), c = (int)(e / m);
            cfms(sh[i + c * n], L.p[i + (long)j * L.ld], sh[j + c * n]);
        }
        __syncthreads();
    }
    // backward
    for (int j = n - 1; j >= 0; --j) {
        const C dinv = cinv(L.p[j + (long)j * L.ld]);
        for (int c = threadIdx.x; c < nc; c += blockDim.x) sh[j + c * n] = cmul(sh[j + c * n], dinv);
        __syncthreads();
        for (long e = threadIdx.x; e < (long)j * nc; e += blockDim.x) {
            const int i = (int)(e % j), c = (int)(e / j);
            cfms(sh[i + c * n], L.p[i + (long)j * L.ld], sh[j + c * n]);
        }
        __syncthreads();
    }
    for (long e = threadIdx.x; e < (long)n * nc; e += blockDim.x) {
        const int i = (int)(e % n), c = (int)(e / n);
        B.p[i + (long)(c0 + c) * B.ld] = sh[e];
    }
}

// C = alpha op(A) op(B) + beta C; 16x16 output tile per CTA, 16-deep K chunks.
constexpr int GT = 16;

template <class C>
__device__ __forceinline__ C ld_op(const MatRefT<C> &M, int op, int i, int j) {
    // element (i, j) of op(M)
    if (op == 0) return M.p[i + (long)j * M.ld];
    C v = M.p[j + (long)i * M.ld];
    return cconj(v);
}

template <class C>
__global__ void __launch_bounds__(GT *GT) k_gemm(const MatRefT<C> *__restrict__ As, int opA,
                                                 const MatRefT<C> *__restrict__ Bs, int opB,
                                                 const MatRefT<C> *__restrict__ Cs, C alpha, C beta, int tiles_m) {
    const MatRefT<C> A = As[blockIdx.y], B = Bs[blockIdx.y], Cm = Cs[blockIdx.y];
    const int M = Cm.rows, N = Cm.cols;
    const int K = (opA == 0) ? A.cols : A.rows;
    const int tm = blockIdx.x % tiles_m, tn = blockIdx.x / tiles_m;
    const int i0 = tm * GT, j0 = tn * GT;
    if (i0 >= M || j0 >= N) return;
    __shared__ C sa[GT][GT + 1], sb[GT][GT + 1];
    const int tx = threadIdx.x % GT, ty = threadIdx.x / GT;
    C acc = czero<C>();
    for (int k0 = 0; k0 < K; k0 += GT) {
        {
            const int i = i0 + tx, k = k0 + ty;
            sa[ty][tx] = (i < M && k < K) ? ld_op(A, opA, i, k) : czero<C>();
            const int kk = k0 + tx, j = j0 + ty;
            sb[ty][tx] = (kk < K && j < N) ? ld_op(B, opB, kk, j) : czero<C>();
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < GT; ++k) cfma(acc, sa[k][tx], sb[ty][k]);
        __syncthreads();
    }
    const int i = i0 + tx, j = j0 + ty;
    if (i < M && j < N) {
        C *c = &Cm.p[i + (long)j * Cm.ld];
        C old = (beta.x != 0 || beta.y != 0) ? *c : czero<C>();
        *c = cadd(cmul(alpha, acc), cmul(beta, old));
    }
}

}  // namespace

int dense_lu(int batch, int max_n, const MatRef *d_A, int *d_piv, const int64_t *d_poff, int *d_info,
             cudaStream_t s) {
    if (batch <= 0) return FDS_OK;
    (void)max_n;
    fds_count_launch(), k_lu<cplx><<<batch, LU_THREADS, 0, s>>>(d_A, d_piv, d_poff, d_info);
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}
// In-place Gauss-Jordan inversion with partial (row) pivoting of each
// complex64 block A[b] (n x n, n <= GJ_MAX_N), held in shared memory by one
// CTA: per step k the pivot row (largest |a_ik|, i >= k) is swapped to k,
// row k becomes its scaled self with 1 / a_kk on the diagonal, every other
// row i loses a_ik times it and gets -a_ik / a_kk in column k (three
// barriers per step: pivot search, the staged column / rows, the update);
// the row swaps are undone as column swaps in reverse order at the end.  X[b] = A[b]^{-1};
// info[b] = first step with a zero or non-finite pivot (0: none).
constexpr int GJ_THREADS = 1024;
__global__ void __launch_bounds__(GJ_THREADS) k_gj_inverse(const MatRefF *__restrict__ As,
                                                          const MatRefF *__restrict__ Xs, int *info) {
    extern __shared__ cplxf gj[];
    const MatRefF A = As[blockIdx.x], X = Xs[blockIdx.x];
    const int n = A.rows, ld = n + 1;   // padded columns
    cplxf *a = gj;                       // n x n, column-major, leading dimension ld
    cplxf *fcol = a + (size_t)ld * n;    // column k before the step
    cplxf *rowk = fcol + n;              // row k after the step
    cplxf *rowold = rowk + n;            // row k before the step
    int *perm = reinterpret_cast<int *>(rowold + n);
    __shared__ int s_p, s_bad;
    const int tid = threadIdx.x;
    for (int e = tid; e < n * n; e += blockDim.x) {
        const int i = e % n, j = e / n;
        a[i + j * ld] = A.p[i + (int64_t)j * A.ld];
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (tid < 32) {
            float best = -1.f;
            int bi = k;
            for (int i = k + tid; i < n; i += 32) {
                const float v = cabs2(a[i + k * ld]);
                if (v > best) { best = v; bi = i; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float v2 = __shfl_xor_sync(0xffffffffu, best, o);
                const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
                if (v2 > best || (v2 == best && i2 < bi)) { best = v2; bi = i2; }
            }
            if (tid == 0) {
                s_p = bi;
                perm[k] = bi;
            }
        }
        __syncthreads();
        // the swap of rows k and p is folded into the two phases below: row
        // k's new values come from row p, row p's from the saved old row k
        const int p = s_p;
        const cplxf d = a[p + k * ld];
        const float m = d.x * d.x + d.y * d.y;
        const bool ok = m > 0.f && isfinite(m);
        const cplxf inv = ok ? mkcf(d.x / m, -d.y / m) : mkcf(0.f, 0.f);
        if (tid == 0 && !ok && !s_bad) s_bad = k + 1;
        for (int t = tid; t < 3 * n; t += blockDim.x) {
            if (t < n) {
                const int r = t == k ? p : (t == p ? k : t);   // row t after the swap
                fcol[t] = t == k ? mkcf(0.f, 0.f) : a[r + k * ld];
            } else if (t < 2 * n) {
                const int c = t - n;
                rowk[c] = c == k ? inv : cmul(a[p + c * ld], inv);
            } else {
                const int c = t - 2 * n;
                rowold[c] = a[k + c * ld];
            }
        }
        __syncthreads();
        for (int e = tid; e < n * n; e += blockDim.x) {
            const int i = e % n, c = e / n;
            cplxf &v = a[i + c * ld];
            if (i == k) {
                v = rowk[c];
            } else {
                const cplxf base = (i == p) ? rowold[c] : v;
                if (c == k) {
                    v = cmul(mkcf(-fcol[i].x, -fcol[i].y), inv);
                } else {
                    cplxf w = base;
                    cfms(w, fcol[i], rowk[c]);
                    v = w;
                }
            }
        }
        __syncthreads();
    }
    // the row swaps of step k become a swap of columns k and perm[k], in reverse order
    for (int k = n - 1; k >= 0; --k) {
        const int p = perm[k];
        if (p != k)
            for (int i = tid; i < n; i += blockDim.x) {
                const cplxf t = a[i + k * ld];
                a[i + k * ld] = a[i + p * ld];
                a[i + p * ld] = t;
            }
        __syncthreads();
    }
    for (int e = tid; e < n * n; e += blockDim.x) {
        const int i = e % n, j = e / n;
        X.p[i + (int64_t)j * X.ld] = a[i + j * ld];
    }
    if (tid == 0) info[blockIdx.x] = s_bad;
}

int dense_lu(int batch, int max_n, const MatRefF *d_A, int *d_piv, const int64_t *d_poff, int *d_info,
             cudaStream_t s) {
    if (batch <= 0) return FDS_OK;
    (void)max_n;
    fds_count_launch(), k_lu<cplxf><<<batch, LU_THREADS, 0, s>>>(d_A, d_piv, d_poff, d_info);
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}

int dense_lu_blocked(int n, cplx *A, int ld, int *d_piv, int *d_info, cudaStream_t s) {
    if (n <= 0) return FDS_OK;
    constexpr int NB = 32;
    FDS_CUDA_TRY(cudaMemsetAsync(d_info, 0, sizeof(int), s));
    std::vector<MatRef> refs;
    for (int k0 = 0; k0 < n; k0 += NB) {
        const int nb = std::min(NB, n - k0), r = n - k0 - nb;
        MatRef L21, U12, A22;
        L21.p = A + (k0 + nb) + (int64_t)k0 * ld;
        L21.rows = r;
        L21.cols = nb;
        L21.ld = ld;
        U12.p = A + k0 + (int64_t)(k0 + nb) * ld;
        U12.rows = nb;
        U12.cols = r;
        U12.ld = ld;
        A22.p = A + (k0 + nb) + (int64_t)(k0 + nb) * ld;
        A22.rows = r;
        A22.cols = r;
        A22.ld = ld;
        refs.push_back(L21);
        refs.push_back(U12);
        refs.push_back(A22);
    }
    DBuf<MatRef> d_refs;
    FDS_TRY(d_refs.upload(refs, s));
    int panel = 0;
    for (int k0 = 0; k0 < n; k0 += NB, ++panel) {
        const int nb = std::min(NB, n - k0), r = n - k0 - nb;
        fds_count_launch(), k_lu_panel<cplx><<<1, LU_THREADS, 0, s>>>(A, n, ld, k0, nb, d_piv, d_info);
        FDS_CUDA_TRY(cudaGetLastError());
        if (r == 0) break;
        fds_count_launch(), k_trsm_l11<cplx><<<(r + 127) / 128, 128, 0, s>>>(A, n, ld, k0, nb);
        FDS_CUDA_TRY(cudaGetLastError());
        const MatRef *R = d_refs.p + 3 * panel;
        FDS_TRY(dense_gemm_rt(1, r, r, R, 0, R + 1, R + 2, mkc(-1.0, 0.0), mkc(1.0, 0.0), s));
    }
    FDS_CUDA_TRY(cudaStreamSynchronize(s));   // the descriptors die with this call
    return FDS_OK;
}

template <class C>
static int lu_solve_t(int batch, int max_rows, int max_cols, const MatRefT<C> *d_LU, const int *d_piv,
                      const int64_t *d_poff, const MatRefT<C> *d_B, cudaStream_t s) {
    if (batch <= 0 || max_rows <= 0 || max_cols <= 0) return FDS_OK;
    // RHS tile width so that rows x rt complex fits in 200 KB of shared memory
    int rt = (int)(200 * 1024 / ((long)sizeof(C) * max_rows));
    if (rt > 32) rt = 32;
    if (rt < 1) return FDS_ERR_ARG;
    size_t smem = (size_t)max_rows * rt * sizeof(C);
    FDS_TRY(ensure_dyn_smem(k_lu_solve<C>, smem));
    dim3 grid((max_cols + rt - 1) / rt, batch);
    fds_count_launch(), k_lu_solve<C><<<grid, SOLVE_THREADS, smem, s>>>(d_LU, d_piv, d_poff, d_B, rt);
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}

template <class C>
static int gemm_t(int batch, int max_m, int max_n, const MatRefT<C> *d_A, int opA, const MatRefT<C> *d_B, int opB,
                  const MatRefT<C> *d_C, C alpha, C beta, cudaStream_t s) {
    if (batch <= 0 || max_m <= 0 || max_n <= 0) return FDS_OK;
    const int tm = (max_m + GT - 1) / GT, tn = (max_n + GT - 1) / GT;
    dim3 grid(tm * tn, batch);
    fds_count_launch(), k_gemm<C><<<grid, GT * GT, 0, s>>>(d_A, opA, d_B, opB, d_C, alpha, beta, tm);
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}

int dense_lu_solve(int batch, int max_rows, int max_cols, const MatRef *d_LU, const int *d_piv,
                   const int64_t *d_poff, const MatRef *d_B, cudaStream_t s) {
    return lu_solve_t<cplx>(batch, max_rows, max_cols, d_LU, d_piv, d_poff, d_B, s);
}
int dense_lu_solve(int batch, int max_rows, int max_cols, const MatRefF *d_LU, const int *d_piv,
                   const int64_t *d_poff, const MatRefF *d_B, cudaStream_t s) {
    return lu_solve_t<cplxf>(batch, max_rows, max_cols, d_LU, d_piv, d_poff, d_B, s);
}
int dense_gemm(int batch, int max_m, int max_n, const MatRef *d_A, int opA, const MatRef *d_B, int opB,
               const MatRef *d_C, cplx alpha, cplx beta, cudaStream_t s) {
    if (opB == 0) return dense_gemm_rt(batch, max_m, max_n, d_A, opA, d_B, d_C, alpha, beta, s);
    return gemm_t<cplx>(batch, max_m, max_n, d_A, opA, d_B, opB, d_C, alpha, beta, s);
}
int dense_gemm(int batch, int max_m, int max_n, const MatRefF *d_A, int opA, const MatRefF *d_B, int opB,
               const MatRefF *d_C, cplxf alpha, cplxf beta, cudaStream_t s) {
    if (opB == 0 && g_c64_tensor && alpha.y == 0.f && beta.y == 0.f)
        return dense_gemm_tc(batch, max_m, max_n, d_A, opA, d_B, d_C, alpha.x, beta.x, nullptr, s);
    if (opB == 0) return dense_gemm_rt(batch, max_m, max_n, d_A, opA, d_B, d_C, alpha, beta, s);
    return gemm_t<cplxf>(batch, max_m, max_n, d_A, opA, d_B, opB, d_C, alpha, beta, s);
}

// Stage entry point: batched LU (see fds.h).
namespace {
__global__ void k_make_refs(int batch, const int32_t *d, const int64_t *off, double *A, MatRef *refs) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    refs[b].p = (cplx *)A + off[b];
    refs[b].rows = d[b];
    refs[b].cols = d[b];
    refs[b].ld = d[b] > 0 ? d[b] : 1;
}
}  // namespace

extern "C" int fds_lu_batched(int32_t batch, const int32_t *d_d, const int64_t *d_off, double *d_A,
                              int32_t *d_piv, const int64_t *d_poff, int32_t *d_info, uint64_t stream) {
    if (batch < 0) return FDS_ERR_ARG;
    if (batch == 0) return FDS_OK;
    if (!d_d || !d_off || !d_A || !d_piv || !d_poff || !d_info) return FDS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    MatRef *refs = nullptr;
    FDS_CUDA_TRY(cudaMallocAsync((void **)&refs, sizeof(MatRef) * batch, s));
    fds_count_launch(), k_make_refs<<<(batch + 127) / 128, 128, 0, s>>>(batch, d_d, d_off, d_A, refs);
    int rc = dense_lu(batch, 0, refs, d_piv, d_poff, d_info, s);
    cudaFreeAsync(refs, s);
    FDS_CUDA_TRY(cudaGetLastError());
    return rc;
}

// ---------------------------------------------------------------------------
// Allocation-free batched LU.  The per-matrix descriptors that fds_lu_batched
// builds in a cudaMallocAsync'd buffer live here in a file-scope device array
// instead; every GPU that loads the library holds it (384 KiB) until exit.
#define FDS_LU_NOALLOC_MAX_BATCH 16384
static __device__ __align__(256) MatRef g_lu_noalloc_refs[FDS_LU_NOALLOC_MAX_BATCH];

namespace {
// Device address of g_lu_noalloc_refs for each device, looked up once per
// device (with that device current) by cudaGetSymbolAddress: in host code the
// array's name is only a host-side stand-in.  The address is kept for the life
// of the process; a cudaDeviceReset() of the device invalidates it.
MatRef *lu_noalloc_scratch(int *err) {
    static std::mutex mu;
    static MatRef *addr[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        *err = FDS_ERR_CUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_lu_noalloc_refs) != cudaSuccess || !p) {
            *err = FDS_ERR_CUDA;
            return nullptr;
        }
        addr[dev] = (MatRef *)p;
    }
    *err = FDS_OK;
    return addr[dev];
}
}  // namespace

extern "C" int fds_lu_batched_noalloc(int32_t batch, const int32_t *d_d, const int64_t *d_off, double *d_A,
                                      int32_t *d_piv, const int64_t *d_poff, int32_t *d_info, uint64_t stream) {
    if (batch < 0 || batch > FDS_LU_NOALLOC_MAX_BATCH) return FDS_ERR_ARG;
    if (batch == 0) return FDS_OK;
    if (!d_d || !d_off || !d_A || !d_piv || !d_poff || !d_info) return FDS_ERR_ARG;
    int err = FDS_OK;
    MatRef *refs = lu_noalloc_scratch(&err);
    if (err != FDS_OK) return err;
    cudaStream_t s = (cudaStream_t)stream;
    fds_count_launch(), k_make_refs<<<(batch + 127) / 128, 128, 0, s>>>(batch, d_d, d_off, d_A, refs);
    FDS_CUDA_TRY(cudaGetLastError());
    return dense_lu(batch, 0, refs, d_piv, d_poff, d_info, s);
}

int dense_inverse_gj(int batch, int max_n, const MatRefF *d_A, const MatRefF *d_X, int *d_info, cudaStream_t s) {
    if (batch <= 0) return FDS_OK;
    if (max_n < 1 || max_n > GJ_MAX_N) return FDS_ERR_ARG;
    const size_t smem = sizeof(cplxf) * ((size_t)(max_n + 1) * max_n + 3 * max_n) + sizeof(int) * max_n;
    FDS_TRY(ensure_dyn_smem(k_gj_inverse, smem));
    fds_count_launch(), k_gj_inverse<<<batch, GJ_THREADS, smem, s>>>(d_A, d_X, d_info);
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}
