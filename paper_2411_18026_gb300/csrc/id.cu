// Batched interpolative decomposition by Householder QR with column pivoting
// (arXiv 2411.18026, Sec. 7.1: M P = Q [R1 R2; 0 R3], ||R3|| ~ 0, V = [I R1^{-1} R2] P^T).
// One CTA per matrix; the matrix stays in global memory (L2), the Householder
// vector, the trailing column norms and the permutation in shared memory.
#include <cmath>

#include "common.cuh"
#include "id.cuh"

namespace {

constexpr int ID_THREADS = 256;
constexpr int ID_WARPS = ID_THREADS / 32;

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Dynamic shared memory: v[m] (cplx), norms2[n] (double), perm[n] (int).
__global__ void __launch_bounds__(ID_THREADS) k_cpqr_id(const int *__restrict__ ms, const int *__restrict__ ns,
                                                        const int64_t *__restrict__ offs, cplx *__restrict__ Yall,
                                                        double tol, int *__restrict__ ranks,
                                                        int *__restrict__ perms, const int64_t *__restrict__ poffs,
                                                        cplx *__restrict__ Tall, const int64_t *__restrict__ toffs,
                                                        const int *__restrict__ sel) {
    extern __shared__ double smem[];
    const int b = sel ? sel[blockIdx.x] : blockIdx.x;
    const int m = ms[b], n = ns[b];
    cplx *Y = Yall + offs[b];
    cplx *v = (cplx *)smem;
    double *nrm = (double *)(v + m);
    int *perm = (int *)(nrm + n);
    __shared__ double r_val[ID_THREADS];
    __shared__ int r_idx[ID_THREADS];
    __shared__ int s_k, s_stop, s_p;
    __shared__ double s_alpha, s_r11;
    __shared__ cplx s_phase;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    for (int j = threadIdx.x; j < n; j += blockDim.x) perm[j] = j;
    for (int c = warp; c < n; c += ID_WARPS) {
        double s = 0.0;
        for (int i = lane; i < m; i += 32) s += cabs2(Y[i + (long)c * m]);
        s = wsum(s);
        if (lane == 0) nrm[c] = s;
    }
    if (threadIdx.x == 0) { s_k = 0; s_stop = 0; s_r11 = 0.0; }
    __syncthreads();
    const int kmax = min(m, n);
    for (int j = 0; j < kmax; ++j) {
        // pivot: largest remaining norm, ties to the lowest index
        double best = -1.0;
        int bi = n;
        for (int c = j + threadIdx.x; c < n; c += blockDim.x) {
            if (nrm[c] > best) { best = nrm[c]; bi = c; }
        }
        r_val[threadIdx.x] = best;
        r_idx[threadIdx.x] = bi;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) {
                double v2 = r_val[threadIdx.x + o];
                int i2 = r_idx[threadIdx.x + o];
                if (v2 > r_val[threadIdx.x] || (v2 == r_val[threadIdx.x] && i2 < r_idx[threadIdx.x])) {
                    r_val[threadIdx.x] = v2;
                    r_idx[threadIdx.x] = i2;
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const int p = r_idx[0] < n ? r_idx[0] : j;
            const double alpha = sqrt(fmax(r_val[0], 0.0));
            if (j == 0) s_r11 = alpha;
            s_p = p;
            s_alpha = alpha;
            s_stop = (alpha == 0.0 || alpha <= tol * s_r11) ? 1 : 0;
        }
        __syncthreads();
        if (s_stop) break;
        const int p = s_p;
        if (p != j) {
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                cplx t = Y[i + (long)j * m];
                Y[i + (long)j * m] = Y[i + (long)p * m];
                Y[i + (long)p * m] = t;
            }
            if (threadIdx.x == 0) {
                int t = perm[j]; perm[j] = perm[p]; perm[p] = t;
                double tn = nrm[j]; nrm[j] = nrm[p]; nrm[p] = tn;
            }
        }
        __syncthreads();
        // Householder vector v = x + phase(x0) alpha e_0 on rows j..m-1
        const double alpha = s_alpha;
        if (threadIdx.x == 0) {
            cplx x0 = Y[j + (long)j * m];
            double a0 = sqrt(cabs2(x0));
            s_phase = a0 > 0.0 ? mkc(x0.x / a0, x0.y / a0) : mkc(1.0, 0.0);
        }
        __syncthreads();
        const cplx ph = s_phase;
        for (int i = j + threadIdx.x; i < m; i += blockDim.x) {
            cplx x = Y[i + (long)j * m];
            if (i == j) x = cadd(x, cscale(ph, alpha));
            v[i] = x;
        }
        __syncthreads();
        double vn2 = 0.0;
        {
            // |v|^2 = 2 alpha (alpha + |x0|)
            cplx x0 = Y[j + (long)j * m];
            vn2 = 2.0 * alpha * (alpha + sqrt(cabs2(x0)));
        }
        const double tau = 2.0 / vn2;
        __syncthreads();
        // apply H = I - tau v v^H to columns j+1..n-1 and refresh their norms
        for (int c = j + 1 + warp; c < n; c += ID_WARPS) {
            cplx *col = Y + (long)c * m;
            double sr = 0.0, si = 0.0;
            for (int i = j + lane; i < m; i += 32) {
                cplx a = col[i];
                cplx vi = v[i];
                // conj(v_i) a
                sr += vi.x * a.x + vi.y * a.y;
                si += vi.x * a.y - vi.y * a.x;
            }
            sr = wsum(sr);
            si = wsum(si);
            const cplx s = mkc(tau * sr, tau * si);
            double nn = 0.0;
            for (int i = j + lane; i < m; i += 32) {
                cplx a = col[i];
                cfms(a, s, v[i]);
                col[i] = a;
                if (i > j) nn += cabs2(a);
            }
            nn = wsum(nn);
            if (lane == 0) nrm[c] = nn;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            Y[j + (long)j * m] = cscale(ph, -alpha);   // R_jj
            s_k = j + 1;
        }
        __syncthreads();
    }
    __syncthreads();
    const int k = s_k;
    int *pout = perms + poffs[b];
    for (int j = threadIdx.x; j < n; j += blockDim.x) pout[j] = perm[j];
    if (threadIdx.x == 0) ranks[b] = k;
    // T = R1^{-1} R2 by back substitution, one thread per column of R2
    cplx *T = Tall + toffs[b];
    for (int c = threadIdx.x; c < n - k; c += blockDim.x) {
        const int col = k + c;
        for (int i = k - 1; i >= 0; --i) {
            cplx acc = Y[i + (long)col * m];
            for (int l = i + 1; l < k; ++l) cfms(acc, Y[i + (long)l * m], T[l + (long)c * k]);
            T[i + (long)c * k] = cdiv(acc, Y[i + (long)i * m]);
        }
    }
}

}  // namespace

int id_batched(int batch, int max_m, int max_n, const int *d_m, const int *d_n, const int64_t *d_off, cplx *d_Y,
               double tol, int *d_rank, int *d_perm, const int64_t *d_poff, cplx *d_T, const int64_t *d_toff,
               cudaStream_t s, const int *d_sel) {
    if (batch <= 0) return FDS_OK;
    size_t smem = (size_t)max_m * sizeof(cplx) + (size_t)max_n * (sizeof(double) + sizeof(int)) + 16;
    if (smem > 220 * 1024) return FDS_ERR_ARG;
    FDS_TRY(ensure_dyn_smem(k_cpqr_id, smem));
    fds_count_launch(), k_cpqr_id<<<batch, ID_THREADS, smem, s>>>(d_m, d_n, d_off, d_Y, tol, d_rank, d_perm, d_poff, d_T, d_toff,
                                                                      d_sel);
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}

extern "C" int fds_id_batched(int32_t batch, const int32_t *d_m, const int32_t *d_n, const int64_t *d_off,
                              double *d_Y, double tol, int32_t *d_rank, int32_t *d_perm, const int64_t *d_poff,
                              double *d_T, const int64_t *d_toff, uint64_t stream) {
    if (batch < 0 || !(tol >= 0.0 && tol < 1.0)) return FDS_ERR_ARG;
    if (batch == 0) return FDS_OK;
    if (!d_m || !d_n || !d_off || !d_Y || !d_rank || !d_perm || !d_poff || !d_T || !d_toff) return FDS_ERR_ARG;
    // sizes are needed on the host for the shared-memory budget
    cudaStream_t s = (cudaStream_t)stream;
    int *hm = new int[batch], *hn = new int[batch];
    cudaError_t e1 = cudaMemcpyAsync(hm, d_m, sizeof(int) * batch, cudaMemcpyDeviceToHost, s);
    cudaError_t e2 = cudaMemcpyAsync(hn, d_n, sizeof(int) * batch, cudaMemcpyDeviceToHost, s);
    cudaError_t e3 = cudaStreamSynchronize(s);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        delete[] hm;
        delete[] hn;
        return FDS_ERR_CUDA;
    }
    int mm = 1, mn = 1;
    for (int b = 0; b < batch; ++b) {
        if (hm[b] < 0 || hn[b] < 0) { delete[] hm; delete[] hn; return FDS_ERR_ARG; }
        mm = hm[b] > mm ? hm[b] : mm;
        mn = hn[b] > mn ? hn[b] : mn;
    }
    delete[] hm;
    delete[] hn;
    return id_batched(batch, mm, mn, d_m, d_n, d_off, (cplx *)d_Y, tol, d_rank, d_perm, d_poff, (cplx *)d_T, d_toff,
                      s);
}
