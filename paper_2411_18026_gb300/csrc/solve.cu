// Multi-RHS solve sweep (arXiv 2411.18026 Sec. 6.2 upward, Sec. 6.3 top and
// downward):
//   up    z_i = A_i^{-1} f_i,  f~_i = A~_i V_i z_i,  parent f by eq. (rhs_rearrangement)
//   top   x = A_top^{-1} f_top
//   down  y_i from the parent x (eqs. (xtoy1)-(xtoy2)),
//         x_i = z_i - W_i (f~_i - A~_i y_i) with W_i = A_i^{-1} U_i   (eq. (down_comv))
// Right-hand sides are processed in column chunks; all arithmetic in the
// batched kernels of dense.cu and the gathers below.
#include <algorithm>

#include "fds_internal.cuh"
#include "prof.cuh"

namespace {

constexpr int CHUNK = 256;

__global__ void k_vec_refs(int nb, cplx *base, const int64_t *__restrict__ off, int cols, int64_t ld, MatRef *out) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    out[b].p = base + off[b];
    out[b].rows = (int)(off[b + 1] - off[b]);
    out[b].cols = cols;
    out[b].ld = (int)ld;
}

// leaf vector <- global natural-order vector (gather) or back (scatter)
__global__ void k_leaf_gather(const int *__restrict__ gidx, int64_t D, int N, const cplx *__restrict__ src,
                              int64_t lds, cplx *dst, int cols, int dir) {
    const int64_t tot = D * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = e % D, c = e / D;
        const int64_t g = gidx[q] + c * lds;
        if (dir == 0) dst[q + c * D] = src[g];
        else ((cplx *)src)[g] = dst[q + c * D];
    }
}

// child skeleton vector (R x cols) <-> parent DOF vector (Dp x cols)
// dir 0: parent[pos] = child  (upward scatter of f~)
// dir 1: child = parent[pos]  (downward gather of y)
__global__ void k_child_parent(int nb, const int64_t *__restrict__ roff, const int *__restrict__ k1,
                               const int *__restrict__ pos1, const int *__restrict__ pos2,
                               const int64_t *__restrict__ pdoff, cplx *child, int64_t ldc, cplx *parent,
                               int64_t ldp, int cols, int dir) {
    const int b = blockIdx.x;
    const int64_t o = roff[b];
    const int r = (int)(roff[b + 1] - o);
    const int64_t pb = pdoff[b >> 1];
    const int kk = k1[b], p1 = pos1[b], p2 = pos2[b];
    for (int64_t e = threadIdx.x; e < (int64_t)r * cols; e += blockDim.x) {
        const int q = (int)(e % r);
        const int64_t c = e / r;
        const int64_t pr = pb + (q < kk ? p1 + q : p2 + (q - kk));
        if (dir == 0) parent[pr + c * ldp] = child[o + q + c * ldc];
        else child[o + q + c * ldc] = parent[pr + c * ldp];
    }
}

int grow(DBuf<cplx> &b, size_t n) {
    if (b.n >= n && b.p) return FDS_OK;
    return b.alloc(n);
}

}  // namespace

int fds_solve_impl(fds_handle *h, cplx *d_rhs, int nrhs, cudaStream_t s) {
    if (nrhs <= 0) return FDS_OK;
    const int L = h->L, l0 = h->l0, N = h->N;
    const int64_t ld_rhs = 2LL * N;
    const int ncmax = std::min(nrhs, CHUNK);
    // workspace
    if ((int)h->wz.size() != L + 1) {
        h->wz = std::vector<DBuf<cplx>>(L + 1);
        h->wf = std::vector<DBuf<cplx>>(L + 1);
        h->wt = std::vector<DBuf<cplx>>(L + 1);
    }
    for (int l = L; l > l0; --l) {
        Level &C = h->lv[l];
        FDS_TRY(grow(h->wz[l], (size_t)C.D * ncmax));
        FDS_TRY(grow(h->wf[l], (size_t)std::max<int64_t>(C.Rtot, 1) * ncmax));
        FDS_TRY(grow(h->wt[l], (size_t)std::max<int64_t>(C.Rtot, 1) * ncmax));
    }
    FDS_TRY(grow(h->wtop, (size_t)h->Dtop * ncmax));
    int maxnb = 1;
    for (int l = L; l >= l0; --l) maxnb = std::max(maxnb, h->lv[l].nb);
    if (h->wrefs.n < (size_t)4 * maxnb) FDS_TRY(h->wrefs.alloc((size_t)4 * maxnb));
    MatRef *rZ = h->wrefs.p, *rF = rZ + maxnb, *rT = rF + maxnb, *rX = rT + maxnb;

    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    for (int c0 = 0; c0 < nrhs; c0 += CHUNK) {
        const int nc = std::min(CHUNK, nrhs - c0);
        cplx *rhs = d_rhs + (int64_t)c0 * ld_rhs;
        // leaf gather
        Level &Lf = h->lv[L];
        cplx *leafv = (L > l0) ? h->wz[L].p : h->wtop.p;
        fds_count_launch(), k_leaf_gather<<<1024, 256, 0, s>>>(h->d_leaf_gidx.p, Lf.D, N, rhs, ld_rhs, leafv, nc, 0);
        FDS_CUDA_TRY(cudaGetLastError());
        // upward
        for (int l = L; l > l0; --l) {
            Level &C = h->lv[l];
            Level &Pn = h->lv[l - 1];
            const int nb = C.nb;
            cplx *Z = h->wz[l].p, *F = h->wf[l].p, *U = h->wt[l].p;
            fds_count_launch(), k_vec_refs<<<(nb + 127) / 128, 128, 0, s>>>(nb, Z, C.d_doff.p, nc, C.D, rZ);
            fds_count_launch(), k_vec_refs<<<(nb + 127) / 128, 128, 0, s>>>(nb, U, C.d_roff.p, nc, std::max<int64_t>(C.Rtot, 1), rT);
            fds_count_launch(), k_vec_refs<<<(nb + 127) / 128, 128, 0, s>>>(nb, F, C.d_roff.p, nc, std::max<int64_t>(C.Rtot, 1), rF);
            {
                ProfScope ps("a6.up_lu_solve", s);
                ps.flops = 8.0 * C.sum_d2 * nc;
                ps.bytes = 16.0 * C.sum_d2 + 32.0 * C.D * nc;
                FDS_TRY(dense_lu_solve(nb, C.dmax, nc, C.rLU.p, C.piv.p, C.d_offpiv.p, rZ, s));
            }
            {
                ProfScope ps("a6.up_apply", s);
                ps.flops = 8.0 * (C.sum_rd + C.sum_r2) * nc;
                ps.bytes = 16.0 * (C.sum_rd + C.sum_r2) + 16.0 * (C.D + 2.0 * C.Rtot) * nc;
                FDS_TRY(dense_gemm(nb, C.rmax, nc, C.rV.p, 0, rZ, 0, rT, mkc(1, 0), mkc(0, 0), s));
                FDS_TRY(dense_gemm(nb, C.rmax, nc, C.rAt.p, 0, rT, 0, rF, mkc(1, 0), mkc(0, 0), s));
            }
            cplx *par = (l - 1 > l0) ? h->wz[l - 1].p : h->wtop.p;
            const int64_t ldp = (l - 1 > l0) ? Pn.D : h->Dtop;
            fds_count_launch(), k_child_parent<<<nb, 256, 0, s>>>(nb, C.d_roff.p, C.d_k1.p, C.d_par_pos1.p, C.d_par_pos2.p, Pn.d_doff.p, F,
                                              std::max<int64_t>(C.Rtot, 1), par, ldp, nc, 0);
            FDS_CUDA_TRY(cudaGetLastError());
        }
        // top
        {
            MatRef tv;
            tv.p = h->wtop.p;
            tv.rows = (int)h->Dtop;
            tv.cols = nc;
            tv.ld = (int)std::max<int64_t>(h->Dtop, 1);
            FDS_CUDA_TRY(cudaMemcpyAsync(rX, &tv, sizeof(MatRef), cudaMemcpyHostToDevice, s));
            ProfScope ps("a6.top_solve", s);
            ps.flops = 8.0 * (double)h->Dtop * h->Dtop * nc;
            ps.bytes = 16.0 * (double)h->Dtop * h->Dtop;
            FDS_TRY(dense_lu_solve(1, (int)h->Dtop, nc, h->rtop.p, h->ptop.p, h->d_ptop_off.p, rX, s));
        }
        // downward
        for (int l = l0 + 1; l <= L; ++l) {
            Level &C = h->lv[l];
            Level &Pn = h->lv[l - 1];
            const int nb = C.nb;
            cplx *Z = h->wz[l].p, *F = h->wf[l].p, *Y = h->wt[l].p;
            cplx *par = (l - 1 > l0) ? h->wz[l - 1].p : h->wtop.p;
            const int64_t ldp = (l - 1 > l0) ? Pn.D : h->Dtop;
            const int64_t ldr = std::max<int64_t>(C.Rtot, 1);
            fds_count_launch(), k_child_parent<<<nb, 256, 0, s>>>(nb, C.d_roff.p, C.d_k1.p, C.d_par_pos1.p, C.d_par_pos2.p, Pn.d_doff.p, Y,
                                              ldr, par, ldp, nc, 1);
            fds_count_launch(), k_vec_refs<<<(nb + 127) / 128, 128, 0, s>>>(nb, Z, C.d_doff.p, nc, C.D, rZ);
            fds_count_launch(), k_vec_refs<<<(nb + 127) / 128, 128, 0, s>>>(nb, Y, C.d_roff.p, nc, ldr, rT);
            fds_count_launch(), k_vec_refs<<<(nb + 127) / 128, 128, 0, s>>>(nb, F, C.d_roff.p, nc, ldr, rF);
            FDS_CUDA_TRY(cudaGetLastError());
            // F <- f~ - A~ y ;  Z <- z - W F
            ProfScope ps("a6.down_apply", s);
            ps.flops = 8.0 * (C.sum_r2 + C.sum_rd) * nc;
            ps.bytes = 16.0 * (C.sum_r2 + C.sum_rd) + 16.0 * (2.0 * C.D + 2.0 * C.Rtot) * nc;
            FDS_TRY(dense_gemm(nb, C.rmax, nc, C.rAt.p, 0, rT, 0, rF, mkc(-1, 0), mkc(1, 0), s));
            FDS_TRY(dense_gemm(nb, C.dmax, nc, C.rW.p, 0, rF, 0, rZ, mkc(-1, 0), mkc(1, 0), s));
        }
        cplx *leafx = (L > l0) ? h->wz[L].p : h->wtop.p;
        fds_count_launch(), k_leaf_gather<<<1024, 256, 0, s>>>(h->d_leaf_gidx.p, Lf.D, N, rhs, ld_rhs, leafx, nc, 1);
        FDS_CUDA_TRY(cudaGetLastError());
    }
    cudaEventRecord(e1, s);
    FDS_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    h->solve_ms = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return FDS_OK;
}
