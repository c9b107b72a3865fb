// Multi-RHS solve sweep (arXiv 2411.18026 Sec. 6.2 upward, Sec. 6.3 top and
// downward):
//   up    z_i = A_i^{-1} f_i (a GEMM with the A_i^{-1} formed at build),
//         f~_i = A~_i V_i z_i,  parent f by eq. (rhs_rearrangement)
//   top   x = A_top^{-1} f_top
//   down  y_i from the parent x (eqs. (xtoy1)-(xtoy2)),
//         x_i = z_i - W_i (f~_i - A~_i y_i) with W_i = A_i^{-1} U_i   (eq. (down_comv))
// Right-hand sides are processed in column chunks; all arithmetic in the
// batched kernels of dense.cu / gemm.cu and the gathers below.  The sweep is
// written once for complex128 factors (FDS_FP64) and complex64 copies
// (FDS_MIXED); the top system is solved with the FP64 LU in both.
#include <algorithm>

#include "fds_internal.cuh"
#include "prof.cuh"
#include "solve.cuh"
#include "vapply.cuh"

namespace {

template <class C>
__global__ void k_vec_refs(int nb, C *base, const int64_t *__restrict__ off, int cols, int64_t ld,
                           MatRefT<C> *out) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    out[b].p = base + off[b];
    out[b].rows = (int)(off[b + 1] - off[b]);
    out[b].cols = cols;
    out[b].ld = (int)ld;
}

// leaf vector <- global natural-order vector (gather) or back (scatter)
__global__ void k_leaf_gather(const int *__restrict__ gidx, int64_t D, const cplx *__restrict__ src, int64_t lds,
                              cplx *dst, int cols, int dir) {
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
template <class C>
__global__ void k_child_parent(int nb, const int64_t *__restrict__ roff, const int *__restrict__ k1,
                               const int *__restrict__ pos1, const int *__restrict__ pos2,
                               const int64_t *__restrict__ pdoff, C *child, int64_t ldc, C *parent, int64_t ldp,
                               int cols, int dir) {
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

template <class A, class B>
__global__ void k_convert(const A *__restrict__ src, B *dst, int64_t rows, int64_t lds, int64_t ldd, int cols) {
    const int64_t tot = rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % rows, c = e / rows;
        const A v = src[i + c * lds];
        dst[i + c * ldd].x = v.x;
        dst[i + c * ldd].y = v.y;
    }
}

template <class T>
int grow(DBuf<T> &b, size_t n) {
    if (b.n >= n && b.p) return FDS_OK;
    return b.alloc(n);
}

// Factor and workspace views of one precision.
template <class C>
struct View;

template <>
struct View<cplx> {
    static const MatRef *Ainv(const Level &v) { return v.rAinv.p; }
    static const MatRef *W(const Level &v) { return v.rW.p; }
    static const MatRef *At(const Level &v) { return v.rAt.p; }
    static const MatRef *V(const Level &v) { return v.rV.p; }
    static const cplx *Tm(const Level &v) { return v.T.p; }
    static std::vector<DBuf<cplx>> &z(fds_handle *h) { return h->wz; }
    static std::vector<DBuf<cplx>> &f(fds_handle *h) { return h->wf; }
    static std::vector<DBuf<cplx>> &t(fds_handle *h) { return h->wt; }
    static std::vector<DBuf<cplx>> &r(fds_handle *h) { return h->wr; }
    static DBuf<cplx> &wtop(fds_handle *h) { return h->wtop; }
    static DBuf<MatRef> &refs(fds_handle *h) { return h->wrefs; }
    static cplx one() { return mkc(1, 0); }
};

template <>
struct View<cplxf> {
    static const MatRefF *Ainv(const Level &v) { return v.rAinvf.p; }
    static const MatRefF *W(const Level &v) { return v.rWf.p; }
    static const MatRefF *At(const Level &v) { return v.rAtf.p; }
    static const MatRefF *V(const Level &v) { return v.rVf.p; }
    static const cplxf *Tm(const Level &v) { return v.Tf.p; }
    static std::vector<DBuf<cplxf>> &z(fds_handle *h) { return h->wzf; }
    static std::vector<DBuf<cplxf>> &f(fds_handle *h) { return h->wff; }
    static std::vector<DBuf<cplxf>> &t(fds_handle *h) { return h->wtf; }
    static std::vector<DBuf<cplxf>> &r(fds_handle *h) { return h->wrf; }
    static DBuf<cplxf> &wtop(fds_handle *h) { return h->wtopf; }
    static DBuf<MatRefF> &refs(fds_handle *h) { return h->wrefsf; }
    static cplxf one() { return mkcf(1, 0); }
};

}  // namespace

int fds_max_cells(const fds_handle *h) {
    int m = 1;
    for (int l = h->L; l >= h->l0; --l) m = std::max(m, h->lv[l].nb);
    return m;
}

// Levels l0 < l <= lsplit run in complex128, levels above lsplit in the
// precision of the mixed sweep (complex64); the top solve is FP64.
int sweep_split(const fds_handle *h) {
    if (h->opt.precision != FDS_MIXED || h->L == h->l0) return h->L;
    // the build decided per level (Level::c64; complex128 levels form a prefix
    // below the top): by sweep_fp64_levels, or automatically complex128 for
    // the levels holding at most 1/8 of the leaf DOFs
    int ls = h->l0;
    for (int l = h->l0 + 1; l <= h->L; ++l)
        if (!h->lv[l].c64) ls = l;
    return ls;
}

template <class C>
int workspace_levels(fds_handle *h, int ncmax, int lo, int hi, bool top) {
    typedef View<C> Vw;
    const int L = h->L;
    auto &wz = Vw::z(h), &wf = Vw::f(h), &wt = Vw::t(h), &wr = Vw::r(h);
    if ((int)wz.size() != L + 1) {
        wz = std::vector<DBuf<C>>(L + 1);
        wf = std::vector<DBuf<C>>(L + 1);
        wt = std::vector<DBuf<C>>(L + 1);
    }
    if ((int)wr.size() != L + 1) wr = std::vector<DBuf<C>>(L + 1);
    for (int l = hi; l >= lo && l > h->l0; --l) {
        Level &Cv = h->lv[l];
        FDS_TRY(grow(wz[l], (size_t)Cv.D * ncmax));
        FDS_TRY(grow(wr[l], (size_t)Cv.D * ncmax));
        FDS_TRY(grow(wf[l], (size_t)std::max<int64_t>(Cv.Rtot, 1) * ncmax));
        FDS_TRY(grow(wt[l], (size_t)std::max<int64_t>(Cv.Rtot, 1) * ncmax));
    }
    if (top) FDS_TRY(grow(Vw::wtop(h), (size_t)std::max<int64_t>(h->Dtop, 1) * ncmax));
    const int maxnb = fds_max_cells(h);
    if (Vw::refs(h).n < (size_t)4 * maxnb) FDS_TRY(Vw::refs(h).alloc((size_t)4 * maxnb));
    return FDS_OK;
}

int sweep_workspace(fds_handle *h, int ncmax) {
    const int ls = sweep_split(h);
    FDS_TRY(workspace_levels<cplx>(h, ncmax, h->l0 + 1, ls, true));
    if (ls < h->L || (h->opt.precision == FDS_MIXED)) {
        // complex64 levels, the boundary level's vectors and the top in complex64
        FDS_TRY(workspace_levels<cplxf>(h, ncmax, ls, h->L, true));
    }
    return FDS_OK;
}

template <class C>
C *sweep_leaf_in(fds_handle *h) {
    return (h->L > h->l0) ? View<C>::r(h)[h->L].p : View<C>::wtop(h).p;
}

template <class C>
C *sweep_leaf_out(fds_handle *h) {
    return (h->L > h->l0) ? View<C>::z(h)[h->L].p : View<C>::wtop(h).p;
}

namespace {

// Upward step of level l: z_i = A_i^{-1} f_i, f~_i = A~_i V_i z_i, scattered
// into the parent's right-hand side (level l-1 vector of type C, or the top).
template <class C>
int up_level(fds_handle *h, int l, int nc, cudaStream_t s) {
    typedef View<C> Vw;
    const int l0 = h->l0;
    const C one = Vw::one(), zero = czero<C>();
    const int maxnb = fds_max_cells(h);
    MatRefT<C> *rZ = Vw::refs(h).p, *rF = rZ + maxnb, *rT = rF + maxnb;
    auto &wz = Vw::z(h), &wf = Vw::f(h), &wt = Vw::t(h), &wr = Vw::r(h);
    const double esz = sizeof(C);
    Level &Cv = h->lv[l];
    Level &Pn = h->lv[l - 1];
    const int nb = Cv.nb;
    const int64_t ldr = std::max<int64_t>(Cv.Rtot, 1);
    C *Z = wz[l].p, *F = wf[l].p, *U = wt[l].p, *Rh = wr[l].p;
    fds_count_launch(), k_vec_refs<C><<<(nb + 127) / 128, 128, 0, s>>>(nb, Rh, Cv.d_doff.p, nc, Cv.D, rF);
    fds_count_launch(), k_vec_refs<C><<<(nb + 127) / 128, 128, 0, s>>>(nb, Z, Cv.d_doff.p, nc, Cv.D, rZ);
    {
        ProfScope ps("a6.up_a_inverse", s);
        ps.flops = 8.0 * Cv.sum_d2 * nc;
        ps.bytes = esz * Cv.sum_d2 + 2 * esz * Cv.D * nc;
        FDS_TRY(dense_gemm(nb, Cv.dmax, nc, Vw::Ainv(Cv), 0, rF, 0, rZ, one, zero, s));
    }
    fds_count_launch(), k_vec_refs<C><<<(nb + 127) / 128, 128, 0, s>>>(nb, U, Cv.d_roff.p, nc, ldr, rT);
    fds_count_launch(), k_vec_refs<C><<<(nb + 127) / 128, 128, 0, s>>>(nb, F, Cv.d_roff.p, nc, ldr, rF);
    {
        // U = V z through V = [I T] P^T, then f~ = A~ U
        ProfScope ps("a6.up_apply", s);
        ps.flops = 8.0 * (Cv.sum_tm + Cv.sum_r2) * nc;
        ps.bytes = esz * (Cv.sum_tm + Cv.sum_r2) + esz * (Cv.D + 2.0 * Cv.Rtot) * nc;
        FDS_TRY(apply_V<C>(h, Cv, Vw::Tm(Cv), Z, Cv.D, U, ldr, nc, s));
        FDS_TRY(dense_gemm(nb, Cv.rmax, nc, Vw::At(Cv), 0, rT, 0, rF, one, zero, s));
    }
    C *par = (l - 1 > l0) ? wr[l - 1].p : Vw::wtop(h).p;
    const int64_t ldp = (l - 1 > l0) ? Pn.D : h->Dtop;
    fds_count_launch(), k_child_parent<C><<<nb, 256, 0, s>>>(nb, Cv.d_roff.p, Cv.d_k1.p, Cv.d_par_pos1.p,
                                                             Cv.d_par_pos2.p, Pn.d_doff.p, F, ldr, par, ldp, nc, 0);
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}

// Downward step of level l: y_i from the parent's solution, then
// x_i = z_i - W_i (f~_i - A~_i y_i).
template <class C>
int down_level(fds_handle *h, int l, int nc, cudaStream_t s) {
    typedef View<C> Vw;
    const int l0 = h->l0;
    const C one = Vw::one();
    C mone = one;
    mone.x = -mone.x;
    const int maxnb = fds_max_cells(h);
    MatRefT<C> *rZ = Vw::refs(h).p, *rF = rZ + maxnb, *rT = rF + maxnb;
    auto &wz = Vw::z(h), &wf = Vw::f(h), &wt = Vw::t(h);
    const double esz = sizeof(C);
    Level &Cv = h->lv[l];
    Level &Pn = h->lv[l - 1];
    const int nb = Cv.nb;
    C *Z = wz[l].p, *F = wf[l].p, *Y = wt[l].p;
    C *par = (l - 1 > l0) ? wz[l - 1].p : Vw::wtop(h).p;
    const int64_t ldp = (l - 1 > l0) ? Pn.D : h->Dtop;
    const int64_t ldr = std::max<int64_t>(Cv.Rtot, 1);
    fds_count_launch(), k_child_parent<C><<<nb, 256, 0, s>>>(nb, Cv.d_roff.p, Cv.d_k1.p, Cv.d_par_pos1.p,
                                                             Cv.d_par_pos2.p, Pn.d_doff.p, Y, ldr, par, ldp, nc, 1);
    fds_count_launch(), k_vec_refs<C><<<(nb + 127) / 128, 128, 0, s>>>(nb, Z, Cv.d_doff.p, nc, Cv.D, rZ);
    fds_count_launch(), k_vec_refs<C><<<(nb + 127) / 128, 128, 0, s>>>(nb, Y, Cv.d_roff.p, nc, ldr, rT);
    fds_count_launch(), k_vec_refs<C><<<(nb + 127) / 128, 128, 0, s>>>(nb, F, Cv.d_roff.p, nc, ldr, rF);
    FDS_CUDA_TRY(cudaGetLastError());
    ProfScope ps("a6.down_apply", s);
    ps.flops = 8.0 * (Cv.sum_r2 + Cv.sum_rd) * nc;
    ps.bytes = esz * (Cv.sum_r2 + Cv.sum_rd) + esz * (2.0 * Cv.D + 2.0 * Cv.Rtot) * nc;
    FDS_TRY(dense_gemm(nb, Cv.rmax, nc, Vw::At(Cv), 0, rT, 0, rF, mone, one, s));
    FDS_TRY(dense_gemm(nb, Cv.dmax, nc, Vw::W(Cv), 0, rF, 0, rZ, mone, one, s));
    return FDS_OK;
}

template <class A, class B>
int convert_vec(const A *src, B *dst, int64_t rows, int nc, cudaStream_t s) {
    const int64_t ld = std::max<int64_t>(rows, 1);
    fds_count_launch(), k_convert<A, B><<<256, 256, 0, s>>>(src, dst, rows, ld, ld, nc);
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}

int top_solve(fds_handle *h, int nc, cudaStream_t s) {
    const int64_t ldt = std::max<int64_t>(h->Dtop, 1);
    MatRef tv;
    tv.p = h->wtop.p;
    tv.rows = (int)h->Dtop;
    tv.cols = nc;
    tv.ld = (int)ldt;
    MatRef *rX = h->wrefs.p + 3 * fds_max_cells(h);
    FDS_CUDA_TRY(cudaMemcpyAsync(rX, &tv, sizeof(tv), cudaMemcpyHostToDevice, s));
    ProfScope ps("a6.top_solve", s);
    ps.flops = 8.0 * (double)h->Dtop * h->Dtop * nc;
    ps.bytes = 16.0 * (double)h->Dtop * h->Dtop;
    return dense_lu_solve(1, (int)h->Dtop, nc, h->rtop.p, h->ptop.p, h->d_ptop_off.p, rX, s);
}

}  // namespace

// One sweep over nc columns: the right-hand sides are in sweep_leaf_in of the
// leaf level's precision, the solution is left in sweep_leaf_out.
int sweep_chunk(fds_handle *h, int nc, cudaStream_t s) {
    const int L = h->L, l0 = h->l0;
    const int ls = sweep_split(h);
    const bool mixed = h->opt.precision == FDS_MIXED;
    for (int l = L; l > l0; --l) {
        if (l > ls) FDS_TRY(up_level<cplxf>(h, l, nc, s));
        else FDS_TRY(up_level<cplx>(h, l, nc, s));
        if (l == ls + 1) {
            // complex64 right-hand side of level ls (or the top) -> complex128
            if (ls > l0) FDS_TRY(convert_vec(h->wrf[ls].p, h->wr[ls].p, h->lv[ls].D, nc, s));
            else FDS_TRY(convert_vec(h->wtopf.p, h->wtop.p, h->Dtop, nc, s));
        }
    }
    if (mixed && L == l0) FDS_TRY(convert_vec(h->wtopf.p, h->wtop.p, h->Dtop, nc, s));
    FDS_TRY(top_solve(h, nc, s));
    if (mixed && L == l0) FDS_TRY(convert_vec(h->wtop.p, h->wtopf.p, h->Dtop, nc, s));
    for (int l = l0 + 1; l <= L; ++l) {
        if (l == ls + 1) {
            // complex128 solution of level ls (or the top) -> complex64
            if (ls > l0) FDS_TRY(convert_vec(h->wz[ls].p, h->wzf[ls].p, h->lv[ls].D, nc, s));
            else FDS_TRY(convert_vec(h->wtop.p, h->wtopf.p, h->Dtop, nc, s));
        }
        if (l > ls) FDS_TRY(down_level<cplxf>(h, l, nc, s));
        else FDS_TRY(down_level<cplx>(h, l, nc, s));
    }
    return FDS_OK;
}

template cplx *sweep_leaf_in<cplx>(fds_handle *);
template cplxf *sweep_leaf_in<cplxf>(fds_handle *);
template cplx *sweep_leaf_out<cplx>(fds_handle *);
template cplxf *sweep_leaf_out<cplxf>(fds_handle *);

int fds_solve_impl(fds_handle *h, cplx *d_rhs, int nrhs, cudaStream_t s) {
    if (nrhs <= 0) return FDS_OK;
    if (h->opt.precision == FDS_MIXED) return fds_solve_mixed_impl(h, d_rhs, nrhs, s);
    const int N = h->N;
    const int64_t ld_rhs = 2LL * N;
    const int ncmax = std::min(nrhs, SOLVE_CHUNK);
    FDS_TRY(sweep_workspace(h, ncmax));
    const Level &Lf = h->lv[h->L];
    cplx *leaf_in = sweep_leaf_in<cplx>(h), *leaf_out = sweep_leaf_out<cplx>(h);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    for (int c0 = 0; c0 < nrhs; c0 += SOLVE_CHUNK) {
        const int nc = std::min(SOLVE_CHUNK, nrhs - c0);
        cplx *rhs = d_rhs + (int64_t)c0 * ld_rhs;
        fds_count_launch(), k_leaf_gather<<<1024, 256, 0, s>>>(h->d_leaf_gidx.p, Lf.D, rhs, ld_rhs, leaf_in, nc, 0);
        FDS_CUDA_TRY(cudaGetLastError());
        FDS_TRY(sweep_chunk(h, nc, s));
        fds_count_launch(), k_leaf_gather<<<1024, 256, 0, s>>>(h->d_leaf_gidx.p, Lf.D, rhs, ld_rhs, leaf_out, nc, 1);
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
