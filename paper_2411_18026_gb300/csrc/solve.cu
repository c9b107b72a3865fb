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
        if (!FDS_IN_RANGE(gidx[q], D)) continue;
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
        if (!FDS_IN_RANGE(pr - pb, pdoff[(b >> 1) + 1] - pb)) continue;
        if (dir == 0) parent[pr + c * ldp] = child[o + q + c * ldc];
        else child[o + q + c * ldc] = parent[pr + c * ldp];
    }
}

// precision changes of vector entries: complex128, complex64, float pair
__device__ __forceinline__ void cvt(const cplx &a, cplx &b) { b = a; }
__device__ __forceinline__ void cvt(const cplx &a, cplxf &b) { b = to_c64(a); }
__device__ __forceinline__ void cvt(const cplxf &a, cplx &b) { b = to_c128(a); }
__device__ __forceinline__ void cvt(const cplx &a, float4 &b) {
    const float rh = (float)a.x, ih = (float)a.y;
    b = make_float4(rh, ih, (float)(a.x - (double)rh), (float)(a.y - (double)ih));
}
__device__ __forceinline__ void cvt(const float4 &a, cplx &b) { b = mkc((double)a.x + a.z, (double)a.y + a.w); }
__device__ __forceinline__ void cvt(const cplxf &a, float4 &b) { b = make_float4(a.x, a.y, 0.f, 0.f); }
__device__ __forceinline__ void cvt(const float4 &a, cplxf &b) { b = mkcf(a.x + a.z, a.y + a.w); }

template <class A, class B>
__global__ void k_convert(const A *__restrict__ src, B *dst, int64_t rows, int64_t lds, int64_t ldd, int cols) {
    const int64_t tot = rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % rows, c = e / rows;
        cvt(src[i + c * lds], dst[i + c * ldd]);
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
    static const cplxf *Tm(const Level &v) { return v.Tf.p; }
    static std::vector<DBuf<cplxf>> &z(fds_handle *h) { return h->wzf; }
    static std::vector<DBuf<cplxf>> &f(fds_handle *h) { return h->wff; }
    static std::vector<DBuf<cplxf>> &t(fds_handle *h) { return h->wtf; }
    static std::vector<DBuf<cplxf>> &r(fds_handle *h) { return h->wrf; }
    static DBuf<cplxf> &wtop(fds_handle *h) { return h->wtopf; }
    static DBuf<MatRefF> &refs(fds_handle *h) { return h->wrefsf; }
    static cplxf one() { return mkcf(1, 0); }
};

template <>
struct View<float4> {
    static const MatRefP *Ainv(const Level &v) { return v.rAinvp.p; }
    static const MatRefP *W(const Level &v) { return v.rWp.p; }
    static const MatRefP *At(const Level &v) { return v.rAtp.p; }
    static const float4 *Tm(const Level &v) { return v.Tp.p; }
    static std::vector<DBuf<float4>> &z(fds_handle *h) { return h->wzq; }
    static std::vector<DBuf<float4>> &f(fds_handle *h) { return h->wfq; }
    static std::vector<DBuf<float4>> &t(fds_handle *h) { return h->wtq; }
    static std::vector<DBuf<float4>> &r(fds_handle *h) { return h->wrq; }
    static DBuf<float4> &wtop(fds_handle *h) { return h->wtopq; }
    static DBuf<MatRefP> &refs(fds_handle *h) { return h->wrefsq; }
    static float4 one() { return make_float4(1.f, 0.f, 0.f, 0.f); }
};

}  // namespace

int fds_max_cells(const fds_handle *h) {
    int m = 1;
    for (int l = h->L; l >= h->l0; --l) m = std::max(m, h->lv[l].nb);
    return m;
}

// Arithmetic of each level's sweep: FDS_FP64 complex128 throughout; FDS_MIXED
// complex64 for the levels the build marked (Level::c64, a suffix ending at
// the leaves) and, for the others, complex128 or (sweep_ff) float pairs.
int level_prec(const fds_handle *h, int l) {
    if (h->opt.precision != FDS_MIXED) return PREC_C128;
    if (h->lv[l].c64) return PREC_C64;
    return h->opt.sweep_ff ? PREC_FF : PREC_C128;
}

int sweep_split(const fds_handle *h) {
    if (h->opt.precision != FDS_MIXED || h->L == h->l0) return h->L;
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
    if (Vw::refs(h).n < (size_t)4 * maxnb + 2) FDS_TRY(Vw::refs(h).alloc((size_t)4 * maxnb + 2));
    return FDS_OK;
}

template <class C>
int workspace_prec(fds_handle *h, int ncmax, int prec) {
    // the levels of this precision, the level (or top) above each of them and
    // the top vector, which may carry a converted copy at a precision change
    const int L = h->L, l0 = h->l0;
    FDS_TRY(workspace_levels<C>(h, ncmax, L + 1, L, true));    // top vector and descriptors
    for (int l = L; l > l0; --l) {
        const bool mine = level_prec(h, l) == prec;
        const bool above = l < L && level_prec(h, l + 1) == prec;   // parent of a level of this precision
        if (mine || above) FDS_TRY(workspace_levels<C>(h, ncmax, l, l, false));
    }
    return FDS_OK;
}

int sweep_workspace(fds_handle *h, int ncmax) {
    FDS_TRY(vapply_workspace(h));
    FDS_TRY(workspace_prec<cplx>(h, ncmax, PREC_C128));
    FDS_TRY(grow(h->wtop2, (size_t)std::max<int64_t>(h->Dtop, 1) * ncmax));
    if (h->opt.precision == FDS_MIXED) {
        FDS_TRY(workspace_prec<cplxf>(h, ncmax, PREC_C64));
        if (h->opt.sweep_ff) FDS_TRY(workspace_prec<float4>(h, ncmax, PREC_FF));
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

// vector of level l (l > l0) or of the top (l = l0) in precision C:
// which 0 = right-hand side, 1 = solution
template <class C>
C *level_vec(fds_handle *h, int l, int which) {
    if (l == h->l0) return View<C>::wtop(h).p;
    return which ? View<C>::z(h)[l].p : View<C>::r(h)[l].p;
}

template <class A, class B>
int convert_level(fds_handle *h, int l, int which, int nc, cudaStream_t s) {
    const int64_t rows = l == h->l0 ? h->Dtop : h->lv[l].D;
    const int64_t ld = std::max<int64_t>(rows, 1);
    fds_count_launch(), k_convert<A, B><<<256, 256, 0, s>>>(level_vec<A>(h, l, which), level_vec<B>(h, l, which),
                                                           rows, ld, ld, nc);
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}

// vector of level l (or the top) from precision pa to pb
int convert_prec(fds_handle *h, int l, int which, int pa, int pb, int nc, cudaStream_t s) {
    if (pa == pb) return FDS_OK;
    if (pa == PREC_C64 && pb == PREC_C128) return convert_level<cplxf, cplx>(h, l, which, nc, s);
    if (pa == PREC_C128 && pb == PREC_C64) return convert_level<cplx, cplxf>(h, l, which, nc, s);
    if (pa == PREC_C64 && pb == PREC_FF) return convert_level<cplxf, float4>(h, l, which, nc, s);
    if (pa == PREC_FF && pb == PREC_C64) return convert_level<float4, cplxf>(h, l, which, nc, s);
    if (pa == PREC_FF && pb == PREC_C128) return convert_level<float4, cplx>(h, l, which, nc, s);
    if (pa == PREC_C128 && pb == PREC_FF) return convert_level<cplx, float4>(h, l, which, nc, s);
    return FDS_ERR_ARG;
}

}  // namespace

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


__global__ void k_top_refs(MatRef *rX, cplx *a, cplx *b, int rows, int cols, int ld) {
    if (threadIdx.x < 2) {
        MatRef r;
        r.p = threadIdx.x ? b : a;
        r.rows = rows;
        r.cols = cols;
        r.ld = ld;
        rX[threadIdx.x] = r;
    }
}

// x_top = A_top^{-1} f_top (Sec. 6.3) as one GEMM with the inverse formed at build
int top_solve(fds_handle *h, int nc, cudaStream_t s) {
    const int64_t ldt = std::max<int64_t>(h->Dtop, 1);
    MatRef *rX = h->wrefs.p + 3 * fds_max_cells(h);
    fds_count_launch(), k_top_refs<<<1, 32, 0, s>>>(rX, h->wtop.p, h->wtop2.p, (int)h->Dtop, nc, (int)ldt);
    FDS_CUDA_TRY(cudaGetLastError());
    ProfScope ps("a6.top_solve", s);
    ps.flops = 8.0 * (double)h->Dtop * h->Dtop * nc;
    ps.bytes = 16.0 * (double)h->Dtop * h->Dtop;
    FDS_TRY(dense_gemm(1, (int)h->Dtop, nc, h->rtop_inv.p, 0, rX, 0, rX + 1, mkc(1.0, 0.0), mkc(0.0, 0.0), s));
    FDS_CUDA_TRY(cudaMemcpyAsync(h->wtop.p, h->wtop2.p, sizeof(cplx) * ldt * nc, cudaMemcpyDeviceToDevice, s));
    return FDS_OK;
}

// Woodbury sweep of the original Martinsson–Rokhlin form (FDS_VARIANT_MR2005,
// complex128): up f~_i = F_i f_i into the parent's right-hand side; down
// x_i = G_i f_i + E_i y_i, y_i from the parent's solution.
int up_level_mr2005(fds_handle *h, int l, int nc, cudaStream_t s) {
    const int maxnb = fds_max_cells(h);
    MatRef *rR = h->wrefs.p, *rF = rR + maxnb;
    Level &Cv = h->lv[l];
    Level &Pn = h->lv[l - 1];
    const int nb = Cv.nb;
    const int64_t ldr = std::max<int64_t>(Cv.Rtot, 1);
    cplx *Rh = h->wr[l].p, *F = h->wf[l].p;
    fds_count_launch(), k_vec_refs<cplx><<<(nb + 127) / 128, 128, 0, s>>>(nb, Rh, Cv.d_doff.p, nc, Cv.D, rR);
    fds_count_launch(), k_vec_refs<cplx><<<(nb + 127) / 128, 128, 0, s>>>(nb, F, Cv.d_roff.p, nc, ldr, rF);
    {
        ProfScope ps("a6.mr2005_up", s);
        ps.flops = 8.0 * Cv.sum_rd * nc;
        ps.bytes = 16.0 * Cv.sum_rd + 16.0 * (Cv.D + Cv.Rtot) * nc;
        FDS_TRY(dense_gemm(nb, Cv.rmax, nc, Cv.rmrF.p, 0, rR, 0, rF, mkc(1, 0), mkc(0, 0), s));
    }
    cplx *par = (l - 1 > h->l0) ? h->wr[l - 1].p : h->wtop.p;
    const int64_t ldp = (l - 1 > h->l0) ? Pn.D : h->Dtop;
    fds_count_launch(), k_child_parent<cplx><<<nb, 256, 0, s>>>(nb, Cv.d_roff.p, Cv.d_k1.p, Cv.d_par_pos1.p,
                                                                Cv.d_par_pos2.p, Pn.d_doff.p, F, ldr, par, ldp, nc, 0);
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}

int down_level_mr2005(fds_handle *h, int l, int nc, cudaStream_t s) {
    const int maxnb = fds_max_cells(h);
    MatRef *rR = h->wrefs.p, *rZ = rR + maxnb, *rY = rZ + maxnb;
    Level &Cv = h->lv[l];
    Level &Pn = h->lv[l - 1];
    const int nb = Cv.nb;
    const int64_t ldr = std::max<int64_t>(Cv.Rtot, 1);
    cplx *Rh = h->wr[l].p, *Z = h->wz[l].p, *Y = h->wt[l].p;
    cplx *par = (l - 1 > h->l0) ? h->wz[l - 1].p : h->wtop.p;
    const int64_t ldp = (l - 1 > h->l0) ? Pn.D : h->Dtop;
    fds_count_launch(), k_child_parent<cplx><<<nb, 256, 0, s>>>(nb, Cv.d_roff.p, Cv.d_k1.p, Cv.d_par_pos1.p,
                                                                Cv.d_par_pos2.p, Pn.d_doff.p, Y, ldr, par, ldp, nc, 1);
    fds_count_launch(), k_vec_refs<cplx><<<(nb + 127) / 128, 128, 0, s>>>(nb, Rh, Cv.d_doff.p, nc, Cv.D, rR);
    fds_count_launch(), k_vec_refs<cplx><<<(nb + 127) / 128, 128, 0, s>>>(nb, Z, Cv.d_doff.p, nc, Cv.D, rZ);
    fds_count_launch(), k_vec_refs<cplx><<<(nb + 127) / 128, 128, 0, s>>>(nb, Y, Cv.d_roff.p, nc, ldr, rY);
    FDS_CUDA_TRY(cudaGetLastError());
    ProfScope ps("a6.mr2005_down", s);
    ps.flops = 8.0 * (Cv.sum_d2 + Cv.sum_rd) * nc;
    ps.bytes = 16.0 * (Cv.sum_d2 + Cv.sum_rd) + 16.0 * (2.0 * Cv.D + Cv.Rtot) * nc;
    FDS_TRY(dense_gemm(nb, Cv.dmax, nc, Cv.rmrG.p, 0, rR, 0, rZ, mkc(1, 0), mkc(0, 0), s));
    FDS_TRY(dense_gemm(nb, Cv.dmax, nc, Cv.rmrE.p, 0, rY, 0, rZ, mkc(1, 0), mkc(1, 0), s));
    return FDS_OK;
}

}  // namespace

// One sweep over nc columns: the right-hand sides are in sweep_leaf_in of the
// leaf level's precision, the solution is left in sweep_leaf_out.
int sweep_chunk(fds_handle *h, int nc, cudaStream_t s) {
    const int L = h->L, l0 = h->l0;
    auto prec = [&](int l) { return l == l0 ? PREC_C128 : level_prec(h, l); };
    auto up = [&](int l) -> int {
        switch (prec(l)) {
            case PREC_C64: return up_level<cplxf>(h, l, nc, s);
            case PREC_FF: return up_level<float4>(h, l, nc, s);
            default: return up_level<cplx>(h, l, nc, s);
        }
    };
    auto down = [&](int l) -> int {
        switch (prec(l)) {
            case PREC_C64: return down_level<cplxf>(h, l, nc, s);
            case PREC_FF: return down_level<float4>(h, l, nc, s);
            default: return down_level<cplx>(h, l, nc, s);
        }
    };
    if (h->opt.variant == FDS_VARIANT_MR2005 && L > l0) {
        for (int l = L; l > l0; --l) FDS_TRY(up_level_mr2005(h, l, nc, s));
        FDS_TRY(top_solve(h, nc, s));
        for (int l = l0 + 1; l <= L; ++l) FDS_TRY(down_level_mr2005(h, l, nc, s));
        return FDS_OK;
    }
    if (L == l0) {
        // one cell: the leaf vector is the top vector, held in the leaf precision
        const int pl = h->opt.precision == FDS_MIXED ? PREC_C64 : PREC_C128;
        FDS_TRY(convert_prec(h, l0, 0, pl, PREC_C128, nc, s));
        FDS_TRY(top_solve(h, nc, s));
        return convert_prec(h, l0, 0, PREC_C128, pl, nc, s);
    }
    for (int l = L; l > l0; --l) {
        FDS_TRY(up(l));
        // the parent's right-hand side arrives in this level's precision
        FDS_TRY(convert_prec(h, l - 1, 0, prec(l), prec(l - 1), nc, s));
    }
    FDS_TRY(top_solve(h, nc, s));
    for (int l = l0 + 1; l <= L; ++l) {
        FDS_TRY(convert_prec(h, l - 1, 1, prec(l - 1), prec(l), nc, s));
        FDS_TRY(down(l));
    }
    return FDS_OK;
}

namespace {

// addresses of every buffer a sweep touches: a graph captured against one
// layout must not be replayed after the workspace was regrown
uint64_t workspace_hash(const fds_handle *h) {
    uint64_t x = 1469598103934665603ull;
    auto mix = [&](const void *p, size_t n) {
        x = (x ^ (uint64_t)(uintptr_t)p) * 1099511628211ull;
        x = (x ^ (uint64_t)n) * 1099511628211ull;
    };
    auto vec = [&](const auto &v) {
        for (const auto &b : v) mix(b.p, b.n);
    };
    vec(h->wz); vec(h->wf); vec(h->wt); vec(h->wr);
    vec(h->wzf); vec(h->wff); vec(h->wtf); vec(h->wrf);
    vec(h->wzq); vec(h->wfq); vec(h->wtq); vec(h->wrq);
    mix(h->wtop.p, h->wtop.n); mix(h->wtop2.p, h->wtop2.n); mix(h->wtopf.p, h->wtopf.n);
    mix(h->wtopq.p, h->wtopq.n); mix(h->wrefs.p, h->wrefs.n); mix(h->wrefsf.p, h->wrefsf.n);
    mix(h->wrefsq.p, h->wrefsq.n); mix(h->wvref.p, h->wvref.n);
    return x;
}

bool capturable(cudaStream_t s) {
    if (s == 0 || s == cudaStreamLegacy || s == cudaStreamPerThread) return false;
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &st) == cudaSuccess && st == cudaStreamCaptureStatusNone;
}

}  // namespace

int sweep_chunk_run(fds_handle *h, int nc, cudaStream_t s) {
    if (!h->opt.use_graph || !capturable(s)) return sweep_chunk(h, nc, s);
    const uint64_t hash = workspace_hash(h);
    fds_handle::SweepGraph *g = nullptr;
    for (auto &e : h->sweep_graphs)
        if (e.first == nc) g = &e.second;
    if (g && g->exec && g->ws_hash == hash) {
        fds_count_launch();
        FDS_CUDA_TRY(cudaGraphLaunch(g->exec, s));
        return FDS_OK;
    }
    // capture the sweep (the workspace is allocated before any sweep, so the
    // captured launches allocate nothing), then replay it; if anything in it
    // cannot be captured, this sweep runs as plain launches
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return sweep_chunk(h, nc, s);
    }
    int rc;
    {
        ProfCaptureScope pc;
        rc = sweep_chunk(h, nc, s);
    }
    const cudaError_t ec = cudaStreamEndCapture(s, &graph);
    cudaGraphExec_t exec = nullptr;
    const bool ok = rc == FDS_OK && ec == cudaSuccess && graph && workspace_hash(h) == hash &&
                    cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
        cudaGetLastError();
        if (exec) cudaGraphExecDestroy(exec);
        return sweep_chunk(h, nc, s);
    }
    if (!g) {
        h->sweep_graphs.push_back({nc, fds_handle::SweepGraph{}});
        g = &h->sweep_graphs.back().second;
    }
    if (g->exec) cudaGraphExecDestroy(g->exec);
    g->exec = exec;
    g->ws_hash = hash;
    fds_count_launch();
    FDS_CUDA_TRY(cudaGraphLaunch(g->exec, s));
    return FDS_OK;
}

template cplx *sweep_leaf_in<cplx>(fds_handle *);
template cplxf *sweep_leaf_in<cplxf>(fds_handle *);
template float4 *sweep_leaf_in<float4>(fds_handle *);
template cplx *sweep_leaf_out<cplx>(fds_handle *);
template cplxf *sweep_leaf_out<cplxf>(fds_handle *);
template float4 *sweep_leaf_out<float4>(fds_handle *);

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
        FDS_TRY(sweep_chunk_run(h, nc, s));
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
