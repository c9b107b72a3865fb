// Mixed-precision solve (FDS_MIXED): the solve sweep of Sec. 6.2-6.3 runs on
// complex64 copies of the factors and is refined against the compressed
// operator the factorisation inverts, from FP64 entries, applied in FP64 or
// (default) split once into float pairs and applied in double-float
// arithmetic on the FP32 pipe (about 44 significant bits):
//
//   A = D_L + U_L B_L V_L,   B_l = S_{l-1} + U_{l-1} B_{l-1} V_{l-1}  (l > l0+1),
//   B_{l0+1} = S_{l0} + A_top,off
//
// where D_L holds the leaf diagonal blocks A^{J_p J_p} (eq. (block_ax=f)),
// U_l = V_l^H and V_l are the interpolation matrices of level l (Sec. 7.1),
// S_l the sibling blocks of the level-l cells (the off-diagonal blocks of
// eq. (A_rearrangement), original entries between the children's skeletons)
// and A_top,off the original entries between different top cells (Sec. 6.3).
// With x_L = x, the apply is
//   up    x_{l-1} = V_l x_l                        (children -> parent order)
//   top   y_{l0} = (A_top,off + S_{l0}) x_{l0}     (+ D_L x_L instead of S when l0 = L)
//   down  y_l = V_l^H y_{l-1}|_l + S_l x_l,  y_L = V_L^H y_{L-1}|_L + D_L x_L.
// Refinement (per column chunk): x = sweep(f); repeat r = f - A x,
// x += sweep(r) until max_c ||r_c|| / ||f_c|| <= tol.
#include <algorithm>
#include <cmath>

#include "fds_internal.cuh"
#include "prof.cuh"
#include "solve.cuh"
#include "vapply.cuh"
#include "fw_tc.cuh"

namespace {

__global__ void k_to_c64(const cplx *__restrict__ src, cplxf *dst, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = to_c64(src[e]);
}

template <class T>
__global__ void k_refs(int nb, T *base, const int64_t *__restrict__ off, int cols, int64_t ld, MatRefT<T> *out) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    out[b].p = base + off[b];
    out[b].rows = (int)(off[b + 1] - off[b]);
    out[b].cols = cols;
    out[b].ld = (int)ld;
}

// child skeleton vector (R x cols) <-> parent DOF vector (Dp x cols)
// dir 0: parent[pos] = child;  dir 1: child = parent[pos]
template <class T>
__global__ void k_child_parent_t(int nb, const int64_t *__restrict__ roff, const int *__restrict__ k1,
                                 const int *__restrict__ pos1, const int *__restrict__ pos2,
                                 const int64_t *__restrict__ pdoff, T *child, int64_t ldc, T *parent, int64_t ldp,
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

// complex128 -> float pair (re_hi, im_hi, re_lo, im_lo)
__global__ void k_split(const cplx *__restrict__ src, float4 *dst, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const cplx v = src[e];
        const float rh = (float)v.x, ih = (float)v.y;
        dst[e] = make_float4(rh, ih, (float)(v.x - (double)rh), (float)(v.y - (double)ih));
    }
}

__device__ __forceinline__ cplx to_c128(const cplx &v) { return v; }
__device__ __forceinline__ cplx to_c128(const float4 &v) {
    return mkc((double)v.x + (double)v.z, (double)v.y + (double)v.w);
}

// r = f - y in leaf order (y may be null: r = f), stored as complex64 for the
// sweep; norms[2c] += |r|^2, norms[2c+1] += |f|^2 over column c.
__device__ __forceinline__ void put(const cplx &a, cplxf &b) { b = to_c64(a); }
__device__ __forceinline__ void put(const cplx &a, float4 &b) {
    const float rh = (float)a.x, ih = (float)a.y;
    b = make_float4(rh, ih, (float)(a.x - (double)rh), (float)(a.y - (double)ih));
}

// r = f - y for the compact columns c (right-hand side cmap[c]), leaf order,
// with ||r||^2 and ||f||^2 per column
template <class T, class LT>
__global__ void k_residual(const int *__restrict__ gidx, int64_t D, const cplx *__restrict__ F, int64_t ldf,
                           const int *__restrict__ cmap, const T *__restrict__ Y, LT *R, double *norms) {
    const int c = blockIdx.y;
    const int64_t fc = cmap[c];
    double rr = 0.0, ff = 0.0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < D; q += (int64_t)gridDim.x * blockDim.x) {
        if (!FDS_IN_RANGE(gidx[q], D)) continue;
        const cplx f = F[gidx[q] + fc * ldf];
        cplx r = f;
        if (Y) r = csub(f, to_c128(Y[q + c * D]));
        put(r, R[q + c * D]);
        rr += cabs2(r);
        ff += cabs2(f);
    }
    for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_xor_sync(0xffffffffu, rr, o);
        ff += __shfl_xor_sync(0xffffffffu, ff, o);
    }
    __shared__ double sr[32], sf[32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sr[w] = rr; sf[w] = ff; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { a += sr[i]; b += sf[i]; }
        atomicAdd(&norms[2 * c], a);
        atomicAdd(&norms[2 * c + 1], b);
    }
}

// X (+)= dX (complex64 correction), leaf order
template <class LT>
__global__ void k_update(cplx *X, const LT *__restrict__ dX, int64_t n, int set) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const cplx d = to_c128(dX[e]);
        X[e] = set ? d : cadd(X[e], d);
    }
}

// X -= dX in the columns c with undo[c] != 0 (D entries per column): takes
// back the last refinement correction of the columns it did not improve
template <typename LT>
__global__ void k_undo_cols(cplx *X, const LT *__restrict__ dX, int64_t D, int cols, const int *__restrict__ undo) {
    const int64_t n = D * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        if (!undo[e / D]) continue;
        const cplx d = to_c128(dX[e]);
        X[e] = mkc(X[e].x - d.x, X[e].y - d.y);
    }
}

// dst column j = src column perm[j] (D entries per column)
template <class T>
__global__ void k_permute_cols(const T *__restrict__ src, T *dst, int64_t D, const int *__restrict__ perm, int cols) {
    const int64_t n = D * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = src[e % D + (int64_t)perm[e / D] * D];
}

// natural-order right-hand side column cmap[c] <- leaf-order compact column c
__global__ void k_leaf_scatter(const int *__restrict__ gidx, int64_t D, const cplx *__restrict__ X, cplx *out,
                               int64_t ldo, const int *__restrict__ cmap, int cols) {
    const int64_t tot = D * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = e % D, c = e / D;
        if (!FDS_IN_RANGE(gidx[q], D)) continue;
        out[gidx[q] + (int64_t)cmap[c] * ldo] = X[q + c * D];
    }
}

template <class T>
int grow(DBuf<T> &b, size_t n) {
    if (b.n >= n && b.p) return FDS_OK;
    return b.alloc(n);
}

int convert(const DBuf<cplx> &src, DBuf<cplxf> &dst, cudaStream_t s) {
    FDS_TRY(dst.alloc(src.n));
    if (src.n) {
        fds_count_launch(), k_to_c64<<<1024, 256, 0, s>>>(src.p, dst.p, (int64_t)src.n);
        FDS_CUDA_TRY(cudaGetLastError());
    }
    return FDS_OK;
}

// compact sibling blocks from the parent's d x d coupling block
__global__ void k_extract_s(const MatRef *__restrict__ S, const int *__restrict__ sperm,
                            const int64_t *__restrict__ doff, const int *__restrict__ ra,
                            const int *__restrict__ rb, const int64_t *__restrict__ scoff, cplx *out) {
    const int p = blockIdx.x;
    const MatRef M = S[p];
    const int a = ra[p], b = rb[p];
    const int *pm = sperm + doff[p];
    cplx *o0 = out + scoff[2 * p], *o1 = out + scoff[2 * p + 1];
    for (int64_t e = threadIdx.x; e < (int64_t)a * b; e += blockDim.x) {
        const int i = (int)(e % a), j = (int)(e / a);
        o0[i + (int64_t)j * a] = M.p[pm[i] + (int64_t)pm[a + j] * M.ld];
    }
    for (int64_t e = threadIdx.x; e < (int64_t)a * b; e += blockDim.x) {
        const int i = (int)(e % b), j = (int)(e / b);
        o1[i + (int64_t)j * b] = M.p[pm[a + i] + (int64_t)pm[j] * M.ld];
    }
}

template <class T>
__global__ void k_srefs(int nb, const T *Sc, const int64_t *__restrict__ scoff, const int *__restrict__ ra,
                        const int *__restrict__ rb, const int64_t *__restrict__ doff, const int *sperm, const T *x,
                        int64_t ldx, T *y, int64_t ldy, int nc, MatRefT<T> *A, MatRefT<T> *B, MatRefT<T> *Cm,
                        RowMaps *M) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 2 * nb) return;
    const int p = e >> 1, side = e & 1;
    const int a = ra[p], b = rb[p];
    const int rows = side ? b : a, cols = side ? a : b;
    const int *pm = sperm + doff[p];
    A[e].p = (T *)Sc + scoff[e];
    A[e].rows = rows;
    A[e].cols = cols;
    A[e].ld = rows > 1 ? rows : 1;
    B[e].p = (T *)x + doff[p];
    B[e].rows = (int)(doff[p + 1] - doff[p]);
    B[e].cols = nc;
    B[e].ld = (int)ldx;
    Cm[e].p = y + doff[p];
    Cm[e].rows = rows;
    Cm[e].cols = nc;
    Cm[e].ld = (int)ldy;
    M[e].b = side ? pm : pm + a;
    M[e].c = side ? pm + a : pm;
    M[e].cext = (int)(doff[p + 1] - doff[p]);
}

double level_d2(const Level &C) {
    double s = 0;
    for (int b = 0; b < C.nb; ++b) {
        const double d = (double)(C.doff[b + 1] - C.doff[b]);
        s += d * d;
    }
    return s;
}

// The forward operator and its vectors in one arithmetic: complex128 (FP64
// products) or float4 float pairs (double-float products on the FP32 pipe).
template <class T>
struct Fw;

template <>
struct Fw<cplx> {
    static const MatRef *V(const Level &c) { return c.rV.p; }
    static const cplx *Tm(const Level &c) { return c.T.p; }
    static const MatRef *D(const Level &c) { return c.rDfw.p; }
    static const MatRef *S(const Level &c) { return c.rSfw.p; }
    static const cplx *Sc(const Level &c) { return c.Sc.p; }
    static const MatRef *top(const fds_handle *h) { return h->rtop_off.p; }
    static std::vector<DBuf<cplx>> &z(fds_handle *h) { return h->wz; }
    static std::vector<DBuf<cplx>> &t(fds_handle *h) { return h->wt; }
    static std::vector<DBuf<cplx>> &y(fds_handle *h) { return h->wy; }
    static DBuf<cplx> &xtop(fds_handle *h) { return h->wtop; }
    static DBuf<cplx> &ytop(fds_handle *h) { return h->wytop; }
    static DBuf<MatRef> &refs(fds_handle *h) { return h->wrefs; }
    static int gemm(int batch, int m, int n, const MatRef *A, int opA, const MatRef *B, const MatRef *C, int acc,
                    cudaStream_t s) {
        return dense_gemm_rt(batch, m, n, A, opA, B, C, mkc(1, 0), mkc(acc ? 1 : 0, 0), s);
    }
};

template <>
struct Fw<float4> {
    static const MatRefP *V(const Level &c) { return c.rVp.p; }
    static const float4 *Tm(const Level &c) { return c.Tp.p; }
    static const MatRefP *D(const Level &c) { return c.rDp.p; }
    static const MatRefP *S(const Level &c) { return c.rSp.p; }
    static const float4 *Sc(const Level &c) { return c.Scp.p; }
    static const MatRefP *top(const fds_handle *h) { return h->rtop_offp.p; }
    static std::vector<DBuf<float4>> &z(fds_handle *h) { return h->wzp; }
    static std::vector<DBuf<float4>> &t(fds_handle *h) { return h->wtp; }
    static std::vector<DBuf<float4>> &y(fds_handle *h) { return h->wyp; }
    static DBuf<float4> &xtop(fds_handle *h) { return h->wtopp; }
    static DBuf<float4> &ytop(fds_handle *h) { return h->wytopp; }
    static DBuf<MatRefP> &refs(fds_handle *h) { return h->wrefsp; }
    static int gemm(int batch, int m, int n, const MatRefP *A, int opA, const MatRefP *B, const MatRefP *C, int acc,
                    cudaStream_t s) {
        return dense_gemm_ffp(batch, m, n, A, opA, B, C, acc, s);
    }
};

// Forward-apply workspace: x_l (l0 < l < L), skeleton temporaries, y_l, top.
template <class T>
int forward_workspace(fds_handle *h, int ncmax) {
    typedef Fw<T> F;
    const int L = h->L, l0 = h->l0;
    auto &wz = F::z(h), &wt = F::t(h), &wy = F::y(h);
    if ((int)wz.size() != L + 1) wz = std::vector<DBuf<T>>(L + 1);
    if ((int)wt.size() != L + 1) wt = std::vector<DBuf<T>>(L + 1);
    if ((int)wy.size() != L + 1) wy = std::vector<DBuf<T>>(L + 1);
    for (int l = L; l > l0; --l) {
        const Level &C = h->lv[l];
        if (l < L) FDS_TRY(grow(wz[l], (size_t)C.D * ncmax));
        FDS_TRY(grow(wt[l], (size_t)std::max<int64_t>(C.Rtot, 1) * ncmax));
        FDS_TRY(grow(wy[l], (size_t)C.D * ncmax));
    }
    FDS_TRY(grow(F::xtop(h), (size_t)std::max<int64_t>(h->Dtop, 1) * ncmax));
    FDS_TRY(grow(F::ytop(h), (size_t)std::max<int64_t>(h->Dtop, 1) * ncmax));
    const int maxnb = fds_max_cells(h);
    if (F::refs(h).n < (size_t)4 * maxnb + 2) FDS_TRY(F::refs(h).alloc((size_t)4 * maxnb + 2));
    return FDS_OK;
}

// Leaf-order output vector of the forward apply.
template <class T>
T *forward_out(fds_handle *h) {
    return (h->L > h->l0) ? Fw<T>::y(h)[h->L].p : Fw<T>::ytop(h).p;
}

// y_l += S_l x_l through the compact sibling blocks of level l (a parent level)
template <class T>
int apply_S(fds_handle *h, const Level &C, const T *x, int64_t ldx, T *y, int64_t ldy, int nc, cudaStream_t s) {
    const int nb = C.nb;
    if (nb == 0) return FDS_OK;
    const int maxnb = fds_max_cells(h);
    const size_t need = (size_t)2 * maxnb * (3 * sizeof(MatRefT<T>) + sizeof(RowMaps)) + 64;
    if (h->wvref.n < need) FDS_TRY(h->wvref.alloc(need));
    MatRefT<T> *A = reinterpret_cast<MatRefT<T> *>(h->wvref.p);
    MatRefT<T> *B = A + 2 * maxnb, *Cr = B + 2 * maxnb;
    RowMaps *M = reinterpret_cast<RowMaps *>(Cr + 2 * maxnb);
    fds_count_launch(), k_srefs<T><<<(2 * nb + 127) / 128, 128, 0, s>>>(
        nb, Fw<T>::Sc(C), C.d_scoff.p, C.d_ra.p, C.d_rb.p, C.d_doff.p, C.d_sperm.p, x, ldx, y, ldy, nc, A, B, Cr,
        M);
    FDS_CUDA_TRY(cudaGetLastError());
    return dense_gemm_map(2 * nb, std::max(C.srmax, 1), nc, A, 0, B, Cr, M, 1, s);
}

// products on the tensor cores (fw_engine = FDS_FW_TENSOR): float-pair
// vectors, with the plans of every level prepared by fds_mixed_prepare
template <class T>
bool fw_on_tensor(const fds_handle *h) {
    return false;
}
template <>
bool fw_on_tensor<float4>(const fds_handle *h) {
    return h->oz_jobs;
}
inline int oz_run(fds_handle *, const std::vector<OzPlan> &, const cplx *, int64_t, cplx *, int64_t, int,
                  cudaStream_t) {
    return FDS_ERR_STATE;
}
inline int oz_run(fds_handle *h, const std::vector<OzPlan> &P, const float4 *x, int64_t ldx, float4 *y, int64_t ldy,
                  int nc, cudaStream_t s) {
    return oz_plan_apply(h, P, x, ldx, y, ldy, nc, s);
}
inline int oz_leaf(fds_handle *, Level &, const cplx *, cplx *, int64_t, int, cudaStream_t) { return FDS_ERR_STATE; }
inline int oz_leaf(fds_handle *h, Level &C, const float4 *x, float4 *y, int64_t ld, int nc, cudaStream_t s) {
    return oz_leaf_apply(h, C, x, y, ld, nc, s);
}
inline int vskel(const Level &, int, const cplx *, int64_t, cplx *, int64_t, int, cudaStream_t) {
    return FDS_ERR_STATE;
}
inline int vskel(const Level &C, int dir, const float4 *x, int64_t ldx, float4 *y, int64_t ldy, int nc,
                 cudaStream_t s) {
    return vskel_apply<float4>(C, dir, x, ldx, y, ldy, nc, s);
}

// Y = A X for nc leaf-order columns (both D_L x nc, column-major).
template <class T>
int forward_apply(fds_handle *h, const T *X, T *Y, int nc, cudaStream_t s) {
    typedef Fw<T> F;
    const int L = h->L, l0 = h->l0;
    const int maxnb = fds_max_cells(h);
    MatRefT<T> *rZ = F::refs(h).p, *rT = rZ + maxnb, *rY = rT + maxnb, *rX = rY + maxnb;   // rX: 2 slots
    auto &wz = F::z(h), &wt = F::t(h), &wy = F::y(h);
    ProfScope ps("a7.forward_apply", s);
    const bool tc = fw_on_tensor<T>(h);
    double fl = 0;
    // up
    for (int l = L; l > l0; --l) {
        Level &C = h->lv[l];
        Level &Pn = h->lv[l - 1];
        const int nb = C.nb;
        const int64_t ldr = std::max<int64_t>(C.Rtot, 1);
        T *xl = (l == L) ? (T *)X : wz[l].p;
        {
            ProfScope pv("a7.fw_interp_up", s);
            pv.flops = 8.0 * C.sum_tm * nc;
            if (tc) {
                FDS_TRY(vskel(C, 0, xl, C.D, wt[l].p, ldr, nc, s));
                FDS_TRY(oz_run(h, C.oz_up, xl, C.D, wt[l].p, ldr, nc, s));
            } else {
                FDS_TRY(apply_V<T>(h, C, F::Tm(C), xl, C.D, wt[l].p, ldr, nc, s));
            }
        }
        T *par = (l - 1 > l0) ? wz[l - 1].p : F::xtop(h).p;
        const int64_t ldp = (l - 1 > l0) ? Pn.D : h->Dtop;
        fds_count_launch(), k_child_parent_t<T><<<nb, 256, 0, s>>>(nb, C.d_roff.p, C.d_k1.p, C.d_par_pos1.p,
                                                                   C.d_par_pos2.p, Pn.d_doff.p, wt[l].p, ldr, par,
                                                                   ldp, nc, 0);
        FDS_CUDA_TRY(cudaGetLastError());
        fl += 8.0 * C.sum_tm * nc;
    }
    // top: off-diagonal blocks between top cells, then the block diagonal
    {
        Level &Tl = h->lv[l0];
        T *xt = (L > l0) ? F::xtop(h).p : (T *)X;
        T *yt = (L > l0) ? F::ytop(h).p : Y;
        const int ld = (int)std::max<int64_t>(h->Dtop, 1);
        MatRefT<T> hv[2];
        hv[0].p = xt; hv[0].rows = (int)h->Dtop; hv[0].cols = nc; hv[0].ld = ld;
        hv[1].p = yt; hv[1].rows = (int)h->Dtop; hv[1].cols = nc; hv[1].ld = ld;
        ProfScope pt("a7.fw_top", s);
        pt.flops = 8.0 * (double)h->Dtop * h->Dtop * nc;
        FDS_CUDA_TRY(cudaMemcpyAsync(rX, hv, sizeof(hv), cudaMemcpyHostToDevice, s));
        FDS_TRY(F::gemm(1, (int)h->Dtop, nc, F::top(h), 0, rX, rX + 1, 0, s));
        fl += 8.0 * (double)h->Dtop * h->Dtop * nc;
        if (L > l0) {
            if (tc) FDS_TRY(oz_run(h, Tl.oz_sib, xt, h->Dtop, yt, h->Dtop, nc, s));
            else FDS_TRY(apply_S<T>(h, Tl, xt, h->Dtop, yt, h->Dtop, nc, s));
            fl += 8.0 * Tl.sum_s2 * nc;
        } else {
            fds_count_launch(), k_refs<T><<<(Tl.nb + 127) / 128, 128, 0, s>>>(Tl.nb, xt, Tl.d_doff.p, nc, h->Dtop,
                                                                              rZ);
            fds_count_launch(), k_refs<T><<<(Tl.nb + 127) / 128, 128, 0, s>>>(Tl.nb, yt, Tl.d_doff.p, nc, h->Dtop,
                                                                              rY);
            FDS_TRY(F::gemm(Tl.nb, Tl.dmax, nc, F::D(Tl), 0, rZ, rY, 1, s));
            fl += 8.0 * level_d2(Tl) * nc;
        }
    }
    // down
    for (int l = l0 + 1; l <= L; ++l) {
        Level &C = h->lv[l];
        Level &Pn = h->lv[l - 1];
        const int nb = C.nb;
        const int64_t ldr = std::max<int64_t>(C.Rtot, 1);
        T *ypar = (l - 1 > l0) ? wy[l - 1].p : F::ytop(h).p;
        const int64_t ldp = (l - 1 > l0) ? Pn.D : h->Dtop;
        T *yl = (l == L) ? Y : wy[l].p;
        T *xl = (l == L) ? (T *)X : wz[l].p;
        fds_count_launch(), k_child_parent_t<T><<<nb, 256, 0, s>>>(nb, C.d_roff.p, C.d_k1.p, C.d_par_pos1.p,
                                                                   C.d_par_pos2.p, Pn.d_doff.p, wt[l].p, ldr, ypar,
                                                                   ldp, nc, 1);
        {
            ProfScope pv("a7.fw_interp_down", s);
            pv.flops = 8.0 * C.sum_tm * nc;
            if (tc) {
                FDS_TRY(vskel(C, 1, wt[l].p, ldr, yl, C.D, nc, s));
                FDS_TRY(oz_run(h, C.oz_down, wt[l].p, ldr, yl, C.D, nc, s));
            } else {
                FDS_TRY(apply_VH<T>(h, C, F::Tm(C), wt[l].p, ldr, yl, C.D, nc, s));
            }
        }
        if (l < L) {
            ProfScope pss("a7.fw_sibling", s);
            pss.flops = 8.0 * C.sum_s2 * nc;
            if (tc) FDS_TRY(oz_run(h, C.oz_sib, xl, C.D, yl, C.D, nc, s));
            else FDS_TRY(apply_S<T>(h, C, xl, C.D, yl, C.D, nc, s));
            fl += 8.0 * (C.sum_tm + C.sum_s2) * nc;
        } else {
            ProfScope pd("a7.fw_leaf_diag", s);
            pd.flops = 8.0 * level_d2(C) * nc;
            if (tc && C.oz_a.p) {
                FDS_TRY(oz_leaf(h, C, xl, yl, C.D, nc, s));
            } else {
                fds_count_launch(), k_refs<T><<<(nb + 127) / 128, 128, 0, s>>>(nb, yl, C.d_doff.p, nc, C.D, rY);
                fds_count_launch(), k_refs<T><<<(nb + 127) / 128, 128, 0, s>>>(nb, xl, C.d_doff.p, nc, C.D, rZ);
                FDS_CUDA_TRY(cudaGetLastError());
                FDS_TRY(F::gemm(nb, C.dmax, nc, F::D(C), 0, rZ, rY, 1, s));
            }
            fl += 8.0 * (C.sum_tm + level_d2(C)) * nc;
        }
    }
    ps.flops = fl;
    return FDS_OK;
}

int split_blocks(const DBuf<cplx> &src, DBuf<float4> &dst, DBuf<MatRefP> &rdst, const std::vector<int64_t> &off,
                 const std::vector<int> &rows, const std::vector<int> &cols, cudaStream_t s) {
    FDS_TRY(dst.alloc(src.n));
    if (src.n) {
        fds_count_launch(), k_split<<<1024, 256, 0, s>>>(src.p, dst.p, (int64_t)src.n);
        FDS_CUDA_TRY(cudaGetLastError());
    }
    return make_refs_t(rdst, dst.p, off, rows, cols, s);
}

}  // namespace

int fds_keep_blocks(const Level &Lv, DBuf<cplx> &dst, DBuf<MatRef> &rdst, cudaStream_t s) {
    const int64_t n = Lv.offA.empty() ? 0 : Lv.offA[Lv.nb];
    FDS_TRY(dst.alloc((size_t)n));
    if (n) FDS_CUDA_TRY(cudaMemcpyAsync(dst.p, Lv.LU.p, sizeof(cplx) * n, cudaMemcpyDeviceToDevice, s));
    std::vector<int> d(Lv.nb);
    for (int b = 0; b < Lv.nb; ++b) d[b] = Lv.n1[b] + Lv.n2[b];
    return make_refs_t(rdst, dst.p, Lv.offA, d, d, s);
}

// Tensor-core products of level C: the plans of its interpolation blocks
// (up: out[skeleton rows] += T^c x[other rows]; down: y[other rows] =
// T^cH t) and, at the leaf level, the slices of its diagonal blocks for the
// leaf kernel.
int oz_interp_leaf_plans(fds_handle *h, Level &C, bool leaf, cudaStream_t s, int64_t &bytes) {
    std::vector<int> vmap(C.D);
    for (int b = 0; b < C.nb; ++b)
        for (int c = 0; c < 2; ++c) {
            const int n = c ? C.n2[b] : C.n1[b], coff = c ? C.n1[b] : 0;
            for (int q = 0; q < n; ++q) vmap[C.doff[b] + coff + q] = coff + C.perm[C.permoff[2 * b + c] + q];
        }
    std::vector<OzSpec> up, down;
    up.reserve(2 * (size_t)C.nb);
    down.reserve(2 * (size_t)C.nb);
    for (int b = 0; b < C.nb; ++b)
        for (int c = 0; c < 2; ++c) {
            const int n = c ? C.n2[b] : C.n1[b], k = c ? C.k2[b] : C.k1[b], m = n - k;
            const int coff = c ? C.n1[b] : 0;
            const int *vm = vmap.data() + C.doff[b] + coff;
            OzSpec q;
            q.a = C.T.p + C.toff_h[2 * b + c];
            q.lda = std::max(k, 1);
            q.op = 0;              // out (k rows) += T (k x m) x[rest]
            q.m = k;
            q.k = m;
            q.x_row = C.doff[b];
            q.xmap = vm + k;
            q.y_row = C.roff[b] + (c ? C.k1[b] : 0);
            up.push_back(q);
            q.op = 1;              // y[rest] (m rows) = T^H (m x k) t
            q.xmap = nullptr;
            q.m = m;
            q.k = k;
            q.x_row = C.roff[b] + (c ? C.k1[b] : 0);
            q.y_row = C.doff[b];
            q.ymap = vm + k;
            q.set = true;
            down.push_back(q);
        }
    FDS_TRY(oz_plan_build(up, C.oz_up, s));
    FDS_TRY(oz_plan_build(down, C.oz_down, s));
    for (auto *v : {&C.oz_up, &C.oz_down})
        for (const OzPlan &P : *v) bytes += (int64_t)(P.aslices.bytes() + P.rowexp.bytes());
    if (leaf && C.dmax <= 128) {   // larger leaves stay double-float
        FDS_TRY(oz_leaf_prepare(C, C.rDfw.p, s));
        bytes += (int64_t)(C.oz_a.bytes() + C.oz_rowexp.bytes());
    }
    return FDS_OK;
}

int fds_mixed_prepare(fds_handle *h) {
    cudaStream_t s = h->stream;
    const int L = h->L, l0 = h->l0;
    const int ls = sweep_split(h);
    int64_t bytes = 0;
    for (int l = ls; l > l0; --l) {
        const Level &C = h->lv[l];
        bytes += (int64_t)(C.Ainv.bytes() + C.W.bytes() + C.At.bytes() + C.V.bytes() + C.Dfw.bytes() +
                           C.Sfw.bytes());
    }
    for (int l = L; l > ls; --l) {
        Level &C = h->lv[l];
        std::vector<int> dv(C.nb), rv(C.nb);
        for (int b = 0; b < C.nb; ++b) {
            dv[b] = C.n1[b] + C.n2[b];
            rv[b] = C.k1[b] + C.k2[b];
        }
        FDS_TRY(convert(C.T, C.Tf, s));
        if (C.Ainvf.p) {   // merged in complex64 by the build
            bytes += (int64_t)(C.Ainvf.bytes() + C.Wf.bytes() + C.Atf.bytes() + C.Vf.bytes() + C.V.bytes() +
                               C.Dfw.bytes() + C.Sfw.bytes());
            continue;
        }
        FDS_TRY(convert(C.Ainv, C.Ainvf, s));
        FDS_TRY(convert(C.W, C.Wf, s));
        FDS_TRY(convert(C.At, C.Atf, s));
        FDS_TRY(convert(C.V, C.Vf, s));
        FDS_TRY(make_refs_t(C.rAinvf, C.Ainvf.p, C.offA, dv, dv, s));
        FDS_TRY(make_refs_t(C.rWf, C.Wf.p, C.offW, dv, rv, s));
        FDS_TRY(make_refs_t(C.rAtf, C.Atf.p, C.offAt, rv, rv, s));
        FDS_TRY(make_refs_t(C.rVf, C.Vf.p, C.offV, rv, dv, s));
        bytes += (int64_t)(C.Ainvf.bytes() + C.Wf.bytes() + C.Atf.bytes() + C.Vf.bytes() + C.V.bytes() +
                           C.Dfw.bytes() + C.Sfw.bytes());
    }
    bytes += (int64_t)h->lv[l0].Sfw.bytes() + (int64_t)h->lv[l0].Dfw.bytes();
    bytes += (int64_t)(h->Atop.bytes() + h->ptop.bytes() + h->Atop_off.bytes());
    for (int l = ls; l > l0; --l) {
        Level &C = h->lv[l];
        if (level_prec(h, l) != PREC_FF) continue;
        std::vector<int> dv(C.nb), rv(C.nb);
        for (int b = 0; b < C.nb; ++b) {
            dv[b] = C.n1[b] + C.n2[b];
            rv[b] = C.k1[b] + C.k2[b];
        }
        FDS_TRY(split_blocks(C.Ainv, C.Ainvp, C.rAinvp, C.offA, dv, dv, s));
        FDS_TRY(split_blocks(C.W, C.Wp, C.rWp, C.offW, dv, rv, s));
        FDS_TRY(split_blocks(C.At, C.Atp, C.rAtp, C.offAt, rv, rv, s));
    }
    // fw_engine = FDS_FW_TENSOR: every block product of the forward operator
    // (leaf, interpolation, sibling) on the tensor cores
    const bool tensor_fw = h->opt.ir_apply == FDS_APPLY_FF && h->opt.fw_engine == FDS_FW_TENSOR && L > l0;
    // compact sibling blocks of every parent level (l0 .. L-1): child a's and
    // b's skeleton DOFs of the parent, grouped by child
    for (int l = L - 1; l >= l0; --l) {
        Level &Pn = h->lv[l];
        const Level &Ch = h->lv[l + 1];
        if (!Pn.Sfw.p) continue;
        std::vector<int> sperm(Pn.D), ra(Pn.nb), rb(Pn.nb);
        std::vector<int64_t> scoff(2 * (size_t)Pn.nb + 1, 0);
        Pn.srmax = 0;
        Pn.sum_s2 = 0;
        for (int p = 0; p < Pn.nb; ++p) {
            const int a = 2 * p, b = 2 * p + 1;
            const int n1p = Pn.n1[p];
            int q = 0;
            const int64_t o = Pn.doff[p];
            for (int i = 0; i < Ch.k1[a]; ++i) sperm[o + q++] = i;
            for (int i = 0; i < Ch.k2[a]; ++i) sperm[o + q++] = n1p + i;
            for (int i = 0; i < Ch.k1[b]; ++i) sperm[o + q++] = Ch.k1[a] + i;
            for (int i = 0; i < Ch.k2[b]; ++i) sperm[o + q++] = n1p + Ch.k2[a] + i;
            ra[p] = Ch.k1[a] + Ch.k2[a];
            rb[p] = Ch.k1[b] + Ch.k2[b];
            scoff[2 * p + 1] = scoff[2 * p] + (int64_t)ra[p] * rb[p];
            scoff[2 * p + 2] = scoff[2 * p + 1] + (int64_t)ra[p] * rb[p];
            Pn.srmax = std::max(Pn.srmax, std::max(ra[p], rb[p]));
            Pn.sum_s2 += 2.0 * ra[p] * rb[p];
        }
        FDS_TRY(Pn.d_sperm.upload(sperm, s));
        FDS_TRY(Pn.d_ra.upload(ra, s));
        FDS_TRY(Pn.d_rb.upload(rb, s));
        FDS_TRY(Pn.d_scoff.upload(scoff, s));
        FDS_TRY(Pn.Sc.alloc((size_t)std::max<int64_t>(scoff[2 * Pn.nb], 1)));
        if (Pn.d_doff.n < (size_t)Pn.nb + 1) FDS_TRY(Pn.d_doff.upload(Pn.doff, s));
        fds_count_launch(), k_extract_s<<<Pn.nb, 256, 0, s>>>(Pn.rSfw.p, Pn.d_sperm.p, Pn.d_doff.p, Pn.d_ra.p,
                                                              Pn.d_rb.p, Pn.d_scoff.p, Pn.Sc.p);
        FDS_CUDA_TRY(cudaGetLastError());
        if (h->opt.ir_apply == FDS_APPLY_FF) {
            FDS_TRY(Pn.Scp.alloc(Pn.Sc.n));
            fds_count_launch(), k_split<<<1024, 256, 0, s>>>(Pn.Sc.p, Pn.Scp.p, (int64_t)Pn.Sc.n);
            FDS_CUDA_TRY(cudaGetLastError());
        }
        if (tensor_fw) {
            // y_a += S_ab x_b and y_b += S_ba x_a per parent, rows through sperm
            std::vector<OzSpec> sp;
            sp.reserve(2 * (size_t)Pn.nb);
            for (int p = 0; p < Pn.nb; ++p) {
                const int a = ra[p], b = rb[p];
                const int64_t o = Pn.doff[p];
                OzSpec q;
                q.a = Pn.Sc.p + scoff[2 * p];
                q.lda = std::max(a, 1);
                q.m = a;
                q.k = b;
                q.x_row = q.y_row = o;
                q.xmap = sperm.data() + o + a;
                q.ymap = sperm.data() + o;
                sp.push_back(q);
                q.a = Pn.Sc.p + scoff[2 * p + 1];
                q.lda = std::max(b, 1);
                q.m = b;
                q.k = a;
                q.xmap = sperm.data() + o;
                q.ymap = sperm.data() + o + a;
                sp.push_back(q);
            }
            FDS_TRY(oz_plan_build(sp, Pn.oz_sib, s));
            for (const OzPlan &P : Pn.oz_sib) bytes += (int64_t)(P.aslices.bytes() + P.rowexp.bytes());
        }
        bytes += (int64_t)(Pn.Sc.bytes() + Pn.Scp.bytes()) - (int64_t)Pn.Sfw.bytes();
    }
    if (h->opt.ir_apply == FDS_APPLY_FF || h->opt.sweep_ff) {
        for (int l = L; l > l0; --l) {
            Level &C = h->lv[l];
            FDS_TRY(C.Tp.alloc(C.T.n));
            fds_count_launch(), k_split<<<1024, 256, 0, s>>>(C.T.p, C.Tp.p, (int64_t)C.T.n);
            FDS_CUDA_TRY(cudaGetLastError());
        }
    }
    if (h->opt.ir_apply == FDS_APPLY_FF) {
        // the forward operator as float pairs (same bytes as complex128)
        for (int l = L; l >= l0; --l) {
            Level &C = h->lv[l];
            std::vector<int> dv(C.nb), rv(C.nb);
            for (int b = 0; b < C.nb; ++b) {
                dv[b] = C.n1[b] + C.n2[b];
                rv[b] = l > l0 ? C.k1[b] + C.k2[b] : 0;
            }
            if (C.Dfw.p) FDS_TRY(split_blocks(C.Dfw, C.Dp, C.rDp, C.offA, dv, dv, s));
            if (tensor_fw && l > l0) FDS_TRY(oz_interp_leaf_plans(h, C, l == L, s, bytes));

        }
        {
            std::vector<int64_t> off = {0, h->Dtop * h->Dtop};
            std::vector<int> d = {(int)h->Dtop};
            FDS_TRY(split_blocks(h->Atop_off, h->Atop_offp, h->rtop_offp, off, d, d, s));
        }
    }
    if (tensor_fw) h->oz_jobs = true;
    FDS_CUDA_TRY(cudaStreamSynchronize(s));
    for (int l = L; l >= l0; --l) {   // the compact blocks replace the d x d sibling coupling
        Level &C = h->lv[l];
        C.Sfw.release();
        C.rSfw.release();
    }
    if (h->opt.ir_apply == FDS_APPLY_FF) {
        for (int l = L; l >= l0; --l) {
            Level &C = h->lv[l];
            C.Dfw.release();
            C.rDfw.release();
        }
        h->Atop_off.release();
        h->rtop_off.release();
    }
    // the FP64 factors of the complex64 and double-float levels are not used by the mixed solve
    for (int l = L; l > l0; --l) {
        if (level_prec(h, l) == PREC_C128) continue;
        Level &C = h->lv[l];
        C.Ainv.release();
        C.rAinv.release();
        C.W.release();
        C.rW.release();
        C.At.release();
        C.rAt.release();
    }
    h->factor_bytes = bytes;
    return FDS_OK;
}

template <class LT>
int solve_mixed(fds_handle *h, cplx *d_rhs, int nrhs, cudaStream_t s) {
    const int N = h->N, L = h->L;
    const int64_t ld_rhs = 2LL * N;
    const int ncmax = std::min(nrhs, SOLVE_CHUNK);
    const Level &Lf = h->lv[L];
    const int64_t D = Lf.D;
    FDS_TRY(sweep_workspace(h, ncmax));
    const bool refine = h->opt.ir_max_iter > 0;
    const bool ffp = h->opt.ir_apply == FDS_APPLY_FF;
    if (refine) {
        if (ffp) FDS_TRY(forward_workspace<float4>(h, ncmax));
        else FDS_TRY(forward_workspace<cplx>(h, ncmax));
    }
    if (refine && ffp) FDS_TRY(grow(h->wXp, (size_t)D * ncmax));
    FDS_TRY(grow(h->wX, (size_t)D * ncmax));
    if (h->wnorm.n < (size_t)2 * ncmax) FDS_TRY(h->wnorm.alloc((size_t)2 * ncmax));
    LT *leaf_in = sweep_leaf_in<LT>(h), *leaf = sweep_leaf_out<LT>(h);
    cplx *Yleaf = (refine && !ffp) ? forward_out<cplx>(h) : nullptr;
    float4 *Ypleaf = (refine && ffp) ? forward_out<float4>(h) : nullptr;
    std::vector<double> nrm(2 * ncmax);
    int iters = 0;
    double worst = refine ? 0.0 : -1.0;
    bool converged = true;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    if (h->wcmap.n < (size_t)ncmax) FDS_TRY(h->wcmap.alloc((size_t)ncmax));
    if (refine && h->wperm.n < (size_t)D * ncmax * sizeof(cplx))
        FDS_TRY(h->wperm.alloc((size_t)D * ncmax * sizeof(cplx)));
    for (int c0 = 0; c0 < nrhs; c0 += SOLVE_CHUNK) {
        const int nc = std::min(SOLVE_CHUNK, nrhs - c0);
        cplx *F = d_rhs + (int64_t)c0 * ld_rhs;
        const unsigned gx = (unsigned)std::min<int64_t>((D + 255) / 256, 64);
        // the iterate's columns are kept with the columns still refining first:
        // compact column j holds right-hand side cmap[j] of the chunk
        std::vector<int> cmap(nc);
        for (int c = 0; c < nc; ++c) cmap[c] = c;
        FDS_CUDA_TRY(cudaMemcpyAsync(h->wcmap.p, cmap.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, s));
        // x = sweep(f)
        FDS_CUDA_TRY(cudaMemsetAsync(h->wnorm.p, 0, sizeof(double) * 2 * nc, s));
        {
            ProfScope ps("a7.residual", s);
            fds_count_launch(), k_residual<cplx, LT><<<dim3(gx, nc), 256, 0, s>>>(
                h->d_leaf_gidx.p, D, F, ld_rhs, h->wcmap.p, nullptr, leaf_in, h->wnorm.p);
        }
        FDS_CUDA_TRY(cudaGetLastError());
        FDS_TRY(sweep_chunk_run(h, nc, s));
        fds_count_launch(), k_update<LT><<<1024, 256, 0, s>>>(h->wX.p, leaf, D * nc, 1);
        FDS_CUDA_TRY(cudaGetLastError());
        // refinement against the FP64 compressed operator, column by column:
        // a column stops when its residual meets ir_tol, stops contracting or
        // the sweeps run out, and keeps the better of its last two iterates;
        // the forward operator and the sweeps then run on the others only
        int nact = nc;
        std::vector<double> prevc(nc, INFINITY), resc(nc, 0.0);
        for (int it = 0; refine && nact > 0; ++it) {
            if (ffp) {
                fds_count_launch(), k_split<<<1024, 256, 0, s>>>(h->wX.p, h->wXp.p, D * nact);
                FDS_TRY(forward_apply<float4>(h, h->wXp.p, Ypleaf, nact, s));
            } else {
                FDS_TRY(forward_apply<cplx>(h, h->wX.p, Yleaf, nact, s));
            }
            FDS_CUDA_TRY(cudaMemsetAsync(h->wnorm.p, 0, sizeof(double) * 2 * nact, s));
            {
                ProfScope ps("a7.residual", s);
                if (ffp)
                    fds_count_launch(), k_residual<float4, LT><<<dim3(gx, nact), 256, 0, s>>>(
                        h->d_leaf_gidx.p, D, F, ld_rhs, h->wcmap.p, Ypleaf, leaf_in, h->wnorm.p);
                else
                    fds_count_launch(), k_residual<cplx, LT><<<dim3(gx, nact), 256, 0, s>>>(
                        h->d_leaf_gidx.p, D, F, ld_rhs, h->wcmap.p, Yleaf, leaf_in, h->wnorm.p);
            }
            FDS_CUDA_TRY(cudaGetLastError());
            FDS_CUDA_TRY(cudaMemcpyAsync(nrm.data(), h->wnorm.p, sizeof(double) * 2 * nact, cudaMemcpyDeviceToHost, s));
            FDS_CUDA_TRY(cudaStreamSynchronize(s));
            std::vector<int> undo(nact, 0), keep, done;
            bool any_undo = false;
            for (int j = 0; j < nact; ++j) {
                resc[j] = nrm[2 * j + 1] > 0 ? std::sqrt(nrm[2 * j] / nrm[2 * j + 1]) : 0.0;
                if (!(resc[j] == resc[j])) return FDS_ERR_SINGULAR;
                const bool stop = resc[j] <= h->opt.ir_tol || it >= h->opt.ir_max_iter || resc[j] > 0.5 * prevc[j];
                if (!stop) {
                    keep.push_back(j);
                    continue;
                }
                // a correction that made the column worse is taken back
                if (resc[j] > prevc[j]) undo[j] = 1, any_undo = true;
                const double best = std::min(resc[j], prevc[j]);
                worst = std::max(worst, best);
                if (best > h->opt.ir_tol) converged = false;
                iters = std::max(iters, it);
                done.push_back(j);
            }
            if (any_undo) {
                FDS_TRY(grow(h->wundo, (size_t)nact));
                FDS_CUDA_TRY(cudaMemcpyAsync(h->wundo.p, undo.data(), sizeof(int) * nact, cudaMemcpyHostToDevice, s));
                fds_count_launch(), k_undo_cols<LT><<<1024, 256, 0, s>>>(h->wX.p, leaf, D, nact, h->wundo.p);
                FDS_CUDA_TRY(cudaGetLastError());
            }
            const int nkeep = (int)keep.size();
            if (nkeep == 0) {
                FDS_CUDA_TRY(cudaStreamSynchronize(s));   // undo[] is a host vector
                break;
            }
            if (nkeep < nact) {
                // the refining columns first: permute the iterate, the residual and the maps
                std::vector<int> perm(keep);
                perm.insert(perm.end(), done.begin(), done.end());
                std::vector<int> cm(nact);
                std::vector<double> pr(nact);
                for (int j = 0; j < nact; ++j) {
                    cm[j] = cmap[perm[j]];
                    pr[j] = resc[perm[j]];
                }
                std::copy(cm.begin(), cm.end(), cmap.begin());
                std::copy(pr.begin(), pr.end(), resc.begin());
                FDS_TRY(grow(h->wundo, (size_t)nact));
                FDS_CUDA_TRY(cudaMemcpyAsync(h->wundo.p, perm.data(), sizeof(int) * nact, cudaMemcpyHostToDevice, s));
                cplx *tx = reinterpret_cast<cplx *>(h->wperm.p);
                fds_count_launch(), k_permute_cols<cplx><<<1024, 256, 0, s>>>(h->wX.p, tx, D, h->wundo.p, nact);
                FDS_CUDA_TRY(cudaMemcpyAsync(h->wX.p, tx, sizeof(cplx) * D * nact, cudaMemcpyDeviceToDevice, s));
                LT *tr = reinterpret_cast<LT *>(h->wperm.p);
                fds_count_launch(), k_permute_cols<LT><<<1024, 256, 0, s>>>(leaf_in, tr, D, h->wundo.p, nkeep);
                FDS_CUDA_TRY(cudaMemcpyAsync(leaf_in, tr, sizeof(LT) * D * nkeep, cudaMemcpyDeviceToDevice, s));
                FDS_CUDA_TRY(cudaMemcpyAsync(h->wcmap.p, cmap.data(), sizeof(int) * nact, cudaMemcpyHostToDevice, s));
                FDS_CUDA_TRY(cudaGetLastError());
                FDS_CUDA_TRY(cudaStreamSynchronize(s));   // perm, cmap: host vectors
            }
            nact = nkeep;
            for (int j = 0; j < nact; ++j) prevc[j] = resc[j];
            FDS_TRY(sweep_chunk_run(h, nact, s));
            fds_count_launch(), k_update<LT><<<1024, 256, 0, s>>>(h->wX.p, leaf, D * nact, 0);
            FDS_CUDA_TRY(cudaGetLastError());
        }
        fds_count_launch(), k_leaf_scatter<<<1024, 256, 0, s>>>(h->d_leaf_gidx.p, D, h->wX.p, F, ld_rhs, h->wcmap.p,
                                                                 nc);
        FDS_CUDA_TRY(cudaGetLastError());
    }
    cudaEventRecord(e1, s);
    FDS_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    h->solve_ms = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->ir_iters = iters;
    h->ir_residual = worst;
    return converged ? FDS_OK : FDS_ERR_NOT_CONVERGED;
}

int fds_solve_mixed_impl(fds_handle *h, cplx *d_rhs, int nrhs, cudaStream_t s) {
    C64EngineScope eng(h->opt.c64_engine == FDS_C64_TENSOR);
    // the refinement's sweep vectors are in the leaf level's precision
    const int rc = (h->L > h->l0 && level_prec(h, h->L) == PREC_FF) ? solve_mixed<float4>(h, d_rhs, nrhs, s)
                                                                   : solve_mixed<cplxf>(h, d_rhs, nrhs, s);
    if (h->oz_jobs) {
        int st = 0, st2 = 0;
        FDS_TRY(ozj_status_take(s, &st));
        FDS_TRY(oz_status_take(s, &st2));
        st |= st2;
        if (st) {
            fds_set_error_detail("tensor-core forward operator: wait on a pipeline barrier timed out");
            return FDS_ERR_TIMEOUT;
        }
    }
    if (h->opt.c64_engine != FDS_C64_TENSOR) return rc;
    int st = 0;
    const int rs = tc_status_take(s, &st);
    if (st) {
        fds_set_error_detail("tensor-core GEMM: wait on the MMA barrier timed out");
        return FDS_ERR_TIMEOUT;
    }
    return rc != FDS_OK ? rc : rs;
}
