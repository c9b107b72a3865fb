// The interpolation matrices of a level applied through their structure
// (Sec. 7.1: V^c = [I  T^c] P^T per cell and component): V x copies the
// skeleton entries of x and adds T^c times the remaining entries; V^H t
// scatters t to the skeleton entries and T^{cH} t to the others.  The T part
// is one batched GEMM over all (cell, component) pairs with a row gather of
// B (V x) or a row scatter of C (V^H t); the dense V_i is never read.
#include <algorithm>

#include "fds_internal.cuh"
#include "solve.cuh"
#include "vapply.cuh"

namespace {

template <class T>
__global__ void k_vrefs(int nb, int dir, const T *Tb, const int64_t *__restrict__ toff, const int *__restrict__ k1,
                        const int *__restrict__ k2, const int *__restrict__ n1, const int *__restrict__ n2,
                        const int64_t *__restrict__ doff, const int64_t *__restrict__ roff, const int *vmap,
                        const T *src, int64_t lds, T *dst, int64_t ldd, int nc, MatRefT<T> *A, MatRefT<T> *B,
                        MatRefT<T> *Cm, RowMaps *M) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 2 * nb) return;
    const int b = e >> 1, c = e & 1;
    const int k = c ? k2[b] : k1[b], n = c ? n2[b] : n1[b], m = n - k;
    const int coff = c ? n1[b] : 0;
    const int64_t ooff = roff[b] + (c ? k1[b] : 0);
    const int *vm = vmap + doff[b] + coff;
    A[e].p = (T *)Tb + toff[e];
    A[e].rows = k;
    A[e].cols = m;
    A[e].ld = k > 1 ? k : 1;
    if (dir == 0) {       // out[skeleton rows] += T x[rest]
        B[e].p = (T *)src + doff[b];
        B[e].rows = (int)(doff[b + 1] - doff[b]);
        B[e].ld = (int)lds;
        Cm[e].p = dst + ooff;
        Cm[e].rows = k;
        Cm[e].ld = (int)ldd;
        M[e].b = vm + k;
        M[e].c = nullptr;
        M[e].cext = 0;
    } else {              // y[rest] = T^H t
        B[e].p = (T *)src + ooff;
        B[e].rows = k;
        B[e].ld = (int)lds;
        Cm[e].p = dst + doff[b];
        Cm[e].rows = m;
        Cm[e].ld = (int)ldd;
        M[e].b = nullptr;
        M[e].c = vm + k;
        M[e].cext = (int)(doff[b + 1] - doff[b]);
    }
    B[e].cols = nc;
    Cm[e].cols = nc;
}

// skeleton entries: dir 0 out[k rows] = x[skeleton], dir 1 y[skeleton] = t[k rows]
template <class T>
__global__ void k_vskel(int dir, const int *__restrict__ k1, const int *__restrict__ k2, const int *__restrict__ n1,
                        const int64_t *__restrict__ doff, const int64_t *__restrict__ roff,
                        const int *__restrict__ vmap, const T *__restrict__ src, int64_t lds, T *dst, int64_t ldd,
                        int nc) {
    const int b = blockIdx.x;
    const int ka = k1[b], kt = ka + k2[b];
    for (int64_t e = threadIdx.x; e < (int64_t)kt * nc; e += blockDim.x) {
        const int q = (int)(e % kt);
        const int64_t col = e / kt;
        const int c = q < ka ? 0 : 1;
        const int qq = c ? q - ka : q;
        const int li = vmap[doff[b] + (c ? n1[b] : 0) + qq];
        if (!FDS_IN_RANGE(li, doff[b + 1] - doff[b])) continue;
        const int64_t cell = doff[b] + li;
        const int64_t skel = roff[b] + q;
        if (dir == 0) dst[skel + col * ldd] = src[cell + col * lds];
        else dst[cell + col * ldd] = src[skel + col * lds];
    }
}

size_t vref_bytes(const fds_handle *h, size_t ref_size) {
    return (size_t)2 * fds_max_cells(h) * (3 * ref_size + sizeof(RowMaps)) + 64;
}

template <class T>
int vapply(fds_handle *h, const Level &C, const T *Tb, int dir, const T *src, int64_t lds, T *dst, int64_t ldd,
           int nc, cudaStream_t s) {
    const int nb = C.nb;
    if (nb == 0 || nc == 0) return FDS_OK;
    const int maxnb = fds_max_cells(h);
    const size_t need = vref_bytes(h, sizeof(MatRefT<T>));
    if (h->wvref.n < need) FDS_TRY(h->wvref.alloc(need));
    MatRefT<T> *A = reinterpret_cast<MatRefT<T> *>(h->wvref.p);
    MatRefT<T> *B = A + 2 * maxnb, *Cr = B + 2 * maxnb;
    RowMaps *M = reinterpret_cast<RowMaps *>(Cr + 2 * maxnb);
    fds_count_launch(), k_vskel<T><<<nb, 256, 0, s>>>(dir, C.d_k1.p, C.d_k2.p, C.d_n1.p, C.d_doff.p, C.d_roff.p,
                                                      C.d_vmap.p, src, lds, dst, ldd, nc);
    fds_count_launch(), k_vrefs<T><<<(2 * nb + 127) / 128, 128, 0, s>>>(
        nb, dir, Tb, C.d_toff.p, C.d_k1.p, C.d_k2.p, C.d_n1.p, C.d_n2.p, C.d_doff.p, C.d_roff.p, C.d_vmap.p, src,
        lds, dst, ldd, nc, A, B, Cr, M);
    FDS_CUDA_TRY(cudaGetLastError());
    const int maxm = dir == 0 ? C.kmax : C.dmax;
    return dense_gemm_map(2 * nb, std::max(maxm, 1), nc, A, dir == 0 ? 0 : 2, B, Cr, M, dir == 0 ? 1 : 0, s);
}

}  // namespace

template <class T>
int vskel_apply(const Level &C, int dir, const T *src, int64_t lds, T *dst, int64_t ldd, int nc, cudaStream_t s) {
    if (C.nb == 0 || nc == 0) return FDS_OK;
    fds_count_launch(), k_vskel<T><<<C.nb, 256, 0, s>>>(dir, C.d_k1.p, C.d_k2.p, C.d_n1.p, C.d_doff.p, C.d_roff.p,
                                                        C.d_vmap.p, src, lds, dst, ldd, nc);
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}
template int vskel_apply<float4>(const Level &, int, const float4 *, int64_t, float4 *, int64_t, int, cudaStream_t);

template <class T>
int apply_V(fds_handle *h, const Level &C, const T *Tb, const T *x, int64_t ldx, T *out, int64_t ldo, int nc,
            cudaStream_t s) {
    return vapply<T>(h, C, Tb, 0, x, ldx, out, ldo, nc, s);
}

int vapply_workspace(fds_handle *h) {
    const size_t need = std::max(vref_bytes(h, sizeof(MatRefT<cplx>)), vref_bytes(h, sizeof(MatRefT<float4>)));
    return h->wvref.n < need ? h->wvref.alloc(need) : FDS_OK;
}

template <class T>
int apply_VH(fds_handle *h, const Level &C, const T *Tb, const T *t, int64_t ldt, T *y, int64_t ldy, int nc,
             cudaStream_t s) {
    return vapply<T>(h, C, Tb, 1, t, ldt, y, ldy, nc, s);
}

template int apply_V<cplx>(fds_handle *, const Level &, const cplx *, const cplx *, int64_t, cplx *, int64_t, int,
                           cudaStream_t);
template int apply_V<cplxf>(fds_handle *, const Level &, const cplxf *, const cplxf *, int64_t, cplxf *, int64_t,
                            int, cudaStream_t);
template int apply_V<float4>(fds_handle *, const Level &, const float4 *, const float4 *, int64_t, float4 *, int64_t,
                             int, cudaStream_t);
template int apply_VH<cplx>(fds_handle *, const Level &, const cplx *, const cplx *, int64_t, cplx *, int64_t, int,
                            cudaStream_t);
template int apply_VH<float4>(fds_handle *, const Level &, const float4 *, const float4 *, int64_t, float4 *,
                              int64_t, int, cudaStream_t);
