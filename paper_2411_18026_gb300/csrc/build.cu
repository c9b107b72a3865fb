// Factorisation (build) of the fast direct solver, arXiv 2411.18026 Sec. 7.3:
//   1-2  binary tree over the boundary nodes and leaf index sequences J_p (Sec. 5.1)
//   3    for l = L .. l0+1: proxy compression (Sec. 7.1/7.2) -> U_i, V_i, J~_i;
//        A_i^{-1} (LU), A_i^{-1} U_i, A~_i = (V_i A_i^{-1} U_i)^{-1} (Sec. 6.2);
//        parent blocks by eq. (A_rearrangement)
//   4    dense LU of the level-l0 system (Sec. 6.3).
// The host plans sizes and index lists level by level; every arithmetic step
// runs in the kernels below or in kernel_eval / id / dense.
#include <algorithm>
#include <cmath>

#include "fds_internal.cuh"
#include "id.cuh"
#include "kernel_eval.cuh"
#include "mlp.cuh"
#include "prof.cuh"

namespace {

using namespace fdsk;

// ------------------------------------------------------------- geometry (a0)
// Cell circle: centre of the bounding box of the hat supports of nodes
// lo..hi-1 (polygon vertices lo-1..hi), radius = largest vertex distance.
__global__ void k_box_circles(int nb, const int *__restrict__ lo, const int *__restrict__ hi,
                              const double *__restrict__ xy, int N, double *cx, double *cy, double *R) {
    const int b = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= nb) return;
    const int a = lo[b] - 1, e = hi[b];
    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
    for (int v = a + lane; v <= e; v += 32) {
        int s = ((v % N) + N) % N;
        double x = xy[2 * s], y = xy[2 * s + 1];
        xmin = fmin(xmin, x); xmax = fmax(xmax, x);
        ymin = fmin(ymin, y); ymax = fmax(ymax, y);
    }
    for (int o = 16; o > 0; o >>= 1) {
        xmin = fmin(xmin, __shfl_xor_sync(0xffffffffu, xmin, o));
        xmax = fmax(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
        ymin = fmin(ymin, __shfl_xor_sync(0xffffffffu, ymin, o));
        ymax = fmax(ymax, __shfl_xor_sync(0xffffffffu, ymax, o));
    }
    const double c0 = 0.5 * (xmin + xmax), c1 = 0.5 * (ymin + ymax);
    double r2 = 0.0;
    for (int v = a + lane; v <= e; v += 32) {
        int s = ((v % N) + N) % N;
        double dx = xy[2 * s] - c0, dy = xy[2 * s + 1] - c1;
        r2 = fmax(r2, dx * dx + dy * dy);
    }
    for (int o = 16; o > 0; o >>= 1) r2 = fmax(r2, __shfl_xor_sync(0xffffffffu, r2, o));
    if (lane == 0) {
        cx[b] = c0;
        cy[b] = c1;
        R[b] = sqrt(r2);
    }
}

// Proxy polygon of each cell: m' counter-clockwise vertices on the circle of
// radius Rp about the cell centre (Sec. 7.1, Fig. domain_proxy).
__global__ void k_proxy_nodes(const double *__restrict__ cx, const double *__restrict__ cy,
                              const double *__restrict__ Rp, const int *__restrict__ m,
                              const int64_t *__restrict__ off, double *out) {
    const int b = blockIdx.x;
    const int mb = m[b];
    for (int k = threadIdx.x; k < mb; k += blockDim.x) {
        double s, c;
        sincospi(2.0 * k / mb, &s, &c);
        out[2 * (off[b] + k)] = cx[b] + Rp[b] * c;
        out[2 * (off[b] + k) + 1] = cy[b] + Rp[b] * s;
    }
}

__device__ __forceinline__ double seg_dist(double px, double py, double ax, double ay, double bx, double by) {
    double ux = bx - ax, uy = by - ay;
    double t = ((px - ax) * ux + (py - ay) * uy) / (ux * ux + uy * uy);
    t = fmin(1.0, fmax(0.0, t));
    double dx = ax + t * ux - px, dy = ay + t * uy - py;
    return sqrt(dx * dx + dy * dy);
}

// Near field of cell i: active nodes of the other cells of the level whose
// hat support meets the closed proxy disk.  mode 0 counts, mode 1 fills.
__global__ void k_near(int nb, const double *__restrict__ cx, const double *__restrict__ cy,
                       const double *__restrict__ R, const double *__restrict__ Rp,
                       const int64_t *__restrict__ uoff, const int *__restrict__ unode,
                       const int *__restrict__ upos1, const int *__restrict__ upos2,
                       const double *__restrict__ xy, int N, int mode, int *count,
                       const int64_t *__restrict__ noff, int *nnode, int *nmask) {
    const int i = blockIdx.x;
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const double ci0 = cx[i], ci1 = cy[i], rp = Rp[i];
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
        if (j == i) continue;
        double dx = cx[j] - ci0, dy = cy[j] - ci1;
        if (sqrt(dx * dx + dy * dy) > rp + R[j]) continue;
        for (int64_t u = uoff[j]; u < uoff[j + 1]; ++u) {
            const int s = unode[u];
            const int sp = (s == 0) ? N - 1 : s - 1, sn = (s + 1 == N) ? 0 : s + 1;
            double d1 = seg_dist(ci0, ci1, xy[2 * sp], xy[2 * sp + 1], xy[2 * s], xy[2 * s + 1]);
            double d2 = seg_dist(ci0, ci1, xy[2 * s], xy[2 * s + 1], xy[2 * sn], xy[2 * sn + 1]);
            if (fmin(d1, d2) <= rp) {
                int slot = atomicAdd(&cnt, 1);
                if (mode == 1) {
                    nnode[noff[i] + slot] = s;
                    nmask[noff[i] + slot] = (upos1[u] >= 0 ? 1 : 0) | (upos2[u] >= 0 ? 2 : 0);
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (mode == 0) count[i] = cnt;
        else {
            // deterministic order: insertion sort by node index
            const int64_t o = noff[i];
            for (int a = 1; a < cnt; ++a) {
                int kn = nnode[o + a], km = nmask[o + a];
                int p = a - 1;
                while (p >= 0 && nnode[o + p] > kn) {
                    nnode[o + p + 1] = nnode[o + p];
                    nmask[o + p + 1] = nmask[o + p];
                    --p;
                }
                nnode[o + p + 1] = kn;
                nmask[o + p + 1] = km;
            }
        }
    }
}

// --------------------------------------------------- ID matrices (a1 -> a2)
struct YDesc {
    const int64_t *yoff;     // 2 nb: offset of Y_{b,c}
    const int *ym;           // nb: rows of Y_b (same for both components)
    const int *mp;           // nb: proxy vertices m'
    const int *nnd;          // nb: near DOF rows
    const int64_t *pxoff;    // nb: proxy vertex offset
    const double *pxy;       // proxy vertices
    const int64_t *uoff;
    const int *unode, *upos1, *upos2;
    const int64_t *noff;     // nb+1 near entries
    const int *nnode, *nmask, *nrow;
};

// ---- tile jobs: each CTA evaluates a tile of at most TILE x TILE hats
struct LeafJob {
    int b, I, J;
};
struct YJob {
    int b, kind, r0, u0;   // kind 0: proxy vertices r0.., kind 1: near entries r0..
};
struct GJob {
    int g, roff, nr, coff, nc;
};

// Leaf diagonal blocks A_p = A^{J_p J_p} (eq. (block_ax=f)): tile (I, J) of
// the cell's hats, I <= J; off-diagonal tiles also write the transposed tile.
__global__ void __launch_bounds__(FDS_TILE_THREADS) k_tiles_leaf(PhysDev P, const int *__restrict__ lo, const int *__restrict__ hi,
                                                    const double *__restrict__ xy, int N, const MatRef *A,
                                                    const LeafJob *__restrict__ jobs) {
    __shared__ TileSmem S;
    const LeafJob jb = jobs[blockIdx.x];
    const int base = lo[jb.b], n = hi[jb.b] - base;
    load_rules(S.G, 0);
    tile_zero(S);
    if (threadIdx.x == 0) {
        S.R.nh = min(TILE, n - jb.I * TILE);
        S.C.nh = min(TILE, n - jb.J * TILE);
        for (int k = 0; k < S.R.nh; ++k) S.R.hats[k] = base + jb.I * TILE + k;
        for (int k = 0; k < S.C.nh; ++k) S.C.hats[k] = base + jb.J * TILE + k;
        tile_side_build(S.R, N);
        tile_side_build(S.C, N);
    }
    __syncthreads();
    const bool diag = jb.I == jb.J;
    tile_eval(P, S, xy, N, xy, N, true, !diag, diag);
    __syncthreads();
    if (diag) {
        tile_fold(S);
        __syncthreads();
    }
    const MatRef M = A[jb.b];
    for (int e = threadIdx.x; e < S.R.nh * S.C.nh * 4; e += blockDim.x) {
        const int r = e % S.R.nh, c = (e / S.R.nh) % S.C.nh, ij = e / (S.R.nh * S.C.nh);
        const int i = ij >> 1, j = ij & 1;
        const int rl = jb.I * TILE + r, cl = jb.J * TILE + c;
        const double m = (i == j) ? 0.5 * mass_entry(xy, N, S.R.hats[r], S.C.hats[c]) : 0.0;
        cplx v = tile_f(S, r, c, i, j);
        v.x += m;
        M.p[(rl + i * n) + (int64_t)(cl + j * n) * M.ld] = v;
        if (!diag) {
            cplx w = tile_r(S, c, r, i, j);
            w.x += m;
            M.p[(cl + i * n) + (int64_t)(rl + j * n) * M.ld] = w;
        }
    }
}

// Rows of the ID matrices Y^c (Sec. 7.1 eq. (mv): M^V = A^{J' J}; Sec. 7.2:
// M^U = A^{J J'} stacked as (M^U)^H): tile of proxy vertices (cross rule) or
// near-field hats (boundary rule) against the cell's hats; the transposed
// entries of the same quadrature points give the M^U rows.
__global__ void __launch_bounds__(FDS_TILE_THREADS) k_tiles_y(PhysDev P, YDesc D, const double *__restrict__ xy, int N, cplx *Y,
                                                 const YJob *__restrict__ jobs) {
    __shared__ TileSmem S;
    __shared__ int rowv[TILE][2], colp[TILE][2];
    const YJob jb = jobs[blockIdx.x];
    const int b = jb.b, mp = D.mp[b];
    const int64_t uo0 = D.uoff[b];
    const int nu = (int)(D.uoff[b + 1] - uo0);
    const bool prox = jb.kind == 0;
    load_rules(S.G, prox ? 2 : 0);
    tile_zero(S);
    if (threadIdx.x == 0) {
        if (prox) {
            S.R.nh = min(TILE, mp - jb.r0);
            for (int k = 0; k < S.R.nh; ++k) {
                S.R.hats[k] = jb.r0 + k;
                rowv[k][0] = jb.r0 + k;
                rowv[k][1] = jb.r0 + k + mp;
            }
        } else {
            const int64_t n0 = D.noff[b];
            const int nn = (int)(D.noff[b + 1] - n0);
            S.R.nh = min(TILE, nn - jb.r0);
            for (int k = 0; k < S.R.nh; ++k) {
                const int64_t q = n0 + jb.r0 + k;
                S.R.hats[k] = D.nnode[q];
                const int mask = D.nmask[q], rb = 2 * mp + D.nrow[q];
                rowv[k][0] = (mask & 1) ? rb : -1;
                rowv[k][1] = (mask & 2) ? rb + (mask & 1) : -1;
            }
        }
        S.C.nh = min(TILE, nu - jb.u0);
        for (int k = 0; k < S.C.nh; ++k) {
            S.C.hats[k] = D.unode[uo0 + jb.u0 + k];
            colp[k][0] = D.upos1[uo0 + jb.u0 + k];
            colp[k][1] = D.upos2[uo0 + jb.u0 + k];
        }
        tile_side_build(S.R, prox ? mp : N);
        tile_side_build(S.C, N);
    }
    __syncthreads();
    const double *X = prox ? D.pxy + 2 * D.pxoff[b] : xy;
    const int NX = prox ? mp : N;
    tile_eval(P, S, X, NX, xy, N, !prox, true, false);
    __syncthreads();
    const int m = D.ym[b];
    const int uoff = 2 * mp + D.nnd[b];
    for (int e = threadIdx.x; e < S.R.nh * S.C.nh * 4; e += blockDim.x) {
        const int r = e % S.R.nh, c = (e / S.R.nh) % S.C.nh, ij = e / (S.R.nh * S.C.nh);
        const int i = ij >> 1, j = ij & 1;
        const double ms = (!prox && i == j) ? 0.5 * mass_entry(xy, N, S.R.hats[r], S.C.hats[c]) : 0.0;
        // forward: test = row item (component i), trial = cell hat (component j) -> Y^j
        if (rowv[r][i] >= 0 && colp[c][j] >= 0) {
            cplx v = tile_f(S, r, c, i, j);
            v.x += ms;
            Y[D.yoff[2 * b + j] + rowv[r][i] + (int64_t)colp[c][j] * m] = v;
        }
        // transposed: test = cell hat (component i), trial = row item (component j) -> conj into Y^i
        if (colp[c][i] >= 0 && rowv[r][j] >= 0) {
            cplx w = tile_r(S, c, r, i, j);
            w.x += ms;
            Y[D.yoff[2 * b + i] + uoff + rowv[r][j] + (int64_t)colp[c][i] * m] = cconj(w);
        }
    }
}

// Blocks of original entries between two disjoint hat lists of a group:
// sibling blocks R of eq. (A_rearrangement) and the off-diagonal blocks of the
// top system.  Items carry the matrix index of each component (or -1).
__global__ void __launch_bounds__(FDS_TILE_THREADS) k_tiles_group(PhysDev P, const int *__restrict__ gnode,
                                                     const int *__restrict__ gi1, const int *__restrict__ gi2,
                                                     const double *__restrict__ xy, int N, const MatRef *M,
                                                     const GJob *__restrict__ jobs) {
    __shared__ TileSmem S;
    __shared__ int ri[TILE][2], ci[TILE][2];
    const GJob jb = jobs[blockIdx.x];
    load_rules(S.G, 0);
    tile_zero(S);
    if (threadIdx.x == 0) {
        S.R.nh = jb.nr;
        S.C.nh = jb.nc;
        for (int k = 0; k < jb.nr; ++k) {
            S.R.hats[k] = gnode[jb.roff + k];
            ri[k][0] = gi1[jb.roff + k];
            ri[k][1] = gi2[jb.roff + k];
        }
        for (int k = 0; k < jb.nc; ++k) {
            S.C.hats[k] = gnode[jb.coff + k];
            ci[k][0] = gi1[jb.coff + k];
            ci[k][1] = gi2[jb.coff + k];
        }
        tile_side_build(S.R, N);
        tile_side_build(S.C, N);
    }
    __syncthreads();
    tile_eval(P, S, xy, N, xy, N, true, true, false);
    __syncthreads();
    const MatRef A = M[jb.g];
    for (int e = threadIdx.x; e < S.R.nh * S.C.nh * 4; e += blockDim.x) {
        const int r = e % S.R.nh, c = (e / S.R.nh) % S.C.nh, ij = e / (S.R.nh * S.C.nh);
        const int i = ij >> 1, j = ij & 1;
        const double ms = (i == j) ? 0.5 * mass_entry(xy, N, S.R.hats[r], S.C.hats[c]) : 0.0;
        if (ri[r][i] >= 0 && ci[c][j] >= 0) {
            cplx v = tile_f(S, r, c, i, j);
            v.x += ms;
            A.p[ri[r][i] + (int64_t)ci[c][j] * A.ld] = v;
        }
        if (ci[c][i] >= 0 && ri[r][j] >= 0) {
            cplx w = tile_r(S, c, r, i, j);
            w.x += ms;
            A.p[ci[c][i] + (int64_t)ri[r][j] * A.ld] = w;
        }
    }
}

// V_i = blockdiag(V^1, V^2), V^c = [I T^c] P^T  (k^c x n^c), dense r x d.
__global__ void k_make_V(const MatRef *__restrict__ Vs, const int *__restrict__ n1, const int *__restrict__ n2,
                         const int *__restrict__ k1, const int *__restrict__ k2, const int *__restrict__ perm,
                         const int64_t *__restrict__ poff, const cplx *__restrict__ T,
                         const int64_t *__restrict__ toff) {
    const int b = blockIdx.x;
    const MatRef V = Vs[b];
    for (int64_t e = threadIdx.x; e < (int64_t)V.rows * V.cols; e += blockDim.x)
        V.p[(e % V.rows) + (e / V.rows) * V.ld] = mkc(0, 0);
    __syncthreads();
    for (int c = 0; c < 2; ++c) {
        const int n = c ? n2[b] : n1[b], k = c ? k2[b] : k1[b];
        const int r0 = c ? k1[b] : 0, c0 = c ? n1[b] : 0;
        const int *pm = perm + poff[2 * b + c];
        const cplx *Tc = T + toff[2 * b + c];
        for (int q = threadIdx.x; q < k; q += blockDim.x) V.p[(r0 + q) + (int64_t)(c0 + pm[q]) * V.ld] = mkc(1, 0);
        for (int64_t e = threadIdx.x; e < (int64_t)k * (n - k); e += blockDim.x) {
            const int q = (int)(e % k), l = (int)(e / k);
            V.p[(r0 + q) + (int64_t)(c0 + pm[k + l]) * V.ld] = Tc[q + (int64_t)l * k];
        }
    }
}

// W = V^H (d x r) as the right-hand side of A_i W = U_i, U_i = V_i^H.
template <class C>
__global__ void k_conj_transpose(const MatRefT<C> *__restrict__ Src, const MatRefT<C> *__restrict__ Dst) {
    const MatRefT<C> S = Src[blockIdx.x], D = Dst[blockIdx.x];
    for (int64_t e = threadIdx.x; e < (int64_t)S.rows * S.cols; e += blockDim.x) {
        const int i = (int)(e % S.rows), j = (int)(e / S.rows);
        D.p[j + (int64_t)i * D.ld] = cconj(S.p[i + (int64_t)j * S.ld]);
    }
}

template <class C>
__global__ void k_set_identity(const MatRefT<C> *__restrict__ Ms) {
    const MatRefT<C> M = Ms[blockIdx.x];
    for (int64_t e = threadIdx.x; e < (int64_t)M.rows * M.cols; e += blockDim.x) {
        const int i = (int)(e % M.rows), j = (int)(e / M.rows);
        C v = czero<C>();
        if (i == j) v.x = 1;
        M.p[i + (int64_t)j * M.ld] = v;
    }
}

// element-wise precision change of a contiguous buffer
template <class A, class B>
__global__ void k_cast(const A *__restrict__ src, B *dst, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        dst[e].x = src[e].x;
        dst[e].y = src[e].y;
    }
}

// float pairs (float4: re_hi, im_hi, re_lo, im_lo) from complex128 / complex64
template <class A>
__global__ void k_to_ff(const A *__restrict__ src, float4 *dst, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const double re = src[e].x, im = src[e].y;
        const float rh = (float)re, ih = (float)im;
        dst[e] = make_float4(rh, ih, (float)(re - (double)rh), (float)(im - (double)ih));
    }
}

// complex64 (rounded) or complex128 from float pairs
template <class B>
__global__ void k_from_ff(const float4 *__restrict__ src, B *dst, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = src[e];
        dst[e].x = (double)v.x + (double)v.z;
        dst[e].y = (double)v.y + (double)v.w;
    }
}

// X1 = X0 + D (float pairs X0, complex64 correction D): the float-pair sum
// (renormalised) and its complex64 rounding
__global__ void k_ff_add_c64(const float4 *__restrict__ x0, const cplxf *__restrict__ d, float4 *x1, cplxf *x1f,
                             int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = x0[e];
        const cplxf b = d[e];
        float h[2] = {a.x, a.y}, l[2] = {a.z, a.w};
        const float c[2] = {b.x, b.y};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const float s = h[q] + c[q], bb = s - h[q];
            const float err = (h[q] - (s - bb)) + (c[q] - bb) + l[q];
            h[q] = s + err;
            l[q] = err - (h[q] - s);
        }
        x1[e] = make_float4(h[0], h[1], l[0], l[1]);
        x1f[e] = mkcf(h[0] + l[0], h[1] + l[1]);
    }
}

// R = I - R on every block (float pairs)
__global__ void k_ff_identity_minus(const MatRefP *__restrict__ Ms) {
    const MatRefP M = Ms[blockIdx.x];
    for (int64_t e = threadIdx.x; e < (int64_t)M.rows * M.cols; e += blockDim.x) {
        const int i = (int)(e % M.rows), j = (int)(e / M.rows);
        float4 &v = M.p[i + (int64_t)j * M.ld];
        float rh = -v.x, rl = -v.z;
        if (i == j) {
            // 1 - (h + l): two-sum of 1 and -h, then the low parts (Knuth)
            const float s1 = 1.0f + rh, bb = s1 - 1.0f;
            const float err = (1.0f - (s1 - bb)) + (rh - bb);
            const float lo = err + rl;
            rh = s1 + lo;
            rl = lo - (rh - s1);
        }
        v = make_float4(rh, -v.y, rl, -v.w);
    }
}

__global__ void k_zero(cplx *p, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        p[e] = mkc(0, 0);
}

// Place the children's A~ blocks into the parent block (eq. (A_rearrangement)):
// child skeleton index q -> parent row q < k1 ? pos1 + q : pos2 + (q - k1).
__global__ void k_place_children(const MatRef *__restrict__ Atc, const int *__restrict__ k1c,
                                 const int *__restrict__ pos1, const int *__restrict__ pos2,
                                 const MatRef *__restrict__ Apar) {
    const int ch = blockIdx.x;   // child index at the lower level
    const MatRef S = Atc[ch], D = Apar[ch >> 1];
    const int k1 = k1c[ch], p1 = pos1[ch], p2 = pos2[ch];
    for (int64_t e = threadIdx.x; e < (int64_t)S.rows * S.cols; e += blockDim.x) {
        const int i = (int)(e % S.rows), j = (int)(e / S.rows);
        const int pi = i < k1 ? p1 + i : p2 + (i - k1);
        const int pj = j < k1 ? p1 + j : p2 + (j - k1);
        D.p[pi + (int64_t)pj * D.ld] = S.p[i + (int64_t)j * S.ld];
    }
}

// Copy diagonal blocks of the top level into the top matrix.
__global__ void k_place_top(const MatRef *__restrict__ Ab, const int64_t *__restrict__ doff, MatRef top) {
    const int b = blockIdx.x;
    const MatRef S = Ab[b];
    const int64_t o = doff[b];
    for (int64_t e = threadIdx.x; e < (int64_t)S.rows * S.cols; e += blockDim.x) {
        const int i = (int)(e % S.rows), j = (int)(e / S.rows);
        top.p[(o + i) + (o + j) * top.ld] = S.p[i + (int64_t)j * S.ld];
    }
}

// Counts the quadrature points of the a1 launches inside a ProfScope (only
// while timing is enabled; synchronises the stream to read the count).
struct PointCount {
    bool on;
    cudaStream_t s;
    explicit PointCount(cudaStream_t st) : on(prof_enabled()), s(st) {
        if (!on) return;
        const unsigned long long z = 0;
        const int one = 1;
        cudaMemcpyToSymbolAsync(d_quad_points, &z, sizeof(z), 0, cudaMemcpyHostToDevice, s);
        cudaMemcpyToSymbolAsync(d_count_points, &one, sizeof(one), 0, cudaMemcpyHostToDevice, s);
    }
    double read() {
        if (!on) return 0.0;
        unsigned long long v = 0;
        const int zero = 0;
        cudaMemcpyFromSymbolAsync(&v, d_quad_points, sizeof(v), 0, cudaMemcpyDeviceToHost, s);
        cudaMemcpyToSymbolAsync(d_count_points, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, s);
        cudaStreamSynchronize(s);
        return (double)v;
    }
};

int sync_check(cudaStream_t s) {
    FDS_CUDA_TRY(cudaStreamSynchronize(s));
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}

template <class T>
int d2h(std::vector<T> &h, const T *d, size_t n, cudaStream_t s) {
    h.resize(n);
    if (n) FDS_CUDA_TRY(cudaMemcpyAsync(h.data(), d, n * sizeof(T), cudaMemcpyDeviceToHost, s));
    return FDS_OK;
}

// Fill per-cell MatRefs for a level buffer with square/rect blocks.
int make_refs(DBuf<MatRef> &dst, cplx *base, const std::vector<int64_t> &off, const std::vector<int> &rows,
              const std::vector<int> &cols, cudaStream_t s) {
    std::vector<MatRef> h(rows.size());
    for (size_t b = 0; b < rows.size(); ++b) {
        h[b].p = base + off[b];
        h[b].rows = rows[b];
        h[b].cols = cols[b];
        h[b].ld = std::max(rows[b], 1);
    }
    return dst.upload(h, s);
}

// Build the union node list of a level from its per-component DOF lists.
void build_union(Level &L) {
    L.uoff.assign(L.nb + 1, 0);
    L.unode.clear(); L.upos1.clear(); L.upos2.clear(); L.utag.clear();
    for (int b = 0; b < L.nb; ++b) {
        const int *d = L.dof_node.data() + L.doff[b];
        std::vector<std::pair<int, int>> items;   // (node, comp/pos code)
        std::vector<int> nodes;
        for (int q = 0; q < L.n1[b]; ++q) nodes.push_back(d[q]);
        for (int q = 0; q < L.n2[b]; ++q) nodes.push_back(d[L.n1[b] + q]);
        std::vector<int> uniq = nodes;
        std::sort(uniq.begin(), uniq.end());
        uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
        std::vector<int> p1(uniq.size(), -1), p2(uniq.size(), -1);
        for (int q = 0; q < L.n1[b]; ++q) {
            size_t k = std::lower_bound(uniq.begin(), uniq.end(), d[q]) - uniq.begin();
            p1[k] = q;
        }
        for (int q = 0; q < L.n2[b]; ++q) {
            size_t k = std::lower_bound(uniq.begin(), uniq.end(), d[L.n1[b] + q]) - uniq.begin();
            p2[k] = q;
        }
        for (size_t k = 0; k < uniq.size(); ++k) {
            L.unode.push_back(uniq[k]);
            L.upos1.push_back(p1[k]);
            L.upos2.push_back(p2[k]);
            L.utag.push_back(0);
        }
        L.uoff[b + 1] = (int64_t)L.unode.size();
    }
}

void finish_offsets(Level &L) {
    L.doff.assign(L.nb + 1, 0);
    L.dmax = 0;
    for (int b = 0; b < L.nb; ++b) {
        L.doff[b + 1] = L.doff[b] + L.n1[b] + L.n2[b];
        L.dmax = std::max(L.dmax, L.n1[b] + L.n2[b]);
    }
    L.D = L.doff[L.nb];
}

// Matrices A_b (d x d) of a level, allocated contiguously.
int alloc_level_A(Level &L, cudaStream_t s) {
    L.offA.assign(L.nb + 1, 0);
    std::vector<int> d(L.nb);
    for (int b = 0; b < L.nb; ++b) {
        d[b] = L.n1[b] + L.n2[b];
        L.offA[b + 1] = L.offA[b] + (int64_t)d[b] * d[b];
    }
    FDS_TRY(L.LU.alloc(L.offA[L.nb]));
    FDS_TRY(make_refs(L.rLU, L.LU.p, L.offA, d, d, s));
    return FDS_OK;
}

// Original-entry blocks between the tagged parts of each group (tags
// ascending: every pair of distinct tags tA < tB is evaluated once, both
// orientations).  Items of group g occupy [goff[g], goff[g+1]) sorted by tag.
int launch_group_blocks(fds_handle *h, const char *name, const std::vector<int64_t> &goff,
                        const std::vector<int> &gnode, const std::vector<int> &gtag, const std::vector<int> &grow1,
                        const std::vector<int> &grow2, const MatRef *d_M, cudaStream_t s) {
    const int ng = (int)goff.size() - 1;
    if (ng <= 0 || gnode.empty()) return FDS_OK;
    std::vector<GJob> jobs;
    for (int g = 0; g < ng; ++g) {
        // split the group's items into runs of equal tag
        std::vector<std::pair<int64_t, int64_t>> runs;
        for (int64_t u = goff[g]; u < goff[g + 1];) {
            int64_t v = u;
            while (v < goff[g + 1] && gtag[v] == gtag[u]) ++v;
            runs.push_back({u, v});
            u = v;
        }
        for (size_t a = 0; a < runs.size(); ++a)
            for (size_t b = a + 1; b < runs.size(); ++b)
                for (int64_t r0 = runs[a].first; r0 < runs[a].second; r0 += TILE)
                    for (int64_t c0 = runs[b].first; c0 < runs[b].second; c0 += TILE) {
                        GJob j;
                        j.g = g;
                        j.roff = (int)r0;
                        j.nr = (int)std::min<int64_t>(TILE, runs[a].second - r0);
                        j.coff = (int)c0;
                        j.nc = (int)std::min<int64_t>(TILE, runs[b].second - c0);
                        jobs.push_back(j);
                    }
    }
    if (jobs.empty()) return FDS_OK;
    DBuf<int> d_gnode, d_g1, d_g2;
    DBuf<GJob> d_jobs;
    FDS_TRY(d_gnode.upload(gnode, s));
    FDS_TRY(d_g1.upload(grow1, s));
    FDS_TRY(d_g2.upload(grow2, s));
    FDS_TRY(d_jobs.upload(jobs, s));
    PointCount pc(s);
    ProfScope ps(name, s);
    fds_count_launch(), k_tiles_group<<<(unsigned)jobs.size(), FDS_TILE_THREADS, 0, s>>>(h->P, d_gnode.p, d_g1.p, d_g2.p,
                                                                          h->d_xy.p, h->N, d_M, d_jobs.p);
    FDS_CUDA_TRY(cudaGetLastError());
    ps.units = pc.read();
    return sync_check(s);   // the temporaries above are freed on return
}

}  // namespace

// ------------------------------------------------------------------ build
// Woodbury form of the original Martinsson–Rokhlin elimination (the method
// the paper's variant is compared with, Sec. 6 introduction): with
// A~_i = (V_i A_i^{-1} U_i)^{-1},
//   A^{-1} = G + E (A~ + B~)^{-1} F,  E_i = A_i^{-1} U_i A~_i,
//   F_i = A~_i V_i A_i^{-1},  G_i = A_i^{-1} - E_i V_i A_i^{-1},
// B~ the coupling between the skeletons (the same compressed system as the
// LU variant).  Four GEMMs per cell beyond the LU variant's products.
int mr2005_level_factors(fds_handle *h, Level &C, const std::vector<int> &dv, const std::vector<int> &rv,
                         cudaStream_t s) {
    const int nb = C.nb;
    double fl_e = 0, fl_q = 0, fl_f = 0, fl_g = 0;
    for (int b = 0; b < nb; ++b) {
        const double d = dv[b], r = rv[b];
        fl_e += 8.0 * d * r * r;
        fl_q += 8.0 * r * d * d;
        fl_f += 8.0 * r * r * d;
        fl_g += 8.0 * d * r * d;
    }
    DBuf<cplx> Q;
    DBuf<MatRef> rQ;
    FDS_TRY(C.mrE.alloc(C.offW[nb]));
    FDS_TRY(C.mrF.alloc(C.offV[nb]));
    FDS_TRY(C.mrG.alloc(C.offA[nb]));
    FDS_TRY(Q.alloc(C.offV[nb]));
    FDS_TRY(make_refs_t(C.rmrE, C.mrE.p, C.offW, dv, rv, s));
    FDS_TRY(make_refs_t(C.rmrF, C.mrF.p, C.offV, rv, dv, s));
    FDS_TRY(make_refs_t(C.rmrG, C.mrG.p, C.offA, dv, dv, s));
    FDS_TRY(make_refs_t(rQ, Q.p, C.offV, rv, dv, s));
    const cplx one = mkc(1, 0), zero = mkc(0, 0), mone = mkc(-1, 0);
    ProfScope ps("a3.mr2005_products", s);
    ps.flops = fl_e + fl_q + fl_f + fl_g;
    // E = W A~ ; Q = V A^{-1} ; F = A~ Q ; G = A^{-1} - E Q
    FDS_TRY(dense_gemm(nb, C.dmax, C.rmax, C.rW.p, 0, C.rAt.p, 0, C.rmrE.p, one, zero, s));
    FDS_TRY(dense_gemm(nb, C.rmax, C.dmax, C.rV.p, 0, C.rAinv.p, 0, rQ.p, one, zero, s));
    FDS_TRY(dense_gemm(nb, C.rmax, C.dmax, C.rAt.p, 0, rQ.p, 0, C.rmrF.p, one, zero, s));
    FDS_CUDA_TRY(cudaMemcpyAsync(C.mrG.p, C.Ainv.p, sizeof(cplx) * C.offA[nb], cudaMemcpyDeviceToDevice, s));
    FDS_TRY(dense_gemm(nb, C.dmax, C.dmax, C.rmrE.p, 0, rQ.p, 0, C.rmrG.p, mone, one, s));
    FDS_TRY(sync_check(s));
    h->factor_bytes += (int64_t)(C.mrE.bytes() + C.mrF.bytes() + C.mrG.bytes());
    return FDS_OK;
}

// ID tolerance of level l: tol at the leaves, tol * tol_decay^(L - l) above,
// but not below 1e-15 (FP64 rounding of the proxy matrices) unless tol is
static double level_tol(const fds_handle *h, int l) {
    const double t = h->tol * std::pow(h->opt.tol_decay, (double)(h->L - l));
    return std::max(t, std::min(h->tol, 1e-15));
}

int fds_build_impl(fds_handle *h) {
    cudaStream_t s = h->stream;
    C64EngineScope eng(h->opt.c64_engine == FDS_C64_TENSOR);
    FDS_TRY(ensure_gauss_tables());
    const int N = h->N;
    const int leaf = h->opt.leaf_size;
    // tree depth: smallest L with ceil(N / 2^L) <= leaf; halving split
    int L = 0;
    while (((N + (1 << L) - 1) >> L) > leaf) ++L;
    h->L = L;
    // top_level < 0 counts up from the leaves: -1 is the single-level variant
    // of Sec. 8.1 (Table tab:error_single), l0 = L - 1
    h->l0 = h->opt.top_level >= 0 ? std::min(h->opt.top_level, L) : std::max(L + h->opt.top_level, 0);
    h->ranges.assign(L + 1, {});
    h->ranges[0].push_back({0, N});
    for (int l = 0; l < L; ++l)
        for (auto &r : h->ranges[l]) {
            int mid = r.first + (r.second - r.first) / 2;
            h->ranges[l + 1].push_back({r.first, mid});
            h->ranges[l + 1].push_back({mid, r.second});
        }
    h->lv.clear();
    h->lv.resize(L + 1);
    FDS_TRY(h->d_xy.upload(h->xy, s));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);

    // leaf level DOFs: contiguous ranges, comp-1 block then comp-2 block
    {
        Level &Lf = h->lv[L];
        Lf.nb = (int)h->ranges[L].size();
        Lf.n1.resize(Lf.nb);
        Lf.n2.resize(Lf.nb);
        Lf.dof_node.clear();
        for (int b = 0; b < Lf.nb; ++b) {
            auto r = h->ranges[L][b];
            Lf.n1[b] = Lf.n2[b] = r.second - r.first;
            for (int c = 0; c < 2; ++c)
                for (int v = r.first; v < r.second; ++v) Lf.dof_node.push_back(v);
        }
        finish_offsets(Lf);
        build_union(Lf);
        FDS_TRY(alloc_level_A(Lf, s));
        std::vector<int> gidx(Lf.D);
        for (int b = 0; b < Lf.nb; ++b)
            for (int q = 0; q < Lf.n1[b] + Lf.n2[b]; ++q)
                gidx[Lf.doff[b] + q] = Lf.dof_node[Lf.doff[b] + q] + (q < Lf.n1[b] ? 0 : N);
        FDS_TRY(h->d_leaf_gidx.upload(gidx, s));
        std::vector<int> lo(Lf.nb), hi(Lf.nb);
        int nmax = 0;
        for (int b = 0; b < Lf.nb; ++b) {
            lo[b] = h->ranges[L][b].first;
            hi[b] = h->ranges[L][b].second;
            nmax = std::max(nmax, hi[b] - lo[b]);
        }
        DBuf<int> d_lo, d_hi;
        FDS_TRY(d_lo.upload(lo, s));
        FDS_TRY(d_hi.upload(hi, s));
        std::vector<LeafJob> jobs;
        for (int b = 0; b < Lf.nb; ++b) {
            const int T = (hi[b] - lo[b] + TILE - 1) / TILE;
            for (int I = 0; I < T; ++I)
                for (int J = I; J < T; ++J) jobs.push_back(LeafJob{b, I, J});
        }
        DBuf<LeafJob> d_jobs;
        FDS_TRY(d_jobs.upload(jobs, s));
        {
            PointCount pc(s);
            ProfScope ps("a1.leaf_blocks", s);
            fds_count_launch(), k_tiles_leaf<<<(unsigned)jobs.size(), FDS_TILE_THREADS, 0, s>>>(h->P, d_lo.p, d_hi.p, h->d_xy.p, N,
                                                                                 Lf.rLU.p, d_jobs.p);
            ps.units = pc.read();
        }
        FDS_CUDA_TRY(cudaGetLastError());
        if (fds_fault_nan_fires()) {
            // injected fault: a NaN in the first leaf's diagonal block
            const cplx bad = mkc(std::nan(""), 0.0);
            FDS_CUDA_TRY(cudaMemcpyAsync(Lf.LU.p, &bad, sizeof(cplx), cudaMemcpyHostToDevice, s));
            FDS_CUDA_TRY(cudaStreamSynchronize(s));
        }
        if (h->opt.precision == FDS_MIXED) FDS_TRY(fds_keep_blocks(Lf, Lf.Dfw, Lf.rDfw, s));
        FDS_TRY(sync_check(s));
    }

    for (int l = L; l > h->l0; --l) {
        Level &C = h->lv[l];
        const int nb = C.nb;
        // ---- cell circles and proxy polygons (a0)
        {
            std::vector<int> lo(nb), hi(nb);
            for (int b = 0; b < nb; ++b) { lo[b] = h->ranges[l][b].first; hi[b] = h->ranges[l][b].second; }
            DBuf<int> d_lo, d_hi;
            DBuf<double> d_cx, d_cy, d_R;
            FDS_TRY(d_lo.upload(lo, s));
            FDS_TRY(d_hi.upload(hi, s));
            FDS_TRY(d_cx.alloc(nb));
            FDS_TRY(d_cy.alloc(nb));
            FDS_TRY(d_R.alloc(nb));
            {
                ProfScope ps("a0.cell_circles", s);
                fds_count_launch(), k_box_circles<<<ceil_div_u((long)nb * 32, 256), 256, 0, s>>>(nb, d_lo.p, d_hi.p, h->d_xy.p, N,
                                                                             d_cx.p, d_cy.p, d_R.p);
            }
            FDS_CUDA_TRY(cudaGetLastError());
            FDS_TRY(d2h(C.cx, d_cx.p, nb, s));
            FDS_TRY(d2h(C.cy, d_cy.p, nb, s));
            FDS_TRY(d2h(C.R, d_R.p, nb, s));
            FDS_TRY(sync_check(s));
        }
        C.Rp.resize(nb);
        C.mprox.resize(nb);
        for (int b = 0; b < nb; ++b) {
            C.Rp[b] = h->opt.proxy_ratio * C.R[b];
            C.mprox[b] = std::max(h->opt.proxy_points, (int)std::ceil(2.0 * h->P.kT * C.Rp[b] + 30.0));
        }
        std::vector<int64_t> pxoff(nb + 1, 0);
        for (int b = 0; b < nb; ++b) pxoff[b + 1] = pxoff[b] + C.mprox[b];
        DBuf<double> d_cx, d_cy, d_R, d_Rp, d_pxy;
        DBuf<int> d_mp;
        DBuf<int64_t> d_pxoff;
        FDS_TRY(d_cx.upload(C.cx, s));
        FDS_TRY(d_cy.upload(C.cy, s));
        FDS_TRY(d_R.upload(C.R, s));
        FDS_TRY(d_Rp.upload(C.Rp, s));
        FDS_TRY(d_mp.upload(C.mprox, s));
        FDS_TRY(d_pxoff.upload(pxoff, s));
        FDS_TRY(d_pxy.alloc(2 * pxoff[nb]));
        fds_count_launch(), k_proxy_nodes<<<nb, 128, 0, s>>>(d_cx.p, d_cy.p, d_Rp.p, d_mp.p, d_pxoff.p, d_pxy.p);
        FDS_CUDA_TRY(cudaGetLastError());
        // ---- union lists on the device
        FDS_TRY(C.d_uoff.upload(C.uoff, s));
        FDS_TRY(C.d_unode.upload(C.unode, s));
        FDS_TRY(C.d_upos1.upload(C.upos1, s));
        FDS_TRY(C.d_upos2.upload(C.upos2, s));
        // ---- near field
        DBuf<int> d_cnt;
        FDS_TRY(d_cnt.alloc(nb));
        {
            ProfScope ps("a0.near_field", s);
            fds_count_launch(), k_near<<<nb, 128, 0, s>>>(nb, d_cx.p, d_cy.p, d_R.p, d_Rp.p, C.d_uoff.p, C.d_unode.p, C.d_upos1.p,
                                      C.d_upos2.p, h->d_xy.p, N, 0, d_cnt.p, nullptr, nullptr, nullptr);
        }
        FDS_CUDA_TRY(cudaGetLastError());
        std::vector<int> cnt;
        FDS_TRY(d2h(cnt, d_cnt.p, nb, s));
        FDS_TRY(sync_check(s));
        std::vector<int64_t> noff(nb + 1, 0);
        for (int b = 0; b < nb; ++b) noff[b + 1] = noff[b] + cnt[b];
        DBuf<int64_t> d_noff;
        DBuf<int> d_nnode, d_nmask;
        FDS_TRY(d_noff.upload(noff, s));
        FDS_TRY(d_nnode.alloc(noff[nb]));
        FDS_TRY(d_nmask.alloc(noff[nb]));
        {
            ProfScope ps("a0.near_field", s);
            fds_count_launch(), k_near<<<nb, 128, 0, s>>>(nb, d_cx.p, d_cy.p, d_R.p, d_Rp.p, C.d_uoff.p, C.d_unode.p, C.d_upos1.p,
                                      C.d_upos2.p, h->d_xy.p, N, 1, d_cnt.p, d_noff.p, d_nnode.p, d_nmask.p);
        }
        FDS_CUDA_TRY(cudaGetLastError());
        std::vector<int> nmask;
        FDS_TRY(d2h(nmask, d_nmask.p, noff[nb], s));
        FDS_TRY(sync_check(s));
        // ---- Y layout: [2m' proxy V][nnd near V][2m' proxy U][nnd near U] rows
        std::vector<int> nrow(noff[nb]), nnd(nb), ym(nb), idm(2 * nb), idn(2 * nb);
        std::vector<int64_t> yoff(2 * nb + 1, 0), toff(2 * nb + 1, 0), poff(2 * nb + 1, 0);
        int maxm = 1, maxn = 1;
        int64_t maxjp = 0, maxjn = 0;
        for (int b = 0; b < nb; ++b) {
            int rb = 0;
            for (int64_t k = noff[b]; k < noff[b + 1]; ++k) {
                nrow[k] = rb;
                rb += (nmask[k] & 1) + ((nmask[k] >> 1) & 1);
            }
            nnd[b] = rb;
            ym[b] = 4 * C.mprox[b] + 2 * rb;
            maxm = std::max(maxm, ym[b]);
            const int64_t nu = C.uoff[b + 1] - C.uoff[b];
            maxjp = std::max(maxjp, (int64_t)C.mprox[b] * nu);
            maxjn = std::max(maxjn, (noff[b + 1] - noff[b]) * nu);
            for (int c = 0; c < 2; ++c) {
                const int n = c ? C.n2[b] : C.n1[b];
                idm[2 * b + c] = ym[b];
                idn[2 * b + c] = n;
                maxn = std::max(maxn, n);
                yoff[2 * b + c + 1] = yoff[2 * b + c] + (int64_t)ym[b] * n;
                toff[2 * b + c + 1] = toff[2 * b + c] + (int64_t)n * n / 4 + 1;
                poff[2 * b + c + 1] = poff[2 * b + c] + n;
            }
        }
        DBuf<cplx> d_Y, d_T;
        DBuf<int64_t> d_yoff, d_toff, d_poff;
        DBuf<int> d_ym, d_nnd, d_nrow, d_idm, d_idn, d_rank, d_perm;
        FDS_TRY(d_Y.alloc(yoff[2 * nb]));
        FDS_TRY(d_T.alloc(toff[2 * nb]));
        FDS_TRY(d_yoff.upload(yoff, s));
        FDS_TRY(d_toff.upload(toff, s));
        FDS_TRY(d_poff.upload(poff, s));
        FDS_TRY(d_ym.upload(ym, s));
        FDS_TRY(d_nnd.upload(nnd, s));
        FDS_TRY(d_nrow.upload(nrow, s));
        FDS_TRY(d_idm.upload(idm, s));
        FDS_TRY(d_idn.upload(idn, s));
        FDS_TRY(d_rank.alloc(2 * nb));
        FDS_TRY(d_perm.alloc(poff[2 * nb]));
        YDesc D;
        D.yoff = d_yoff.p; D.ym = d_ym.p; D.mp = d_mp.p; D.nnd = d_nnd.p; D.pxoff = d_pxoff.p; D.pxy = d_pxy.p;
        D.uoff = C.d_uoff.p; D.unode = C.d_unode.p; D.upos1 = C.d_upos1.p; D.upos2 = C.d_upos2.p;
        D.noff = d_noff.p; D.nnode = d_nnode.p; D.nmask = d_nmask.p; D.nrow = d_nrow.p;
        // ---- kernel evaluation (a1)
        for (int kind = 0; kind < 2; ++kind) {
            std::vector<YJob> jobs;
            for (int b = 0; b < nb; ++b) {
                const int nu = (int)(C.uoff[b + 1] - C.uoff[b]);
                const int nrows = kind == 0 ? C.mprox[b] : (int)(noff[b + 1] - noff[b]);
                for (int u0 = 0; u0 < nu; u0 += TILE)
                    for (int r0 = 0; r0 < nrows; r0 += TILE) jobs.push_back(YJob{b, kind, r0, u0});
            }
            DBuf<YJob> d_jobs;
            FDS_TRY(d_jobs.upload(jobs, s));
            if (!jobs.empty()) {
                PointCount pc(s);
                ProfScope ps(kind == 0 ? "a1.proxy_rows" : "a1.near_rows", s);
                fds_count_launch(), k_tiles_y<<<(unsigned)jobs.size(), FDS_TILE_THREADS, 0, s>>>(h->P, D, h->d_xy.p, N, d_Y.p,
                                                                                   d_jobs.p);
                ps.units = pc.read();
            }
            FDS_CUDA_TRY(cudaGetLastError());
            FDS_TRY(sync_check(s));
        }
        // ---- interpolative decomposition (a2; a2' with the learned rank)
        const bool learned = h->opt.rank_mode == FDS_RANK_LEARNED;
        const double tol_l = level_tol(h, l);
        std::vector<int> h_fail_flags;   // learned: the (cell, component) IDs redone by the adaptive CPQR
        DBuf<float> d_feat;
        if (learned || h->opt.record_features) {
            std::vector<int> lo(nb), hi(nb);
            for (int b = 0; b < nb; ++b) { lo[b] = h->ranges[l][b].first; hi[b] = h->ranges[l][b].second; }
            DBuf<int> d_lo, d_hi, d_fn1, d_fn2;
            FDS_TRY(d_lo.upload(lo, s));
            FDS_TRY(d_hi.upload(hi, s));
            FDS_TRY(d_fn1.upload(C.n1, s));
            FDS_TRY(d_fn2.upload(C.n2, s));
            FDS_TRY(d_feat.alloc((size_t)2 * nb * FDS_MLP_NIN));
            ProfScope ps("a2.features", s);
            FDS_TRY(level_features(nb, d_lo.p, d_hi.p, h->d_xy.p, N, d_R.p, d_fn1.p, d_fn2.p, d_nnd.p, L - l,
                                   h->P.kT, h->P.kL, tol_l, d_feat.p, s));
            FDS_TRY(sync_check(s));
        }
        if (learned) {
            DBuf<float> d_frac;
            DBuf<int> d_fail;
            FDS_TRY(d_frac.alloc((size_t)2 * nb));
            FDS_TRY(d_fail.alloc((size_t)2 * nb));
            {
                ProfScope ps("a2.rank_mlp", s);
                FDS_TRY(mlp_forward(h->d_mlp.p, d_feat.p, 2 * nb, d_frac.p, s));
            }
            {
                ProfScope ps("a2.id_sketch", s);
                FDS_TRY(id_sketched(2 * nb, maxm, d_idm.p, d_idn.p, d_yoff.p, d_Y.p, d_frac.p, h->opt.sketch_extra,
                                    tol_l, d_rank.p, d_perm.p, d_poff.p, d_T.p, d_toff.p, d_fail.p,
                                    0x5eed2411ULL ^ ((unsigned long long)l << 40), s));
            }
            std::vector<int> fail;
            FDS_TRY(d2h(fail, d_fail.p, 2 * nb, s));
            FDS_TRY(sync_check(s));
            h_fail_flags = fail;
            std::vector<int> sel;
            for (int b = 0; b < 2 * nb; ++b)
                if (fail[b]) sel.push_back(b);
            h->id_sketched += 2 * nb - (int64_t)sel.size();
            h->id_fallback += (int64_t)sel.size();
            if (!sel.empty()) {
                DBuf<int> d_sel;
                FDS_TRY(d_sel.upload(sel, s));
                ProfScope ps("a2.id_cpqr", s);
                FDS_TRY(id_batched((int)sel.size(), maxm, maxn, d_idm.p, d_idn.p, d_yoff.p, d_Y.p, tol_l, d_rank.p,
                                   d_perm.p, d_poff.p, d_T.p, d_toff.p, s, d_sel.p));
                FDS_TRY(sync_check(s));
            }
        } else {
            ProfScope ps("a2.id_cpqr", s);
            FDS_TRY(id_batched(2 * nb, maxm, maxn, d_idm.p, d_idn.p, d_yoff.p, d_Y.p, tol_l, d_rank.p, d_perm.p,
                               d_poff.p, d_T.p, d_toff.p, s));
        }
        std::vector<int> rank;
        FDS_TRY(d2h(rank, d_rank.p, 2 * nb, s));
        FDS_TRY(d2h(C.perm, d_perm.p, poff[2 * nb], s));
        FDS_TRY(sync_check(s));
        if (prof_enabled()) {
            // algorithmic work of the Householder CPQR that ran, m x n to rank k:
            // 8 (2 m n k - k^2 (m + n) + 2 k^3 / 3) real flops per matrix
            std::vector<char> ran(2 * nb, learned ? 0 : 1);
            if (learned)
                for (int b = 0; b < 2 * nb; ++b) ran[b] = h_fail_flags.empty() ? 0 : h_fail_flags[b];
            double fl = 0;
            for (int b = 0; b < 2 * nb; ++b) {
                if (!ran[b]) continue;
                const double m = idm[b], n = idn[b], k = rank[b];
                fl += 8.0 * (2.0 * m * n * k - k * k * (m + n) + 2.0 * k * k * k / 3.0);
            }
            prof_add_work("a2.id_cpqr", fl, 0, 0);
        }
        if (h->opt.record_features) {
            std::vector<float> f;
            FDS_TRY(d2h(f, d_feat.p, (size_t)2 * nb * FDS_MLP_NIN, s));
            FDS_TRY(sync_check(s));
            for (int b = 0; b < 2 * nb; ++b) {
                const int n = (b & 1) ? C.n2[b >> 1] : C.n1[b >> 1];
                if (n <= 0) continue;
                h->feat_rows.insert(h->feat_rows.end(), f.begin() + (size_t)b * FDS_MLP_NIN,
                                    f.begin() + (size_t)(b + 1) * FDS_MLP_NIN);
                h->frac_rows.push_back((float)rank[b] / (float)n);
            }
        }
        C.permoff = poff;
        C.k1.resize(nb);
        C.k2.resize(nb);
        C.roff.assign(nb + 1, 0);
        C.rmax = 0;
        for (int b = 0; b < nb; ++b) {
            C.k1[b] = rank[2 * b];
            C.k2[b] = rank[2 * b + 1];
            C.roff[b + 1] = C.roff[b] + C.k1[b] + C.k2[b];
            C.rmax = std::max(C.rmax, C.k1[b] + C.k2[b]);
        }
        C.Rtot = C.roff[nb];
        // ---- merge (a3): LU(A_i), W = A_i^{-1} V_i^H, S = V_i W, A~ = S^{-1}
        std::vector<int> dv(nb), rv(nb);
        C.offV.assign(nb + 1, 0);
        C.offAt.assign(nb + 1, 0);
        C.offpiv.assign(nb + 1, 0);
        C.sum_d2 = C.sum_rd = C.sum_r2 = 0;
        for (int b = 0; b < nb; ++b) {
            dv[b] = C.n1[b] + C.n2[b];
            rv[b] = C.k1[b] + C.k2[b];
            C.sum_d2 += (double)dv[b] * dv[b];
            C.sum_rd += (double)rv[b] * dv[b];
            C.sum_r2 += (double)rv[b] * rv[b];
            C.offV[b + 1] = C.offV[b] + (int64_t)rv[b] * dv[b];
            C.offAt[b + 1] = C.offAt[b] + (int64_t)rv[b] * rv[b];
            C.offpiv[b + 1] = C.offpiv[b] + dv[b];
        }
        C.offW = C.offV;
        // FDS_MIXED: the lower levels, whose sweep runs in complex64, are merged
        // in complex64 too (decided from the top down so that the complex128
        // levels stay a prefix below the top)
        C.c64 = false;
        if (h->opt.precision == FDS_MIXED && h->opt.sweep_ff < 2 && !h->fp64_reached) {
            if (h->opt.sweep_fp64_levels >= 0) C.c64 = l > std::min(L - 1, h->l0 + h->opt.sweep_fp64_levels);
            else C.c64 = (l == L) || 8 * C.D > h->lv[L].D;
            if (!C.c64) h->fp64_reached = true;
        }
        // merged in complex64 (else FP64, converted later): every complex64
        // level, or the lowest merge_c64_levels of them
        const bool merge64 = C.c64 && h->opt.merge_c64 &&
                             (h->opt.merge_c64_levels <= 0 || l > L - h->opt.merge_c64_levels);
        FDS_TRY(C.V.alloc(C.offV[nb]));
        FDS_TRY(C.At.alloc(C.offAt[nb]));
        FDS_TRY(C.piv.alloc(C.offpiv[nb]));
        FDS_TRY(C.d_offpiv.upload(C.offpiv, s));
        FDS_TRY(make_refs(C.rV, C.V.p, C.offV, rv, dv, s));
        FDS_TRY(make_refs(C.rAt, C.At.p, C.offAt, rv, rv, s));
        if (!merge64) {
            FDS_TRY(C.W.alloc(C.offW[nb]));
            FDS_TRY(make_refs(C.rW, C.W.p, C.offW, dv, rv, s));
        }
        DBuf<cplx> S;
        DBuf<MatRef> rS;
        if (!merge64) {
            FDS_TRY(S.alloc(C.offAt[nb]));
            FDS_TRY(make_refs(rS, S.p, C.offAt, rv, rv, s));
        }
        DBuf<int> d_n1, d_n2;
        FDS_TRY(d_n1.upload(C.n1, s));
        FDS_TRY(d_n2.upload(C.n2, s));
        FDS_TRY(C.d_k1.upload(C.k1, s));
        FDS_TRY(C.d_k2.upload(C.k2, s));
        fds_count_launch(), k_make_V<<<nb, 256, 0, s>>>(C.rV.p, d_n1.p, d_n2.p, C.d_k1.p, C.d_k2.p, d_perm.p, d_poff.p, d_T.p,
                                    d_toff.p);
        FDS_CUDA_TRY(cudaGetLastError());
        // keep T and the permuted DOF order for the structured V of the solve
        {
            std::vector<int> vmap(C.D);
            C.kmax = 0;
            C.sum_tm = 0;
            for (int b = 0; b < nb; ++b)
                for (int c = 0; c < 2; ++c) {
                    const int n = c ? C.n2[b] : C.n1[b], k = c ? C.k2[b] : C.k1[b];
                    const int coff = c ? C.n1[b] : 0;
                    for (int q = 0; q < n; ++q) vmap[C.doff[b] + coff + q] = coff + C.perm[C.permoff[2 * b + c] + q];
                    C.kmax = std::max(C.kmax, k);
                    C.sum_tm += (double)k * (n - k);
                }
            FDS_TRY(C.d_vmap.upload(vmap, s));
            FDS_TRY(C.d_toff.upload(toff, s));
            C.toff_h = toff;
            FDS_TRY(C.d_n1.upload(C.n1, s));
            FDS_TRY(C.d_n2.upload(C.n2, s));
            C.T = std::move(d_T);
        }
        DBuf<int> info;
        FDS_TRY(info.alloc(nb));
        double fl_lu = 0, fl_w = 0, fl_s = 0, fl_slu = 0, fl_at = 0;
        for (int b = 0; b < nb; ++b) {
            const double d = dv[b], r = rv[b];
            fl_lu += 8.0 / 3.0 * d * d * d;
            fl_w += 8.0 * d * d * r;
            fl_s += 8.0 * r * d * r;
            fl_slu += 8.0 / 3.0 * r * r * r;
            fl_at += 8.0 * r * r * r;
        }
        DBuf<int> spiv, info2;
        DBuf<int64_t> d_sp;
        std::vector<int64_t> spoff(nb + 1, 0);
        for (int b = 0; b < nb; ++b) spoff[b + 1] = spoff[b] + rv[b];
        FDS_TRY(spiv.alloc(spoff[nb]));
        FDS_TRY(d_sp.upload(spoff, s));
        FDS_TRY(info2.alloc(nb));
        if (merge64) {
            // first inverses in complex64 (Gauss-Jordan in shared memory for
            // blocks of order <= GJ_MAX_N, else LU and solves), each refined
            // by one Newton step whose residual is formed in double-float
            // arithmetic (float pairs on the FP32 pipe):
            //   X1 = X0 + X0 (I - A X0)   against the FP64 blocks A,
            //   W = X1 V^H, S = V W       (complex64),
            //   A~ = Y0 + Y0 (I - S Y0)   Y0 a complex64 inverse of S.
            // The refined inverses, rounded to complex64 for the sweep, are as
            // accurate as FP64 ones rounded (without the steps the first
            // solve's residual is ~1000x larger and the refinement needs one
            // more sweep); A~ goes to the parent in complex128.
            const int64_t nA = C.offA[nb], nV = C.offV[nb], nS = C.offAt[nb];
            DBuf<cplxf> LUf, Sf;
            DBuf<MatRefF> rLUf, rSf;
            FDS_TRY(LUf.alloc(nA));
            FDS_TRY(C.Vf.alloc(nV));
            FDS_TRY(C.Wf.alloc(nV));
            FDS_TRY(C.Ainvf.alloc(nA));
            FDS_TRY(C.Atf.alloc(nS));
            FDS_TRY(Sf.alloc(nS));
            FDS_TRY(make_refs_t(rLUf, LUf.p, C.offA, dv, dv, s));
            FDS_TRY(make_refs_t(C.rVf, C.Vf.p, C.offV, rv, dv, s));
            FDS_TRY(make_refs_t(C.rWf, C.Wf.p, C.offW, dv, rv, s));
            FDS_TRY(make_refs_t(C.rAinvf, C.Ainvf.p, C.offA, dv, dv, s));
            FDS_TRY(make_refs_t(C.rAtf, C.Atf.p, C.offAt, rv, rv, s));
            FDS_TRY(make_refs_t(rSf, Sf.p, C.offAt, rv, rv, s));
            // double-float work buffers: A, X0, R, X1 (d x d); S, Y0, RS, Y1 (r x r)
            // (nS, nV <= nA: the r x r and d x r blocks fit the d x d complex64 buffers below)
            DBuf<float4> Ap, Xp, Rp, X1p, Sp, Yp, RSp, Y1p;
            DBuf<MatRefP> rAp, rXp, rRp, rX1p, rSp, rYp, rRSp, rY1p;
            for (auto *b : {&Ap, &Xp, &Rp, &X1p}) FDS_TRY(b->alloc(nA));
            for (auto *b : {&Sp, &Yp, &RSp, &Y1p}) FDS_TRY(b->alloc(nS));
            // complex64 residual and correction of the Newton steps (d x d, reused for r x r)
            DBuf<cplxf> Rf, Df;
            DBuf<MatRefF> rRf, rDf, rRSf, rDSf;
            FDS_TRY(Rf.alloc(nA));
            FDS_TRY(Df.alloc(nA));
            FDS_TRY(make_refs_t(rRf, Rf.p, C.offA, dv, dv, s));
            FDS_TRY(make_refs_t(rDf, Df.p, C.offA, dv, dv, s));
            FDS_TRY(make_refs_t(rAp, Ap.p, C.offA, dv, dv, s));
            FDS_TRY(make_refs_t(rXp, Xp.p, C.offA, dv, dv, s));
            FDS_TRY(make_refs_t(rRp, Rp.p, C.offA, dv, dv, s));
            FDS_TRY(make_refs_t(rX1p, X1p.p, C.offA, dv, dv, s));
            FDS_TRY(make_refs_t(rSp, Sp.p, C.offAt, rv, rv, s));
            FDS_TRY(make_refs_t(rYp, Yp.p, C.offAt, rv, rv, s));
            FDS_TRY(make_refs_t(rRSp, RSp.p, C.offAt, rv, rv, s));
            FDS_TRY(make_refs_t(rY1p, Y1p.p, C.offAt, rv, rv, s));
            fds_count_launch(), k_cast<cplx, cplxf><<<1024, 256, 0, s>>>(C.LU.p, LUf.p, nA);
            fds_count_launch(), k_cast<cplx, cplxf><<<1024, 256, 0, s>>>(C.V.p, C.Vf.p, nV);
            fds_count_launch(), k_to_ff<cplx><<<1024, 256, 0, s>>>(C.LU.p, Ap.p, nA);
            FDS_CUDA_TRY(cudaGetLastError());
            if (C.dmax <= GJ_MAX_N) {
                // the first inverse by Gauss-Jordan in shared memory (no LU is kept)
                ProfScope ps("a3.merge_a_inverse", s);
                ps.flops = fl_lu * 3.0;
                FDS_TRY(dense_inverse_gj(nb, C.dmax, rLUf.p, C.rAinvf.p, info.p, s));
            } else {
                {
                    ProfScope ps("a3.merge_lu", s);
                    ps.flops = fl_lu;
                    FDS_TRY(dense_lu(nb, C.dmax, rLUf.p, C.piv.p, C.d_offpiv.p, info.p, s));
                }
                fds_count_launch(), k_set_identity<cplxf><<<nb, 256, 0, s>>>(C.rAinvf.p);
                FDS_CUDA_TRY(cudaGetLastError());
                ProfScope ps("a3.merge_a_inverse", s);
                ps.flops = fl_lu * 3.0;
                FDS_TRY(dense_lu_solve(nb, C.dmax, C.dmax, rLUf.p, C.piv.p, C.d_offpiv.p, C.rAinvf.p, s));
            }
            {
                // X1 = X0 + X0 (I - A X0) in double-float, rounded to complex64
                ProfScope ps("a3.merge_refine", s);
                ps.flops = fl_lu * 6.0;   // two d^3 complex products per cell
                fds_count_launch(), k_to_ff<cplxf><<<1024, 256, 0, s>>>(C.Ainvf.p, Xp.p, nA);
                FDS_CUDA_TRY(cudaGetLastError());
                FDS_TRY(dense_gemm_ffp(nb, C.dmax, C.dmax, rAp.p, 0, rXp.p, rRp.p, 0, s));
                fds_count_launch(), k_ff_identity_minus<<<nb, 256, 0, s>>>(rRp.p);
                // the correction X0 R (~|R| |X0|) needs complex64 accuracy only
                fds_count_launch(), k_from_ff<cplxf><<<1024, 256, 0, s>>>(Rp.p, Rf.p, nA);
                FDS_CUDA_TRY(cudaGetLastError());
                FDS_TRY(dense_gemm_rt(nb, C.dmax, C.dmax, C.rAinvf.p, 0, rRf.p, rDf.p, mkcf(1, 0), mkcf(0, 0), s));
                fds_count_launch(), k_ff_add_c64<<<1024, 256, 0, s>>>(Xp.p, Df.p, X1p.p, C.Ainvf.p, nA);
                FDS_CUDA_TRY(cudaGetLastError());
            }
            {
                // W = A^{-1} U = X1 V^H (complex64, V^H staged in the correction buffer)
                ProfScope ps("a3.merge_w_solve", s);
                ps.flops = fl_w;
                DBuf<MatRefF> rVHf;
                FDS_TRY(make_refs_t(rVHf, Df.p, C.offW, dv, rv, s));
                fds_count_launch(), k_conj_transpose<cplxf><<<nb, 256, 0, s>>>(C.rVf.p, rVHf.p);
                FDS_CUDA_TRY(cudaGetLastError());
                FDS_TRY(dense_gemm_rt(nb, C.dmax, C.rmax, C.rAinvf.p, 0, rVHf.p, C.rWf.p, mkcf(1, 0), mkcf(0, 0), s));
                FDS_CUDA_TRY(cudaStreamSynchronize(s));   // rVHf is freed on leaving the block
            }
            {
                ProfScope ps("a3.merge_s_gemm", s);
                ps.flops = fl_s;
                FDS_TRY(dense_gemm_rt(nb, C.rmax, C.rmax, C.rVf.p, 0, C.rWf.p, rSf.p, mkcf(1, 0), mkcf(0, 0), s));
                fds_count_launch(), k_to_ff<cplxf><<<1024, 256, 0, s>>>(Sf.p, Sp.p, nS);
                FDS_CUDA_TRY(cudaGetLastError());
            }
            if (C.rmax <= GJ_MAX_N) {
                ProfScope ps("a3.merge_inverse", s);
                ps.flops = fl_at + fl_slu;
                FDS_TRY(dense_inverse_gj(nb, C.rmax, rSf.p, C.rAtf.p, info2.p, s));
            } else {
                {
                    ProfScope ps("a3.merge_s_lu", s);
                    ps.flops = fl_slu;
                    FDS_TRY(dense_lu(nb, C.rmax, rSf.p, spiv.p, d_sp.p, info2.p, s));
                }
                fds_count_launch(), k_set_identity<cplxf><<<nb, 256, 0, s>>>(C.rAtf.p);
                FDS_CUDA_TRY(cudaGetLastError());
                ProfScope ps("a3.merge_inverse", s);
                ps.flops = fl_at;
                FDS_TRY(dense_lu_solve(nb, C.rmax, C.rmax, rSf.p, spiv.p, d_sp.p, C.rAtf.p, s));
            }
            {
                // A~ = Y0 + Y0 (I - S Y0) in double-float: complex64 for the sweep, complex128 for the parent
                ProfScope ps("a3.merge_refine", s);
                ps.flops = fl_at * 2.0;
                fds_count_launch(), k_to_ff<cplxf><<<1024, 256, 0, s>>>(C.Atf.p, Yp.p, nS);
                FDS_CUDA_TRY(cudaGetLastError());
                FDS_TRY(dense_gemm_ffp(nb, C.rmax, C.rmax, rSp.p, 0, rYp.p, rRSp.p, 0, s));
                fds_count_launch(), k_ff_identity_minus<<<nb, 256, 0, s>>>(rRSp.p);
                fds_count_launch(), k_from_ff<cplxf><<<1024, 256, 0, s>>>(RSp.p, Rf.p, nS);
                FDS_CUDA_TRY(cudaGetLastError());
                FDS_TRY(make_refs_t(rRSf, Rf.p, C.offAt, rv, rv, s));
                FDS_TRY(make_refs_t(rDSf, Df.p, C.offAt, rv, rv, s));
                FDS_TRY(dense_gemm_rt(nb, C.rmax, C.rmax, C.rAtf.p, 0, rRSf.p, rDSf.p, mkcf(1, 0), mkcf(0, 0), s));
                fds_count_launch(), k_ff_add_c64<<<1024, 256, 0, s>>>(Yp.p, Df.p, Y1p.p, C.Atf.p, nS);
                fds_count_launch(), k_from_ff<cplx><<<1024, 256, 0, s>>>(Y1p.p, C.At.p, nS);
                FDS_CUDA_TRY(cudaGetLastError());
            }
            FDS_CUDA_TRY(cudaStreamSynchronize(s));   // the work buffers are freed on leaving the block
        } else {
            {
                ProfScope ps("a3.merge_lu", s);
                ps.flops = fl_lu;
                FDS_TRY(dense_lu(nb, C.dmax, C.rLU.p, C.piv.p, C.d_offpiv.p, info.p, s));
            }
            fds_count_launch(), k_conj_transpose<cplx><<<nb, 256, 0, s>>>(C.rV.p, C.rW.p);
            FDS_CUDA_TRY(cudaGetLastError());
            {
                ProfScope ps("a3.merge_w_solve", s);
                ps.flops = fl_w;
                FDS_TRY(dense_lu_solve(nb, C.dmax, C.rmax, C.rLU.p, C.piv.p, C.d_offpiv.p, C.rW.p, s));
            }
            // A_i^{-1} for the solve sweep (Sec. 7.3 step 3(b)), from the LU factors
            // by a solve against the identity; the LU itself is not kept
            FDS_TRY(C.Ainv.alloc(C.offA[nb]));
            FDS_TRY(make_refs(C.rAinv, C.Ainv.p, C.offA, dv, dv, s));
            fds_count_launch(), k_set_identity<cplx><<<nb, 256, 0, s>>>(C.rAinv.p);
            FDS_CUDA_TRY(cudaGetLastError());
            {
                ProfScope ps("a3.merge_a_inverse", s);
                ps.flops = fl_lu * 3.0;
                FDS_TRY(dense_lu_solve(nb, C.dmax, C.dmax, C.rLU.p, C.piv.p, C.d_offpiv.p, C.rAinv.p, s));
            }
            {
                ProfScope ps("a3.merge_s_gemm", s);
                ps.flops = fl_s;
                FDS_TRY(dense_gemm(nb, C.rmax, C.rmax, C.rV.p, 0, C.rW.p, 0, rS.p, mkc(1, 0), mkc(0, 0), s));
            }
            {
                ProfScope ps("a3.merge_s_lu", s);
                ps.flops = fl_slu;
                FDS_TRY(dense_lu(nb, C.rmax, rS.p, spiv.p, d_sp.p, info2.p, s));
            }
            fds_count_launch(), k_set_identity<cplx><<<nb, 256, 0, s>>>(C.rAt.p);
            FDS_CUDA_TRY(cudaGetLastError());
            {
                ProfScope ps("a3.merge_inverse", s);
                ps.flops = fl_at;
                FDS_TRY(dense_lu_solve(nb, C.rmax, C.rmax, rS.p, spiv.p, d_sp.p, C.rAt.p, s));
            }
        }
        std::vector<int> hinfo, hinfo2;
        FDS_TRY(d2h(hinfo, info.p, nb, s));
        FDS_TRY(d2h(hinfo2, info2.p, nb, s));
        FDS_TRY(sync_check(s));
        for (int b = 0; b < nb; ++b)
            if (hinfo[b] || hinfo2[b]) return FDS_ERR_SINGULAR;
        if (h->opt.variant == FDS_VARIANT_MR2005) FDS_TRY(mr2005_level_factors(h, C, dv, rv, s));
        C.LU.release();
        C.rLU.release();
        C.piv.release();
        h->factor_bytes += (int64_t)(C.Ainv.bytes() + C.V.bytes() + C.W.bytes() + C.At.bytes() + C.Ainvf.bytes() +
                                     C.Wf.bytes() + C.Atf.bytes() + C.Vf.bytes());

        // ---- parent level (eq. (A_rearrangement)): DOFs = children's skeletons
        Level &Pn = h->lv[l - 1];
        Pn.nb = nb / 2;
        Pn.n1.assign(Pn.nb, 0);
        Pn.n2.assign(Pn.nb, 0);
        Pn.dof_node.clear();
        C.par_pos1.assign(nb, 0);
        C.par_pos2.assign(nb, 0);
        for (int p = 0; p < Pn.nb; ++p) {
            const int a = 2 * p, bb = 2 * p + 1;
            Pn.n1[p] = C.k1[a] + C.k1[bb];
            Pn.n2[p] = C.k2[a] + C.k2[bb];
            C.par_pos1[a] = 0;
            C.par_pos1[bb] = C.k1[a];
            C.par_pos2[a] = Pn.n1[p];
            C.par_pos2[bb] = Pn.n1[p] + C.k2[a];
            for (int c = 0; c < 2; ++c)
                for (int ch : {a, bb}) {
                    const int k = c ? C.k2[ch] : C.k1[ch];
                    const int base = (int)C.doff[ch] + (c ? C.n1[ch] : 0);
                    const int *pm = C.perm.data() + C.permoff[2 * ch + c];
                    for (int q = 0; q < k; ++q) Pn.dof_node.push_back(C.dof_node[base + pm[q]]);
                }
        }
        finish_offsets(Pn);
        build_union(Pn);
        FDS_TRY(C.d_par_pos1.upload(C.par_pos1, s));
        FDS_TRY(C.d_par_pos2.upload(C.par_pos2, s));
        FDS_TRY(C.d_doff.upload(C.doff, s));
        FDS_TRY(C.d_roff.upload(C.roff, s));
        FDS_TRY(alloc_level_A(Pn, s));
        fds_count_launch(), k_zero<<<1024, 256, 0, s>>>(Pn.LU.p, Pn.offA[Pn.nb]);
        FDS_CUDA_TRY(cudaGetLastError());
        // sibling blocks R (group = parent, tags = child index) first, then the
        // children's A~ blocks on the diagonal (disjoint positions); between
        // the two the parent blocks hold exactly the sibling coupling S of the
        // compressed forward operator
        std::vector<int64_t> goff(Pn.nb + 1, 0);
        std::vector<int> gnode, gtag, g1, g2;
        for (int p = 0; p < Pn.nb; ++p) {
            for (int64_t u = Pn.uoff[p]; u < Pn.uoff[p + 1]; ++u) {
                const int pos1 = Pn.upos1[u], pos2 = Pn.upos2[u];
                // which child: a's DOFs occupy [0, k1_a) in comp 1 and [0, k2_a) in comp 2
                int tag = 1;
                if ((pos1 >= 0 && pos1 < C.k1[2 * p]) || (pos2 >= 0 && pos2 < C.k2[2 * p])) tag = 0;
                gnode.push_back(Pn.unode[u]);
                gtag.push_back(tag);
                g1.push_back(pos1);
                g2.push_back(pos2 >= 0 ? Pn.n1[p] + pos2 : -1);
                Pn.utag[u] = tag;
            }
            goff[p + 1] = (int64_t)gnode.size();
        }
        FDS_TRY(launch_group_blocks(h, "a1.sibling_blocks", goff, gnode, gtag, g1, g2, Pn.rLU.p, s));
        if (h->opt.precision == FDS_MIXED) FDS_TRY(fds_keep_blocks(Pn, Pn.Sfw, Pn.rSfw, s));
        fds_count_launch(), k_place_children<<<nb, 256, 0, s>>>(C.rAt.p, C.d_k1.p, C.d_par_pos1.p, C.d_par_pos2.p, Pn.rLU.p);
        FDS_CUDA_TRY(cudaGetLastError());
    }

    // ---- top level (Sec. 6.3): dense system over the cells of level l0
    {
        Level &T = h->lv[h->l0];
        h->Dtop = T.D;
        FDS_TRY(h->Atop.alloc((size_t)h->Dtop * h->Dtop));
        fds_count_launch(), k_zero<<<1024, 256, 0, s>>>(h->Atop.p, h->Dtop * h->Dtop);
        MatRef top;
        top.p = h->Atop.p;
        top.rows = top.cols = (int)h->Dtop;
        top.ld = (int)std::max<int64_t>(h->Dtop, 1);
        FDS_TRY(T.d_doff.upload(T.doff, s));
        std::vector<int64_t> goff = {0};
        std::vector<int> gnode, gtag, g1, g2;
        for (int b = 0; b < T.nb; ++b)
            for (int64_t u = T.uoff[b]; u < T.uoff[b + 1]; ++u) {
                gnode.push_back(T.unode[u]);
                gtag.push_back(b);
                g1.push_back(T.upos1[u] >= 0 ? (int)T.doff[b] + T.upos1[u] : -1);
                g2.push_back(T.upos2[u] >= 0 ? (int)T.doff[b] + T.n1[b] + T.upos2[u] : -1);
            }
        goff.push_back((int64_t)gnode.size());
        std::vector<MatRef> ht = {top};
        FDS_TRY(h->rtop.upload(ht, s));
        // off-diagonal blocks between top cells, then the cells' own blocks
        if (T.nb > 1) FDS_TRY(launch_group_blocks(h, "a1.top_blocks", goff, gnode, gtag, g1, g2, h->rtop.p, s));
        if (h->opt.precision == FDS_MIXED) {
            FDS_TRY(h->Atop_off.alloc((size_t)h->Dtop * h->Dtop));
            FDS_CUDA_TRY(cudaMemcpyAsync(h->Atop_off.p, h->Atop.p, h->Atop.bytes(), cudaMemcpyDeviceToDevice, s));
            MatRef off = top;
            off.p = h->Atop_off.p;
            std::vector<MatRef> ho = {off};
            FDS_TRY(h->rtop_off.upload(ho, s));
        }
        fds_count_launch(), k_place_top<<<T.nb, 256, 0, s>>>(T.rLU.p, T.d_doff.p, top);
        FDS_CUDA_TRY(cudaGetLastError());
        std::vector<int64_t> po = {0, h->Dtop};
        FDS_TRY(h->d_ptop_off.upload(po, s));
        FDS_TRY(h->ptop.alloc(h->Dtop));
        FDS_TRY(h->d_info.alloc(1));
        {
            ProfScope ps("a4.top_lu", s);
            ps.flops = 8.0 / 3.0 * (double)h->Dtop * h->Dtop * h->Dtop;
            if (h->Dtop > 128)
                FDS_TRY(dense_lu_blocked((int)h->Dtop, h->Atop.p, top.ld, h->ptop.p, h->d_info.p, s));
            else
                FDS_TRY(dense_lu(1, (int)h->Dtop, h->rtop.p, h->ptop.p, h->d_ptop_off.p, h->d_info.p, s));
        }
        std::vector<int> hinfo;
        FDS_TRY(d2h(hinfo, h->d_info.p, 1, s));
        FDS_TRY(sync_check(s));
        if (hinfo[0]) return FDS_ERR_SINGULAR;
        // A_top^{-1} from the LU, so that each top solve of the sweep is one GEMM
        {
            ProfScope ps("a4.top_inverse", s);
            ps.flops = 8.0 * (double)h->Dtop * h->Dtop * h->Dtop;
            FDS_TRY(h->Atop_inv.alloc((size_t)h->Dtop * h->Dtop));
            MatRef inv = top;
            inv.p = h->Atop_inv.p;
            std::vector<MatRef> hi = {inv};
            FDS_TRY(h->rtop_inv.upload(hi, s));
            fds_count_launch(), k_set_identity<cplx><<<1, 256, 0, s>>>(h->rtop_inv.p);
            FDS_CUDA_TRY(cudaGetLastError());
            FDS_TRY(dense_lu_solve(1, (int)h->Dtop, (int)h->Dtop, h->rtop.p, h->ptop.p, h->d_ptop_off.p,
                                   h->rtop_inv.p, s));
        }
        h->factor_bytes += (int64_t)(h->Atop.bytes() + h->ptop.bytes() + h->Atop_inv.bytes());
        // the top level's per-cell A blocks are no longer needed
        if (h->l0 < L || T.nb > 0) {
            T.LU.release();
            T.rLU.release();
        }
        FDS_TRY(T.d_doff.upload(T.doff, s));
    }
    if (h->opt.precision == FDS_MIXED) {
        // complex64 / float-pair copies of the factors, the forward operator's blocks and their tensor-core slices
        ProfScope ps("a4.mixed_prepare", h->stream);
        FDS_TRY(fds_mixed_prepare(h));
    }
    // the solve applies V through T (vapply.cu): the dense V_i are not kept
    FDS_TRY(sync_check(s));
    for (int l = L; l > h->l0; --l) {
        Level &C = h->lv[l];
        h->factor_bytes -= (int64_t)(C.V.bytes() + C.Vf.bytes());
        h->factor_bytes += (int64_t)(C.T.bytes() + C.Tf.bytes() + C.Tp.bytes());
        C.V.release();
        C.rV.release();
        C.Vf.release();
        C.rVf.release();
        C.Vp.release();
        C.rVp.release();
    }
    cudaEventRecord(e1, s);
    FDS_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    h->build_ms = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (h->opt.precision == FDS_MIXED && h->opt.merge_c64 && h->opt.c64_engine == FDS_C64_TENSOR) {
        int st = 0;
        FDS_TRY(tc_status_take(s, &st));
        if (st) {
            fds_set_error_detail("tensor-core GEMM: wait on the MMA barrier timed out");
            return FDS_ERR_TIMEOUT;
        }
    }
    return FDS_OK;
}
