// Register-tiled batched complex GEMM, C = alpha op(A) B + beta C, for the
// solve sweep and the forward operator.  One CTA computes a 16 MI x 16 TJ
// tile of one matrix of the batch (MI = 2, 3 or 4 row groups, picked per
// launch from the largest row count); 256 threads, each an MI x TJ
// micro-tile with rows tx + 16 i and columns ty + 16 j (conflict-free
// shared-memory reads), K in steps of 16 staged in shared memory.
//
// Three arithmetics share the tiling:
//   Arith64   complex64 loads, FP32 FMA
//   Arith128  complex128 loads, FP64 FMA
//   ArithFFP3 operands stored as float pairs (hi + lo), products and sums in
//             double-float arithmetic on the FP32 pipe: a x = ah xh +
//             (err(ah xh) + ah xl + al xh) with err() from one FMA (Dekker's
//             product), accumulation by Knuth's TwoSum, and Gauss's
//             three-product complex multiply; about 44 bits of significand
//             at 36 FP32 instructions per complex multiply-add, against FP64
//             at 1/64 of the FP32 rate on this GPU.
#include "dense.cuh"
#include "fds_internal.cuh"

namespace {

constexpr int BK = 16, NT = 256;
// columns per thread of the float-pair kernel at 4 row groups (register budget)
#ifndef FDS_FFP_TJ4
#define FDS_FFP_TJ4 2
#endif
#ifndef FDS_C64_TJ4
#define FDS_C64_TJ4 4
#endif

// ---------------------------------------------------------------- arithmetics
struct Arith64 {
    typedef cplxf G;      // global element
    typedef cplxf SA;     // staged element of op(A)
    typedef cplxf SB;     // staged element of B
    typedef cplxf Acc;
    __device__ static SA stage_a(G v, bool cj) { return cj ? cconj(v) : v; }
    __device__ static SB stage_b(G v) { return v; }
    __device__ static SA za() { return mkcf(0.f, 0.f); }
    __device__ static SB zb() { return mkcf(0.f, 0.f); }
    __device__ static void zero(Acc &a) { a = mkcf(0.f, 0.f); }
    __device__ static void mac(Acc &c, const SA &a, const SB &b) { cfma(c, a, b); }
    __device__ static G finish(const Acc &c, G alpha, G beta, const G *old) {
        G r = cmul(alpha, c);
        if (old) r = cadd(r, cmul(beta, *old));
        return r;
    }
};

struct Arith128 {
    typedef cplx G;
    typedef cplx SA;
    typedef cplx SB;
    typedef cplx Acc;
    __device__ static SA stage_a(G v, bool cj) { return cj ? cconj(v) : v; }
    __device__ static SB stage_b(G v) { return v; }
    __device__ static SA za() { return mkc(0.0, 0.0); }
    __device__ static SB zb() { return mkc(0.0, 0.0); }
    __device__ static void zero(Acc &a) { a = mkc(0.0, 0.0); }
    __device__ static void mac(Acc &c, const SA &a, const SB &b) { cfma(c, a, b); }
    __device__ static G finish(const Acc &c, G alpha, G beta, const G *old) {
        G r = cmul(alpha, c);
        if (old) r = cadd(r, cmul(beta, *old));
        return r;
    }
};

// float pair h + l of a double (|l| <= ulp(h)/2)
struct ff {
    float h, l;
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// acc += x y (the xl yl term is below the pair's precision)
__device__ __forceinline__ void ff_mac(ff &acc, const ff &x, const ff &y) {
    const float ph = x.h * y.h;
    const float pl = fmaf(x.h, y.l, fmaf(x.l, y.h, fmaf(x.h, y.h, -ph)));
    float s, e;
    two_sum(acc.h, ph, s, e);
    acc.h = s;
    acc.l += e + pl;
}


// Operands already held as float pairs (float4 = re_hi, im_hi, re_lo, im_lo):
// the constant operators are split once, the vectors stay split, so no FP64
// instruction is issued (ArithFFP3 below).  alpha = 1 or -1 (sign of
// alpha.x); beta = 0 or 1.
__device__ __forceinline__ ff ff_norm(ff a) {
    const float h = a.h + a.l;
    return ff{h, a.l - (h - a.h)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    float s, e;
    two_sum(a.h, b.h, s, e);
    return ff_norm(ff{s, e + (a.l + b.l)});
}

// Float-pair operands with Gauss's three-product complex multiply:
//   (a + i b)(c + i d) = (k1 - k3) + i (k1 + k2),
//   k1 = c (a + b),  k2 = a (d - c),  k3 = b (c + d),
// the sums a + b (per staged element of op(A)) and d - c, c + d (per staged
// element of B) formed once when the tile is staged and reused by every
// product of the tile: 36 FP32 instructions per complex multiply-add.
struct ArithFFP3 {
    typedef float4 G;
    struct SA {
        ff a, b, s;     // re, im, re + im
    };
    struct SB {
        ff c, dm, dp;   // re, im - re, re + im
    };
    struct Acc {
        ff k1, k2, k3;
    };
    __device__ static SA stage_a(G v, bool cj) {
        const ff a{v.x, v.z}, b = cj ? ff{-v.y, -v.w} : ff{v.y, v.w};
        return SA{a, b, ff_add(a, b)};
    }
    __device__ static SB stage_b(G v) {
        const ff c{v.x, v.z}, d{v.y, v.w};
        return SB{c, ff_add(d, ff{-c.h, -c.l}), ff_add(c, d)};
    }
    __device__ static SA za() { return SA{{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}}; }
    __device__ static SB zb() { return SB{{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}}; }
    __device__ static void zero(Acc &x) { x = Acc{{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}}; }
    __device__ static void mac(Acc &x, const SA &a, const SB &b) {
        ff_mac(x.k1, b.c, a.s);
        ff_mac(x.k2, a.a, b.dm);
        ff_mac(x.k3, a.b, b.dp);
    }
    __device__ static G finish(const Acc &x, G alpha, G, const G *old) {
        const ff k1 = ff_norm(x.k1), k2 = ff_norm(x.k2), k3 = ff_norm(x.k3);
        ff re = ff_add(k1, ff{-k3.h, -k3.l}), im = ff_add(k1, k2);
        if (alpha.x < 0.f) {   // alpha = -1
            re = ff{-re.h, -re.l};
            im = ff{-im.h, -im.l};
        }
        if (old) {
            re = ff_add(re, ff{old->x, old->z});
            im = ff_add(im, ff{old->y, old->w});
        }
        return make_float4(re.h, im.h, re.l, im.l);
    }
};

// TJ columns per thread (CTA tile 64 x 16 TJ)
// Optional row maps (maps nullable, and each pointer nullable): B's row k is
// read from row bmap[k], C's row i is written to row cmap[i].
template <class Ar, int TJ, int MI>
__global__ void __launch_bounds__(NT) k_gemm_rt(const MatRefT<typename Ar::G> *__restrict__ As, int opA,
                                                const MatRefT<typename Ar::G> *__restrict__ Bs,
                                                const MatRefT<typename Ar::G> *__restrict__ Cs,
                                                typename Ar::G alpha, typename Ar::G beta, int use_beta,
                                                int tiles_m, const RowMaps *__restrict__ maps) {
    typedef typename Ar::G G;
    typedef typename Ar::SA SA;
    typedef typename Ar::SB SB;
    const MatRefT<G> A = As[blockIdx.y], B = Bs[blockIdx.y], Cm = Cs[blockIdx.y];
    const int *bmap = maps ? maps[blockIdx.y].b : nullptr;
    const int *cmap = maps ? maps[blockIdx.y].c : nullptr;
    const int M = Cm.rows, N = Cm.cols;
    const int K = (opA == 0) ? A.cols : A.rows;
    constexpr int BN = 16 * TJ, BMt = 16 * MI;
    const int i0 = (blockIdx.x % tiles_m) * BMt, j0 = (blockIdx.x / tiles_m) * BN;
    if (i0 >= M || j0 >= N) return;
    __shared__ SA sa[BK][BMt];
    __shared__ SB sb[BK][16 * TJ];
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    typename Ar::Acc acc[MI][TJ];
#pragma unroll
    for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int j = 0; j < TJ; ++j) Ar::zero(acc[i][j]);
    for (int k0 = 0; k0 < K; k0 += BK) {
        // stage op(A)[i0:i0+BMt, k0:k0+16] as sa[k][i]
        if (opA == 0) {
#pragma unroll
            for (int q = 0; q < MI; ++q) {
                const int e = t + NT * q, i = e % BMt, k = e / BMt;
                const int gi = i0 + i, gk = k0 + k;
                sa[k][i] = (gi < M && gk < K) ? Ar::stage_a(A.p[gi + (int64_t)gk * A.ld], false) : Ar::za();
            }
        } else {
#pragma unroll
            for (int q = 0; q < MI; ++q) {
                const int k = t & 15, i = (t >> 4) + 16 * q;
                const int gi = i0 + i, gk = k0 + k;
                sa[k][i] = (gi < M && gk < K) ? Ar::stage_a(A.p[gk + (int64_t)gi * A.ld], true) : Ar::za();
            }
        }
        // stage B[k0:k0+16, j0:j0+BN] as sb[k][j]
#pragma unroll
        for (int q = 0; q < TJ; ++q) {
            const int k = t & 15, j = (t >> 4) + 16 * q;
            const int gk = k0 + k, gj = j0 + j;
            sb[k][j] = (gk < K && gj < N) ? Ar::stage_b(B.p[(bmap ? bmap[gk] : gk) + (int64_t)gj * B.ld]) : Ar::zb();
        }
        __syncthreads();
        const int kmax = min(BK, K - k0);
        for (int k = 0; k < kmax; ++k) {
            SA a[MI];
            SB b[TJ];
#pragma unroll
            for (int i = 0; i < MI; ++i) a[i] = sa[k][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < TJ; ++j) b[j] = sb[k][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < MI; ++i)
#pragma unroll
                for (int j = 0; j < TJ; ++j) Ar::mac(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int j = 0; j < TJ; ++j) {
            const int gi = i0 + tx + 16 * i, gj = j0 + ty + 16 * j;
            if (gi < M && gj < N) {
                G *c = &Cm.p[(cmap ? cmap[gi] : gi) + (int64_t)gj * Cm.ld];
                *c = Ar::finish(acc[i][j], alpha, beta, use_beta ? c : nullptr);
            }
        }
}

template <class Ar, int TJ, int MI>
int launch_t(int batch, int max_m, int max_n, const MatRefT<typename Ar::G> *d_A, int opA,
             const MatRefT<typename Ar::G> *d_B, const MatRefT<typename Ar::G> *d_C, typename Ar::G alpha,
             typename Ar::G beta, cudaStream_t s, const RowMaps *maps) {
    constexpr int BN = 16 * TJ, BMt = 16 * MI;
    const int tm = (max_m + BMt - 1) / BMt, tn = (max_n + BN - 1) / BN;
    const int use_beta = (beta.x != 0 || beta.y != 0) ? 1 : 0;
    dim3 grid(tm * tn, batch);
    fds_count_launch(),
        k_gemm_rt<Ar, TJ, MI><<<grid, NT, 0, s>>>(d_A, opA, d_B, d_C, alpha, beta, use_beta, tm, maps);
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}

// Tile height 32, 48 or 64 rows, whichever pads the largest row count of the
// batch least (ties to the taller tile); the column width keeps about the
// same number of products per thread (TJ2, TJ3, TJ4 for 2, 3, 4 row groups).
template <class Ar, int TJ4, int TJ3, int TJ2>
int launch(int batch, int max_m, int max_n, const MatRefT<typename Ar::G> *d_A, int opA,
           const MatRefT<typename Ar::G> *d_B, const MatRefT<typename Ar::G> *d_C, typename Ar::G alpha,
           typename Ar::G beta, cudaStream_t s, const RowMaps *maps = nullptr) {
    if (batch <= 0 || max_m <= 0 || max_n <= 0) return FDS_OK;
    if (opA != 0 && opA != 2) return FDS_ERR_ARG;
    int best = 4, pad = 1 << 30;
    for (int mi = 4; mi >= 2; --mi) {
        const int p = (max_m + 16 * mi - 1) / (16 * mi) * 16 * mi;
        if (p < pad) {
            pad = p;
            best = mi;
        }
    }
    if (best == 2) return launch_t<Ar, TJ2, 2>(batch, max_m, max_n, d_A, opA, d_B, d_C, alpha, beta, s, maps);
    if (best == 3) return launch_t<Ar, TJ3, 3>(batch, max_m, max_n, d_A, opA, d_B, d_C, alpha, beta, s, maps);
    return launch_t<Ar, TJ4, 4>(batch, max_m, max_n, d_A, opA, d_B, d_C, alpha, beta, s, maps);
}

}  // namespace

int dense_gemm_rt(int batch, int max_m, int max_n, const MatRef *d_A, int opA, const MatRef *d_B, const MatRef *d_C,
                  cplx alpha, cplx beta, cudaStream_t s) {
    return launch<Arith128, 4, 4, 8>(batch, max_m, max_n, d_A, opA, d_B, d_C, alpha, beta, s);
}

int dense_gemm_rt(int batch, int max_m, int max_n, const MatRefF *d_A, int opA, const MatRefF *d_B,
                  const MatRefF *d_C, cplxf alpha, cplxf beta, cudaStream_t s) {
    return launch<Arith64, FDS_C64_TJ4, 4, 8>(batch, max_m, max_n, d_A, opA, d_B, d_C, alpha, beta, s);
}

int dense_gemm_ffp(int batch, int max_m, int max_n, const MatRefT<float4> *d_A, int opA, const MatRefT<float4> *d_B,
                   const MatRefT<float4> *d_C, int accumulate, cudaStream_t s) {
    return launch<ArithFFP3, FDS_FFP_TJ4, 3, 4>(batch, max_m, max_n, d_A, opA, d_B, d_C, make_float4(1.f, 0.f, 0.f, 0.f),
                                make_float4(accumulate ? 1.f : 0.f, 0.f, 0.f, 0.f), s);
}

int dense_gemm_map(int batch, int max_m, int max_n, const MatRef *d_A, int opA, const MatRef *d_B, const MatRef *d_C,
                   const RowMaps *d_maps, int accumulate, cudaStream_t s) {
    return launch<Arith128, 4, 4, 8>(batch, max_m, max_n, d_A, opA, d_B, d_C, mkc(1, 0), mkc(accumulate ? 1 : 0, 0), s,
                               d_maps);
}
int dense_gemm_map(int batch, int max_m, int max_n, const MatRefF *d_A, int opA, const MatRefF *d_B,
                   const MatRefF *d_C, const RowMaps *d_maps, int accumulate, cudaStream_t s) {
    if (g_c64_tensor)
        return dense_gemm_tc(batch, max_m, max_n, d_A, opA, d_B, d_C, 1.f, accumulate ? 1.f : 0.f, d_maps, s);
    return launch<Arith64, FDS_C64_TJ4, 4, 8>(batch, max_m, max_n, d_A, opA, d_B, d_C, mkcf(1, 0), mkcf(accumulate ? 1 : 0, 0), s,
                              d_maps);
}
int dense_gemm_map(int batch, int max_m, int max_n, const MatRefP *d_A, int opA, const MatRefP *d_B,
                   const MatRefP *d_C, const RowMaps *d_maps, int accumulate, cudaStream_t s) {
    return launch<ArithFFP3, FDS_FFP_TJ4, 3, 4>(batch, max_m, max_n, d_A, opA, d_B, d_C, make_float4(1.f, 0.f, 0.f, 0.f),
                                make_float4(accumulate ? 1.f : 0.f, 0.f, 0.f, 0.f), s, d_maps);
}

int dense_gemm(int batch, int max_m, int max_n, const MatRefP *d_A, int opA, const MatRefP *d_B, int opB,
               const MatRefP *d_C, float4 alpha, float4 beta, cudaStream_t s) {
    if (opB != 0) return FDS_ERR_ARG;
    return launch<ArithFFP3, FDS_FFP_TJ4, 3, 4>(batch, max_m, max_n, d_A, opA, d_B, d_C, alpha, beta, s);
}
