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
#include <atomic>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>

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
    static constexpr int ID = 0;
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
    static constexpr int ID = 1;
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
    static constexpr int ID = 2;
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
    // rows padded by one element: the staging stores walk K across threads
    __shared__ SA sa[BK][BMt + 1];
    __shared__ SB sb[BK][16 * TJ + 1];
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
            const int rk = (gk < K && gj < N) ? (bmap ? bmap[gk] : gk) : -1;
            sb[k][j] = (rk >= 0 && FDS_IN_RANGE(rk, B.rows)) ? Ar::stage_b(B.p[rk + (int64_t)gj * B.ld]) : Ar::zb();
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
                const int ri = cmap ? cmap[gi] : gi;
                if (!FDS_IN_RANGE(ri, cmap ? maps[blockIdx.y].cext : M)) continue;
                G *c = &Cm.p[ri + (int64_t)gj * Cm.ld];
                *c = Ar::finish(acc[i][j], alpha, beta, use_beta ? c : nullptr);
            }
        }
}

// complex64 with op(A) = A: the same tiles, summation order and results as
// k_gemm_rt, with the K slabs copied global -> shared by cp.async into two
// buffers (the next slab lands while the current one is multiplied; no
// staging registers, so the occupancy stays that of k_gemm_rt)
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem, int bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem), "r"(bytes)
                 : "memory");
}

template <int TJ, int MI>
__global__ void __launch_bounds__(NT) k_gemm_c64_async(const MatRefT<cplxf> *__restrict__ As,
                                                      const MatRefT<cplxf> *__restrict__ Bs,
                                                      const MatRefT<cplxf> *__restrict__ Cs, cplxf alpha,
                                                      cplxf beta, int use_beta, int tiles_m,
                                                      const RowMaps *__restrict__ maps) {
    const MatRefT<cplxf> A = As[blockIdx.y], B = Bs[blockIdx.y], Cm = Cs[blockIdx.y];
    const int *bmap = maps ? maps[blockIdx.y].b : nullptr;
    const int *cmap = maps ? maps[blockIdx.y].c : nullptr;
    const int M = Cm.rows, N = Cm.cols, K = A.cols;
    constexpr int BN = 16 * TJ, BMt = 16 * MI;
    const int i0 = (blockIdx.x % tiles_m) * BMt, j0 = (blockIdx.x / tiles_m) * BN;
    if (i0 >= M || j0 >= N) return;
    // rows padded by one element: the B copies walk K across threads
    __shared__ __align__(16) cplxf sa[2][BK][BMt + 1];
    __shared__ __align__(16) cplxf sb[2][BK][16 * TJ + 1];
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    auto issue = [&](int k0, int buf) {
#pragma unroll
        for (int q = 0; q < MI; ++q) {
            const int e = t + NT * q, i = e % BMt, k = e / BMt;
            const int gi = i0 + i, gk = k0 + k;
            const bool in = gi < M && gk < K;
            cp_async8(&sa[buf][k][i], in ? (const void *)(A.p + gi + (int64_t)gk * A.ld) : (const void *)A.p,
                      in ? 8 : 0);
        }
#pragma unroll
        for (int q = 0; q < TJ; ++q) {
            const int k = t & 15, j = (t >> 4) + 16 * q;
            const int gk = k0 + k, gj = j0 + j;
            const int rk = (gk < K && gj < N) ? (bmap ? bmap[gk] : gk) : -1;
            const bool in = rk >= 0 && FDS_IN_RANGE(rk, B.rows);
            cp_async8(&sb[buf][k][j], in ? (const void *)(B.p + rk + (int64_t)gj * B.ld) : (const void *)B.p,
                      in ? 8 : 0);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    cplxf acc[MI][TJ];
#pragma unroll
    for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int j = 0; j < TJ; ++j) acc[i][j] = mkcf(0.f, 0.f);
    if (K > 0) issue(0, 0);
    for (int k0 = 0, buf = 0; k0 < K; k0 += BK, buf ^= 1) {
        if (k0 + BK < K) {
            issue(k0 + BK, buf ^ 1);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        const int kmax = min(BK, K - k0);
        for (int k = 0; k < kmax; ++k) {
            cplxf a[MI], b[TJ];
#pragma unroll
            for (int i = 0; i < MI; ++i) a[i] = sa[buf][k][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < TJ; ++j) b[j] = sb[buf][k][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < MI; ++i)
#pragma unroll
                for (int j = 0; j < TJ; ++j) cfma(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int j = 0; j < TJ; ++j) {
            const int gi = i0 + tx + 16 * i, gj = j0 + ty + 16 * j;
            if (gi < M && gj < N) {
                const int ri = cmap ? cmap[gi] : gi;
                if (!FDS_IN_RANGE(ri, cmap ? maps[blockIdx.y].cext : M)) continue;
                cplxf *c = &Cm.p[ri + (int64_t)gj * Cm.ld];
                cplxf r = cmul(alpha, acc[i][j]);
                if (use_beta) r = cadd(r, cmul(beta, *c));
                *c = r;
            }
        }
}

template <class Ar, int TJ, int MI>
void launch_kernel(dim3 grid, cudaStream_t s, const MatRefT<typename Ar::G> *d_A, int opA,
                   const MatRefT<typename Ar::G> *d_B, const MatRefT<typename Ar::G> *d_C, typename Ar::G alpha,
                   typename Ar::G beta, int use_beta, int tm, const RowMaps *maps) {
    k_gemm_rt<Ar, TJ, MI><<<grid, NT, 0, s>>>(d_A, opA, d_B, d_C, alpha, beta, use_beta, tm, maps);
}
// complex64 products with op(A) = A take the cp.async kernel
template <>
void launch_kernel<Arith64, 4, 4>(dim3 grid, cudaStream_t s, const MatRefT<cplxf> *d_A, int opA,
                                  const MatRefT<cplxf> *d_B, const MatRefT<cplxf> *d_C, cplxf alpha, cplxf beta,
                                  int use_beta, int tm, const RowMaps *maps) {
    if (opA == 0) k_gemm_c64_async<4, 4><<<grid, NT, 0, s>>>(d_A, d_B, d_C, alpha, beta, use_beta, tm, maps);
    else k_gemm_rt<Arith64, 4, 4><<<grid, NT, 0, s>>>(d_A, opA, d_B, d_C, alpha, beta, use_beta, tm, maps);
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
        launch_kernel<Ar, TJ, MI>(grid, s, d_A, opA, d_B, d_C, alpha, beta, use_beta, tm, maps);
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}

// ---------------------------------------------------------------- autotuner
// Tile shapes (row groups MI x columns per thread TJ) chosen by timing: the
// first launch of a shape class (arithmetic, op(A), row count in steps of 16,
// column and batch counts by powers of two, row maps or not) whose result
// does not depend on C's old contents (beta = 0) runs every candidate shape
// on its stream (CUDA events, best of two), keeps the fastest in a
// process-wide table and leaves C as any candidate computes it (the K loop
// order is the same for every shape, so the results are identical).  Other
// launches use the table, or the rule below while their class is untuned.
struct TuneKey {
    int arith, opA, mb, nb, bb, mapped;
    bool operator<(const TuneKey &o) const {
        const int a[6] = {arith, opA, mb, nb, bb, mapped}, b[6] = {o.arith, o.opA, o.mb, o.nb, o.bb, o.mapped};
        for (int i = 0; i < 6; ++i)
            if (a[i] != b[i]) return a[i] < b[i];
        return false;
    }
};
struct TuneVal {
    int mi, tj;
    float best_us, rule_us;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;
std::atomic<int> g_tune_on{0};

int ceil_log2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

template <class Ar>
using LaunchFn = int (*)(int, int, int, const MatRefT<typename Ar::G> *, int, const MatRefT<typename Ar::G> *,
                         const MatRefT<typename Ar::G> *, typename Ar::G, typename Ar::G, cudaStream_t,
                         const RowMaps *);

// candidate shapes per arithmetic (register budgets: the float-pair
// accumulators are three pairs per output)
template <class Ar>
struct Cands;
template <>
struct Cands<Arith64> {
    static constexpr int n = 6;
    static constexpr int mi[n] = {4, 4, 3, 3, 2, 2}, tj[n] = {4, 2, 4, 2, 8, 4};
    static LaunchFn<Arith64> fn(int c);
};
template <>
struct Cands<Arith128> {
    static constexpr int n = 5;
    static constexpr int mi[n] = {4, 4, 3, 2, 2}, tj[n] = {4, 2, 4, 8, 4};
    static LaunchFn<Arith128> fn(int c);
};
template <>
struct Cands<ArithFFP3> {
    static constexpr int n = 5;
    static constexpr int mi[n] = {4, 3, 3, 2, 2}, tj[n] = {2, 4, 2, 4, 2};
    static LaunchFn<ArithFFP3> fn(int c);
};

// Tile height 32, 48 or 64 rows, whichever pads the largest row count of the
// batch least (ties to the taller tile); the column width keeps about the
// same number of products per thread (TJ2, TJ3, TJ4 for 2, 3, 4 row groups).
template <class Ar, int TJ4, int TJ3, int TJ2>
int launch(int batch, int max_m, int max_n, const MatRefT<typename Ar::G> *d_A, int opA,
           const MatRefT<typename Ar::G> *d_B, const MatRefT<typename Ar::G> *d_C, typename Ar::G alpha,
           typename Ar::G beta, cudaStream_t s, const RowMaps *maps = nullptr);

template <class Ar, int TJ4, int TJ3, int TJ2>
int launch_rule(int batch, int max_m, int max_n, const MatRefT<typename Ar::G> *d_A, int opA,
                const MatRefT<typename Ar::G> *d_B, const MatRefT<typename Ar::G> *d_C, typename Ar::G alpha,
                typename Ar::G beta, cudaStream_t s, const RowMaps *maps) {
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

// time one launch on stream s (ms); negative on failure
template <class F>
float time_launch(cudaStream_t s, F &&f) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -1.f;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return -1.f;
    }
    float ms = -1.f;
    cudaEventRecord(e0, s);
    const int rc = f();
    cudaEventRecord(e1, s);
    if (rc == FDS_OK && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc == FDS_OK ? ms : -1.f;
}

template <class Ar, int TJ4, int TJ3, int TJ2>
int launch(int batch, int max_m, int max_n, const MatRefT<typename Ar::G> *d_A, int opA,
           const MatRefT<typename Ar::G> *d_B, const MatRefT<typename Ar::G> *d_C, typename Ar::G alpha,
           typename Ar::G beta, cudaStream_t s, const RowMaps *maps) {
    if (batch <= 0 || max_m <= 0 || max_n <= 0) return FDS_OK;
    if (opA != 0 && opA != 2) return FDS_ERR_ARG;
    if (!g_tune_on.load(std::memory_order_relaxed))
        return launch_rule<Ar, TJ4, TJ3, TJ2>(batch, max_m, max_n, d_A, opA, d_B, d_C, alpha, beta, s, maps);
    const TuneKey key{Ar::ID, opA, (max_m + 15) / 16, ceil_log2(max_n), ceil_log2(batch), maps ? 1 : 0};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            for (int c = 0; c < Cands<Ar>::n; ++c)
                if (Cands<Ar>::mi[c] == it->second.mi && Cands<Ar>::tj[c] == it->second.tj)
                    return Cands<Ar>::fn(c)(batch, max_m, max_n, d_A, opA, d_B, d_C, alpha, beta, s, maps);
        }
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const bool use_beta = !(beta.x == 0 && beta.y == 0);
    if (use_beta || cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
        return launch_rule<Ar, TJ4, TJ3, TJ2>(batch, max_m, max_n, d_A, opA, d_B, d_C, alpha, beta, s, maps);
    TuneVal v{0, 0, 1e30f, -1.f};
    for (int rep = 0; rep < 2; ++rep) {
        const float r = time_launch(s, [&] {
            return launch_rule<Ar, TJ4, TJ3, TJ2>(batch, max_m, max_n, d_A, opA, d_B, d_C, alpha, beta, s, maps);
        });
        if (r < 0) return FDS_ERR_CUDA;
        v.rule_us = v.rule_us < 0 ? 1e3f * r : fminf(v.rule_us, 1e3f * r);
        for (int c = 0; c < Cands<Ar>::n; ++c) {
            const float t = time_launch(s, [&] {
                return Cands<Ar>::fn(c)(batch, max_m, max_n, d_A, opA, d_B, d_C, alpha, beta, s, maps);
            });
            if (t < 0) return FDS_ERR_CUDA;
            if (1e3f * t < v.best_us) v = TuneVal{Cands<Ar>::mi[c], Cands<Ar>::tj[c], 1e3f * t, v.rule_us};
        }
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = v;
    return FDS_OK;
}

#define FDS_CAND(Ar, MI, TJ) &launch_t<Ar, TJ, MI>
LaunchFn<Arith64> Cands<Arith64>::fn(int c) {
    static const LaunchFn<Arith64> f[n] = {FDS_CAND(Arith64, 4, 4), FDS_CAND(Arith64, 4, 2), FDS_CAND(Arith64, 3, 4),
                                           FDS_CAND(Arith64, 3, 2), FDS_CAND(Arith64, 2, 8), FDS_CAND(Arith64, 2, 4)};
    return f[c];
}
LaunchFn<Arith128> Cands<Arith128>::fn(int c) {
    static const LaunchFn<Arith128> f[n] = {FDS_CAND(Arith128, 4, 4), FDS_CAND(Arith128, 4, 2),
                                            FDS_CAND(Arith128, 3, 4), FDS_CAND(Arith128, 2, 8),
                                            FDS_CAND(Arith128, 2, 4)};
    return f[c];
}
LaunchFn<ArithFFP3> Cands<ArithFFP3>::fn(int c) {
    static const LaunchFn<ArithFFP3> f[n] = {FDS_CAND(ArithFFP3, 4, 2), FDS_CAND(ArithFFP3, 3, 4),
                                             FDS_CAND(ArithFFP3, 3, 2), FDS_CAND(ArithFFP3, 2, 4),
                                             FDS_CAND(ArithFFP3, 2, 2)};
    return f[c];
}
#undef FDS_CAND

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

extern "C" void fds_autotune_enable(int32_t on) { g_tune_on.store(on ? 1 : 0); }

extern "C" void fds_autotune_reset(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
}

extern "C" int fds_autotune_report(char *buf, int32_t cap) {
    static const char *names[3] = {"c64", "c128", "ff"};
    std::lock_guard<std::mutex> lk(g_tune_mu);
    std::string out;
    char line[160];
    for (auto &kv : g_tune) {
        const TuneKey &k = kv.first;
        snprintf(line, sizeof(line), "%s %d %d %d %d %d %d %d %.3f %.3f\n", names[k.arith], k.opA, 16 * k.mb,
                 1 << k.nb, 1 << k.bb, k.mapped, kv.second.mi, kv.second.tj, kv.second.best_us, kv.second.rule_us);
        out += line;
    }
    if (buf && cap > 0) {
        const size_t n = out.size() < (size_t)(cap - 1) ? out.size() : (size_t)(cap - 1);
        memcpy(buf, out.data(), n);
        buf[n] = 0;
    }
    return (int)out.size() + 1;
}
