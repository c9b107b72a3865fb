// Register-tiled batched complex GEMM, C = alpha op(A) B + beta C, for the
// solve sweep and the forward operator.  One CTA computes a 64 x 16 TJ tile
// of one matrix of the batch; 256 threads, each a 4 x TJ micro-tile with rows
// tx + 16 i and columns ty + 16 j (conflict-free shared-memory reads), K in
// steps of 16 staged in shared memory.  TJ = 4 for complex64/128, 2 for the
// double-float variant (register budget).
//
// Three arithmetics share the tiling:
//   Arith64  complex64 loads, FP32 FMA
//   Arith128 complex128 loads, FP64 FMA
//   ArithFF  complex128 loads split into float pairs (hi + lo) when staged,
//            products and sums in double-float arithmetic on the FP32 pipe:
//            a x = ah xh + (err(ah xh) + ah xl + al xh) with err() from one
//            FMA (Dekker's product), accumulation by Knuth's TwoSum; about
//            44 bits of significand at 1/5 the FP32 rate, against 1/64 for
//            FP64 on this GPU.
#include "dense.cuh"

namespace {

constexpr int BM = 64, BK = 16, NT = 256;

// ---------------------------------------------------------------- arithmetics
struct Arith64 {
    typedef cplxf G;      // global element
    typedef cplxf S;      // staged element
    typedef cplxf Acc;
    __device__ static S stage(G v) { return v; }
    __device__ static S szero() { return mkcf(0.f, 0.f); }
    __device__ static void zero(Acc &a) { a = mkcf(0.f, 0.f); }
    __device__ static S conj(S v) { return cconj(v); }
    __device__ static void mac(Acc &c, const S &a, const S &b) { cfma(c, a, b); }
    __device__ static G finish(const Acc &c, G alpha, G beta, const G *old) {
        G r = cmul(alpha, c);
        if (old) r = cadd(r, cmul(beta, *old));
        return r;
    }
};

struct Arith128 {
    typedef cplx G;
    typedef cplx S;
    typedef cplx Acc;
    __device__ static S stage(G v) { return v; }
    __device__ static S szero() { return mkc(0.0, 0.0); }
    __device__ static void zero(Acc &a) { a = mkc(0.0, 0.0); }
    __device__ static S conj(S v) { return cconj(v); }
    __device__ static void mac(Acc &c, const S &a, const S &b) { cfma(c, a, b); }
    __device__ static G finish(const Acc &c, G alpha, G beta, const G *old) {
        G r = cmul(alpha, c);
        if (old) r = cadd(r, cmul(beta, *old));
        return r;
    }
};

// float pair: value = h + l, |l| <= ulp(h)/2
struct ffc {
    float rh, ih, rl, il;
};
struct ffacc {
    float rh, rl, ih, il;
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// acc += x y (x = xh + xl, y = yh + yl; the xl yl term is below the pair's precision)
__device__ __forceinline__ void ff_mac(float &sh, float &sl, float xh, float xl, float yh, float yl) {
    const float ph = xh * yh;
    const float pl = fmaf(xh, yl, fmaf(xl, yh, fmaf(xh, yh, -ph)));
    float s, e;
    two_sum(sh, ph, s, e);
    sh = s;
    sl += e + pl;
}

struct ArithFF {
    typedef cplx G;
    typedef ffc S;
    typedef ffacc Acc;
    __device__ static S stage(G v) {
        S r;
        r.rh = (float)v.x;
        r.rl = (float)(v.x - (double)r.rh);
        r.ih = (float)v.y;
        r.il = (float)(v.y - (double)r.ih);
        return r;
    }
    __device__ static S szero() { return S{0.f, 0.f, 0.f, 0.f}; }
    __device__ static void zero(Acc &a) { a = Acc{0.f, 0.f, 0.f, 0.f}; }
    __device__ static S conj(S v) {
        v.ih = -v.ih;
        v.il = -v.il;
        return v;
    }
    __device__ static void mac(Acc &c, const S &a, const S &b) {
        // re += ar br - ai bi ; im += ar bi + ai br
        ff_mac(c.rh, c.rl, a.rh, a.rl, b.rh, b.rl);
        ff_mac(c.rh, c.rl, -a.ih, -a.il, b.ih, b.il);
        ff_mac(c.ih, c.il, a.rh, a.rl, b.ih, b.il);
        ff_mac(c.ih, c.il, a.ih, a.il, b.rh, b.rl);
    }
    __device__ static G finish(const Acc &c, G alpha, G beta, const G *old) {
        const G v = mkc((double)c.rh + (double)c.rl, (double)c.ih + (double)c.il);
        G r = cmul(alpha, v);
        if (old) r = cadd(r, cmul(beta, *old));
        return r;
    }
};

// TJ columns per thread (CTA tile 64 x 16 TJ)
template <class Ar, int TJ>
__global__ void __launch_bounds__(NT) k_gemm_rt(const MatRefT<typename Ar::G> *__restrict__ As, int opA,
                                                const MatRefT<typename Ar::G> *__restrict__ Bs,
                                                const MatRefT<typename Ar::G> *__restrict__ Cs,
                                                typename Ar::G alpha, typename Ar::G beta, int use_beta,
                                                int tiles_m) {
    typedef typename Ar::G G;
    typedef typename Ar::S S;
    const MatRefT<G> A = As[blockIdx.y], B = Bs[blockIdx.y], Cm = Cs[blockIdx.y];
    const int M = Cm.rows, N = Cm.cols;
    const int K = (opA == 0) ? A.cols : A.rows;
    constexpr int BN = 16 * TJ;
    const int i0 = (blockIdx.x % tiles_m) * BM, j0 = (blockIdx.x / tiles_m) * BN;
    if (i0 >= M || j0 >= N) return;
    __shared__ S sa[BK][BM], sb[BK][16 * TJ];
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    typename Ar::Acc acc[4][TJ];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TJ; ++j) Ar::zero(acc[i][j]);
    for (int k0 = 0; k0 < K; k0 += BK) {
        // stage op(A)[i0:i0+64, k0:k0+16] as sa[k][i]
        if (opA == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = t & 63, k = (t >> 6) + 4 * q;
                const int gi = i0 + i, gk = k0 + k;
                sa[k][i] = (gi < M && gk < K) ? Ar::stage(A.p[gi + (int64_t)gk * A.ld]) : Ar::szero();
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = t & 15, i = (t >> 4) + 16 * q;
                const int gi = i0 + i, gk = k0 + k;
                sa[k][i] = (gi < M && gk < K) ? Ar::conj(Ar::stage(A.p[gk + (int64_t)gi * A.ld])) : Ar::szero();
            }
        }
        // stage B[k0:k0+16, j0:j0+BN] as sb[k][j]
#pragma unroll
        for (int q = 0; q < TJ; ++q) {
            const int k = t & 15, j = (t >> 4) + 16 * q;
            const int gk = k0 + k, gj = j0 + j;
            sb[k][j] = (gk < K && gj < N) ? Ar::stage(B.p[gk + (int64_t)gj * B.ld]) : Ar::szero();
        }
        __syncthreads();
        const int kmax = min(BK, K - k0);
        for (int k = 0; k < kmax; ++k) {
            S a[4], b[TJ];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sa[k][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < TJ; ++j) b[j] = sb[k][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < TJ; ++j) Ar::mac(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TJ; ++j) {
            const int gi = i0 + tx + 16 * i, gj = j0 + ty + 16 * j;
            if (gi < M && gj < N) {
                G *c = &Cm.p[gi + (int64_t)gj * Cm.ld];
                *c = Ar::finish(acc[i][j], alpha, beta, use_beta ? c : nullptr);
            }
        }
}

template <class Ar, int TJ>
int launch(int batch, int max_m, int max_n, const MatRefT<typename Ar::G> *d_A, int opA,
           const MatRefT<typename Ar::G> *d_B, const MatRefT<typename Ar::G> *d_C, typename Ar::G alpha,
           typename Ar::G beta, cudaStream_t s) {
    if (batch <= 0 || max_m <= 0 || max_n <= 0) return FDS_OK;
    if (opA != 0 && opA != 2) return FDS_ERR_ARG;
    constexpr int BN = 16 * TJ;
    const int tm = (max_m + BM - 1) / BM, tn = (max_n + BN - 1) / BN;
    const int use_beta = (beta.x != 0 || beta.y != 0) ? 1 : 0;
    dim3 grid(tm * tn, batch);
    fds_count_launch(), k_gemm_rt<Ar, TJ><<<grid, NT, 0, s>>>(d_A, opA, d_B, d_C, alpha, beta, use_beta, tm);
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}

}  // namespace

int dense_gemm_rt(int batch, int max_m, int max_n, const MatRef *d_A, int opA, const MatRef *d_B, const MatRef *d_C,
                  cplx alpha, cplx beta, cudaStream_t s) {
    return launch<Arith128, 4>(batch, max_m, max_n, d_A, opA, d_B, d_C, alpha, beta, s);
}

int dense_gemm_rt(int batch, int max_m, int max_n, const MatRefF *d_A, int opA, const MatRefF *d_B,
                  const MatRefF *d_C, cplxf alpha, cplxf beta, cudaStream_t s) {
    return launch<Arith64, 4>(batch, max_m, max_n, d_A, opA, d_B, d_C, alpha, beta, s);
}

int dense_gemm_ff(int batch, int max_m, int max_n, const MatRef *d_A, int opA, const MatRef *d_B, const MatRef *d_C,
                  cplx alpha, cplx beta, cudaStream_t s) {
    return launch<ArithFF, 2>(batch, max_m, max_n, d_A, opA, d_B, d_C, alpha, beta, s);
}
