// Batched complex64 GEMM on the 5th-generation tensor cores (tcgen05,
// kind::f16 with bf16 inputs), the mixed-precision merge/sweep products of
// Sec. 7 at fp32 accuracy with fp32 accumulation:
//
//   C_e = alpha op(A_e) B_e + beta C_e     (op = identity or conjugate transpose)
//
// A complex product is one real product of twice the size: with x stored as
// interleaved (re, im) pairs, the column of x is already the real vector
// [x_r(0), x_i(0), x_r(1), ...], and op(A) becomes the real matrix whose 2x2
// block (i, k) is [[a_r, -a_i], [a_i, a_r]].  Every fp32 operand v is split
// into three bf16 pieces v = p0 + p1 + p2 (p0 = bf16(v), p1 = bf16(v - p0),
// p2 = bf16(v - p0 - p1); each difference is exact in fp32), which hold 24
// bits of v; the six products p_i q_j with i + j <= 2 leave out terms below
// 2^-24 of |v||w|, and bf16 x bf16 products are exact in the fp32
// accumulator, so the result carries fp32 rounding only.
//
// Tile: 128 real rows (64 complex rows of C) x 128 right-hand-side columns,
// accumulated in TMEM (128 lanes x 128 fp32 columns).  K advances in stages
// of 64 reals (32 complex), one 128-byte row of bf16 per tile row: the 256
// threads load stage k+1 into registers while the tensor core works on stage
// k, then expand, split and store it into 128-byte-swizzled K-major tiles of
// the free stage buffer; one thread issues the MMAs and commits them to that
// buffer's mbarrier.  Every wait is bounded: after about two seconds the
// kernel records a status, waits (bounded again) for its own MMAs, frees its
// TMEM and returns.
#include <algorithm>
#include <cstdint>
#include <vector>

#include <cuda_bf16.h>

#include "common.cuh"
#include "dense.cuh"
#include "fds_internal.cuh"

namespace {

constexpr int TC_BM = 128;          // real rows of a tile
constexpr int TC_BN = 128;          // columns of a tile
constexpr int TC_THREADS = 256;
constexpr int TC_STAGES = 2;
constexpr int TC_KC = 32;           // complex K per stage (64 reals = one 128-byte bf16 row)
constexpr int TC_PIECES = 3;
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;

struct TcLayout {
    static constexpr int A_BYTES = TC_BM * 128;     // one piece: rows x 128 B
    static constexpr int B_BYTES = TC_BN * 128;
    static constexpr int STAGE = TC_PIECES * (A_BYTES + B_BYTES);
    static constexpr int TOTAL = TC_STAGES * STAGE + 1024 + 64;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 B apart (tile bases are 1024-byte aligned)
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)(1024u >> 4) << 32;   // stride between 8-row groups
    d |= (uint64_t)1 << 46;              // descriptor version of this architecture
    d |= (uint64_t)2 << 61;              // 128-byte swizzle
    return d;
}

// instruction descriptor: fp32 accumulator, bf16 A and B, both K-major, M 128
__device__ __forceinline__ uint32_t idesc_bf16() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_BN >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
}

// byte offset of 16-byte chunk c (0..7) of row r in a 128-byte-swizzled tile
__device__ __forceinline__ uint32_t sw128_off(int r, int c) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
}

// three bf16 pieces of v (bit patterns)
__device__ __forceinline__ void split3(float v, uint32_t (&p)[TC_PIECES]) {
    const __nv_bfloat16 b0 = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(b0);
    const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(b1);
    const __nv_bfloat16 b2 = __float2bfloat16_rn(r2);
    p[0] = __bfloat16_as_ushort(b0);
    p[1] = __bfloat16_as_ushort(b1);
    p[2] = __bfloat16_as_ushort(b2);
}

__device__ __forceinline__ uint32_t pk(uint32_t lo, uint32_t hi) { return lo | (hi << 16); }

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_try(bar, parity)) return true;   // the common case: no timer read
    const unsigned long long t0 = global_ns();
    while (!mbar_try(bar, parity))
        if (global_ns() - t0 > TC_WAIT_NS) return false;
    return true;
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// One stage of operands in registers: per thread 2 A items (4 complex entries
// of one row of op(A)) and 4 B items (4 consecutive complex rows of one column).
constexpr int TC_AIT = TC_BM / 2 * (TC_KC / 4) / TC_THREADS;   // 2
constexpr int TC_BIT = TC_BN * (TC_KC / 4) / TC_THREADS;       // 4

struct Stage {
    float2 a[TC_AIT][4];
    float2 b[TC_BIT][4];
};

__device__ __forceinline__ void a_item(int it, int opA, int &li, int &q) {
    if (opA == 0) {   // consecutive threads: consecutive rows (contiguous in column-major A)
        li = it & 63;
        q = it >> 6;
    } else {          // consecutive threads: consecutive k (contiguous rows of A^H)
        q = it & 7;
        li = it >> 3;
    }
}

__device__ __forceinline__ void load_stage(Stage &S, const MatRefF &A, const MatRefF &B, const int *bmap, int opA,
                                           int Mc, int N, int Kc, int ci0, int j0, int k0, int tid) {
#pragma unroll
    for (int u = 0; u < TC_AIT; ++u) {
        int li, q;
        a_item(tid + u * TC_THREADS, opA, li, q);
        const int ci = ci0 + li, ck = k0 + 4 * q;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            float2 v = make_float2(0.f, 0.f);
            if (ci < Mc && ck + t < Kc)
                v = opA == 0 ? A.p[ci + (int64_t)(ck + t) * A.ld] : A.p[ck + t + (int64_t)ci * A.ld];
            S.a[u][t] = v;
        }
    }
#pragma unroll
    for (int u = 0; u < TC_BIT; ++u) {
        const int it = tid + u * TC_THREADS;
        const int c = it & 7, n = it >> 3;
        const int col = j0 + n, ck = k0 + 4 * c;
        const cplxf *bc = B.p + (int64_t)col * B.ld;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            float2 v = make_float2(0.f, 0.f);
            if (col < N && ck + t < Kc) {
                const int rk = bmap ? bmap[ck + t] : ck + t;
                if (FDS_IN_RANGE(rk, B.rows)) v = bc[rk];
            }
            S.b[u][t] = v;
        }
    }
}

__device__ __forceinline__ void store_stage(const Stage &S, unsigned char *buf, int opA, int tid) {
    unsigned char *ap = buf, *bp = buf + TC_PIECES * TcLayout::A_BYTES;
#pragma unroll
    for (int u = 0; u < TC_AIT; ++u) {
        int li, q;
        a_item(tid + u * TC_THREADS, opA, li, q);
        uint32_t pr[4][TC_PIECES], pi[4][TC_PIECES];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            split3(S.a[u][t].x, pr[t]);
            split3(S.a[u][t].y, pi[t]);
        }
        const uint32_t ore = sw128_off(2 * li, q), oim = sw128_off(2 * li + 1, q);
#pragma unroll
        for (int s = 0; s < TC_PIECES; ++s) {
            uint4 re, im;
            if (opA == 0) {   // rows [a_r, -a_i ...] and [a_i, a_r ...]
                re = make_uint4(pk(pr[0][s], pi[0][s] ^ 0x8000u), pk(pr[1][s], pi[1][s] ^ 0x8000u),
                                pk(pr[2][s], pi[2][s] ^ 0x8000u), pk(pr[3][s], pi[3][s] ^ 0x8000u));
                im = make_uint4(pk(pi[0][s], pr[0][s]), pk(pi[1][s], pr[1][s]), pk(pi[2][s], pr[2][s]),
                                pk(pi[3][s], pr[3][s]));
            } else {          // conjugate: [a_r, a_i ...] and [-a_i, a_r ...]
                re = make_uint4(pk(pr[0][s], pi[0][s]), pk(pr[1][s], pi[1][s]), pk(pr[2][s], pi[2][s]),
                                pk(pr[3][s], pi[3][s]));
                im = make_uint4(pk(pi[0][s] ^ 0x8000u, pr[0][s]), pk(pi[1][s] ^ 0x8000u, pr[1][s]),
                                pk(pi[2][s] ^ 0x8000u, pr[2][s]), pk(pi[3][s] ^ 0x8000u, pr[3][s]));
            }
            *reinterpret_cast<uint4 *>(ap + s * TcLayout::A_BYTES + ore) = re;
            *reinterpret_cast<uint4 *>(ap + s * TcLayout::A_BYTES + oim) = im;
        }
    }
#pragma unroll
    for (int u = 0; u < TC_BIT; ++u) {
        const int it = tid + u * TC_THREADS;
        const int c = it & 7, n = it >> 3;
        uint32_t pr[4][TC_PIECES], pi[4][TC_PIECES];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            split3(S.b[u][t].x, pr[t]);
            split3(S.b[u][t].y, pi[t]);
        }
        const uint32_t o = sw128_off(n, c);
#pragma unroll
        for (int s = 0; s < TC_PIECES; ++s)
            *reinterpret_cast<uint4 *>(bp + s * TcLayout::B_BYTES + o) =
                make_uint4(pk(pr[0][s], pi[0][s]), pk(pr[1][s], pi[1][s]), pk(pr[2][s], pi[2][s]),
                           pk(pr[3][s], pi[3][s]));
    }
}

}  // namespace

__device__ int g_tc_status;   // 1 once a tensor-core GEMM gave up waiting on its MMAs
__device__ int g_tc_fault;    // injected fault: the next launch's first CTA issues no MMAs

namespace {

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gemm_tc(const MatRefF *__restrict__ As, int opA, const MatRefF *__restrict__ Bs,
              const MatRefF *__restrict__ Cs, float alpha, float beta, int tiles_m,
              const RowMaps *__restrict__ maps) {
    typedef TcLayout Lay;
    extern __shared__ unsigned char tc_raw[];
    const MatRefF A = As[blockIdx.y], B = Bs[blockIdx.y], Cm = Cs[blockIdx.y];
    const int *bmap = maps ? maps[blockIdx.y].b : nullptr;
    const int *cmap = maps ? maps[blockIdx.y].c : nullptr;
    const int Mc = Cm.rows, N = Cm.cols;
    const int Kc = (opA == 0) ? A.cols : A.rows;
    const int i0 = (blockIdx.x % tiles_m) * TC_BM, j0 = (blockIdx.x / tiles_m) * TC_BN;
    if (i0 >= 2 * Mc || j0 >= N) return;

    const uint32_t raw = smem_u32(tc_raw);
    const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
    unsigned char *base = tc_raw + pad;
    const uint32_t sbase = raw + pad;
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + TC_STAGES * Lay::STAGE);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + TC_STAGES);
    const int tid = threadIdx.x, warp = tid >> 5;

    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bars + s)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TC_BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    const int nch = (Kc + TC_KC - 1) / TC_KC;
    const int ci0 = i0 >> 1;
    bool bad = false;
    int committed = -1;   // last stage whose MMAs were committed
    // injected stall: the first CTA issues no MMAs, so its completion waits run out
    const bool stall = tid == 0 && blockIdx.x == 0 && blockIdx.y == 0 && atomicExch(&g_tc_fault, 0) != 0;
    Stage S;
    if (nch > 0) load_stage(S, A, B, bmap, opA, Mc, N, Kc, ci0, j0, 0, tid);
    for (int kc = 0; kc < nch; ++kc) {
        const int buf = kc & 1;
        if (kc >= TC_STAGES) {
            const bool ok = mbar_wait(smem_u32(bars + buf), (uint32_t)(((kc - TC_STAGES) >> 1) & 1));
            if (__syncthreads_or(!ok)) {
                bad = true;
                break;
            }
        }
        store_stage(S, base + buf * Lay::STAGE, opA, tid);
        if (kc + 1 < nch) load_stage(S, A, B, bmap, opA, Mc, N, Kc, ci0, j0, (kc + 1) * TC_KC, tid);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0 && !stall) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t idesc = idesc_bf16();
            const uint32_t sa = sbase + buf * Lay::STAGE;
            const uint32_t sb = sa + TC_PIECES * Lay::A_BYTES;
            const int nks = min(4, (2 * (Kc - kc * TC_KC) + 15) / 16);   // k-steps of 16 reals holding data
            for (int ks = 0; ks < nks; ++ks) {
                const uint32_t o = 32u * ks;
                // smallest terms first: (2,0) (1,1) (0,2) (1,0) (0,1) (0,0)
                const int pa[6] = {2, 1, 0, 1, 0, 0}, pb[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
                for (int t = 0; t < 6; ++t)
                    mma_bf16(tmem, sw128_desc(sa + pa[t] * Lay::A_BYTES + o),
                             sw128_desc(sb + pb[t] * Lay::B_BYTES + o), idesc, (kc | ks | t) ? 1u : 0u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(bars + buf))
                         : "memory");
            committed = kc;
        }
    }
    if (!bad && nch > 0) {
        const int kl = nch - 1;
        const bool ok = mbar_wait(smem_u32(bars + (kl & 1)), (uint32_t)((kl >> 1) & 1));
        bad = __syncthreads_or(!ok);
    }
    if (bad) {
        if (tid == 0) {
            atomicExch(&g_tc_status, 1);
            // the last committed stage (bounded again) before the TMEM is freed
            if (committed >= 0)
                mbar_wait(smem_u32(bars + (committed & 1)), (uint32_t)((committed >> 1) & 1));
        }
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int q = warp & 3, half = warp >> 2;
        const int rr = i0 + q * 32 + (tid & 31);
        const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16);
        bool row_ok = rr < 2 * Mc;
        float *cp = nullptr;
        if (row_ok) {
            const int ci = rr >> 1;
            const int ri = cmap ? cmap[ci] : ci;
            row_ok = FDS_IN_RANGE(ri, cmap ? maps[blockIdx.y].cext : Mc);
            if (row_ok) cp = reinterpret_cast<float *>(Cm.p) + 2 * (int64_t)ri + (rr & 1);
        }
        for (int cb = half * (TC_BN / 2); cb < (half + 1) * (TC_BN / 2); cb += 16) {
            if (j0 + cb >= N) break;
            float v[16], old[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) old[j] = 0.f;
            if (row_ok && beta != 0.f) {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (j0 + cb + j < N) old[j] = cp[2 * (int64_t)(j0 + cb + j) * Cm.ld];
            }
            if (nch > 0) {
                tmem_ld16(tq + (uint32_t)cb, v);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = 0.f;
            }
            if (row_ok) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = j0 + cb + j;
                    if (col < N) cp[2 * (int64_t)col * Cm.ld] = alpha * v[j] + beta * old[j];
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_BN));
}

}  // namespace

int dense_gemm_tc(int batch, int max_m, int max_n, const MatRefF *d_A, int opA, const MatRefF *d_B,
                  const MatRefF *d_C, float alpha, float beta, const RowMaps *d_maps, cudaStream_t s) {
    if (batch <= 0 || max_m <= 0 || max_n <= 0) return FDS_OK;
    if (opA != 0 && opA != 2) return FDS_ERR_ARG;
    if (batch > 65535) return FDS_ERR_ARG;
    const int tm = (2 * max_m + TC_BM - 1) / TC_BM, tn = (max_n + TC_BN - 1) / TC_BN;
    constexpr int smem = TcLayout::TOTAL;
    FDS_TRY(ensure_dyn_smem(k_gemm_tc, smem));
    dim3 grid(tm * tn, batch);
    fds_count_launch(), k_gemm_tc<<<grid, TC_THREADS, smem, s>>>(d_A, opA, d_B, d_C, alpha, beta, tm, d_maps);
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}

int tc_status_take(cudaStream_t s, int *status) {
    int v = 0, zero = 0;
    FDS_CUDA_TRY(cudaMemcpyFromSymbolAsync(&v, g_tc_status, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    FDS_CUDA_TRY(cudaStreamSynchronize(s));
    if (v) FDS_CUDA_TRY(cudaMemcpyToSymbolAsync(g_tc_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
    *status = v;
    return FDS_OK;
}

int tc_fault_arm(int on) {
    const int v = on ? 1 : 0;
    FDS_CUDA_TRY(cudaMemcpyToSymbol(g_tc_fault, &v, sizeof(int)));
    return FDS_OK;
}

// ------------------------------------------------------------------ stage entry
namespace {
__global__ void k_cgemm_refs(int batch, const int *m, const int *n, const int *k, const int64_t *aoff,
                             const int64_t *boff, const int64_t *coff, const float *A, const float *B, float *C,
                             int opA, MatRefF *rA, MatRefF *rB, MatRefF *rC) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    const int ar = opA ? k[b] : m[b], ac = opA ? m[b] : k[b];
    rA[b].p = (cplxf *)(A + 2 * aoff[b]);
    rA[b].rows = ar;
    rA[b].cols = ac;
    rA[b].ld = ar > 1 ? ar : 1;
    rB[b].p = (cplxf *)(B + 2 * boff[b]);
    rB[b].rows = k[b];
    rB[b].cols = n[b];
    rB[b].ld = k[b] > 1 ? k[b] : 1;
    rC[b].p = (cplxf *)(C + 2 * coff[b]);
    rC[b].rows = m[b];
    rC[b].cols = n[b];
    rC[b].ld = m[b] > 1 ? m[b] : 1;
}
}  // namespace

extern "C" int fds_cgemm_c64_batched(int32_t batch, const int32_t *m, const int32_t *n, const int32_t *k,
                                     const int64_t *aoff, const int64_t *boff, const int64_t *coff,
                                     const float *d_A, const float *d_B, float *d_C, int32_t opA, float alpha,
                                     float beta, int32_t engine, uint64_t stream) {
    if (batch < 0 || batch > 65535) return FDS_ERR_ARG;
    if (batch == 0) return FDS_OK;
    if (!m || !n || !k || !aoff || !boff || !coff || !d_A || !d_B || !d_C) return FDS_ERR_ARG;
    if ((opA != 0 && opA != 2) || (engine != FDS_C64_SIMT && engine != FDS_C64_TENSOR)) return FDS_ERR_ARG;
    int max_m = 0, max_n = 0;
    for (int b = 0; b < batch; ++b) {
        if (m[b] < 0 || n[b] < 0 || k[b] < 0 || aoff[b] < 0 || boff[b] < 0 || coff[b] < 0) return FDS_ERR_ARG;
        max_m = std::max(max_m, m[b]);
        max_n = std::max(max_n, n[b]);
    }
    cudaStream_t s = (cudaStream_t)stream;
    DBuf<int> dm, dn, dk;
    DBuf<int64_t> da, db, dc;
    DBuf<MatRefF> refs;
    FDS_TRY(dm.upload(std::vector<int>(m, m + batch), s));
    FDS_TRY(dn.upload(std::vector<int>(n, n + batch), s));
    FDS_TRY(dk.upload(std::vector<int>(k, k + batch), s));
    FDS_TRY(da.upload(std::vector<int64_t>(aoff, aoff + batch), s));
    FDS_TRY(db.upload(std::vector<int64_t>(boff, boff + batch), s));
    FDS_TRY(dc.upload(std::vector<int64_t>(coff, coff + batch), s));
    FDS_TRY(refs.alloc(3 * (size_t)batch));
    fds_count_launch(), k_cgemm_refs<<<(batch + 127) / 128, 128, 0, s>>>(
        batch, dm.p, dn.p, dk.p, da.p, db.p, dc.p, d_A, d_B, d_C, opA, refs.p, refs.p + batch, refs.p + 2 * batch);
    FDS_CUDA_TRY(cudaGetLastError());
    int rc;
    if (engine == FDS_C64_TENSOR) {
        rc = dense_gemm_tc(batch, max_m, max_n, refs.p, opA, refs.p + batch, refs.p + 2 * batch, alpha, beta,
                           nullptr, s);
    } else {
        rc = dense_gemm_rt(batch, max_m, max_n, refs.p, opA, refs.p + batch, refs.p + 2 * batch, mkcf(alpha, 0.f),
                           mkcf(beta, 0.f), s);
    }
    FDS_CUDA_TRY(cudaStreamSynchronize(s));
    if (rc != FDS_OK) return rc;
    if (engine == FDS_C64_TENSOR) {
        int st = 0;
        FDS_TRY(tc_status_take(s, &st));
        if (st) return FDS_ERR_TIMEOUT;
    }
    return FDS_OK;
}
