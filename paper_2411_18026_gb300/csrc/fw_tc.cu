// Leaf diagonal blocks of the FP64 compressed forward operator (the residual
// r = f - A x of the mixed-precision refinement) on the 5th-generation tensor
// cores, with FP64-level accuracy from bf16 products (an Ozaki-type split):
//
//   y_b += D_b x_b   for every leaf b (D_b: d_b x d_b complex, d_b <= 128).
//
// Real form: D_b is the 2d x 2d real matrix of 2 x 2 blocks [[a_r, -a_i],
// [a_i, a_r]], x the interleaved (re, im) vector.  Each real row r of D_b is
// scaled by 2^e_r (e_r from frexp of the row's largest entry) and cut into
// six slices s_0..s_5: v = D_rk / 2^e_r in (-1, 1), s_i = trunc(256 v_i),
// v_{i+1} = 256 v_i - s_i, so D_rk = 2^e_r sum_i s_i 2^(-8(i+1)) with every
// s_i an integer of at most 8 bits (exact in bf16); slice i is stored times
// 2^(-8i).  Each column c of x is cut the same way with its own exponent.
// The product needs the 21 slice pairs with i + j <= 5 (the others are below
// 2^-48 of |D| |x|).  The tensor core's fp32 accumulation keeps about 24 bits
// below the running sum's leading bit, so a sum is exact only while its
// terms' granularity fits that window.  Each pair with i + j <= 2 therefore
// has an fp32 accumulator of its own in tensor memory (a sum of K <= 256
// products of two 8-bit integers, scaled by one power of two: exact); the
// pairs with i + j = 3 share one (its truncation lies near 2^-38 of the
// result), those with i + j >= 4 another (measured with one accumulator for
// every i + j >= 2: 3.6e-10 of |D| |x|; with two slices per operand every
// accumulator is exact).  The epilogue adds the eight in FP64, scales by
// 2^(e_r + f_c - 16) and adds the result to y (float pairs, the refinement's
// forward-operator format).
//
// Kernel: one CTA per (leaf, 128 real rows, 64 columns); eight accumulators
// of 64 fp32 columns fill the 512 tensor-memory columns.  Two rings of
// operand tiles (A slice tiles, 128 rows x 64 K, and x slice tiles, 64 rows x
// 64 K, of bf16, stored pre-swizzled so that each is one bulk copy) fed by
// one producer thread with cp.async.bulk and mbarrier transaction counts;
// the pairs are ordered by the A slice, so each A tile is loaded once per K
// chunk and serves 6 - i products.  One thread issues tcgen05.mma
// (kind::f16, bf16, M 128, N 64, K 16) into the accumulator of the pair and
// commits each x tile (and each A tile after its last product) back to the
// producer.  Every wait is bounded: after about two seconds the kernel
// records a status, waits (bounded again) for its own MMAs, frees its TMEM
// and returns.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include <cuda_bf16.h>

#include "common.cuh"
#include "fds_internal.cuh"
#include "fw_tc.cuh"

namespace {

constexpr int OZ_SLICES = 6;
constexpr int OZ_TILE = 128 * 128;     // bytes of one 128 x 64 bf16 tile (A)
constexpr int OZ_BN = 64;              // columns of x per CTA
constexpr int OZ_XTILE = OZ_BN * 128;  // bytes of one 64 x 64 bf16 tile (x)
constexpr int OZ_NA = 6;               // ring of A slice tiles (16 KB each)
constexpr int OZ_NX = 2;               // x buffers, each the six slice tiles of one K chunk (48 KB)
constexpr int OZ_THREADS = 128;
constexpr int OZ_KC = 4;               // 64-wide K chunks of a 256-real K
constexpr int OZ_ACC = 8;
constexpr unsigned long long OZ_WAIT_NS = 2000000000ull;

struct OzLayout {
    static constexpr int XBUF = OZ_SLICES * OZ_XTILE;               // one K chunk of x slices
    static constexpr int XOFF = OZ_NA * OZ_TILE;                    // x buffers after the A ring
    static constexpr int RINGS = XOFF + OZ_NX * XBUF;
    static constexpr int NBAR = 2 * OZ_NA + 2 * OZ_NX + 1;          // full/empty of both rings, done
    static constexpr int TOTAL = RINGS + 1024 + 8 * NBAR + 512;     // + TMEM slot, flag, 64 exponents
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// K-major operand tile, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// fp32 accumulator, bf16 A and B, both K-major, N 64, M 128
__device__ __forceinline__ uint32_t idesc_bf16_m128_n64() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_BN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// byte offset of element (row r, k) in a 128 x 64 bf16 tile with 128-byte swizzle
__device__ __forceinline__ uint32_t sw_elem(int r, int k) {
    const int c = k >> 3;
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4) + (k & 7) * 2);
}

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
        if (global_ns() - t0 > OZ_WAIT_NS) return false;
    return true;
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// a 32-lane x 16-column tensor-memory load without its wait (several loads, then one tcgen05.wait::ld)
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// 2^k as a float for -126 <= k <= 127 (exact scaling by multiplication)
__device__ __forceinline__ float pow2f(int k) {
    k = max(-126, min(127, k));
    return __uint_as_float((uint32_t)(k + 127) << 23);
}

// error-free float sum: s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// (rh, rl) = (ah, al) + (bh, bl) in float-pair arithmetic (~46 bits)
__device__ __forceinline__ void ff_add(float ah, float al, float bh, float bl, float &rh, float &rl) {
    float s, e;
    two_sum_f(ah, bh, s, e);
    e += al + bl;
    rh = s + e;
    rl = e - (rh - s);
}

// accumulator of pair (i, j): one each for i + j <= 2, then i + j = 3, then i + j >= 4
__device__ __forceinline__ int pair_acc(int i, int j) {
    const int g = i + j;
    if (g == 0) return 0;
    if (g == 1) return i == 0 ? 1 : 2;
    if (g == 2) return 3 + i;
    return g == 3 ? 6 : 7;
}

// The products of operator slice I with vector slices j = 0 .. 5 - I for one
// K chunk (nks k-steps of 16): descriptors da (slice I's tile) and db[j]
// (the chunk's vector slice tiles) advance by 32 bytes (2 in the address
// field) per k-step; pair (I, j) accumulates into group pair_acc(I, j) of
// the set at tacc (ncol columns per group) and overwrites it when it is the
// group's first pair of the item's first chunk.  All indexes are
// compile-time constants, so each MMA costs a few instructions to issue.
template <int I>
__device__ __forceinline__ void mma_slice(uint32_t tacc, uint32_t ncol, uint64_t da, const uint64_t (&db)[6],
                                          uint32_t idesc, int nks, bool first_chunk) {
#pragma unroll
    for (int j = 0; j < 6 - I; ++j) {
        const int g = pair_acc(I, j);
        // first pair of its group in issue order (i outer, j inner): (0, 0..4), (1, 0), (1, 1), (2, 0)
        const bool grp_first = (I == 0 && j <= 4) || (I == 1 && j <= 1) || (I == 2 && j == 0);
        const uint32_t d = tacc + (uint32_t)g * ncol;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)
            if (ks < nks)
                mma_bf16(d, da + 2ull * ks, db[j] + 2ull * ks, idesc,
                         (first_chunk && ks == 0 && grp_first) ? 0u : 1u);
    }
}

__device__ __forceinline__ void mma_slice_rt(int i, uint32_t tacc, uint32_t ncol, uint64_t da,
                                             const uint64_t (&db)[6], uint32_t idesc, int nks, bool first_chunk) {
    switch (i) {
        case 0: mma_slice<0>(tacc, ncol, da, db, idesc, nks, first_chunk); break;
        case 1: mma_slice<1>(tacc, ncol, da, db, idesc, nks, first_chunk); break;
        case 2: mma_slice<2>(tacc, ncol, da, db, idesc, nks, first_chunk); break;
        case 3: mma_slice<3>(tacc, ncol, da, db, idesc, nks, first_chunk); break;
        case 4: mma_slice<4>(tacc, ncol, da, db, idesc, nks, first_chunk); break;
        default: mma_slice<5>(tacc, ncol, da, db, idesc, nks, first_chunk); break;
    }
}

// Six slices of v = a 2^-e (|v| < 1): s_i = trunc(256 v_i), v_{i+1} =
// 256 v_i - s_i (v_0 = v), slice i stored times 2^(-8i) (exact in bf16).
// Computed from the bits of a: q = trunc(|v| 2^48) by an integer shift of
// a's 53-bit significand, s_i = bits 40 - 8i .. 47 - 8i of q with a's sign
// (the same values as the FP64 recurrence, whose steps are all exact, on
// the integer pipe instead of the slow FP64 one).
__device__ __forceinline__ void cut6_bits(double a, int e, unsigned short (&out)[OZ_SLICES]) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(a);
    const int ex = (int)((b >> 52) & 2047ull);
    unsigned long long q = 0;
    if (ex != 0) {   // zero or subnormal: below 2^-1022, no bit at 2^-48 of v
        const unsigned long long mant = (b & ((1ull << 52) - 1ull)) | (1ull << 52);   // |a| = mant 2^(ex - 1075)
        const int sh = 1027 - ex + e;                                               // |v| 2^48 = mant 2^-sh
        q = sh >= 64 ? 0ull : (sh > 0 ? (mant >> sh) : (mant << min(-sh, 11)));
    }
    if (q >= (1ull << 48)) q = (1ull << 48) - 1;   // |v| < 1
    const bool neg = (b >> 63) != 0ull;
    float sc = 1.0f;
#pragma unroll
    for (int i = 0; i < OZ_SLICES; ++i) {
        const uint32_t chunk = (uint32_t)((q >> (40 - 8 * i)) & 255ull);
        const float t = (__uint_as_float(0x4B000000u | chunk) - 8388608.0f) * sc;
        out[i] = __bfloat16_as_ushort(__float2bfloat16_rn(neg ? -t : t));
        sc *= 1.0f / 256.0f;
    }
}

// ------------------------------------------------------------------ slicing
// A slices: one warp per real row r of one leaf block; tiles at
// base + (((b * 2 + mt) * OZ_KC + kc) * OZ_SLICES + i) * OZ_TILE; exponent per row.
__global__ void k_oz_slice_a(int nb, const MatRef *__restrict__ D, unsigned char *slices, int *rowexp) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= nb * 256) return;
    const int b = warp >> 8, r = warp & 255;
    const MatRef A = D[b];
    const int d = A.rows;
    const int i = r >> 1;
    const bool im_row = r & 1;
    // row r of the real form: k = 2 l -> (re ? a_r : a_i), k = 2 l + 1 -> (re ? -a_i : a_r)
    double m = 0.0;
    if (i < d)
        for (int l = lane; l < d; l += 32) {
            const cplx a = A.p[i + (int64_t)l * A.ld];
            m = fmax(m, fmax(fabs(a.x), fabs(a.y)));
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    int e = 0;
    if (m > 0.0) frexp(m, &e);
    if (lane == 0) rowexp[b * 256 + r] = e;
    const int mt = r >> 7, rr = r & 127;
    for (int k = lane; k < 256; k += 32) {
        double v = 0.0;
        const int l = k >> 1;
        if (i < d && l < d) {
            const cplx a = A.p[i + (int64_t)l * A.ld];
            v = !im_row ? ((k & 1) ? -a.y : a.x) : ((k & 1) ? a.x : a.y);
        }
        unsigned short s[OZ_SLICES];
        cut6_bits(v, e, s);
        const int kc = k >> 6;
        unsigned char *t = slices + (size_t)(((b * 2 + mt) * OZ_KC + kc) * OZ_SLICES) * OZ_TILE;
        const uint32_t off = sw_elem(rr, k & 63);
#pragma unroll
        for (int q = 0; q < OZ_SLICES; ++q) *reinterpret_cast<unsigned short *>(t + (size_t)q * OZ_TILE + off) = s[q];
    }
}

// trunc(|f| 2^sh) as an integer (|f| 2^sh < 2^48), from the bits of f
// (integer instructions only: 64-bit conversions run on the slow FP64 pipe)
__device__ __forceinline__ unsigned long long fixed48(float f, int sh) {
    const uint32_t b = __float_as_uint(f);
    const int ex = (int)((b >> 23) & 255u);
    if (ex == 0) return 0ull;                         // zero or subnormal: below 2^-126
    const uint32_t mant = (b & 0x7FFFFFu) | 0x800000u;    // |f| = mant 2^(ex - 150)
    const int s = ex - 150 + sh;
    if (s >= 0) return (unsigned long long)mant << s;
    if (s <= -24) return 0ull;
    return (unsigned long long)(mant >> (-s));
}

// six slices of the float pair (h, l) scaled by 2^-e (|h + l| < 2^e), from
// the 48-bit integer q = trunc(h 2^(48-e)) + trunc(l 2^(48-e)): slice i is
// bits 40 - 8i .. 47 - 8i of |q|, with q's sign, times 2^(-8i)
__device__ __forceinline__ void cut6_pair(float h, float l, int e, unsigned short (&out)[OZ_SLICES]) {
    const long long qh = (long long)fixed48(h, 48 - e), ql = (long long)fixed48(l, 48 - e);
    const long long q = (h < 0.f ? -qh : qh) + (l < 0.f ? -ql : ql);
    const bool neg = q < 0;
    unsigned long long m = (unsigned long long)(neg ? -q : q);
    if (m >= (1ull << 48)) m = (1ull << 48) - 1;   // |h + l| within one unit of 2^e
    float sc = 1.0f;
#pragma unroll
    for (int i = 0; i < OZ_SLICES; ++i) {
        // the 8-bit chunk as a float: OR it into the mantissa of 2^23 (exact)
        const uint32_t chunk = (uint32_t)((m >> (40 - 8 * i)) & 255ull);
        const float t = (__uint_as_float(0x4B000000u | chunk) - 8388608.0f) * sc;
        out[i] = __bfloat16_as_ushort(__float2bfloat16_rn(neg ? -t : t));
        sc *= 1.0f / 256.0f;
    }
}

// x slices: one warp per (leaf b, column c); the leaf's rows are
// xin[doff[b] .. doff[b] + d) of column c (float pairs); 64-column tiles at
// base + (((b * ntile + nt) * OZ_KC + kc) * OZ_SLICES + j) * OZ_XTILE.
__global__ void k_oz_slice_x(int nb, const int64_t *__restrict__ doff, const float4 *__restrict__ x, int64_t ldx,
                             int nc, int ntile, unsigned char *slices, int *colexp) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int cols = ntile * OZ_BN;
    if (warp >= nb * cols) return;
    const int b = warp / cols, c = warp % cols;
    const int64_t o = doff[b];
    const int d = (int)(doff[b + 1] - o);
    float m = 0.f;
    if (c < nc)
        for (int l = lane; l < d; l += 32) {
            const float4 v = x[o + l + (int64_t)c * ldx];
            m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
        }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, s));
    // 2^e > |h| (1 + 2^-23) >= |h + l|
    int e = 0;
    if (m > 0.f) {
        frexpf(m, &e);
        if (m >= ldexpf(1.0f - 1.0f / (1 << 20), e)) ++e;
    }
    if (lane == 0) colexp[b * cols + c] = e;
    const int nt = c / OZ_BN, n = c % OZ_BN;
    for (int k = lane; k < 256; k += 32) {
        const int l = k >> 1;
        float h = 0.f, lo = 0.f;
        if (c < nc && l < d) {
            const float4 q = x[o + l + (int64_t)c * ldx];
            h = (k & 1) ? q.y : q.x;
            lo = (k & 1) ? q.w : q.z;
        }
        unsigned short s[OZ_SLICES];
        cut6_pair(h, lo, e, s);
        const int kc = k >> 6;
        unsigned char *t = slices + (size_t)(((b * ntile + nt) * OZ_KC + kc) * OZ_SLICES) * OZ_XTILE;
        const uint32_t off = sw_elem(n, k & 63);
#pragma unroll
        for (int q = 0; q < OZ_SLICES; ++q)
            *reinterpret_cast<unsigned short *>(t + (size_t)q * OZ_XTILE + off) = s[q];
    }
}

}  // namespace

__device__ int g_oz_status;   // 1 once a leaf-block tensor-core product gave up waiting
__device__ int g_oz_fault;    // injected fault: the next launch's first CTA issues no copies

namespace {

// ------------------------------------------------------------------ product
__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_oz_leaf(int nb, int ntile, const int64_t *__restrict__ doff, const unsigned char *__restrict__ aslices,
              const int *__restrict__ rowexp, const unsigned char *__restrict__ xslices,
              const int *__restrict__ colexp, float4 *y, int64_t ldy, int nc) {
    extern __shared__ unsigned char oz_raw[];
    const int tile = blockIdx.x;
    const int b = tile / (2 * ntile), mt = (tile / ntile) & 1, nt = tile % ntile;
    const int64_t o = doff[b];
    const int d = (int)(doff[b + 1] - o);
    if (2 * d <= mt * 128) return;     // no rows of this leaf in the lower half
    const uint32_t raw = smem_u32(oz_raw);
    const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
    const uint32_t sbase = raw + pad;
    uint64_t *bars = reinterpret_cast<uint64_t *>(oz_raw + pad + OzLayout::RINGS);
    // A ring: full bars[q], empty bars[OZ_NA + q]; x ring: full bars[2 OZ_NA + q],
    // empty bars[2 OZ_NA + OZ_NX + q]; done: bars[NBAR - 1]
    uint64_t *fullA = bars, *emptyA = bars + OZ_NA, *fullX = bars + 2 * OZ_NA, *emptyX = fullX + OZ_NX;
    uint64_t *donebar = bars + OzLayout::NBAR - 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + OzLayout::NBAR);
    int *sflag = reinterpret_cast<int *>(tslot + 1);
    int *s_colexp = sflag + 1;   // exponents of this CTA's 64 columns
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid < OZ_BN) {
        const int c = nt * OZ_BN + tid;
        s_colexp[tid] = c < nc ? colexp[b * (ntile * OZ_BN) + c] : 0;
    }
    if (tid == 0) {
        for (int s = 0; s < OzLayout::NBAR; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bars + s)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *sflag = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const int nkc = (2 * d + 63) / 64;
    const unsigned char *abase = aslices + (size_t)((b * 2 + mt) * OZ_KC) * OZ_SLICES * OZ_TILE;
    const unsigned char *xbase = xslices + (size_t)((b * ntile + nt) * OZ_KC) * OZ_SLICES * OZ_XTILE;
    if (tid == 0) {
        // producer: per K chunk kc the six x slice tiles (x buffer kc % 2),
        // then the A slice tiles A_0 .. A_5 of kc through the A ring; a buffer
        // or slot is refilled once the MMAs that read it have completed (their
        // commit on its empty barrier).  With the injected stall the first
        // CTA issues nothing and its MMA thread's wait runs out.
        const bool stall = blockIdx.x == 0 && atomicExch(&g_oz_fault, 0) != 0;
        int ua = 0;
        for (int kc = 0; kc < nkc && !stall; ++kc) {
            if (*(volatile int *)sflag) break;
            const int qx = kc % OZ_NX;
            if (kc >= OZ_NX && !mbar_wait(smem_u32(emptyX + qx), (uint32_t)(((kc / OZ_NX) - 1) & 1))) {
                atomicExch(sflag, 1);
                break;
            }
            const uint32_t fx = smem_u32(fullX + qx);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fx), "r"(OzLayout::XBUF)
                         : "memory");
            for (int j = 0; j < OZ_SLICES; ++j)
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        sbase + OzLayout::XOFF + qx * OzLayout::XBUF + j * OZ_XTILE),
                    "l"(xbase + (size_t)(kc * OZ_SLICES + j) * OZ_XTILE), "r"(OZ_XTILE), "r"(fx)
                    : "memory");
            for (int i = 0; i < OZ_SLICES; ++i, ++ua) {
                const int qa = ua % OZ_NA;
                if (ua >= OZ_NA && !mbar_wait(smem_u32(emptyA + qa), (uint32_t)(((ua / OZ_NA) - 1) & 1))) {
                    atomicExch(sflag, 1);
                    break;
                }
                const uint32_t fa = smem_u32(fullA + qa);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fa), "r"(OZ_TILE)
                             : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        sbase + qa * OZ_TILE),
                    "l"(abase + (size_t)(kc * OZ_SLICES + i) * OZ_TILE), "r"(OZ_TILE), "r"(fa)
                    : "memory");
            }
        }
    } else if (tid == 32) {
        // MMA issuer: for each K chunk and A slice i, the products with x
        // slices j = 0 .. 5 - i into the accumulator of (i, j)
        const uint32_t idesc = idesc_bf16_m128_n64();
        int ua = 0;
        bool ok = true;
        for (int kc = 0; kc < nkc && ok; ++kc) {
            const int qx = kc % OZ_NX;
            if (!mbar_wait(smem_u32(fullX + qx), (uint32_t)((kc / OZ_NX) & 1)) || *(volatile int *)sflag) {
                ok = false;
                break;
            }
            const int kin = min(64, 2 * d - kc * 64);   // reals of this chunk holding data
            const int nks = (kin + 15) / 16;
            uint64_t db[OZ_SLICES];
#pragma unroll
            for (int j = 0; j < OZ_SLICES; ++j)
                db[j] = sw128_desc(sbase + OzLayout::XOFF + qx * OzLayout::XBUF + j * OZ_XTILE);
            for (int i = 0; i < OZ_SLICES; ++i, ++ua) {
                const int qa = ua % OZ_NA;
                if (!mbar_wait(smem_u32(fullA + qa), (uint32_t)((ua / OZ_NA) & 1))) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                mma_slice_rt(i, tmem, OZ_BN, sw128_desc(sbase + qa * OZ_TILE), db, idesc, nks, kc == 0);
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(emptyA + qa))
                             : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(emptyX + qx))
                         : "memory");
        }
        if (!ok) atomicExch(sflag, 1);
        // all MMAs issued so far complete -> done
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(donebar))
                     : "memory");
    }
    __syncwarp();
    const bool done_ok = mbar_wait(smem_u32(donebar), 0u);
    const int bad = __syncthreads_or(!done_ok || *(volatile int *)sflag);
    if (bad) {
        if (tid == 0) {
            atomicExch(&g_oz_status, 1);
            // the MMAs issued before the give-up (committed to done) complete
            // before the tensor memory is freed (bounded again)
            mbar_wait(smem_u32(donebar), 0u);
        }
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int lane = tid & 31;
        const int r = mt * 128 + warp * 32 + lane;            // real row of the leaf block
        const uint32_t tq = tmem + ((uint32_t)(warp * 32) << 16);
        const int er = rowexp[b * 256 + r];
        const float rs1 = pow2f(er / 2), rs2 = pow2f(er - er / 2);   // 2^e_r in two exact factors
        for (int cb = 0; cb < OZ_BN; cb += 16) {
            const int c0 = nt * OZ_BN + cb;
            if (c0 >= nc) break;
            // 2^(f_c - 16) of column c0 + j in two exact factors, held by lane j
            const int fj = (lane < 16 && c0 + lane < nc) ? s_colexp[cb + lane] - 16 : 0;
            const float cs1 = pow2f(fj / 2), cs2 = pow2f(fj - fj / 2);
            uint32_t raw[OZ_ACC][16];
#pragma unroll
            for (int g = 0; g < OZ_ACC; ++g) tmem_ld16_nowait(tq + (uint32_t)(g * OZ_BN + cb), raw[g]);
            // the y entries of this chunk, loaded while the tensor-memory loads land
            float4 ycur[16];
            const bool wr = !(lane & 1) && r < 2 * d;
#pragma unroll
            for (int j = 0; j < 16; ++j)
                ycur[j] = (wr && c0 + j < nc) ? y[o + (r >> 1) + (int64_t)(c0 + j) * ldy] : make_float4(0.f, 0.f, 0.f, 0.f);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float v[OZ_ACC][16];
#pragma unroll
            for (int g = 0; g < OZ_ACC; ++g)
#pragma unroll
                for (int j = 0; j < 16; ++j) v[g][j] = __uint_as_float(raw[g][j]);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int c = c0 + j;
                // float-pair sum of the eight accumulators: the six exact ones
                // (pairs with i + j <= 2) by error-free two-sums, the two
                // rounded ones (i + j >= 3, below 2^-24 of the result) into
                // the low part
                float h = v[0][j], lo = 0.f, e;
#pragma unroll
                for (int g = 1; g < 6; ++g) {
                    two_sum_f(h, v[g][j], h, e);
                    lo += e;
                }
                lo += v[6][j] + v[7][j];
                // scale by 2^(e_r + f_c - 16) in exact power-of-two steps
                const float a1 = __shfl_sync(0xffffffffu, cs1, j), a2 = __shfl_sync(0xffffffffu, cs2, j);
                h = c < nc ? (((h * rs1) * rs2) * a1) * a2 : 0.f;
                lo = c < nc ? (((lo * rs1) * rs2) * a1) * a2 : 0.f;
                const float oh = __shfl_xor_sync(0xffffffffu, h, 1);   // the partner real row
                const float ol = __shfl_xor_sync(0xffffffffu, lo, 1);
                if (wr && c < nc) {
                    float rh, rl, ih, il;
                    ff_add(ycur[j].x, ycur[j].z, h, lo, rh, rl);
                    ff_add(ycur[j].y, ycur[j].w, oh, ol, ih, il);
                    y[o + (r >> 1) + (int64_t)c * ldy] = make_float4(rh, ih, rl, il);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

}  // namespace

namespace {

// ------------------------------------------------------------------ general block products
// The same split for any batch of jobs y[ymap] (+)= op(A_e) x[xmap]
// (leaf blocks, the interpolation blocks T^c and T^cH, the sibling blocks),
// op(A_e) m x k complex with k <= 128 per launch: a persistent kernel, one
// CTA per SM, looping over work items (job, 128-real row tile, 32-column
// tile).  Warp roles: warps 0-3 drain tensor memory (thread t owns row t of
// the tile), warp 4 loads (one thread, cp.async.bulk into a ring of operator
// slice tiles and a ring of vector slice buffers), warp 5 issues the MMAs
// (one thread).  Tensor memory holds two sets of the eight accumulators (32
// columns each), so the MMAs of one item run while the epilogue drains the
// previous one.
constexpr int OZJ_BN = 32;                     // columns per work item
constexpr int OZJ_XTILE = OZJ_BN * 128;        // one 32 x 64 bf16 vector slice tile
constexpr int OZJ_NA = 8;                      // operator slice ring (16 KB slots)
constexpr int OZJ_NX = 3;                      // vector slice buffers (six tiles of one K chunk each)
constexpr int OZJ_THREADS = 192;

struct OzjLayout {
    static constexpr int XBUF = OZ_SLICES * OZJ_XTILE;
    static constexpr int XOFF = OZJ_NA * OZ_TILE;
    static constexpr int RINGS = XOFF + OZJ_NX * XBUF;
    // fullA, emptyA, fullX, emptyX, tfull[2], tempty[2], done
    static constexpr int NBAR = 2 * OZJ_NA + 2 * OZJ_NX + 5;
    static constexpr int TOTAL = RINGS + 1024 + 8 * NBAR + 64;
};

struct OzSrc {
    const cplx *a;   // the stored block
    int lda;
    int op;          // 0: op(A) = A (m x k); 1: op(A) = A^H of the stored k x m block
};

// fp32 accumulator, bf16 A and B, both K-major, M 128, N n
__device__ __forceinline__ uint32_t idesc_bf16_m128(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// operator slices of every job: block j of the grid, its warps over the
// job's nmt * 128 real rows (rows and K positions beyond the job are zero)
__global__ void k_ozj_slice_a(const OzJob *__restrict__ jobs, const OzSrc *__restrict__ src,
                              unsigned char *slices, int *rowexp) {
    const OzJob J = jobs[blockIdx.x];
    const OzSrc S = src[blockIdx.x];
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int K = J.nkc * 64;
    for (int r = threadIdx.x >> 5; r < J.nmt * 128; r += nw) {
        const int i = r >> 1;
        const bool im_row = r & 1, valid = i < J.m;
        double mx = 0.0;
        if (valid)
            for (int l = lane; l < J.k; l += 32) {
                const cplx a = S.op ? S.a[l + (int64_t)i * S.lda] : S.a[i + (int64_t)l * S.lda];
                mx = fmax(mx, fmax(fabs(a.x), fabs(a.y)));
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        int e = 0;
        if (mx > 0.0) frexp(mx, &e);
        if (lane == 0) rowexp[J.rexp + r] = e;
        const int mt = r >> 7, rr = r & 127;
        for (int kk = lane; kk < K; kk += 32) {
            const int l = kk >> 1;
            double v = 0.0;
            if (valid && l < J.k) {
                cplx a = S.op ? S.a[l + (int64_t)i * S.lda] : S.a[i + (int64_t)l * S.lda];
                if (S.op) a.y = -a.y;
                v = !im_row ? ((kk & 1) ? -a.y : a.x) : ((kk & 1) ? a.x : a.y);
            }
            unsigned short s[OZ_SLICES];
            cut6_bits(v, e, s);
            unsigned char *t = slices + (size_t)(J.a_tile + (int64_t)(mt * J.nkc + (kk >> 6)) * OZ_SLICES) * OZ_TILE;
            const uint32_t off = sw_elem(rr, kk & 63);
#pragma unroll
            for (int q = 0; q < OZ_SLICES; ++q)
                *reinterpret_cast<unsigned short *>(t + (size_t)q * OZ_TILE + off) = s[q];
        }
    }
}

// vector slices of every job for this application: block (j, 8-column
// group), one warp per column; the job's rows of x are gathered through its
// map; colexp[j * cols + c] receives the column's exponent
__global__ void k_ozj_slice_x(const OzJob *__restrict__ jobs, const int *__restrict__ maps,
                              const float4 *__restrict__ x, int64_t ldx, int nc, int ntile,
                              unsigned char *slices, int *colexp) {
    const int jb = blockIdx.x;
    const OzJob J = jobs[jb];
    const int lane = threadIdx.x & 31;
    const int cols = ntile * OZJ_BN;
    const int c = blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= cols) return;
    const bool live = c < nc;
    float m = 0.f;
    if (live)
        for (int l = lane; l < J.k; l += 32) {
            const int64_t row = J.x_row + (J.xmap >= 0 ? maps[J.xmap + l] : l);
            const float4 v = x[row + (int64_t)c * ldx];
            m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
        }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, s));
    int e = 0;
    if (m > 0.f) {
        frexpf(m, &e);
        if (m >= ldexpf(1.0f - 1.0f / (1 << 20), e)) ++e;
    }
    if (lane == 0) colexp[(int64_t)jb * cols + c] = e;
    const int nt = c / OZJ_BN, n = c % OZJ_BN;
    const int K = J.nkc * 64;
    for (int kk = lane; kk < K; kk += 32) {
        const int l = kk >> 1;
        float h = 0.f, lo = 0.f;
        if (live && l < J.k) {
            const float4 q = x[J.x_row + (J.xmap >= 0 ? maps[J.xmap + l] : l) + (int64_t)c * ldx];
            h = (kk & 1) ? q.y : q.x;
            lo = (kk & 1) ? q.w : q.z;
        }
        unsigned short s[OZ_SLICES];
        cut6_pair(h, lo, e, s);
        unsigned char *t =
            slices + (size_t)((J.x_tile * ntile + (int64_t)nt * J.nkc + (kk >> 6)) * OZ_SLICES) * OZJ_XTILE;
        const uint32_t off = sw_elem(n, kk & 63);
#pragma unroll
        for (int q = 0; q < OZ_SLICES; ++q)
            *reinterpret_cast<unsigned short *>(t + (size_t)q * OZJ_XTILE + off) = s[q];
    }
}

}  // namespace

__device__ int g_ozj_status;   // 1 once a general block product gave up waiting
__device__ int g_ozj_fault;    // injected fault: the next launch's first CTA issues no copies

namespace {

__global__ void __launch_bounds__(OZJ_THREADS, 1)
    k_ozj(const OzJob *__restrict__ jobs, const int2 *__restrict__ tiles, int nitems, int ntile,
          const int *__restrict__ maps, const unsigned char *__restrict__ aslices, const int *__restrict__ rowexp,
          const unsigned char *__restrict__ xslices, const int *__restrict__ colexp, float4 *y, int64_t ldy,
          int nc) {
    extern __shared__ unsigned char ozj_raw[];
    const uint32_t raw = smem_u32(ozj_raw);
    const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
    const uint32_t sbase = raw + pad;
    uint64_t *bars = reinterpret_cast<uint64_t *>(ozj_raw + pad + OzjLayout::RINGS);
    uint64_t *fullA = bars, *emptyA = bars + OZJ_NA, *fullX = bars + 2 * OZJ_NA, *emptyX = fullX + OZJ_NX;
    uint64_t *tfull = emptyX + OZJ_NX, *tempty = tfull + 2, *donebar = tempty + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + OzjLayout::NBAR);
    int *sflag = reinterpret_cast<int *>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cols = ntile * OZJ_BN;
    if (tid == 0) {
        for (int q = 0; q < OzjLayout::NBAR; ++q) {
            // tempty: one arrival per epilogue warp; the others: one arrival (+ bytes)
            const int cnt = (q == 2 * OZJ_NA + 2 * OZJ_NX + 2 || q == 2 * OZJ_NA + 2 * OZJ_NX + 3) ? 4 : 1;
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bars + q)), "r"(cnt));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *sflag = 0;
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    if (warp == 4) {
        if (lane == 0) {
            // producer: per item and K chunk, the six vector slice tiles into
            // a buffer, then the operator slice tiles A_0 .. A_5 through the ring
            const bool stall = blockIdx.x == 0 && atomicExch(&g_ozj_fault, 0) != 0;
            int ua = 0, ux = 0;
            int2 tl = blockIdx.x < nitems ? tiles[blockIdx.x / ntile] : make_int2(0, 0);
            OzJob J = jobs[tl.x];
            for (int it = blockIdx.x; it < nitems && !stall; it += gridDim.x) {
                const int nt = it % ntile;
                // the next item's tile, loaded while this item's copies are issued
                const int itn = it + gridDim.x;
                const int2 tln = itn < nitems ? tiles[itn / ntile] : tl;
                const unsigned char *ab = aslices + (size_t)(J.a_tile + (int64_t)tl.y * J.nkc * OZ_SLICES) * OZ_TILE;
                const unsigned char *xb =
                    xslices + (size_t)((J.x_tile * ntile + (int64_t)nt * J.nkc) * OZ_SLICES) * OZJ_XTILE;
                bool ok = true;
                for (int kc = 0; kc < J.nkc && ok; ++kc) {
                    if (*(volatile int *)sflag) { ok = false; break; }
                    const int qx = ux % OZJ_NX;
                    if (ux >= OZJ_NX && !mbar_wait(smem_u32(emptyX + qx), (uint32_t)(((ux / OZJ_NX) - 1) & 1))) {
                        ok = false;
                        break;
                    }
                    const uint32_t fx = smem_u32(fullX + qx);
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fx),
                                 "r"(OzjLayout::XBUF)
                                 : "memory");
                    for (int j = 0; j < OZ_SLICES; ++j)
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
                            "[%3];" ::"r"(sbase + OzjLayout::XOFF + qx * OzjLayout::XBUF + j * OZJ_XTILE),
                            "l"(xb + (size_t)(kc * OZ_SLICES + j) * OZJ_XTILE), "r"(OZJ_XTILE), "r"(fx)
                            : "memory");
                    ++ux;
                    for (int i = 0; i < OZ_SLICES; ++i) {
                        const int qa = ua % OZJ_NA;
                        if (ua >= OZJ_NA && !mbar_wait(smem_u32(emptyA + qa), (uint32_t)(((ua / OZJ_NA) - 1) & 1))) {
                            ok = false;
                            break;
                        }
                        const uint32_t fa = smem_u32(fullA + qa);
                        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fa), "r"(OZ_TILE)
                                     : "memory");
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
                            "[%3];" ::"r"(sbase + qa * OZ_TILE),
                            "l"(ab + (size_t)(kc * OZ_SLICES + i) * OZ_TILE), "r"(OZ_TILE), "r"(fa)
                            : "memory");
                        ++ua;
                    }
                }
                if (!ok) {
                    atomicExch(sflag, 1);
                    break;
                }
                tl = tln;
                J = jobs[tl.x];
            }
            // every copy issued has landed before the CTA may exit (bounded)
            for (int q = 0; q < OZJ_NA && q < ua; ++q) {
                const int last = q + ((ua - 1 - q) / OZJ_NA) * OZJ_NA;   // last use of slot q
                mbar_wait(smem_u32(fullA + q), (uint32_t)((last / OZJ_NA) & 1));
            }
            for (int q = 0; q < OZJ_NX && q < ux; ++q) {
                const int last = q + ((ux - 1 - q) / OZJ_NX) * OZJ_NX;
                mbar_wait(smem_u32(fullX + q), (uint32_t)((last / OZJ_NX) & 1));
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {
            // MMA issuer: item it accumulates into tensor-memory set it % 2
            // once the epilogue has drained that set's previous item
            const uint32_t idesc = idesc_bf16_m128(OZJ_BN);
            int ua = 0, ux = 0, n = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x, ++n) {
                const OzJob J = jobs[tiles[it / ntile].x];
                const int tb = n & 1;
                if (n >= 2 && !mbar_wait(smem_u32(tempty + tb), (uint32_t)(((n >> 1) - 1) & 1))) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t tacc = tmem + (uint32_t)(tb * OZ_ACC * OZJ_BN);
                for (int kc = 0; kc < J.nkc && ok; ++kc) {
                    const int qx = ux % OZJ_NX;
                    if (!mbar_wait(smem_u32(fullX + qx), (uint32_t)((ux / OZJ_NX) & 1)) || *(volatile int *)sflag) {
                        ok = false;
                        break;
                    }
                    // k-steps of 16 reals holding data (one zero step for a job without columns)
                    const int kin = min(64, 2 * J.k - kc * 64);
                    const int nks = max(1, (kin + 15) / 16);
                    uint64_t db[OZ_SLICES];
#pragma unroll
                    for (int j = 0; j < OZ_SLICES; ++j)
                        db[j] = sw128_desc(sbase + OzjLayout::XOFF + qx * OzjLayout::XBUF + j * OZJ_XTILE);
                    for (int i = 0; i < OZ_SLICES; ++i) {
                        const int qa = ua % OZJ_NA;
                        if (!mbar_wait(smem_u32(fullA + qa), (uint32_t)((ua / OZJ_NA) & 1))) {
                            ok = false;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        mma_slice_rt(i, tacc, OZJ_BN, sw128_desc(sbase + qa * OZ_TILE), db, idesc, nks, kc == 0);
                        asm volatile(
                            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                smem_u32(emptyA + qa))
                            : "memory");
                        ++ua;
                    }
                    if (!ok) break;
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(emptyX + qx))
                                 : "memory");
                    ++ux;
                }
                if (!ok) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(tfull + tb))
                             : "memory");
            }
            if (!ok) atomicExch(sflag, 1);
            // all MMAs issued have completed before the tensor memory is freed (bounded)
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(donebar))
                         : "memory");
            mbar_wait(smem_u32(donebar), 0u);
        }
    } else {
        // epilogue: thread t owns real row t of the item's row tile
        int n = 0;
        for (int it = blockIdx.x; it < nitems; it += gridDim.x, ++n) {
            const int tb = n & 1;
            // the item's description, loaded while its MMAs run
            const int2 tl = tiles[it / ntile];
            const int nt = it % ntile;
            const OzJob J = jobs[tl.x];
            const int r = tl.y * 128 + warp * 32 + lane;   // real row of op(A_e)
            const bool valid = r < 2 * J.m;
            const bool live = __any_sync(0xffffffffu, valid);   // the warp holds rows of the job
            const int er = rowexp[J.rexp + r];
            const int64_t yr = valid ? J.y_row + (J.ymap >= 0 ? maps[J.ymap + (r >> 1)] : (r >> 1)) : 0;
            const bool set = J.flags & 1;
            const float rs1 = pow2f(er / 2), rs2 = pow2f(er - er / 2);   // 2^e_r in two exact factors
            const int *ce = colexp + (int64_t)tl.x * cols;
            bool ok = mbar_wait(smem_u32(tfull + tb), (uint32_t)((n >> 1) & 1)) && !*(volatile int *)sflag;
            ok = __all_sync(0xffffffffu, ok);   // the warp leaves together (its loads and shuffles are warp-wide)
            if (!ok) {
                if (lane == 0) atomicExch(sflag, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t tq = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(tb * OZ_ACC * OZJ_BN);
            for (int cb = 0; cb < OZJ_BN; cb += 16) {
                const int c0 = nt * OZJ_BN + cb;
                // 2^(f_c - 16) of column c0 + j in two exact factors, held by lane j
                const int fj = (lane < 16 && c0 + lane < nc) ? ce[c0 + lane] - 16 : 0;
                const float cs1 = pow2f(fj / 2), cs2 = pow2f(fj - fj / 2);
                uint32_t rw[OZ_ACC][16];
                float4 ycur[16];
                const bool wr = !(lane & 1) && valid;
                if (live) {
#pragma unroll
                    for (int g = 0; g < OZ_ACC; ++g) tmem_ld16_nowait(tq + (uint32_t)(g * OZJ_BN + cb), rw[g]);
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        ycur[j] = (wr && !set && c0 + j < nc) ? y[yr + (int64_t)(c0 + j) * ldy]
                                                              : make_float4(0.f, 0.f, 0.f, 0.f);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                }
                if (cb + 16 == OZJ_BN) {
                    // the set is in registers: hand it back to the MMA issuer
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0)
                        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(tempty + tb))
                                     : "memory");
                }
                if (!live) continue;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int c = c0 + j;
                    float h = __uint_as_float(rw[0][j]), lo = 0.f, e;
#pragma unroll
                    for (int g = 1; g < 6; ++g) {
                        two_sum_f(h, __uint_as_float(rw[g][j]), h, e);
                        lo += e;
                    }
                    lo += __uint_as_float(rw[6][j]) + __uint_as_float(rw[7][j]);
                    const float a1 = __shfl_sync(0xffffffffu, cs1, j), a2 = __shfl_sync(0xffffffffu, cs2, j);
                    h = (((h * rs1) * rs2) * a1) * a2;
                    lo = (((lo * rs1) * rs2) * a1) * a2;
                    const float oh = __shfl_xor_sync(0xffffffffu, h, 1);   // the partner real row
                    const float ol = __shfl_xor_sync(0xffffffffu, lo, 1);
                    if (wr && c < nc) {
                        float rh, rl, ih, il;
                        ff_add(ycur[j].x, ycur[j].z, h, lo, rh, rl);
                        ff_add(ycur[j].y, ycur[j].w, oh, ol, ih, il);
                        y[yr + (int64_t)c * ldy] = make_float4(rh, ih, rl, il);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0 && *(volatile int *)sflag) atomicExch(&g_ozj_status, 1);
    if (warp == 4) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            n = v;
        else
            n = 1;
    }
    return n;
}

}  // namespace

int oz_plan_build(const std::vector<OzSpec> &specs, std::vector<OzPlan> &passes, cudaStream_t s) {
    passes.clear();
    int maxk = 0;
    for (const OzSpec &q : specs) {
        if (q.m < 0 || q.k < 0 || (q.m > 0 && !q.a && q.k > 0)) return FDS_ERR_ARG;
        maxk = std::max(maxk, q.k);
    }
    const int npass = std::max(1, (maxk + 127) / 128);
    for (int p = 0; p < npass; ++p) {
        std::vector<OzJob> jobs;
        std::vector<int2> tiles;
        std::vector<int> maps;
        std::vector<OzSrc> src;
        int64_t atile = 0, xg = 0, rexp = 0;
        double fl = 0;
        for (const OzSpec &q : specs) {
            const int k0 = 128 * p;
            if (q.m == 0 || (p > 0 && k0 >= q.k)) continue;
            const int kp = std::max(0, std::min(128, q.k - k0));
            if (kp == 0 && !q.set) continue;   // nothing to add
            OzJob J;
            J.m = q.m;
            J.k = kp;
            J.nmt = (2 * q.m + 127) / 128;
            J.nkc = std::max(1, (2 * kp + 63) / 64);
            J.a_tile = atile;
            atile += (int64_t)J.nmt * J.nkc * OZ_SLICES;
            J.x_tile = xg;
            xg += J.nkc;
            J.rexp = (int32_t)rexp;
            rexp += (int64_t)J.nmt * 128;
            J.x_row = q.x_row + (q.xmap ? 0 : k0);
            J.xmap = -1;
            if (q.xmap && kp > 0) {
                J.xmap = (int32_t)maps.size();
                maps.insert(maps.end(), q.xmap + k0, q.xmap + k0 + kp);
            }
            J.y_row = q.y_row;
            J.ymap = -1;
            if (q.ymap) {
                J.ymap = (int32_t)maps.size();
                maps.insert(maps.end(), q.ymap, q.ymap + q.m);
            }
            J.flags = (q.set && p == 0) ? 1 : 0;
            OzSrc S;
            S.a = q.a ? (q.op ? q.a + k0 : q.a + (int64_t)k0 * q.lda) : nullptr;
            S.lda = q.lda;
            S.op = q.op;
            for (int mt = 0; mt < J.nmt; ++mt) tiles.push_back(make_int2((int)jobs.size(), mt));
            jobs.push_back(J);
            src.push_back(S);
            fl += 8.0 * q.m * kp;
        }
        if (jobs.empty()) continue;
        if (rexp > 2147483647LL || maps.size() > 2147483647ULL || jobs.size() > 2147483647ULL) return FDS_ERR_ARG;
        OzPlan P;
        P.njobs = (int)jobs.size();
        P.ntiles = (int)tiles.size();
        P.xgroups = xg;
        P.flops = fl;
        if (maps.empty()) maps.push_back(0);
        FDS_TRY(P.jobs.upload(jobs, s));
        FDS_TRY(P.tiles.upload(tiles, s));
        FDS_TRY(P.maps.upload(maps, s));
        FDS_TRY(P.aslices.alloc((size_t)atile * OZ_TILE));
        FDS_TRY(P.rowexp.alloc((size_t)rexp));
        DBuf<OzSrc> d_src;
        FDS_TRY(d_src.upload(src, s));
        fds_count_launch(), k_ozj_slice_a<<<P.njobs, 256, 0, s>>>(P.jobs.p, d_src.p, P.aslices.p, P.rowexp.p);
        FDS_CUDA_TRY(cudaGetLastError());
        FDS_CUDA_TRY(cudaStreamSynchronize(s));   // d_src is freed on return
        passes.push_back(std::move(P));
    }
    return FDS_OK;
}

int oz_plan_apply(fds_handle *h, const std::vector<OzPlan> &passes, const float4 *x, int64_t ldx, float4 *y,
                  int64_t ldy, int nc, cudaStream_t s) {
    if (nc <= 0) return FDS_OK;
    const int ntile = (nc + OZJ_BN - 1) / OZJ_BN;
    const int cols = ntile * OZJ_BN;
    if (cols / 8 > 65535) return FDS_ERR_ARG;
    for (const OzPlan &P : passes) {
        const size_t xs = (size_t)P.xgroups * ntile * OZ_SLICES * OZJ_XTILE;
        if (h->oz_x.n < xs) FDS_TRY(h->oz_x.alloc(xs));
        if (h->oz_colexp.n < (size_t)P.njobs * cols) FDS_TRY(h->oz_colexp.alloc((size_t)P.njobs * cols));
        fds_count_launch(), k_ozj_slice_x<<<dim3(P.njobs, cols / 8), 256, 0, s>>>(
            P.jobs.p, P.maps.p, x, ldx, nc, ntile, h->oz_x.p, h->oz_colexp.p);
        FDS_CUDA_TRY(cudaGetLastError());
        const int64_t items = (int64_t)P.ntiles * ntile;
        if (items > 2147483647LL) return FDS_ERR_ARG;
        constexpr int smem = OzjLayout::TOTAL;
        FDS_TRY(ensure_dyn_smem(k_ozj, smem));
        const int grid = (int)std::min<int64_t>(items, sm_count());
        fds_count_launch(), k_ozj<<<grid, OZJ_THREADS, smem, s>>>(P.jobs.p, P.tiles.p, (int)items, ntile, P.maps.p,
                                                                  P.aslices.p, P.rowexp.p, h->oz_x.p,
                                                                  h->oz_colexp.p, y, ldy, nc);
        FDS_CUDA_TRY(cudaGetLastError());
    }
    return FDS_OK;
}

int ozj_status_take(cudaStream_t s, int *status) {
    int v = 0, zero = 0;
    FDS_CUDA_TRY(cudaMemcpyFromSymbolAsync(&v, g_ozj_status, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    FDS_CUDA_TRY(cudaStreamSynchronize(s));
    if (v) FDS_CUDA_TRY(cudaMemcpyToSymbolAsync(g_ozj_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
    *status = v;
    return FDS_OK;
}

int ozj_fault_arm(int on) {
    const int v = on ? 1 : 0;
    FDS_CUDA_TRY(cudaMemcpyToSymbol(g_ozj_fault, &v, sizeof(int)));
    return FDS_OK;
}

namespace {

int oz_slice_blocks(int nb, const MatRef *d_blocks, DBuf<unsigned char> &aslices, DBuf<int> &rowexp,
                    cudaStream_t s) {
    FDS_TRY(aslices.alloc((size_t)nb * 2 * OZ_KC * OZ_SLICES * OZ_TILE));
    FDS_TRY(rowexp.alloc((size_t)nb * 256));
    const int64_t warps = (int64_t)nb * 256;
    fds_count_launch(), k_oz_slice_a<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(nb, d_blocks, aslices.p,
                                                                                         rowexp.p);
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}

int oz_apply(int nb, const int64_t *d_doff, const unsigned char *aslices, const int *rowexp,
             DBuf<unsigned char> &xs, DBuf<int> &colexp, const float4 *x, float4 *y, int64_t ld, int nc,
             cudaStream_t s) {
    if (nb == 0 || nc == 0) return FDS_OK;
    const int ntile = (nc + OZ_BN - 1) / OZ_BN;
    const size_t need = (size_t)nb * ntile * OZ_KC * OZ_SLICES * OZ_XTILE;
    if (xs.n < need) FDS_TRY(xs.alloc(need));
    if (colexp.n < (size_t)nb * ntile * OZ_BN) FDS_TRY(colexp.alloc((size_t)nb * ntile * OZ_BN));
    const int64_t warps = (int64_t)nb * ntile * OZ_BN;
    fds_count_launch(), k_oz_slice_x<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(nb, d_doff, x, ld, nc,
                                                                                          ntile, xs.p, colexp.p);
    FDS_CUDA_TRY(cudaGetLastError());
    constexpr int smem = OzLayout::TOTAL;
    FDS_TRY(ensure_dyn_smem(k_oz_leaf, smem));
    const int64_t tiles = (int64_t)nb * 2 * ntile;
    if (tiles > 2147483647) return FDS_ERR_ARG;
    fds_count_launch(), k_oz_leaf<<<(unsigned)tiles, OZ_THREADS, smem, s>>>(nb, ntile, d_doff, aslices, rowexp,
                                                                            xs.p, colexp.p, y, ld, nc);
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}

// complex128 <-> float pairs
__global__ void k_oz_to_pairs(const cplx *__restrict__ a, float4 *b, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const cplx v = a[e];
        const float rh = (float)v.x, ih = (float)v.y;
        b[e] = make_float4(rh, ih, (float)(v.x - (double)rh), (float)(v.y - (double)ih));
    }
}
__global__ void k_oz_from_pairs(const float4 *__restrict__ a, cplx *b, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = a[e];
        b[e] = mkc((double)v.x + v.z, (double)v.y + v.w);
    }
}

__global__ void k_oz_block_refs(int nb, cplx *A, const int64_t *__restrict__ aoff, const int64_t *__restrict__ doff,
                                MatRef *out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int d = (int)(doff[b + 1] - doff[b]);
    out[b].p = A + aoff[b];
    out[b].rows = out[b].cols = d;
    out[b].ld = d > 1 ? d : 1;
}

}  // namespace

int oz_leaf_prepare(Level &C, const MatRef *d_blocks, cudaStream_t s) {
    for (int b = 0; b < C.nb; ++b)
        if (C.n1[b] + C.n2[b] > 128) return FDS_ERR_ARG;
    return oz_slice_blocks(C.nb, d_blocks, C.oz_a, C.oz_rowexp, s);
}

int oz_leaf_apply(fds_handle *h, Level &C, const float4 *x, float4 *y, int64_t ld, int nc, cudaStream_t s) {
    return oz_apply(C.nb, C.d_doff.p, C.oz_a.p, C.oz_rowexp.p, h->oz_x, h->oz_colexp, x, y, ld, nc, s);
}

extern "C" int fds_zgemm_blocks_tc(int32_t batch, const int32_t *d, const double *d_A, const double *d_X,
                                   double *d_Y, int32_t nc, uint64_t stream) {
    if (batch < 0 || nc < 0) return FDS_ERR_ARG;
    if (batch == 0 || nc == 0) return FDS_OK;
    if (!d || !d_A || !d_X || !d_Y) return FDS_ERR_ARG;
    std::vector<int64_t> doff(batch + 1, 0), aoff(batch + 1, 0);
    for (int b = 0; b < batch; ++b) {
        if (d[b] < 1 || d[b] > 128) return FDS_ERR_ARG;
        doff[b + 1] = doff[b] + d[b];
        aoff[b + 1] = aoff[b] + (int64_t)d[b] * d[b];
    }
    const int64_t D = doff[batch];
    if ((int64_t)batch * 2 * ((nc + OZ_BN - 1) / OZ_BN) > 2147483647) return FDS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    FDS_TRY(ensure_gauss_tables());
    DBuf<int64_t> d_doff, d_aoff;
    DBuf<MatRef> refs;
    DBuf<float4> xp, yp;
    DBuf<unsigned char> as, xs;
    DBuf<int> rowexp, colexp;
    FDS_TRY(d_doff.upload(doff, s));
    FDS_TRY(d_aoff.upload(aoff, s));
    FDS_TRY(refs.alloc(batch));
    fds_count_launch(), k_oz_block_refs<<<(batch + 127) / 128, 128, 0, s>>>(batch, (cplx *)d_A, d_aoff.p, d_doff.p,
                                                                            refs.p);
    FDS_CUDA_TRY(cudaGetLastError());
    FDS_TRY(xp.alloc((size_t)D * nc));
    FDS_TRY(yp.alloc((size_t)D * nc));
    fds_count_launch(), k_oz_to_pairs<<<1024, 256, 0, s>>>((const cplx *)d_X, xp.p, D * nc);
    fds_count_launch(), k_oz_to_pairs<<<1024, 256, 0, s>>>((const cplx *)d_Y, yp.p, D * nc);
    FDS_CUDA_TRY(cudaGetLastError());
    FDS_TRY(oz_slice_blocks(batch, refs.p, as, rowexp, s));
    FDS_TRY(oz_apply(batch, d_doff.p, as.p, rowexp.p, xs, colexp, xp.p, yp.p, D, nc, s));
    fds_count_launch(), k_oz_from_pairs<<<1024, 256, 0, s>>>(yp.p, (cplx *)d_Y, D * nc);
    FDS_CUDA_TRY(cudaGetLastError());
    FDS_CUDA_TRY(cudaStreamSynchronize(s));
    int st = 0;
    FDS_TRY(oz_status_take(s, &st));
    return st ? FDS_ERR_TIMEOUT : FDS_OK;
}

extern "C" int fds_zgemm_jobs_tc(int32_t njobs, const int32_t *m, const int32_t *k, const int32_t *op,
                                 const int64_t *a_off, const int32_t *lda, const int64_t *x_row,
                                 const int64_t *xmap_off, const int64_t *y_row, const int64_t *ymap_off,
                                 const int32_t *set, const int32_t *maps, const double *d_A, const double *d_X,
                                 int64_t ldx, double *d_Y, int64_t ldy, int32_t nc, uint64_t stream) {
    if (njobs < 0 || nc < 0 || ldx < 1 || ldy < 1) return FDS_ERR_ARG;
    if (njobs == 0 || nc == 0) return FDS_OK;
    if (!m || !k || !op || !a_off || !lda || !x_row || !xmap_off || !y_row || !ymap_off || !set || !d_A || !d_X ||
        !d_Y)
        return FDS_ERR_ARG;
    std::vector<OzSpec> specs(njobs);
    for (int e = 0; e < njobs; ++e) {
        if (m[e] < 0 || k[e] < 0 || (op[e] != 0 && op[e] != 1) || lda[e] < std::max(1, op[e] ? k[e] : m[e]) ||
            a_off[e] < 0 || x_row[e] < 0 || y_row[e] < 0 || ((xmap_off[e] >= 0 || ymap_off[e] >= 0) && !maps))
            return FDS_ERR_ARG;
        OzSpec &q = specs[e];
        q.a = reinterpret_cast<const cplx *>(d_A) + a_off[e];
        q.lda = lda[e];
        q.op = op[e];
        q.m = m[e];
        q.k = k[e];
        q.x_row = x_row[e];
        q.y_row = y_row[e];
        q.xmap = xmap_off[e] >= 0 ? maps + xmap_off[e] : nullptr;
        q.ymap = ymap_off[e] >= 0 ? maps + ymap_off[e] : nullptr;
        q.set = set[e] != 0;
        // every row addressed stays inside X and Y
        for (int l = 0; l < q.k; ++l) {
            const int64_t r = q.x_row + (q.xmap ? q.xmap[l] : l);
            if (r < 0 || r >= ldx) return FDS_ERR_ARG;
        }
        for (int i = 0; i < q.m; ++i) {
            const int64_t r = q.y_row + (q.ymap ? q.ymap[i] : i);
            if (r < 0 || r >= ldy) return FDS_ERR_ARG;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    fds_handle h;   // workspace holder for the vector slices
    std::vector<OzPlan> passes;
    FDS_TRY(oz_plan_build(specs, passes, s));
    DBuf<float4> xp, yp;
    FDS_TRY(xp.alloc((size_t)ldx * nc));
    FDS_TRY(yp.alloc((size_t)ldy * nc));
    fds_count_launch(), k_oz_to_pairs<<<1024, 256, 0, s>>>((const cplx *)d_X, xp.p, ldx * nc);
    fds_count_launch(), k_oz_to_pairs<<<1024, 256, 0, s>>>((const cplx *)d_Y, yp.p, ldy * nc);
    FDS_CUDA_TRY(cudaGetLastError());
    FDS_TRY(oz_plan_apply(&h, passes, xp.p, ldx, yp.p, ldy, nc, s));
    fds_count_launch(), k_oz_from_pairs<<<1024, 256, 0, s>>>(yp.p, (cplx *)d_Y, ldy * nc);
    FDS_CUDA_TRY(cudaGetLastError());
    FDS_CUDA_TRY(cudaStreamSynchronize(s));
    int st = 0;
    FDS_TRY(ozj_status_take(s, &st));
    return st ? FDS_ERR_TIMEOUT : FDS_OK;
}

int oz_status_take(cudaStream_t s, int *status) {
    int v = 0, zero = 0;
    FDS_CUDA_TRY(cudaMemcpyFromSymbolAsync(&v, g_oz_status, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    FDS_CUDA_TRY(cudaStreamSynchronize(s));
    if (v) FDS_CUDA_TRY(cudaMemcpyToSymbolAsync(g_oz_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
    *status = v;
    return FDS_OK;
}

int oz_fault_arm(int on) {
    // both tensor-core product kernels (leaf-block stage entry, general plans)
    const int v = on ? 1 : 0;
    FDS_CUDA_TRY(cudaMemcpyToSymbol(g_oz_fault, &v, sizeof(int)));
    return ozj_fault_arm(on);
}
