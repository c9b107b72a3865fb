// Shared device/host helpers of the GB300 fast direct solver (complex128
// arithmetic on double2, launch checks, Gauss–Legendre tables).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <mutex>

#include "../../include/fds.h"

#ifndef FDS_PI
#define FDS_PI 3.14159265358979323846
#endif

typedef double2 cplx;

__host__ __device__ __forceinline__ cplx mkc(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ cplx cadd(cplx a, cplx b) { return mkc(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ cplx csub(cplx a, cplx b) { return mkc(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ cplx cmul(cplx a, cplx b) {
    return mkc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__host__ __device__ __forceinline__ cplx cmulc(cplx a, cplx b) {
    return mkc(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__host__ __device__ __forceinline__ cplx cconj(cplx a) { return mkc(a.x, -a.y); }
__host__ __device__ __forceinline__ cplx cscale(cplx a, double s) { return mkc(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double cabs2(cplx a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ cplx cneg(cplx a) { return mkc(-a.x, -a.y); }
// acc += a * b
__host__ __device__ __forceinline__ void cfma(cplx &acc, cplx a, cplx b) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
// acc -= a * b
__host__ __device__ __forceinline__ void cfms(cplx &acc, cplx a, cplx b) {
    acc.x = fma(-a.x, b.x, fma(a.y, b.y, acc.x));
    acc.y = fma(-a.x, b.y, fma(-a.y, b.x, acc.y));
}
__host__ __device__ __forceinline__ cplx cinv(cplx a) {
    double d = 1.0 / cabs2(a);
    return mkc(a.x * d, -a.y * d);
}
__host__ __device__ __forceinline__ cplx cdiv(cplx a, cplx b) { return cmul(a, cinv(b)); }

// complex64 (float2) counterparts for the mixed-precision sweep
typedef float2 cplxf;
__host__ __device__ __forceinline__ cplxf mkcf(float r, float i) { return make_float2(r, i); }
__host__ __device__ __forceinline__ cplxf cadd(cplxf a, cplxf b) { return mkcf(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ cplxf csub(cplxf a, cplxf b) { return mkcf(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ cplxf cmul(cplxf a, cplxf b) {
    return mkcf(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ cplxf cconj(cplxf a) { return mkcf(a.x, -a.y); }
__host__ __device__ __forceinline__ float cabs2(cplxf a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ void cfma(cplxf &acc, cplxf a, cplxf b) {
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}
__host__ __device__ __forceinline__ void cfms(cplxf &acc, cplxf a, cplxf b) {
    acc.x = fmaf(-a.x, b.x, fmaf(a.y, b.y, acc.x));
    acc.y = fmaf(-a.x, b.y, fmaf(-a.y, b.x, acc.y));
}
__host__ __device__ __forceinline__ cplxf cinv(cplxf a) {
    float d = 1.0f / cabs2(a);
    return mkcf(a.x * d, -a.y * d);
}
template <class C> __host__ __device__ __forceinline__ C czero();
template <> __host__ __device__ __forceinline__ cplx czero<cplx>() { return mkc(0.0, 0.0); }
template <> __host__ __device__ __forceinline__ cplxf czero<cplxf>() { return mkcf(0.f, 0.f); }
template <> __host__ __device__ __forceinline__ float4 czero<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
__host__ __device__ __forceinline__ cplxf to_c64(cplx a) { return mkcf((float)a.x, (float)a.y); }
__host__ __device__ __forceinline__ cplx to_c128(cplxf a) { return mkc((double)a.x, (double)a.y); }

// Physical constants prepared on the host for one problem.
struct PhysDev {
    double lam, mu, rho, omega;
    double kT, kL;
    double rw2;        // rho omega^2
    double c2;         // 2 / kT^2
    double lhalfT, lhalfL;   // ln(kT/2), ln(kL/2)
    cplx alpha;        // Burton–Miller coupling
    cplx alpha_rw2;    // alpha rho omega^2
    cplx alpha_m2mu;   // -2 mu alpha
};

PhysDev make_physdev(const fds_physics *ph);

// Gauss–Legendre tables on [0,1] for the orders the quadrature rules use.
// Index q holds q nodes; only q in {1..8, 16, 20} are filled.
#define GL_MAXQ 20
#define SER_TERMS 14
struct GaussTables {
    double x[GL_MAXQ + 1][GL_MAXQ];
    double w[GL_MAXQ + 1][GL_MAXQ];
    // ascending-series coefficients of the Bessel functions (see kernel_eval.cuh)
    double sa[SER_TERMS], sb[SER_TERMS], sh[SER_TERMS], sp[SER_TERMS];
};
// Each translation unit that evaluates quadrature owns a copy of the table
// (whole-program compilation, no relocatable device code) and uploads it with
// its own ensure_gauss_tables() before the first launch.
static __constant__ GaussTables c_gauss;
int gauss_tables_host(GaussTables *T);   // fills the host copy (kernel_eval.cu)

// Records the failing CUDA call of this thread (fds_last_error_detail).
void fds_note_cuda_error(cudaError_t e, const char *file, int line);
void fds_set_error_detail(const char *msg);
extern "C" const char *fds_last_error_detail(void);

#define FDS_CUDA_TRY(expr)                                                   \
    do {                                                                     \
        cudaError_t _e = (expr);                                             \
        if (_e != cudaSuccess) {                                             \
            fds_note_cuda_error(_e, __FILE__, __LINE__);                     \
            return (_e == cudaErrorMemoryAllocation) ? FDS_ERR_OOM : FDS_ERR_CUDA; \
        }                                                                    \
    } while (0)

#define FDS_TRY(expr)                \
    do {                             \
        int _r = (expr);             \
        if (_r != FDS_OK) return _r; \
    } while (0)

// Counts kernel launches of this library (fds_launch_count).
void fds_count_launch();

// Bounds checks of the index-mapped gathers and scatters.  In a library built
// with -DFDS_CHECKS, FDS_IN_RANGE(i, n) is false for i outside [0, n), counts
// the miss in a device word of this translation unit, and the caller skips
// the access; fds_bounds_violations() reads and clears every unit's word.
// Without the flag it is the constant true.
int fds_bounds_register(unsigned long long (*take)());
#ifdef FDS_CHECKS
static __device__ unsigned long long g_bounds_miss;
__device__ __forceinline__ bool fds_in_range(long long i, long long n) {
    if (i >= 0 && i < n) return true;
    atomicAdd(&g_bounds_miss, 1ull);
    return false;
}
#define FDS_IN_RANGE(i, n) fds_in_range((long long)(i), (long long)(n))
namespace {
unsigned long long bounds_take_unit() {
    unsigned long long v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_bounds_miss, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (v) cudaMemcpyToSymbol(g_bounds_miss, &z, sizeof(z));
    return v;
}
const int g_bounds_registered = fds_bounds_register(&bounds_take_unit);
}  // namespace
#else
#define FDS_IN_RANGE(i, n) true
#endif

static inline unsigned ceil_div_u(long a, long b) { return (unsigned)((a + b - 1) / b); }

// Raise a kernel's dynamic shared-memory limit to at least `bytes`, never
// lowering it: the attribute is process-wide, so concurrent callers (batched
// builds on several host threads) that each set their own size would
// otherwise shrink it under another's launch.
size_t &dyn_smem_slot(const void *kernel);   // per-kernel current limit (prof.cu), under the lock below
std::mutex &dyn_smem_mutex();

template <class K>
int ensure_dyn_smem(K kernel, size_t bytes) {
    std::lock_guard<std::mutex> lk(dyn_smem_mutex());
    size_t &cur = dyn_smem_slot((const void *)kernel);
    if (bytes <= cur) return FDS_OK;
    FDS_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    cur = bytes;
    return FDS_OK;
}

// Upload this translation unit's Gauss table once per device.
static inline int ensure_gauss_tables() {
    static std::mutex mu;
    static int done[64] = {0};
    int dev = 0;
    FDS_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 64 && done[dev]) return FDS_OK;
    GaussTables T;
    FDS_TRY(gauss_tables_host(&T));
    FDS_CUDA_TRY(cudaMemcpyToSymbol(c_gauss, &T, sizeof(T)));
    if (dev >= 0 && dev < 64) done[dev] = 1;
    return FDS_OK;
}
