// Learned skeleton-rank predictor: a 16 -> 64 -> 64 -> 1 perceptron (tanh
// hidden units) in FP32, with hand-written inference, loss-gradient and Adam
// kernels.  The network maps the geometry features of one (cell, component)
// of a tree level to the fraction k / n of its DOFs that the interpolative
// decomposition of Sec. 7.1-7.2 keeps.
//
// Parameter vector (floats): W1 [64 x 16] row-major, b1 [64], W2 [64 x 64],
// b2 [64], w3 [64], b3, then the input normalisation mu [16], sd [16]
// (u = (x - mu) / sd; not trained).
//
// The gradient is deterministic: each CTA runs its samples in chunks of 32,
// the hidden activations and their back-propagated errors go to shared
// memory, and every thread then accumulates a fixed set of parameters over
// the chunk in sample order; per-CTA partial sums are added in CTA order by
// a second kernel.
#include <vector>

#include "common.cuh"
#include "mlp.cuh"

namespace {

constexpr int NI = FDS_MLP_NIN, NH = 64;
constexpr int OW1 = 0, OB1 = OW1 + NH * NI, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH, OB3 = OW3 + NH;
constexpr int ONORM = OB3 + 1;
static_assert(ONORM == FDS_MLP_NTRAIN, "parameter layout");
static_assert(ONORM + 2 * NI == FDS_MLP_NPARAM, "parameter layout");

constexpr int MT = 256;           // threads per CTA
constexpr int CH = 32;            // samples per chunk
constexpr int PPT = (FDS_MLP_NTRAIN + MT - 1) / MT;   // parameters per thread (21)

struct MlpSmem {
    float W1[NH * NI], b1[NH], W2[NH * NH], b2[NH], w3[NH], b3, mu[NI], sd[NI];
};

__device__ void load_params(MlpSmem &S, const float *__restrict__ p) {
    for (int i = threadIdx.x; i < NH * NI; i += blockDim.x) S.W1[i] = p[OW1 + i];
    for (int i = threadIdx.x; i < NH * NH; i += blockDim.x) S.W2[i] = p[OW2 + i];
    for (int i = threadIdx.x; i < NH; i += blockDim.x) {
        S.b1[i] = p[OB1 + i];
        S.b2[i] = p[OB2 + i];
        S.w3[i] = p[OW3 + i];
    }
    for (int i = threadIdx.x; i < NI; i += blockDim.x) {
        S.mu[i] = p[ONORM + i];
        S.sd[i] = p[ONORM + NI + i];
    }
    if (threadIdx.x == 0) S.b3 = p[OB3];
}

// one thread per sample
__global__ void __launch_bounds__(MT) k_mlp_forward(const float *__restrict__ params, const float *__restrict__ X,
                                                    int n, float *__restrict__ y) {
    __shared__ MlpSmem S;
    load_params(S, params);
    __syncthreads();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    float u[NI], h1[NH];
#pragma unroll
    for (int i = 0; i < NI; ++i) u[i] = (X[(long)b * NI + i] - S.mu[i]) / S.sd[i];
#pragma unroll 4
    for (int j = 0; j < NH; ++j) {
        float a = S.b1[j];
#pragma unroll
        for (int i = 0; i < NI; ++i) a = fmaf(S.W1[j * NI + i], u[i], a);
        h1[j] = tanhf(a);
    }
    float out = S.b3;
    for (int j = 0; j < NH; ++j) {
        float a = S.b2[j];
#pragma unroll
        for (int k = 0; k < NH; ++k) a = fmaf(S.W2[j * NH + k], h1[k], a);
        out = fmaf(S.w3[j], tanhf(a), out);
    }
    y[b] = out;
}

struct GradSmem {
    MlpSmem P;
    float U[CH][NI], H1[CH][NH], H2[CH][NH], D1[CH][NH], D2[CH][NH], dy[CH];
};

// Per-CTA partial gradients of L = (1/n_total) sum (y - t)^2 over the samples
// idx[s] (or s when idx is null) for s in [blockIdx.x * per, (blockIdx.x+1) * per) n [0, n).
__global__ void __launch_bounds__(MT) k_mlp_grad(const float *__restrict__ params, const float *__restrict__ X,
                                                 const float *__restrict__ t, const int *__restrict__ idx, int n,
                                                 int per, float inv_total, float *__restrict__ part,
                                                 float *__restrict__ part_loss) {
    extern __shared__ __align__(16) unsigned char g_raw[];
    GradSmem &S = *reinterpret_cast<GradSmem *>(g_raw);
    load_params(S.P, params);
    float acc[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) acc[q] = 0.f;
    float lsum = 0.f;
    const int s0 = blockIdx.x * per, s1 = min(n, s0 + per);
    __syncthreads();
    for (int c0 = s0; c0 < s1; c0 += CH) {
        const int nb = min(CH, s1 - c0);
        // normalised inputs
        for (int e = threadIdx.x; e < CH * NI; e += blockDim.x) {
            const int b = e / NI, i = e % NI;
            float v = 0.f;
            if (b < nb) {
                const int smp = idx ? idx[c0 + b] : c0 + b;
                v = (X[(long)smp * NI + i] - S.P.mu[i]) / S.P.sd[i];
            }
            S.U[b][i] = v;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < CH * NH; e += blockDim.x) {
            const int b = e / NH, j = e % NH;
            float a = S.P.b1[j];
#pragma unroll
            for (int i = 0; i < NI; ++i) a = fmaf(S.P.W1[j * NI + i], S.U[b][i], a);
            S.H1[b][j] = tanhf(a);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < CH * NH; e += blockDim.x) {
            const int b = e / NH, j = e % NH;
            float a = S.P.b2[j];
            for (int k = 0; k < NH; ++k) a = fmaf(S.P.W2[j * NH + k], S.H1[b][k], a);
            S.H2[b][j] = tanhf(a);
        }
        __syncthreads();
        // output, residual and dL/dy (one warp per sample group)
        if (threadIdx.x < CH) {
            const int b = threadIdx.x;
            float y = S.P.b3;
            for (int j = 0; j < NH; ++j) y = fmaf(S.P.w3[j], S.H2[b][j], y);
            float d = 0.f;
            if (b < nb) {
                const int smp = idx ? idx[c0 + b] : c0 + b;
                const float r = y - t[smp];
                lsum = fmaf(r, r, lsum);
                d = 2.f * r * inv_total;
            }
            S.dy[b] = d;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < CH * NH; e += blockDim.x) {
            const int b = e / NH, j = e % NH;
            const float h = S.H2[b][j];
            S.D2[b][j] = S.dy[b] * S.P.w3[j] * (1.f - h * h);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < CH * NH; e += blockDim.x) {
            const int b = e / NH, k = e % NH;
            float a = 0.f;
            for (int j = 0; j < NH; ++j) a = fmaf(S.D2[b][j], S.P.W2[j * NH + k], a);
            const float h = S.H1[b][k];
            S.D1[b][k] = a * (1.f - h * h);
        }
        __syncthreads();
        // parameter-parallel accumulation in sample order
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            const int p = threadIdx.x + q * MT;
            if (p >= FDS_MLP_NTRAIN) break;
            float g = 0.f;
            if (p < OB1) {
                const int j = p / NI, i = p % NI;
                for (int b = 0; b < CH; ++b) g = fmaf(S.D1[b][j], S.U[b][i], g);
            } else if (p < OW2) {
                const int j = p - OB1;
                for (int b = 0; b < CH; ++b) g += S.D1[b][j];
            } else if (p < OB2) {
                const int j = (p - OW2) / NH, k = (p - OW2) % NH;
                for (int b = 0; b < CH; ++b) g = fmaf(S.D2[b][j], S.H1[b][k], g);
            } else if (p < OW3) {
                const int j = p - OB2;
                for (int b = 0; b < CH; ++b) g += S.D2[b][j];
            } else if (p < OB3) {
                const int j = p - OW3;
                for (int b = 0; b < CH; ++b) g = fmaf(S.dy[b], S.H2[b][j], g);
            } else {
                for (int b = 0; b < CH; ++b) g += S.dy[b];
            }
            acc[q] += g;
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int p = threadIdx.x + q * MT;
        if (p < FDS_MLP_NTRAIN) part[(long)blockIdx.x * FDS_MLP_NTRAIN + p] = acc[q];
    }
    // loss partial: threads 0..CH-1 hold sums; add them in thread order
    __shared__ float ls[CH];
    if (threadIdx.x < CH) ls[threadIdx.x] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f;
        for (int i = 0; i < CH; ++i) a += ls[i];
        part_loss[blockIdx.x] = a;
    }
}

__global__ void k_mlp_reduce(const float *__restrict__ part, const float *__restrict__ part_loss, int nblk,
                             float inv_total, float *__restrict__ grad, float *__restrict__ loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < FDS_MLP_NTRAIN) {
        float g = 0.f;
        for (int b = 0; b < nblk; ++b) g += part[(long)b * FDS_MLP_NTRAIN + p];
        grad[p] = g;
    }
    if (p == 0 && loss) {
        float a = 0.f;
        for (int b = 0; b < nblk; ++b) a += part_loss[b];
        *loss = a * inv_total;
    }
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= FDS_MLP_NTRAIN) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

constexpr int GRAD_PER = 256;     // samples per CTA in the gradient kernel

struct GradWork {
    float *part = nullptr, *ploss = nullptr;
    size_t cap = 0;
    ~GradWork() {
        cudaFree(part);
        cudaFree(ploss);
    }
};

int grad_launch(const float *params, const float *X, const float *t, const int *idx, int n, float *grad,
                float *loss, float *part, float *ploss, cudaStream_t s) {
    const int nblk = (n + GRAD_PER - 1) / GRAD_PER;
    const size_t smem = sizeof(GradSmem);
    FDS_TRY(ensure_dyn_smem(k_mlp_grad, smem));
    const float inv = 1.f / (float)n;
    fds_count_launch(), k_mlp_grad<<<nblk, MT, smem, s>>>(params, X, t, idx, n, GRAD_PER, inv, part, ploss);
    FDS_CUDA_TRY(cudaGetLastError());
    fds_count_launch(), k_mlp_reduce<<<(FDS_MLP_NTRAIN + 255) / 256, 256, 0, s>>>(part, ploss, nblk, inv, grad, loss);
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}

}  // namespace

int mlp_forward(const float *d_params, const float *d_X, int n, float *d_y, cudaStream_t s) {
    if (n <= 0) return FDS_OK;
    fds_count_launch(), k_mlp_forward<<<(n + MT - 1) / MT, MT, 0, s>>>(d_params, d_X, n, d_y);
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}

extern "C" int fds_mlp_forward(const float *d_params, const float *d_X, int32_t n, float *d_y, uint64_t stream) {
    if (n < 0 || (n > 0 && (!d_params || !d_X || !d_y))) return FDS_ERR_ARG;
    return mlp_forward(d_params, d_X, n, d_y, (cudaStream_t)stream);
}

extern "C" int fds_mlp_loss_grad(const float *d_params, const float *d_X, const float *d_t, int32_t n, float *d_grad,
                                 float *d_loss, uint64_t stream) {
    if (n <= 0 || !d_params || !d_X || !d_t || !d_grad) return FDS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int nblk = (n + GRAD_PER - 1) / GRAD_PER;
    float *part = nullptr, *ploss = nullptr;
    FDS_CUDA_TRY(cudaMallocAsync((void **)&part, sizeof(float) * (size_t)nblk * FDS_MLP_NTRAIN, s));
    if (cudaMallocAsync((void **)&ploss, sizeof(float) * nblk, s) != cudaSuccess) {
        cudaFreeAsync(part, s);
        return FDS_ERR_OOM;
    }
    const int rc = grad_launch(d_params, d_X, d_t, nullptr, n, d_grad, d_loss, part, ploss, s);
    cudaFreeAsync(part, s);
    cudaFreeAsync(ploss, s);
    return rc;
}

extern "C" int fds_mlp_adam(float *d_params, const float *d_grad, float *d_m, float *d_v, int32_t step, float lr,
                            float beta1, float beta2, float eps, uint64_t stream) {
    if (!d_params || !d_grad || !d_m || !d_v || step < 1) return FDS_ERR_ARG;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    fds_count_launch(), k_adam<<<(FDS_MLP_NTRAIN + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
        d_params, d_grad, d_m, d_v, lr, beta1, beta2, eps, c1, c2);
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}

extern "C" int fds_mlp_train(float *d_params, const float *d_X, const float *d_t, int32_t n, const int32_t *d_order,
                             int32_t n_order, int32_t batch, float lr, float *d_losses, uint64_t stream) {
    if (n <= 0 || batch <= 0 || n_order < batch || !d_params || !d_X || !d_t || !d_order) return FDS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int steps = n_order / batch;
    const int nblk = (batch + GRAD_PER - 1) / GRAD_PER;
    float *work = nullptr;
    const size_t nw = (size_t)nblk * FDS_MLP_NTRAIN + nblk + 3 * (size_t)FDS_MLP_NTRAIN;
    FDS_CUDA_TRY(cudaMallocAsync((void **)&work, sizeof(float) * nw, s));
    float *part = work, *ploss = part + (size_t)nblk * FDS_MLP_NTRAIN, *grad = ploss + nblk;
    float *m = grad + FDS_MLP_NTRAIN, *v = m + FDS_MLP_NTRAIN;
    int rc = FDS_OK;
    if (cudaMemsetAsync(m, 0, sizeof(float) * 2 * FDS_MLP_NTRAIN, s) != cudaSuccess) rc = FDS_ERR_CUDA;
    for (int st = 0; st < steps && rc == FDS_OK; ++st) {
        rc = grad_launch(d_params, d_X, d_t, d_order + (long)st * batch, batch, grad, d_losses ? d_losses + st : nullptr,
                         part, ploss, s);
        if (rc == FDS_OK) rc = fds_mlp_adam(d_params, grad, m, v, st + 1, lr, 0.9f, 0.999f, 1e-8f, (uint64_t)s);
    }
    cudaFreeAsync(work, s);
    return rc;
}
