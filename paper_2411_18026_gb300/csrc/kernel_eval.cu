// Galerkin kernel evaluation: stage entry points and the shared setup
// (Gauss tables, physical constants).  Device math lives in kernel_eval.cuh.
#include <math.h>
#include <mutex>
#include <string.h>

#include "common.cuh"
#include "kernel_eval.cuh"

PhysDev make_physdev(const fds_physics *ph) {
    PhysDev P;
    P.lam = ph->lambda;
    P.mu = ph->mu;
    P.rho = ph->rho > 0 ? ph->rho : 1.0;
    P.omega = ph->omega;
    // c_L = sqrt((lam + 2 mu)/rho), c_T = sqrt(mu/rho), k = omega / c   (Sec. 2)
    P.kL = P.omega / sqrt((P.lam + 2.0 * P.mu) / P.rho);
    P.kT = P.omega / sqrt(P.mu / P.rho);
    P.rw2 = P.rho * P.omega * P.omega;
    P.c2 = 2.0 / (P.kT * P.kT);
    P.lhalfT = log(0.5 * P.kT);
    P.lhalfL = log(0.5 * P.kL);
    if (ph->alpha_set)
        P.alpha = mkc(ph->alpha_re, ph->alpha_im);
    else
        P.alpha = mkc(0.0, 1.0 / (P.mu * P.kT));   // alpha = i / (mu k_T)
    P.alpha_rw2 = cscale(P.alpha, P.rw2);
    P.alpha_m2mu = cscale(P.alpha, -2.0 * P.mu);
    return P;
}

// Gauss–Legendre nodes on [0,1]: roots of P_q by Newton's method from the
// Chebyshev-like initial guesses, weights 1/((1-x^2) P_q'(x)^2) (mapped).
static void gauss_legendre01(int q, double *x, double *w) {
    for (int i = 0; i < q; ++i) {
        double r = cos(FDS_PI * (4.0 * i + 3.0) / (4.0 * q + 2.0));
        double dp = 1.0;
        for (int it = 0; it < 200; ++it) {
            double p0 = 1.0, p1 = r;
            for (int k = 2; k <= q; ++k) {
                double p2 = ((2.0 * k - 1.0) * r * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = q * (r * p1 - p0) / (r * r - 1.0);
            double step = p1 / dp;
            r -= step;
            if (fabs(step) < 1e-17) break;
        }
        double p0 = 1.0, p1 = r;
        for (int k = 2; k <= q; ++k) {
            double p2 = ((2.0 * k - 1.0) * r * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = q * (r * p1 - p0) / (r * r - 1.0);
        x[i] = 0.5 * (1.0 - r);
        w[i] = 1.0 / ((1.0 - r * r) * dp * dp);
    }
}

int gauss_tables_host(GaussTables *T) {
    static GaussTables cache;
    static bool ready = false;
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    if (!ready) {
        memset(&cache, 0, sizeof(cache));
        for (int q = 1; q <= GL_MAXQ; ++q) gauss_legendre01(q, cache.x[q], cache.w[q]);
        // series coefficients in powers of q = -z^2/4:
        //   sa_m = 1/(m!)^2, sb_m = 1/(m!(m+1)!), sh_m = H_m sa_m,
        //   sp_m = (2 (H_m - gamma) + 1/(m+1)) sb_m,  H_m = 1 + 1/2 + ... + 1/m
        const double g = 0.57721566490153286061;
        double fm = 1.0, hm = 0.0;   // m!, H_m
        for (int m = 0; m < SER_TERMS; ++m) {
            if (m > 0) {
                fm *= m;
                hm += 1.0 / m;
            }
            const double a = 1.0 / (fm * fm), b = 1.0 / (fm * fm * (m + 1.0));
            cache.sa[m] = a;
            cache.sb[m] = b;
            cache.sh[m] = hm * a;
            cache.sp[m] = (2.0 * (hm - g) + 1.0 / (m + 1.0)) * b;
        }
        ready = true;
    }
    *T = cache;
    return FDS_OK;
}

namespace {

using namespace fdsk;

// Stage kernels: one CTA per (row chunk, column chunk) tile; forward entries
// only (the row and column lists may overlap).  Output column-major
// out[(r + i nr) + (c + j nc) * 2 nr].
__global__ void __launch_bounds__(FDS_TILE_THREADS) k_stage_tiles(PhysDev P, const double *__restrict__ X, int NX,
                                                     const int *__restrict__ rows, int nr,
                                                     const double *__restrict__ Y, int NY,
                                                     const int *__restrict__ cols, int nc, int q, int same,
                                                     cplx *out) {
    __shared__ TileSmem S;
    const int r0 = blockIdx.x * TILE, c0 = blockIdx.y * TILE;
    load_rules(S.G, same ? 0 : q);
    tile_zero(S);
    if (threadIdx.x == 0) {
        S.R.nh = min(TILE, nr - r0);
        S.C.nh = min(TILE, nc - c0);
        for (int k = 0; k < S.R.nh; ++k) S.R.hats[k] = rows[r0 + k];
        for (int k = 0; k < S.C.nh; ++k) S.C.hats[k] = cols[c0 + k];
        tile_side_build(S.R, NX);
        tile_side_build(S.C, same ? NX : NY);
    }
    __syncthreads();
    tile_eval(P, S, X, NX, Y, NY, same != 0, false, false);
    __syncthreads();
    const long ld = 2L * nr;
    for (int e = threadIdx.x; e < S.R.nh * S.C.nh * 4; e += blockDim.x) {
        const int r = e % S.R.nh, c = (e / S.R.nh) % S.C.nh, ij = e / (S.R.nh * S.C.nh);
        const int i = ij >> 1, j = ij & 1;
        cplx v = tile_f(S, r, c, i, j);
        if (same && i == j) v.x += 0.5 * mass_entry(X, NX, S.R.hats[r], S.C.hats[c]);
        out[(r0 + r + (long)i * nr) + (c0 + c + (long)j * nc) * ld] = v;
    }
}

bool phys_ok(const fds_physics *ph) {
    return ph && ph->mu > 0 && ph->omega > 0 && ph->lambda + 2.0 * ph->mu > 0;
}

}  // namespace

extern "C" int fds_eval_entries(const fds_physics *ph, const double *d_xy, int32_t n, const int32_t *d_rows,
                                int32_t nr, const int32_t *d_cols, int32_t nc, double *d_out,
                                uint64_t stream) {
    if (!phys_ok(ph) || !d_xy || n < 3 || nr < 0 || nc < 0) return FDS_ERR_ARG;
    if (nr == 0 || nc == 0) return FDS_OK;
    if (!d_rows || !d_cols || !d_out) return FDS_ERR_ARG;
    FDS_TRY(ensure_gauss_tables());
    PhysDev P = make_physdev(ph);
    dim3 grid(ceil_div_u(nr, TILE), ceil_div_u(nc, TILE));
    fds_count_launch(), k_stage_tiles<<<grid, FDS_TILE_THREADS, 0, (cudaStream_t)stream>>>(
        P, d_xy, n, d_rows, nr, d_xy, n, d_cols, nc, 0, 1, (cplx *)d_out);
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}

extern "C" int fds_eval_cross(const fds_physics *ph, const double *d_X, int32_t nx, const int32_t *d_rows,
                              int32_t nr, const double *d_Y, int32_t ny, const int32_t *d_cols, int32_t nc,
                              int32_t q, double *d_out, uint64_t stream) {
    if (!phys_ok(ph) || !d_X || !d_Y || nx < 3 || ny < 3 || nr < 0 || nc < 0 || q < 1 || q > 8)
        return FDS_ERR_ARG;
    if (nr == 0 || nc == 0) return FDS_OK;
    if (!d_rows || !d_cols || !d_out) return FDS_ERR_ARG;
    FDS_TRY(ensure_gauss_tables());
    PhysDev P = make_physdev(ph);
    dim3 grid(ceil_div_u(nr, TILE), ceil_div_u(nc, TILE));
    fds_count_launch(), k_stage_tiles<<<grid, FDS_TILE_THREADS, 0, (cudaStream_t)stream>>>(
        P, d_X, nx, d_rows, nr, d_Y, ny, d_cols, nc, q, 0, (cplx *)d_out);
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}
