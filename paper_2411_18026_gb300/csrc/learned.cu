// Learned-rank interpolative decomposition (extension of Sec. 7.1-7.2).
//
// Features: per (cell, component) of a level, 16 geometry / size features
// from the cell's polygon piece (the hat supports of nodes lo..hi-1, i.e.
// vertices lo-1..hi).
//
// Sketched ID: with the predicted fraction f of the component's n DOFs, the
// stacked proxy matrix Y (m x n) is compressed to s = min(n, ceil(f n) +
// extra) rows by a sparse sign embedding (every row of Y is added, with a
// sign, to 2 sketch rows chosen by the SplitMix64 hash of (matrix, row,
// slot): row floor(h_hi32 s / 2^32), sign from the lowest bit); the sketch Z = Omega Y goes through the same CPQR as the adaptive
// ID (largest remaining column, stop at |R_jj| <= tol |R_11| / 10: the
// sketch underestimates the trailing norms), giving the skeleton columns and
// T = R11^{-1} R12 (on the proxy matrices of this method about 2 more
// skeleton columns per (cell, component) than the adaptive ID).
// The result is accepted when the rank was revealed (k < s, or s = n) and the
// ID residual on Y, max over columns of ||Y[:, c] - Y[:, J] T[:, c]||, is at
// most tol times the largest column norm of Y (what the adaptive CPQR
// guarantees); otherwise the caller reruns the adaptive CPQR on Y.
#include <cmath>

#include "common.cuh"
#include "id.cuh"

namespace {

constexpr int LT = 256;
constexpr int SK_MAXN = 64;      // columns handled by the sketch kernel (n <= 64, else fallback)

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    // Steele, Lea, Flood (2014), SplitMix64 finaliser
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// one warp per cell
__global__ void k_features(int nb, const int *__restrict__ lo, const int *__restrict__ hi,
                           const double *__restrict__ xy, int N, const double *__restrict__ R,
                           const int *__restrict__ n1, const int *__restrict__ n2, const int *__restrict__ nnd,
                           int height, double kT, double kL, double tol, float *__restrict__ feat) {
    const int b = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= nb) return;
    const int a = lo[b] - 1, e = hi[b];      // vertices a..e
    auto vx = [&](int v) { const int q = ((v % N) + N) % N; return xy[2 * q]; };
    auto vy = [&](int v) { const int q = ((v % N) + N) % N; return xy[2 * q + 1]; };
    double arc = 0, sx = 0, sy = 0, sxx = 0, syy = 0, sxy = 0;
    double tsum = 0, tabs = 0, tmax = 0, tsq = 0;
    for (int v = a + lane; v <= e; v += 32) {
        const double x = vx(v), y = vy(v);
        sx += x; sy += y; sxx += x * x; syy += y * y; sxy += x * y;
        if (v < e) arc += hypot(vx(v + 1) - x, vy(v + 1) - y);
        if (v > a && v < e) {
            // turning angle at v between edges (v-1, v) and (v, v+1)
            const double ux = x - vx(v - 1), uy = y - vy(v - 1), wx = vx(v + 1) - x, wy = vy(v + 1) - y;
            const double th = atan2(ux * wy - uy * wx, ux * wx + uy * wy);
            tsum += th; tabs += fabs(th); tsq += th * th; tmax = fmax(tmax, fabs(th));
        }
    }
    arc = wsum(arc); sx = wsum(sx); sy = wsum(sy); sxx = wsum(sxx); syy = wsum(syy); sxy = wsum(sxy);
    tsum = wsum(tsum); tabs = wsum(tabs); tsq = wsum(tsq);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tmax = fmax(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
    if (lane != 0) return;
    const double nv = (double)(e - a + 1), nt = fmax((double)(e - a - 1), 1.0);
    const double mx = sx / nv, my = sy / nv;
    const double cxx = sxx / nv - mx * mx, cyy = syy / nv - my * my, cxy = sxy / nv - mx * my;
    const double tr = cxx + cyy, det = cxx * cyy - cxy * cxy;
    const double disc = sqrt(fmax(0.25 * tr * tr - det, 0.0));
    const double l1 = 0.5 * tr + disc, l2 = fmax(0.5 * tr - disc, 0.0);
    const double chord = hypot(vx(e) - vx(a), vy(e) - vy(a));
    const double diam = 2.0 * R[b];
    const int nodes = hi[b] - lo[b];
    const int d = n1[b] + n2[b];
    for (int c = 0; c < 2; ++c) {
        const int n = c ? n2[b] : n1[b];
        float *f = feat + (long)(2 * b + c) * FDS_MLP_NIN;
        f[0] = (float)height;
        f[1] = (float)log2(fmax((double)n, 1.0));
        f[2] = (float)c;
        f[3] = (float)(kT * diam);
        f[4] = (float)(kL * diam);
        f[5] = (float)(arc / fmax(diam, 1e-300));
        f[6] = (float)(chord / fmax(arc, 1e-300));
        f[7] = (float)(tabs / nt);
        f[8] = (float)tmax;
        f[9] = (float)sqrt(tsq / nt);
        f[10] = (float)tsum;
        f[11] = (float)sqrt(l2 / fmax(l1, 1e-300));
        f[12] = (float)((double)nnd[b] / fmax((double)d, 1.0));
        f[13] = (float)log10(fmax(tol, 1e-300));
        f[14] = (float)((double)n / fmax((double)nodes, 1.0));
        f[15] = (float)(kT * arc / (2.0 * FDS_PI));
    }
}

__global__ void __launch_bounds__(LT) k_sketch_id(const int *__restrict__ ms, const int *__restrict__ ns,
                                                  const int64_t *__restrict__ offs, const cplx *__restrict__ Yall,
                                                  const float *__restrict__ frac, int extra, double tol,
                                                  int *__restrict__ ranks, int *__restrict__ perms,
                                                  const int64_t *__restrict__ poffs, cplx *__restrict__ Tall,
                                                  const int64_t *__restrict__ toffs, int *__restrict__ fail,
                                                  unsigned long long seed) {
    extern __shared__ __align__(16) unsigned char sk_raw[];
    const int b = blockIdx.x;
    const int m = ms[b], n = ns[b];
    const cplx *Y = Yall + offs[b];
    if (n > SK_MAXN || m <= 0 || n <= 0) {
        if (threadIdx.x == 0) fail[b] = (n > 0) ? 1 : 0;
        if (threadIdx.x == 0 && n == 0) ranks[b] = 0;
        return;
    }
    float fr = frac[b];
    if (!(fr == fr)) fr = 1.f;
    fr = fminf(fmaxf(fr, 0.f), 1.f);
    const int s = min(n, (int)ceilf(fr * (float)n) + extra);
    // shared layout: Z[s x n] (column-major), nrm[n], perm[n], bucket lists
    cplx *Z = reinterpret_cast<cplx *>(sk_raw);
    double *nrm = reinterpret_cast<double *>(Z + (size_t)SK_MAXN * SK_MAXN);
    int *perm = reinterpret_cast<int *>(nrm + SK_MAXN);
    int *cnt = perm + SK_MAXN;                   // [SK_MAXN + 1]
    int *lst = cnt + SK_MAXN + 1;                // [2 m] (row << 1 | sign)
    __shared__ double r_val[LT];
    __shared__ int r_idx[LT];
    __shared__ int s_k, s_stop, s_p, s_ok;
    __shared__ double s_alpha, s_r11;
    __shared__ cplx s_phase;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned long long key = seed ^ ((unsigned long long)b << 32);
    // bucket lists in row order: thread q collects the (row, sign) entries of bucket q
    if (threadIdx.x < s) {
        const int q = threadIdx.x;
        int c = 0;
        for (int i = 0; i < m; ++i)
            for (int slot = 0; slot < 2; ++slot) {
                const unsigned long long z = splitmix64(key + 2ULL * (unsigned long long)i + slot);
                if ((int)(((z >> 32) * (unsigned long long)s) >> 32) == q) ++c;
            }
        cnt[q + 1] = c;
    }
    if (threadIdx.x == 0) cnt[0] = 0;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int q = 0; q < s; ++q) cnt[q + 1] += cnt[q];
    __syncthreads();
    if (threadIdx.x < s) {
        const int q = threadIdx.x;
        int o = cnt[q];
        for (int i = 0; i < m; ++i)
            for (int slot = 0; slot < 2; ++slot) {
                const unsigned long long z = splitmix64(key + 2ULL * (unsigned long long)i + slot);
                if ((int)(((z >> 32) * (unsigned long long)s) >> 32) == q) lst[o++] = (i << 1) | (int)(z & 1ULL);
            }
    }
    __syncthreads();
    // Z = Omega Y
    for (int e = threadIdx.x; e < s * n; e += blockDim.x) {
        const int q = e % s, c = e / s;
        double re = 0, im = 0;
        for (int o = cnt[q]; o < cnt[q + 1]; ++o) {
            const int code = lst[o];
            const cplx y = Y[(code >> 1) + (long)c * m];
            if (code & 1) { re -= y.x; im -= y.y; }
            else { re += y.x; im += y.y; }
        }
        Z[q + c * s] = mkc(re, im);
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) perm[j] = j;
    __syncthreads();
    // CPQR of Z (as in the adaptive ID, on the s x n sketch)
    for (int c = warp; c < n; c += LT / 32) {
        double a = 0.0;
        for (int i = lane; i < s; i += 32) a += cabs2(Z[i + c * s]);
        a = wsum(a);
        if (lane == 0) nrm[c] = a;
    }
    if (threadIdx.x == 0) { s_k = 0; s_stop = 0; s_r11 = 0.0; }
    __syncthreads();
    const int kmax = min(s, n);
    // two passes: stop the sketch's CPQR at tol/3 and check the ID on Y; if
    // the check fails, continue the same factorisation down to tol/10 and
    // check again (fewer skeleton columns than a single tol/10 pass)
    for (int pass = 0; pass < 2; ++pass) {
    const double stop_frac = pass == 0 ? (1.0 / 3.0) : 0.1;
    if (threadIdx.x == 0) s_stop = 0;
    __syncthreads();
    for (int j = s_k; j < kmax; ++j) {
        double best = -1.0;
        int bi = n;
        for (int c = j + threadIdx.x; c < n; c += blockDim.x)
            if (nrm[c] > best) { best = nrm[c]; bi = c; }
        r_val[threadIdx.x] = best;
        r_idx[threadIdx.x] = bi;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) {
                const double v2 = r_val[threadIdx.x + o];
                const int i2 = r_idx[threadIdx.x + o];
                if (v2 > r_val[threadIdx.x] || (v2 == r_val[threadIdx.x] && i2 < r_idx[threadIdx.x])) {
                    r_val[threadIdx.x] = v2;
                    r_idx[threadIdx.x] = i2;
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const int p = r_idx[0] < n ? r_idx[0] : j;
            const double alpha = sqrt(fmax(r_val[0], 0.0));
            if (j == 0) s_r11 = alpha;
            s_p = p;
            s_alpha = alpha;
            // a tenth of the tolerance on the sketch: a (k + extra)-row sketch
            // underestimates the trailing norms
            s_stop = (alpha == 0.0 || alpha <= stop_frac * tol * s_r11) ? 1 : 0;
        }
        __syncthreads();
        if (s_stop) break;
        const int p = s_p;
        if (p != j) {
            for (int i = threadIdx.x; i < s; i += blockDim.x) {
                const cplx t = Z[i + j * s];
                Z[i + j * s] = Z[i + p * s];
                Z[i + p * s] = t;
            }
            if (threadIdx.x == 0) {
                const int t = perm[j]; perm[j] = perm[p]; perm[p] = t;
                const double tn = nrm[j]; nrm[j] = nrm[p]; nrm[p] = tn;
            }
        }
        __syncthreads();
        const double alpha = s_alpha;
        if (threadIdx.x == 0) {
            const cplx x0 = Z[j + j * s];
            const double a0 = sqrt(cabs2(x0));
            s_phase = a0 > 0.0 ? mkc(x0.x / a0, x0.y / a0) : mkc(1.0, 0.0);
        }
        __syncthreads();
        const cplx ph = s_phase;
        const cplx x0 = Z[j + j * s];
        const double tau = 2.0 / (2.0 * alpha * (alpha + sqrt(cabs2(x0))));
        __syncthreads();
        // v = Z[j:, j] + ph alpha e_0 (kept in column j until the update is done)
        for (int c = j + 1 + warp; c < n; c += LT / 32) {
            double sr = 0.0, si = 0.0;
            for (int i = j + lane; i < s; i += 32) {
                cplx vi = Z[i + j * s];
                if (i == j) vi = cadd(vi, cscale(ph, alpha));
                const cplx a = Z[i + c * s];
                sr += vi.x * a.x + vi.y * a.y;
                si += vi.x * a.y - vi.y * a.x;
            }
            sr = wsum(sr);
            si = wsum(si);
            const cplx sc = mkc(tau * sr, tau * si);
            double nn = 0.0;
            for (int i = j + lane; i < s; i += 32) {
                cplx vi = Z[i + j * s];
                if (i == j) vi = cadd(vi, cscale(ph, alpha));
                cplx a = Z[i + c * s];
                cfms(a, sc, vi);
                Z[i + c * s] = a;
                if (i > j) nn += cabs2(a);
            }
            nn = wsum(nn);
            if (lane == 0) nrm[c] = nn;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            Z[j + j * s] = cscale(ph, -alpha);
            s_k = j + 1;
        }
        __syncthreads();
    }
    const int k = s_k;
    // T = R11^{-1} R12 (k x (n - k)), one thread per column
    cplx *T = Tall + toffs[b];
    __syncthreads();
    for (int c = threadIdx.x; c < n - k; c += blockDim.x) {
        const int col = k + c;
        for (int i = k - 1; i >= 0; --i) {
            cplx acc = Z[i + col * s];
            for (int l = i + 1; l < k; ++l) cfms(acc, Z[i + l * s], T[l + (long)c * k]);
            T[i + (long)c * k] = cdiv(acc, Z[i + i * s]);
        }
    }
    if (threadIdx.x == 0) s_ok = (k < s || s == n) ? 1 : 0;
    __syncthreads();
    // ID residual on all rows of Y: warp per column, lanes over rows
    double ymax = 0.0, emax = 0.0;
    for (int c = warp; c < n; c += LT / 32) {
        double a = 0.0;
        for (int i = lane; i < m; i += 32) a += cabs2(Y[i + (long)perm[c] * m]);
        ymax = fmax(ymax, wsum(a));
    }
    for (int c = warp; c < n - k; c += LT / 32) {
        double a = 0.0;
        for (int i = lane; i < m; i += 32) {
            cplx e = Y[i + (long)perm[k + c] * m];
            for (int l = 0; l < k; ++l) cfms(e, Y[i + (long)perm[l] * m], T[l + (long)c * k]);
            a += cabs2(e);
        }
        emax = fmax(emax, wsum(a));
    }
    r_val[threadIdx.x] = (lane == 0) ? ymax : 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
        double yy = 0.0;
        for (int w = 0; w < LT / 32; ++w) yy = fmax(yy, r_val[w * 32]);
        s_alpha = yy;
    }
    __syncthreads();
    r_val[threadIdx.x] = (lane == 0) ? emax : 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
        double ee = 0.0;
        for (int w = 0; w < LT / 32; ++w) ee = fmax(ee, r_val[w * 32]);
        // the adaptive ID's guarantee: every residual column <= tol x the largest column of Y
        const int ok = s_ok && (ee <= tol * tol * s_alpha);
        fail[b] = ok ? 0 : 1;
        if (ok) ranks[b] = k;
        s_ok = ok;
    }
    __syncthreads();
    if (s_ok || k >= kmax) break;
    }   // pass
    int *pout = perms + poffs[b];
    for (int j = threadIdx.x; j < n; j += blockDim.x) pout[j] = perm[j];
}

}  // namespace

int level_features(int nb, const int *d_lo, const int *d_hi, const double *d_xy, int N, const double *d_R,
                   const int *d_n1, const int *d_n2, const int *d_nnd, int height, double kT, double kL, double tol,
                   float *d_feat, cudaStream_t s) {
    if (nb <= 0) return FDS_OK;
    fds_count_launch(), k_features<<<(nb * 32 + 255) / 256, 256, 0, s>>>(nb, d_lo, d_hi, d_xy, N, d_R, d_n1, d_n2,
                                                                          d_nnd, height, kT, kL, tol, d_feat);
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}

int id_sketched(int batch, int max_m, const int *d_m, const int *d_n, const int64_t *d_off, const cplx *d_Y,
                const float *d_frac, int extra, double tol, int *d_rank, int *d_perm, const int64_t *d_poff,
                cplx *d_T, const int64_t *d_toff, int *d_fail, unsigned long long seed, cudaStream_t s) {
    if (batch <= 0) return FDS_OK;
    const size_t smem = sizeof(cplx) * SK_MAXN * SK_MAXN + sizeof(double) * SK_MAXN +
                        sizeof(int) * (SK_MAXN + SK_MAXN + 1 + 2 * (size_t)max_m) + 16;
    if (smem > 220 * 1024) return FDS_ERR_ARG;
    FDS_TRY(ensure_dyn_smem(k_sketch_id, smem));
    fds_count_launch(), k_sketch_id<<<batch, LT, smem, s>>>(d_m, d_n, d_off, d_Y, d_frac, extra, tol, d_rank, d_perm,
                                                             d_poff, d_T, d_toff, d_fail, seed);
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}
