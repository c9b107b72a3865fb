// Displacement at points off the boundary from the boundary solution, by the
// integral representation of arXiv 2411.18026 Sec. 3, eq. (integ_rep), for
// the traction-free cavity:
//   u_i(x) = u^I_i(x) - int_Gamma K_ij(x, y) u_j(y) ds(y),
//   K_ij = T^{n_y}_{jk} G_ik = lam n_j d_k G_ik + mu (d_n G_ij + n_k d_j G_ik),
// derivatives in y, z = y - x, G of eq. (funda):
//   G_ik(z) = i/(4 mu) [H0(k_T r) delta_ik + k_T^-2 d_i d_k (H0(k_T r) - H0(k_L r))].
// With D_m = (r^-1 d/dr)^m H0(k r) = (-k/r)^m H_m(k r):
//   d_c G_ik = i/(4 mu) [delta_ik z_c D1_T
//              + k_T^-2 ((delta_ik z_c + delta_ic z_k + delta_kc z_i) (D2_T - D2_L)
//                        + z_i z_k z_c (D3_T - D3_L))].
// u is P1 on each element (nodal values), integrated with the 8-point Gauss
// rule per element.  Direct summation: every point sees every element, the
// kernel of a quadrature point is shared by the right-hand sides of a group.
#include <algorithm>
#include <cmath>
#include <vector>

#include "fds_internal.cuh"
#include "kernel_eval.cuh"
#include "prof.cuh"

namespace {

constexpr int FT = 256;   // threads per CTA (one observation point)
constexpr int RG = 8;     // right-hand sides per CTA

__device__ __forceinline__ double bsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(FT) k_field(PhysDev P, const double *__restrict__ xy, int N,
                                              const cplx *__restrict__ u, int64_t ldu, int nrhs,
                                              const int *__restrict__ kinds, const double *__restrict__ angles,
                                              const double *__restrict__ pts, int npts, cplx *out, int64_t ldo) {
    const int p = blockIdx.x, jb = blockIdx.y * RG;
    const int nj = min(RG, nrhs - jb);
    const double x0 = pts[2 * p], x1 = pts[2 * p + 1];
    const double ikT2 = 1.0 / (P.kT * P.kT);
    cplx acc[RG][2];
#pragma unroll
    for (int j = 0; j < RG; ++j) acc[j][0] = acc[j][1] = mkc(0.0, 0.0);
    for (int e = threadIdx.x; e < N; e += FT) {
        const fdsk::Elem E = fdsk::load_elem(xy, N, e);
        const int e1 = (e + 1 == N) ? 0 : e + 1;
        for (int q = 0; q < 8; ++q) {
            const double sig = c_gauss.x[8][q];
            const double w = c_gauss.w[8][q] * E.h;
            const double z[2] = {E.a.x + sig * E.h * E.t.x - x0, E.a.y + sig * E.h * E.t.y - x1};
            const double r = sqrt(z[0] * z[0] + z[1] * z[1]);
            const double ir = 1.0 / r;
            // H0..H3 at k_T r and k_L r (upward recurrence from H0, H1)
            double DT[4][2], DL[4][2];
            {
                const double zt = P.kT * r, zl = P.kL * r;
                double HT[4][2] = {{j0(zt), y0(zt)}, {j1(zt), y1(zt)}};
                double HL[4][2] = {{j0(zl), y0(zl)}, {j1(zl), y1(zl)}};
                for (int m = 1; m < 3; ++m)
                    for (int c = 0; c < 2; ++c) {
                        HT[m + 1][c] = (2.0 * m / zt) * HT[m][c] - HT[m - 1][c];
                        HL[m + 1][c] = (2.0 * m / zl) * HL[m][c] - HL[m - 1][c];
                    }
                double ft = 1.0, fl = 1.0;
                for (int m = 0; m < 4; ++m) {
                    for (int c = 0; c < 2; ++c) {
                        DT[m][c] = ft * HT[m][c];
                        DL[m][c] = fl * HL[m][c];
                    }
                    ft *= -P.kT * ir;
                    fl *= -P.kL * ir;
                }
            }
            // d_c G_ik without the factor i/(4 mu), then K_ij
            cplx G1[2][2][2];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int k = 0; k < 2; ++k)
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const double t3 = (i == k ? z[c] : 0.0) + (i == c ? z[k] : 0.0) + (k == c ? z[i] : 0.0);
                        const double z3 = z[i] * z[k] * z[c];
                        cplx v;
                        v.x = (i == k ? z[c] * DT[1][0] : 0.0) +
                              ikT2 * (t3 * (DT[2][0] - DL[2][0]) + z3 * (DT[3][0] - DL[3][0]));
                        v.y = (i == k ? z[c] * DT[1][1] : 0.0) +
                              ikT2 * (t3 * (DT[2][1] - DL[2][1]) + z3 * (DT[3][1] - DL[3][1]));
                        G1[i][k][c] = v;
                    }
            const double n[2] = {E.n.x, E.n.y};
            cplx K[2][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const cplx dv = cadd(G1[i][0][0], G1[i][1][1]);
#pragma unroll
                for (int jj = 0; jj < 2; ++jj) {
                    cplx k = cscale(dv, P.lam * n[jj]);
                    k = cadd(k, cscale(cadd(cscale(G1[i][jj][0], n[0]), cscale(G1[i][jj][1], n[1])), P.mu));
                    k = cadd(k, cscale(cadd(cscale(G1[i][0][jj], n[0]), cscale(G1[i][1][jj], n[1])), P.mu));
                    // times i/(4 mu) and the weight
                    K[i][jj] = mkc(-0.25 / P.mu * w * k.y, 0.25 / P.mu * w * k.x);
                }
            }
#pragma unroll
            for (int j = 0; j < RG; ++j) {
                if (j >= nj) break;
                const cplx *uj = u + (int64_t)(jb + j) * ldu;
                const cplx ua = cadd(cscale(uj[e], 1.0 - sig), cscale(uj[e1], sig));
                const cplx ub = cadd(cscale(uj[e + N], 1.0 - sig), cscale(uj[e1 + N], sig));
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    acc[j][i] = cadd(acc[j][i], cmul(K[i][0], ua));
                    acc[j][i] = cadd(acc[j][i], cmul(K[i][1], ub));
                }
            }
        }
    }
    // block reduction: warp sums, then one partial per warp in shared memory
    __shared__ double part[FT / 32][RG * 4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < RG; ++j)
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const double re = bsum(acc[j][i].x), im = bsum(acc[j][i].y);
            if (lane == 0) {
                part[warp][4 * j + 2 * i] = re;
                part[warp][4 * j + 2 * i + 1] = im;
            }
        }
    __syncthreads();
    if (threadIdx.x < nj * 2) {
        const int j = threadIdx.x >> 1, i = threadIdx.x & 1;
        double re = 0.0, im = 0.0;
        for (int w = 0; w < FT / 32; ++w) {
            re += part[w][4 * j + 2 * i];
            im += part[w][4 * j + 2 * i + 1];
        }
        // incident wave: P u = d e^{i k_L d.x}, SV u = d_perp e^{i k_T d.x}
        double sd, cd;
        sincos(angles[jb + j], &sd, &cd);
        const bool sv = kinds[jb + j] != 0;
        const double k = sv ? P.kT : P.kL;
        double sp, cp;
        sincos(k * (cd * x0 + sd * x1), &sp, &cp);
        const double amp = sv ? (i == 0 ? -sd : cd) : (i == 0 ? cd : sd);
        out[p + (int64_t)i * npts + (int64_t)(jb + j) * ldo] = mkc(amp * cp - re, amp * sp - im);
    }
}

}  // namespace

extern "C" int fds_field(fds_handle *h, const double *d_u, int32_t nrhs, const int32_t *kinds,
                         const double *angles, const double *d_pts, int32_t npts, double *d_out, uint64_t stream) {
    if (!h || nrhs < 0 || npts < 0) return FDS_ERR_ARG;
    if (nrhs == 0 || npts == 0) return FDS_OK;
    if (!d_u || !kinds || !angles || !d_pts || !d_out) return FDS_ERR_ARG;
    for (int j = 0; j < nrhs; ++j)
        if ((kinds[j] != 0 && kinds[j] != 1) || !std::isfinite(angles[j])) return FDS_ERR_ARG;
    if (npts > 2147483647 / 2 || (nrhs + RG - 1) / RG > 65535) return FDS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    FDS_TRY(ensure_gauss_tables());
    DBuf<int> dk;
    DBuf<double> da;
    FDS_TRY(dk.upload(std::vector<int>(kinds, kinds + nrhs), s));
    FDS_TRY(da.upload(std::vector<double>(angles, angles + nrhs), s));
    {
        ProfScope ps("f1.field", s);
        ps.units = (double)npts * nrhs;
        dim3 grid(npts, (nrhs + RG - 1) / RG);
        fds_count_launch(), k_field<<<grid, FT, 0, s>>>(h->P, h->d_xy.p, h->N, (const cplx *)d_u, 2LL * h->N, nrhs,
                                                        dk.p, da.p, d_pts, npts, (cplx *)d_out, 2LL * npts);
        FDS_CUDA_TRY(cudaGetLastError());
    }
    FDS_CUDA_TRY(cudaStreamSynchronize(s));
    return FDS_OK;
}
