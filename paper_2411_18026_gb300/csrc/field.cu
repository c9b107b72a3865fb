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
#include "vapply.cuh"

namespace {

constexpr int FT = 256;   // threads per CTA (one observation point)
constexpr int RG = 8;     // right-hand sides per CTA

__device__ __forceinline__ double bsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// K_ij(x, y) w at one quadrature point (z = y - x, element normal n, weight w)
__device__ __forceinline__ void field_kernel(const PhysDev &P, const double z[2], double nx, double ny, double w,
                                             cplx K[2][2]) {
    const double ikT2 = 1.0 / (P.kT * P.kT);
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
                v.x = (i == k ? z[c] * DT[1][0] : 0.0) + ikT2 * (t3 * (DT[2][0] - DL[2][0]) + z3 * (DT[3][0] - DL[3][0]));
                v.y = (i == k ? z[c] * DT[1][1] : 0.0) + ikT2 * (t3 * (DT[2][1] - DL[2][1]) + z3 * (DT[3][1] - DL[3][1]));
                G1[i][k][c] = v;
            }
    const double n[2] = {nx, ny};
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
}

__global__ void __launch_bounds__(FT) k_field(PhysDev P, const double *__restrict__ xy, int N,
                                              const cplx *__restrict__ u, int64_t ldu, int nrhs,
                                              const int *__restrict__ kinds, const double *__restrict__ angles,
                                              const double *__restrict__ pts, int npts, cplx *out, int64_t ldo) {
    const int p = blockIdx.x, jb = blockIdx.y * RG;
    const int nj = min(RG, nrhs - jb);
    const double x0 = pts[2 * p], x1 = pts[2 * p + 1];
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
            cplx K[2][2];
            field_kernel(P, z, E.n.x, E.n.y, w, K);
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

// ------------------------------------------------------------------------
// Proxy-compressed evaluation.  A cell's sources seen from outside its proxy
// circle are represented by its skeleton hats with coefficients u~ = V u
// (the column ID of Sec. 7.1, whose proxy rows test the double-layer field
// of each hat on the proxy circle), recursively u~_parent = V_parent
// [u~_children].  Each point takes, from the cells of level l0 + 1 down, the
// skeleton sum of every cell whose proxy circle it lies outside, and the
// direct sum over the hats of the leaf cells whose proxy circle holds it.
constexpr int JT = 128;   // threads per job
constexpr int SOLVE_CHUNK_FIELD = 256;   // columns per structured V application

// incident wave u^I at every point (out: 2 npts x nrhs)
__global__ void k_field_incident(PhysDev P, const int *__restrict__ kinds, const double *__restrict__ angles,
                                 const double *__restrict__ pts, int npts, int nrhs, cplx *out, int64_t ldo) {
    const int64_t tot = 2LL * npts * nrhs;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(e % npts), i = (int)((e / npts) & 1);
        const int j = (int)(e / (2LL * npts));
        double sd, cd;
        sincos(angles[j], &sd, &cd);
        const bool sv = kinds[j] != 0;
        const double k = sv ? P.kT : P.kL;
        double sp, cp;
        sincos(k * (cd * pts[2 * p] + sd * pts[2 * p + 1]), &sp, &cp);
        const double amp = sv ? (i == 0 ? -sd : cd) : (i == 0 ? cd : sd);
        out[p + (int64_t)i * npts + (int64_t)j * ldo] = mkc(amp * cp, amp * sp);
    }
}

// One job per CTA (x: point, start, count of its hat list): subtracts from
// out the double-layer field at the point of hats e in [start, start+count)
// (node hnode[e], component hcomp[e], coefficient coef[e + j ldc] for
// right-hand side j).  A hat at node s spans element s-1 (weight sigma) and
// element s (weight 1 - sigma); 8 Gauss points per element.
__global__ void __launch_bounds__(JT) k_field_jobs(PhysDev P, const double *__restrict__ xy, int N,
                                                   const int4 *__restrict__ jobs, const int *__restrict__ hnode,
                                                   const unsigned char *__restrict__ hcomp,
                                                   const cplx *__restrict__ coef, int64_t ldc, int nrhs,
                                                   const double *__restrict__ pts, int npts, cplx *out,
                                                   int64_t ldo) {
    const int4 J = jobs[blockIdx.x];
    const int jb = blockIdx.y * RG;
    const int nj = min(RG, nrhs - jb);
    const double x0 = pts[2 * J.x], x1 = pts[2 * J.x + 1];
    cplx acc[RG][2];
#pragma unroll
    for (int j = 0; j < RG; ++j) acc[j][0] = acc[j][1] = mkc(0.0, 0.0);
    for (int q = threadIdx.x; q < J.z * 16; q += JT) {
        const int e = J.y + (q >> 4), half = (q >> 3) & 1, g = q & 7;
        const int node = hnode[e], c = hcomp[e];
        const int el = half ? node : (node == 0 ? N - 1 : node - 1);
        const fdsk::Elem E = fdsk::load_elem(xy, N, el);
        const double sig = c_gauss.x[8][g];
        const double w = c_gauss.w[8][g] * E.h * (half ? 1.0 - sig : sig);
        const double z[2] = {E.a.x + sig * E.h * E.t.x - x0, E.a.y + sig * E.h * E.t.y - x1};
        cplx K[2][2];
        field_kernel(P, z, E.n.x, E.n.y, w, K);
#pragma unroll
        for (int j = 0; j < RG; ++j) {
            if (j >= nj) break;
            const cplx cf = coef[e + (int64_t)(jb + j) * ldc];
            acc[j][0] = cadd(acc[j][0], cmul(K[0][c], cf));
            acc[j][1] = cadd(acc[j][1], cmul(K[1][c], cf));
        }
    }
    __shared__ double part[JT / 32][RG * 4];
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
        for (int w = 0; w < JT / 32; ++w) {
            re += part[w][4 * j + 2 * i];
            im += part[w][4 * j + 2 * i + 1];
        }
        cplx *o = out + J.x + (int64_t)i * npts + (int64_t)(jb + j) * ldo;
        atomicAdd(&o->x, -re);
        atomicAdd(&o->y, -im);
    }
}

// leaf-order coefficients from the natural-order solution (gidx: leaf position -> row)
__global__ void k_field_gather(const int *__restrict__ gidx, int64_t D, const cplx *__restrict__ u, int64_t ldu,
                               cplx *dst, int64_t ldd, int cols) {
    const int64_t tot = D * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = e % D, c = e / D;
        if (!FDS_IN_RANGE(gidx[q], D)) continue;
        dst[q + c * ldd] = u[gidx[q] + c * ldu];
    }
}

// children's skeleton coefficients (skeleton offsets roff, ld ldc) placed in
// the parent's DOF vector (ld ldp) as in eq. (rhs_rearrangement)
__global__ void k_field_to_parent(int nb, const int64_t *__restrict__ roff, const int *__restrict__ k1,
                                  const int *__restrict__ pos1, const int *__restrict__ pos2,
                                  const int64_t *__restrict__ pdoff, const cplx *__restrict__ child, int64_t ldc,
                                  cplx *parent, int64_t ldp, int cols) {
    const int b = blockIdx.x;
    const int64_t o = roff[b];
    const int r = (int)(roff[b + 1] - o);
    const int64_t pb = pdoff[b >> 1];
    for (int64_t e = threadIdx.x; e < (int64_t)r * cols; e += blockDim.x) {
        const int q = (int)(e % r);
        const int64_t c = e / r;
        const int64_t pr = q < k1[b] ? pos1[b] + q : pos2[b] + (q - k1[b]);
        if (!FDS_IN_RANGE(pr, pdoff[(b >> 1) + 1] - pb)) continue;
        parent[pb + pr + c * ldp] = child[o + q + c * ldc];
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

extern "C" int fds_field_compressed(fds_handle *h, const double *d_u, int32_t nrhs, const int32_t *kinds,
                                    const double *angles, const double *d_pts, int32_t npts, double *d_out,
                                    uint64_t stream) {
    if (!h || nrhs < 0 || npts < 0) return FDS_ERR_ARG;
    if (nrhs == 0 || npts == 0) return FDS_OK;
    if (!d_u || !kinds || !angles || !d_pts || !d_out) return FDS_ERR_ARG;
    for (int j = 0; j < nrhs; ++j)
        if ((kinds[j] != 0 && kinds[j] != 1) || !std::isfinite(angles[j])) return FDS_ERR_ARG;
    if (npts > 2147483647 / 2 || (nrhs + RG - 1) / RG > 65535) return FDS_ERR_ARG;
    const int L = h->L, l0 = h->l0, N = h->N;
    if (L == l0) return fds_field(h, d_u, nrhs, kinds, angles, d_pts, npts, d_out, stream);
    for (int l = L; l > l0; --l)
        if (!h->lv[l].T.p) return FDS_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    AllocStreamScope as(s);
    FDS_TRY(ensure_gauss_tables());
    // hat tables: the leaf DOFs, then the skeleton DOFs of levels L .. l0+1
    const Level &Lf = h->lv[L];
    std::vector<int64_t> eoff(L + 2, 0);   // eoff[l]: first entry of level l's skeletons; eoff[L + 1] = 0 (leaves)
    int64_t Etot = Lf.D;
    for (int l = L; l > l0; --l) {
        eoff[l] = Etot;
        Etot += h->lv[l].Rtot;
    }
    std::vector<int> hnode((size_t)Etot);
    std::vector<unsigned char> hcomp((size_t)Etot);
    for (int b = 0; b < Lf.nb; ++b)
        for (int q = 0; q < Lf.n1[b] + Lf.n2[b]; ++q) {
            hnode[Lf.doff[b] + q] = Lf.dof_node[Lf.doff[b] + q];
            hcomp[Lf.doff[b] + q] = q < Lf.n1[b] ? 0 : 1;
        }
    for (int l = L; l > l0; --l) {
        const Level &C = h->lv[l];
        for (int b = 0; b < C.nb; ++b)
            for (int q = 0; q < C.k1[b] + C.k2[b]; ++q) {
                const int c = q < C.k1[b] ? 0 : 1, qq = c ? q - C.k1[b] : q;
                const int pos = (c ? C.n1[b] : 0) + C.perm[C.permoff[2 * b + c] + qq];
                hnode[eoff[l] + C.roff[b] + q] = C.dof_node[C.doff[b] + pos];
                hcomp[eoff[l] + C.roff[b] + q] = (unsigned char)c;
            }
    }
    // jobs: per point, from the cells of level l0 + 1 down
    std::vector<double> pts(2 * (size_t)npts);
    FDS_CUDA_TRY(cudaMemcpyAsync(pts.data(), d_pts, sizeof(double) * pts.size(), cudaMemcpyDeviceToHost, s));
    FDS_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<int4> jobs;
    int64_t hats = 0;
    std::vector<std::pair<int, int>> stack;
    for (int p = 0; p < npts; ++p) {
        const double x0 = pts[2 * p], x1 = pts[2 * p + 1];
        if (!std::isfinite(x0) || !std::isfinite(x1)) return FDS_ERR_ARG;
        stack.clear();
        for (int c = h->lv[l0 + 1].nb - 1; c >= 0; --c) stack.push_back({l0 + 1, c});
        while (!stack.empty()) {
            const int l = stack.back().first, c = stack.back().second;
            stack.pop_back();
            const Level &C = h->lv[l];
            const double dx = x0 - C.cx[c], dy = x1 - C.cy[c];
            if (dx * dx + dy * dy > C.Rp[c] * C.Rp[c]) {
                const int cnt = (int)(C.roff[c + 1] - C.roff[c]);
                if (cnt) jobs.push_back(make_int4(p, (int)(eoff[l] + C.roff[c]), cnt, 0));
                hats += cnt;
            } else if (l == L) {
                const int cnt = (int)(C.doff[c + 1] - C.doff[c]);
                if (cnt) jobs.push_back(make_int4(p, (int)C.doff[c], cnt, 0));
                hats += cnt;
            } else {
                stack.push_back({l + 1, 2 * c + 1});
                stack.push_back({l + 1, 2 * c});
            }
        }
    }
    if (Etot > 2147483647 || jobs.size() > 2147483647u) return FDS_ERR_ARG;
    DBuf<int> d_hnode;
    DBuf<unsigned char> d_hcomp;
    DBuf<int4> d_jobs;
    DBuf<cplx> coef, X[2];
    FDS_TRY(d_hnode.upload(hnode, s));
    FDS_TRY(d_hcomp.upload(hcomp, s));
    FDS_TRY(d_jobs.upload(jobs, s));
    FDS_TRY(coef.alloc((size_t)Etot * nrhs));
    DBuf<int> dk;
    DBuf<double> da;
    FDS_TRY(dk.upload(std::vector<int>(kinds, kinds + nrhs), s));
    FDS_TRY(da.upload(std::vector<double>(angles, angles + nrhs), s));
    ProfScope ps("f1.field_compressed", s);
    ps.units = (double)hats * nrhs;
    // u~ of every compressed level: V_L u_leaf, then V_l [u~ of the children]
    fds_count_launch(), k_field_gather<<<1024, 256, 0, s>>>(h->d_leaf_gidx.p, Lf.D, (const cplx *)d_u, 2LL * N,
                                                            coef.p, Etot, nrhs);
    FDS_CUDA_TRY(cudaGetLastError());
    const cplx *in = coef.p;
    int64_t ldin = Etot;
    for (int l = L; l > l0; --l) {
        Level &C = h->lv[l];
        for (int c0 = 0; c0 < nrhs; c0 += SOLVE_CHUNK_FIELD) {
            const int nc = std::min(SOLVE_CHUNK_FIELD, nrhs - c0);
            FDS_TRY(apply_V<cplx>(h, C, C.T.p, in + c0 * ldin, ldin, coef.p + eoff[l] + c0 * Etot, Etot, nc, s));
        }
        if (l - 1 > l0) {
            Level &Pn = h->lv[l - 1];
            DBuf<cplx> &Xp = X[l & 1];
            FDS_TRY(Xp.alloc((size_t)Pn.D * nrhs));
            fds_count_launch(), k_field_to_parent<<<C.nb, 256, 0, s>>>(C.nb, C.d_roff.p, C.d_k1.p, C.d_par_pos1.p,
                                                                       C.d_par_pos2.p, Pn.d_doff.p,
                                                                       coef.p + eoff[l], Etot, Xp.p, Pn.D, nrhs);
            FDS_CUDA_TRY(cudaGetLastError());
            in = Xp.p;
            ldin = Pn.D;
        }
    }
    fds_count_launch(), k_field_incident<<<256, 256, 0, s>>>(h->P, dk.p, da.p, d_pts, npts, nrhs, (cplx *)d_out,
                                                             2LL * npts);
    FDS_CUDA_TRY(cudaGetLastError());
    if (!jobs.empty()) {
        dim3 grid((unsigned)jobs.size(), (nrhs + RG - 1) / RG);
        fds_count_launch(), k_field_jobs<<<grid, JT, 0, s>>>(h->P, h->d_xy.p, N, d_jobs.p, d_hnode.p, d_hcomp.p,
                                                             coef.p, Etot, nrhs, d_pts, npts, (cplx *)d_out,
                                                             2LL * npts);
        FDS_CUDA_TRY(cudaGetLastError());
    }
    FDS_CUDA_TRY(cudaStreamSynchronize(s));
    return FDS_OK;
}
