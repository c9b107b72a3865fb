// Galerkin load vectors of plane incident waves (arXiv 2411.18026 Sec. 4,
// eq. (gal) right-hand side): f^s_i = int psi^s (u^I_i + alpha T^{n_x}_ij u^I_j) ds.
//   P  wave: u^I = d exp(i k_L d.x),      T u^I = i k_L e (lam n + 2 mu (n.d) d)
//   SV wave: u^I = d_perp exp(i k_T d.x), T u^I = i k_T mu e ((n.d) d_perp + (n.d_perp) d)
// One thread per (node, right-hand side); 8-point Gauss on each element of
// the hat's support.
#include "fds_internal.cuh"
#include "kernel_eval.cuh"
#include "prof.cuh"

namespace {

__global__ void k_rhs(PhysDev P, const double *__restrict__ xy, int N, const int *__restrict__ kinds,
                      const double *__restrict__ angles, int nrhs, cplx *f) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)N * nrhs) return;
    const int s = (int)(e % N), j = (int)(e / N);
    const int kind = kinds[j];
    double sd, cd;
    sincos(angles[j], &sd, &cd);
    const double d0 = cd, d1 = sd, dp0 = -sd, dp1 = cd;
    const double k = kind == 0 ? P.kL : P.kT;
    cplx acc0 = mkc(0, 0), acc1 = mkc(0, 0);
    for (int a = 0; a < 2; ++a) {
        const int el = a == 0 ? (s == 0 ? N - 1 : s - 1) : s;
        const fdsk::Elem E = fdsk::load_elem(xy, N, el);
        // phase k d.x at x = a + sig h t: theta_a + sig phi; exp(i sig phi) by
        // its Taylor polynomial while |phi| < 0.05 (error < 3e-20), else sincos
        double sa, ca;
        sincos(k * (d0 * E.a.x + d1 * E.a.y), &sa, &ca);
        const double phi = k * E.h * (d0 * E.t.x + d1 * E.t.y);
        for (int g = 0; g < 8; ++g) {
            const double sig = c_gauss.x[8][g];
            const double w = c_gauss.w[8][g] * E.h * (a == 0 ? sig : 1.0 - sig);
            const double xg = sig * phi;
            double sx, cx;
            if (fabs(phi) < 0.05) {
                const double x2 = xg * xg;
                cx = 1.0 + x2 * (-1.0 / 2 + x2 * (1.0 / 24 + x2 * (-1.0 / 720 + x2 * (1.0 / 40320))));
                sx = xg * (1.0 + x2 * (-1.0 / 6 + x2 * (1.0 / 120 + x2 * (-1.0 / 5040 + x2 * (1.0 / 362880)))));
            } else {
                sincos(xg, &sx, &cx);
            }
            const cplx ph = mkc(ca * cx - sa * sx, sa * cx + ca * sx);
            const double n0 = E.n.x, n1 = E.n.y;
            cplx u0, u1, t0, t1;
            if (kind == 0) {
                const double nd = n0 * d0 + n1 * d1;
                u0 = cscale(ph, d0);
                u1 = cscale(ph, d1);
                const cplx ik = cmul(mkc(0, k), ph);
                t0 = cscale(ik, P.lam * n0 + 2.0 * P.mu * nd * d0);
                t1 = cscale(ik, P.lam * n1 + 2.0 * P.mu * nd * d1);
            } else {
                const double nd = n0 * d0 + n1 * d1, ndp = n0 * dp0 + n1 * dp1;
                u0 = cscale(ph, dp0);
                u1 = cscale(ph, dp1);
                const cplx ik = cmul(mkc(0, k * P.mu), ph);
                t0 = cscale(ik, nd * dp0 + ndp * d0);
                t1 = cscale(ik, nd * dp1 + ndp * d1);
            }
            acc0 = cadd(acc0, cscale(cadd(u0, cmul(P.alpha, t0)), w));
            acc1 = cadd(acc1, cscale(cadd(u1, cmul(P.alpha, t1)), w));
        }
    }
    f[s + (int64_t)j * 2 * N] = acc0;
    f[s + N + (int64_t)j * 2 * N] = acc1;
}

}  // namespace

int fds_rhs_impl(fds_handle *h, const int *d_kinds, const double *d_angles, int nrhs, cplx *d_f, cudaStream_t s) {
    if (nrhs <= 0) return FDS_OK;
    FDS_TRY(ensure_gauss_tables());
    const int64_t tot = (int64_t)h->N * nrhs;
    ProfScope ps("a5.load_vectors", s);
    ps.units = (double)tot;
    fds_count_launch(), k_rhs<<<ceil_div_u(tot, 256), 256, 0, s>>>(h->P, h->d_xy.p, h->N, d_kinds, d_angles, nrhs, d_f);
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}
