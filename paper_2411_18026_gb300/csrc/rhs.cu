// Galerkin load vectors of plane incident waves (arXiv 2411.18026 Sec. 4,
// eq. (gal) right-hand side): f^s_i = int psi^s (u^I_i + alpha T^{n_x}_ij u^I_j) ds.
//   P  wave: u^I = d exp(i k_L d.x),      T u^I = i k_L e (lam n + 2 mu (n.d) d)
//   SV wave: u^I = d_perp exp(i k_T d.x), T u^I = i k_T mu e ((n.d) d_perp + (n.d_perp) d)
// Each element is integrated once per wave against both of its hats.  Along
// the element the phase is theta_a + sig phi, so the two hat integrals are
// h e^{i theta_a} times
//   S0(phi) = int_0^1 (1 - sig) e^{i sig phi} dsig = sum_n (i phi)^n / (n+2)!,
//   S1(phi) = int_0^1 sig e^{i sig phi} dsig      = sum_n (n+1) (i phi)^n / (n+2)!,
// summed through n = 8 while |phi| < 0.05 (next term below 1e-19); larger
// phase steps use the 8-point Gauss rule.
#include <algorithm>

#include "fds_internal.cuh"
#include "kernel_eval.cuh"
#include "prof.cuh"

namespace {

constexpr int RT = 256;   // nodes per CTA
constexpr int WPB = 4;    // waves per CTA (the element geometry is shared)

// Integrals of one element against its two hats for one wave:
// J[0] = int (1 - sig) g (hat at the element's first node), J[1] = int sig g,
// g = u^I + alpha T u^I, both components.
__device__ __forceinline__ void element_load(const PhysDev &P, const fdsk::Elem &E, int kind, double d0,
                                             double d1, double k, cplx J[2][2]) {
    const double dp0 = -d1, dp1 = d0;
    // phase k d.x at x = a + sig h t: theta_a + sig phi; exp(i sig phi) by its
    // Taylor polynomial while |phi| < 0.05 (error < 3e-20), else sincos
    double sa, ca;
    sincos(k * (d0 * E.a.x + d1 * E.a.y), &sa, &ca);
    const double phi = k * E.h * (d0 * E.t.x + d1 * E.t.y);
    const double n0 = E.n.x, n1 = E.n.y;
    // u = amp * ph, T u = i k tr * ph (per component)
    double amp0, amp1, tr0, tr1, kk;
    if (kind == 0) {
        const double nd = n0 * d0 + n1 * d1;
        amp0 = d0;
        amp1 = d1;
        tr0 = P.lam * n0 + 2.0 * P.mu * nd * d0;
        tr1 = P.lam * n1 + 2.0 * P.mu * nd * d1;
        kk = k;
    } else {
        const double nd = n0 * d0 + n1 * d1, ndp = n0 * dp0 + n1 * dp1;
        amp0 = dp0;
        amp1 = dp1;
        tr0 = nd * dp0 + ndp * d0;
        tr1 = nd * dp1 + ndp * d1;
        kk = k * P.mu;
    }
    // g_c = ph (amp_c + alpha i kk tr_c)
    const cplx ia = cmul(P.alpha, mkc(0.0, kk));
    const cplx c0 = cadd(mkc(amp0, 0.0), cscale(ia, tr0)), c1 = cadd(mkc(amp1, 0.0), cscale(ia, tr1));
    cplx s0 = mkc(0, 0), s1 = mkc(0, 0);      // int (1 - sig) ph, int sig ph
    if (fabs(phi) < 0.05) {
        // even / odd powers of i phi in p = -phi^2; 1/(n+2)! and (n+1)/(n+2)!
        const double p = -phi * phi;
        const double r0 = 1.0 / 2 + p * (1.0 / 24 + p * (1.0 / 720 + p * (1.0 / 40320 + p * (1.0 / 3628800))));
        const double i0 = phi * (1.0 / 6 + p * (1.0 / 120 + p * (1.0 / 5040 + p * (1.0 / 362880))));
        const double r1 = 1.0 / 2 + p * (3.0 / 24 + p * (5.0 / 720 + p * (7.0 / 40320 + p * (9.0 / 3628800))));
        const double i1 = phi * (2.0 / 6 + p * (4.0 / 120 + p * (6.0 / 5040 + p * (8.0 / 362880))));
        const cplx e = mkc(ca * E.h, sa * E.h);
        s0 = cmul(e, mkc(r0, i0));
        s1 = cmul(e, mkc(r1, i1));
    } else {
        for (int g = 0; g < 8; ++g) {
            const double sig = c_gauss.x[8][g];
            const double w = c_gauss.w[8][g] * E.h;
            double sx, cx;
            sincos(sig * phi, &sx, &cx);
            const cplx ph = mkc(ca * cx - sa * sx, sa * cx + ca * sx);
            s0 = cadd(s0, cscale(ph, w * (1.0 - sig)));
            s1 = cadd(s1, cscale(ph, w * sig));
        }
    }
    J[0][0] = cmul(c0, s0);
    J[0][1] = cmul(c1, s0);
    J[1][0] = cmul(c0, s1);
    J[1][1] = cmul(c1, s1);
}

// CTA per (block of RT nodes, WPB right-hand sides): each element of the
// block (plus the element before the block) is loaded once and integrated
// once per wave, then node s sums the contributions of elements s (weight
// 1 - sig) and s - 1 (weight sig).
__global__ void __launch_bounds__(RT) k_rhs(PhysDev P, const double *__restrict__ xy, int N, int nrhs,
                                            const int *__restrict__ kinds, const double *__restrict__ angles,
                                            cplx *f) {
    __shared__ cplx Js[RT + 1][2][2];
    const int s0 = blockIdx.x * RT;
    const int t = threadIdx.x;
    const int s = s0 + t;
    fdsk::Elem E, Eb;
    if (s < N) E = fdsk::load_elem(xy, N, s);
    if (t == 0) Eb = fdsk::load_elem(xy, N, s0 == 0 ? N - 1 : s0 - 1);
    for (int w = 0; w < WPB; ++w) {
        const int j = blockIdx.y * WPB + w;
        if (j >= nrhs) break;
        const int kind = kinds[j];
        double sd, cd;
        sincos(angles[j], &sd, &cd);
        const double k = kind == 0 ? P.kL : P.kT;
        if (s < N) element_load(P, E, kind, cd, sd, k, Js[t + 1]);
        if (t == 0) element_load(P, Eb, kind, cd, sd, k, Js[0]);
        __syncthreads();
        if (s < N) {
            // element s (slot t + 1) carries (1 - sig) for node s, element s - 1 (slot t) carries sig
            f[s + (int64_t)j * 2 * N] = cadd(Js[t][1][0], Js[t + 1][0][0]);
            f[s + N + (int64_t)j * 2 * N] = cadd(Js[t][1][1], Js[t + 1][0][1]);
        }
        __syncthreads();
    }
}

}  // namespace

int fds_rhs_impl(fds_handle *h, const int *d_kinds, const double *d_angles, int nrhs, cplx *d_f, cudaStream_t s) {
    if (nrhs <= 0) return FDS_OK;
    FDS_TRY(ensure_gauss_tables());
    const int64_t tot = (int64_t)h->N * nrhs;
    ProfScope ps("a5.load_vectors", s);
    ps.units = (double)tot;
    for (int c0 = 0; c0 < nrhs; c0 += 65535 * WPB) {   // grid.y limit
        const int nc = std::min(65535 * WPB, nrhs - c0);
        dim3 grid(ceil_div_u(h->N, RT), (nc + WPB - 1) / WPB);
        fds_count_launch(), k_rhs<<<grid, RT, 0, s>>>(h->P, h->d_xy.p, h->N, nc, d_kinds + c0, d_angles + c0,
                                                     d_f + (int64_t)c0 * 2 * h->N);
    }
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}
