// Galerkin load vectors of plane incident waves (arXiv 2411.18026 Sec. 4,
// eq. (gal) right-hand side): f^s_i = int psi^s (u^I_i + alpha T^{n_x}_ij u^I_j) ds.
//   P  wave: u^I = d exp(i k_L d.x),      T u^I = i k_L e (lam n + 2 mu (n.d) d)
//   SV wave: u^I = d_perp exp(i k_T d.x), T u^I = i k_T mu e ((n.d) d_perp + (n.d_perp) d)
// 8-point Gauss on each element, each element integrated once per wave
// against both of its hats.
#include <algorithm>

#include "fds_internal.cuh"
#include "kernel_eval.cuh"
#include "prof.cuh"

namespace {

constexpr int RT = 256;   // nodes per CTA

// Integrals of one element against its two hats for one wave:
// J[0] = int (1 - sig) g (hat at the element's first node), J[1] = int sig g,
// g = u^I + alpha T u^I, both components.
__device__ __forceinline__ void element_load(const PhysDev &P, const double *__restrict__ xy, int N, int el,
                                             int kind, double d0, double d1, double k, cplx J[2][2]) {
    const double dp0 = -d1, dp1 = d0;
    const fdsk::Elem E = fdsk::load_elem(xy, N, el);
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
    for (int g = 0; g < 8; ++g) {
        const double sig = c_gauss.x[8][g];
        const double w = c_gauss.w[8][g] * E.h;
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
        s0 = cadd(s0, cscale(ph, w * (1.0 - sig)));
        s1 = cadd(s1, cscale(ph, w * sig));
    }
    J[0][0] = cmul(c0, s0);
    J[0][1] = cmul(c1, s0);
    J[1][0] = cmul(c0, s1);
    J[1][1] = cmul(c1, s1);
}

// CTA per (block of RT nodes, right-hand side): each element of the block is
// integrated once (plus the element before the block), then node s sums the
// contributions of elements s (weight 1 - sig) and s - 1 (weight sig).
__global__ void __launch_bounds__(RT) k_rhs(PhysDev P, const double *__restrict__ xy, int N,
                                            const int *__restrict__ kinds, const double *__restrict__ angles,
                                            cplx *f) {
    __shared__ cplx Js[RT + 1][2][2];
    const int j = blockIdx.y;
    const int s0 = blockIdx.x * RT;
    const int kind = kinds[j];
    double sd, cd;
    sincos(angles[j], &sd, &cd);
    const double k = kind == 0 ? P.kL : P.kT;
    const int t = threadIdx.x;
    if (s0 + t < N) element_load(P, xy, N, s0 + t, kind, cd, sd, k, Js[t + 1]);
    if (t == 0) element_load(P, xy, N, s0 == 0 ? N - 1 : s0 - 1, kind, cd, sd, k, Js[0]);
    __syncthreads();
    const int s = s0 + t;
    if (s >= N) return;
    // element s (slot t + 1) carries (1 - sig) for node s, element s - 1 (slot t) carries sig
    f[s + (int64_t)j * 2 * N] = cadd(Js[t][1][0], Js[t + 1][0][0]);
    f[s + N + (int64_t)j * 2 * N] = cadd(Js[t][1][1], Js[t + 1][0][1]);
}

}  // namespace

int fds_rhs_impl(fds_handle *h, const int *d_kinds, const double *d_angles, int nrhs, cplx *d_f, cudaStream_t s) {
    if (nrhs <= 0) return FDS_OK;
    FDS_TRY(ensure_gauss_tables());
    const int64_t tot = (int64_t)h->N * nrhs;
    ProfScope ps("a5.load_vectors", s);
    ps.units = (double)tot;
    for (int c0 = 0; c0 < nrhs; c0 += 65535) {   // grid.y limit
        const int nc = std::min(65535, nrhs - c0);
        dim3 grid(ceil_div_u(h->N, RT), nc);
        fds_count_launch(), k_rhs<<<grid, RT, 0, s>>>(h->P, h->d_xy.p, h->N, d_kinds + c0, d_angles + c0,
                                                     d_f + (int64_t)c0 * 2 * h->N);
    }
    FDS_CUDA_TRY(cudaGetLastError());
    return FDS_OK;
}
