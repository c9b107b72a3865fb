// Device-side Galerkin kernel evaluation for the 2D elastodynamic
// Burton–Miller operator D + I_0/2 + alpha N (arXiv 2411.18026, Sec. 3 eq.
// (funda), Sec. 4 eq. (Aijpq)).
//
// Regularised Galerkin forms (tangential derivatives moved onto the P1
// test/trial hats; z = y - x, t = (n_2, -n_1), eps = [[0,1],[-1,0]],
// c = 2/k_T^2, F = g_T - g_L, g_k = (i/4) H0(k r)):
//   D: psi phi  [n^y_j d_i g_L + t^y_j eps_iq d_q g_T]
//      psi phi' -[2 eps_ji g_T + c eps_jp d_p d_i F]
//   N: psi phi  rho w^2 (n^x_i n^y_j g_L + t^x_i t^y_j g_T)
//      psi phi' -2 mu [t^x_i d_j g_T - n^x_i eps_jk d_k g_L]
//      psi' phi -2 mu [n^y_j eps_ik d_k g_L - t^y_j d_i g_T]
//      psi'phi'  2 mu [2 delta_ij g_T + c eps_ik eps_jp d_k d_p F]
// with d_k d_p F = -(i/4) P zh zh + (i/4) Q (2 zh zh - I),
// P = kT^2 H0(kT r) - kL^2 H0(kL r), Q = kT^2 E(kT r) - kL^2 E(kL r),
// E(z) = (z H1(z) + 2i/pi)/z^2.
//
// Quadrature rule per element pair (x on element e, y on element f):
//   self      (u, v) split of the unit square, u = w^5, 20 Gauss nodes in w,
//             4 in v; both triangles (u and -u) at every node -> principal value
//   adjacent  Duffy split at the shared vertex, xi = w^4, 16 x 8 nodes
//   near      midpoint distance < 2.5 max(h): halve both elements, 8x8 per sub-pair
//   mid       < 6 max(h): 8x8;   far: 6x6
//   cross     (proxy polygon vs boundary): fixed q x q.
#pragma once

#include "common.cuh"

namespace fdsk {

// ---------------------------------------------------------------- Bessel
// H0, H1 of the first kind from CUDA's j0/y0/j1/y1, and E(z) with the small-z
// branch from the ascending series of J_1 and Y_1 (Abramowitz & Stegun 9.1.10,
// 9.1.11), which keeps the difference of two E values free of pole cancellation.
struct Hank {
    cplx h0T, h1T, h0L, h1L, eT, eL;
};

__device__ __forceinline__ cplx ehat_series(double z) {
    // sum_{m>=0} t_m (1/2),  S = sum_{m>=0} (psi(m+1) + psi(m+2)) t_m,
    // t_m = (-z^2/4)^m / (m! (m+1)!)
    const double q = -0.25 * z * z;
    double t = 1.0, half_sum = 0.0, S = 0.0;
    double hm = 0.0;   // harmonic number H_m
    const double g = 0.57721566490153286061;
#pragma unroll
    for (int m = 0; m < 11; ++m) {
        // psi(m+1) + psi(m+2) = 2(H_m - g) + 1/(m+1)
        double ps = 2.0 * (hm - g) + 1.0 / (m + 1.0);
        half_sum += 0.5 * t;
        S += ps * t;
        hm += 1.0 / (m + 1.0);
        t *= q / ((m + 1.0) * (m + 2.0));
    }
    double re = half_sum;   // J1(z)/z
    double im = (2.0 / FDS_PI) * log(0.5 * z) * half_sum - S * (0.5 / FDS_PI);
    return mkc(re, im);
}

__device__ __forceinline__ void hankels_at(double z, cplx &h0, cplx &h1, cplx &e) {
    double a0 = j0(z), b0 = y0(z), a1 = j1(z), b1 = y1(z);
    h0 = mkc(a0, b0);
    h1 = mkc(a1, b1);
    if (z < 1.0) {
        e = ehat_series(z);
    } else {
        double iz2 = 1.0 / (z * z);
        e = mkc(z * a1 * iz2, (z * b1 + 2.0 / FDS_PI) * iz2);
    }
}

__device__ __forceinline__ Hank hankels(const PhysDev &P, double r) {
    Hank H;
    hankels_at(P.kT * r, H.h0T, H.h1T, H.eT);
    hankels_at(P.kL * r, H.h0L, H.h1L, H.eL);
    return H;
}

// ---------------------------------------------------------------- kernel
// Weighted kernel contribution: acc_ij += w (b0 K0 + b1 K1 + b2 K2 + b3 K3)
// for the operator D + alpha N at relative position z (test normal nx, trial
// normal ny), with the Hankel values of r = |z| precomputed.
__device__ __forceinline__ void kernel_accum(const PhysDev &P, const Hank &H, double2 z, double r,
                                             double2 nx, double2 ny, double w, double b0, double b1,
                                             double b2, double b3, cplx acc[2][2]) {
    const double ir = 1.0 / r;
    const double zh[2] = {z.x * ir, z.y * ir};
    const double nxv[2] = {nx.x, nx.y}, nyv[2] = {ny.x, ny.y};
    const double txv[2] = {nx.y, -nx.x}, tyv[2] = {ny.y, -ny.x};
    // g = (i/4) H0 ; g' = -(i/4) k H1
    const cplx gT = mkc(-0.25 * H.h0T.y, 0.25 * H.h0T.x);
    const cplx gL = mkc(-0.25 * H.h0L.y, 0.25 * H.h0L.x);
    const cplx gTp = mkc(0.25 * P.kT * H.h1T.y, -0.25 * P.kT * H.h1T.x);
    const cplx gLp = mkc(0.25 * P.kL * H.h1L.y, -0.25 * P.kL * H.h1L.x);
    const double kT2 = P.kT * P.kT, kL2 = P.kL * P.kL;
    const cplx Pf = mkc(kT2 * H.h0T.x - kL2 * H.h0L.x, kT2 * H.h0T.y - kL2 * H.h0L.y);
    const cplx Qf = mkc(kT2 * H.eT.x - kL2 * H.eL.x, kT2 * H.eT.y - kL2 * H.eL.y);
    // HF_ab = (i/4) [ (Q - P) zh_a zh_b - Q delta_ab ] ... written out:
    // -(i/4) P zz + (i/4) Q (2 zz - delta) = (i/4)[(2Q - P) zz - Q delta]
    const cplx iq4 = mkc(-0.25 * Qf.y, 0.25 * Qf.x);                 // (i/4) Q
    const cplx c2qp = mkc(2.0 * Qf.x - Pf.x, 2.0 * Qf.y - Pf.y);
    const cplx i2qp4 = mkc(-0.25 * c2qp.y, 0.25 * c2qp.x);           // (i/4)(2Q - P)
    cplx HF[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            HF[a][b] = cscale(i2qp4, zh[a] * zh[b]);
            if (a == b) HF[a][b] = csub(HF[a][b], iq4);
        }
    cplx dgT[2], dgL[2], edgT[2], edgL[2];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        dgT[a] = cscale(gTp, zh[a]);
        dgL[a] = cscale(gLp, zh[a]);
    }
    // (eps v)_1 = v_2, (eps v)_2 = -v_1
    edgT[0] = dgT[1]; edgT[1] = cneg(dgT[0]);
    edgL[0] = dgL[1]; edgL[1] = cneg(dgL[0]);
    // eps HF eps^T = [[HF22, -HF12], [-HF21, HF11]]
    cplx EHE[2][2] = {{HF[1][1], cneg(HF[0][1])}, {cneg(HF[1][0]), HF[0][0]}};
    // (eps HF)_{ji}: j=1 row [HF21, HF22], j=2 row [-HF11, -HF12]
    cplx EH[2][2] = {{HF[1][0], HF[1][1]}, {cneg(HF[0][0]), cneg(HF[0][1])}};   // EH[j][i]
    const double eps_[2][2] = {{0.0, 1.0}, {-1.0, 0.0}};
    const double c = P.c2, mu2 = 2.0 * P.mu;
    const cplx al = P.alpha;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            cplx D0 = cadd(cscale(dgL[i], nyv[j]), cscale(edgT[i], tyv[j]));
            cplx D1 = cneg(cadd(cscale(gT, 2.0 * eps_[j][i]), cscale(EH[j][i], c)));
            cplx N0 = cscale(cadd(cscale(gL, nxv[i] * nyv[j]), cscale(gT, txv[i] * tyv[j])), P.rw2);
            cplx N1 = cscale(csub(cscale(dgT[j], txv[i]), cscale(edgL[j], nxv[i])), -mu2);
            cplx N2 = cscale(csub(cscale(edgL[i], nyv[j]), cscale(dgT[i], tyv[j])), -mu2);
            cplx N3 = cscale(cadd(cscale(gT, i == j ? 2.0 : 0.0), cscale(EHE[i][j], c)), mu2);
            cplx Dsum = cadd(cscale(D0, b0), cscale(D1, b1));
            cplx Nsum = cadd(cadd(cscale(N0, b0), cscale(N1, b1)), cadd(cscale(N2, b2), cscale(N3, b3)));
            cplx v = cadd(Dsum, cmul(al, Nsum));
            acc[i][j].x = fma(w, v.x, acc[i][j].x);
            acc[i][j].y = fma(w, v.y, acc[i][j].y);
        }
}

// ---------------------------------------------------------------- elements
struct Elem {
    double2 a, t, n;
    double h;
};

__device__ __forceinline__ Elem load_elem(const double *__restrict__ xy, int N, int e) {
    int e1 = (e + 1 == N) ? 0 : e + 1;
    Elem E;
    double ax = xy[2 * e], ay = xy[2 * e + 1];
    double bx = xy[2 * e1], by = xy[2 * e1 + 1];
    double dx = bx - ax, dy = by - ay;
    E.h = sqrt(dx * dx + dy * dy);
    double ih = 1.0 / E.h;
    E.a = make_double2(ax, ay);
    E.t = make_double2(dx * ih, dy * ih);
    E.n = make_double2(-dy * ih, dx * ih);   // tangent rotated by +90 degrees
    return E;
}

enum PairKind { PK_SELF = 0, PK_ADJ_NEXT = 1, PK_ADJ_PREV = 2, PK_NEAR = 3, PK_MID = 4, PK_FAR = 5, PK_CROSS = 6 };

__device__ __forceinline__ int pair_kind(const Elem &E, const Elem &F, int ie, int jf, int N) {
    if (ie == jf) return PK_SELF;
    int in = (ie + 1 == N) ? 0 : ie + 1;
    int jn = (jf + 1 == N) ? 0 : jf + 1;
    if (jf == in) return PK_ADJ_NEXT;
    if (ie == jn) return PK_ADJ_PREV;
    double mx = E.a.x + 0.5 * E.h * E.t.x - (F.a.x + 0.5 * F.h * F.t.x);
    double my = E.a.y + 0.5 * E.h * E.t.y - (F.a.y + 0.5 * F.h * F.t.y);
    double d = sqrt(mx * mx + my * my);
    double L = fmax(E.h, F.h);
    if (d >= 6.0 * L) return PK_FAR;
    if (d >= 2.5 * L) return PK_MID;
    return PK_NEAR;
}

__device__ __forceinline__ int pair_points(int kind, int qcross) {
    switch (kind) {
        case PK_SELF: return 20 * 4;          // each node evaluates the +u and -u points
        case PK_ADJ_NEXT:
        case PK_ADJ_PREV: return 2 * 16 * 8;
        case PK_NEAR: return 4 * 64;
        case PK_MID: return 64;
        case PK_FAR: return 36;
        default: return qcross * qcross;
    }
}

// One quadrature point of the element-pair rule: local coordinates
// (sig on E, tau on F), relative vector z = y - x and weight (incl. h_e h_f).
// For PK_SELF the point p also has a mirror (sig, tau) <-> (tau, sig), z -> -z
// which the caller evaluates with the same weight.
__device__ __forceinline__ void pair_point(int kind, int p, int qcross, const Elem &E, const Elem &F,
                                           double &sig, double &tau, double2 &z, double &w) {
    const double hh = E.h * F.h;
    switch (kind) {
        case PK_SELF: {
            int a = p >> 2, b = p & 3;
            double wv = c_gauss.x[20][a];
            double w2 = wv * wv, w4 = w2 * w2;
            double u = w4 * wv;
            double du = c_gauss.w[20][a] * 5.0 * w4;
            double v = (1.0 - u) * c_gauss.x[4][b];
            w = du * (1.0 - u) * c_gauss.w[4][b] * hh;
            sig = v;
            tau = v + u;
            z = make_double2(u * E.h * E.t.x, u * E.h * E.t.y);
            return;
        }
        case PK_ADJ_NEXT:
        case PK_ADJ_PREV: {
            int tri = p >> 7, rem = p & 127;
            int a = rem >> 3, b = rem & 7;
            double wx = c_gauss.x[16][a];
            double wx2 = wx * wx;
            double xi = wx2 * wx2;
            double dxi = c_gauss.w[16][a] * 4.0 * wx2 * wx;
            double eta = c_gauss.x[8][b];
            double al = tri == 0 ? xi : xi * eta;
            double be = tri == 0 ? xi * eta : xi;
            w = dxi * c_gauss.w[8][b] * xi * hh;
            if (kind == PK_ADJ_NEXT) {
                sig = 1.0 - al;
                tau = be;
                z = make_double2(be * F.h * F.t.x + al * E.h * E.t.x, be * F.h * F.t.y + al * E.h * E.t.y);
            } else {
                sig = al;
                tau = 1.0 - be;
                z = make_double2(-be * F.h * F.t.x - al * E.h * E.t.x, -be * F.h * F.t.y - al * E.h * E.t.y);
            }
            return;
        }
        case PK_NEAR: {
            int sub = p >> 6, rem = p & 63;
            int a = rem >> 3, b = rem & 7;
            double s0 = 0.5 * (sub >> 1), t0 = 0.5 * (sub & 1);
            sig = s0 + 0.5 * c_gauss.x[8][a];
            tau = t0 + 0.5 * c_gauss.x[8][b];
            w = 0.25 * c_gauss.w[8][a] * c_gauss.w[8][b] * hh;
            break;
        }
        case PK_MID: {
            int a = p >> 3, b = p & 7;
            sig = c_gauss.x[8][a];
            tau = c_gauss.x[8][b];
            w = c_gauss.w[8][a] * c_gauss.w[8][b] * hh;
            break;
        }
        case PK_FAR: {
            int a = p / 6, b = p - 6 * (p / 6);
            sig = c_gauss.x[6][a];
            tau = c_gauss.x[6][b];
            w = c_gauss.w[6][a] * c_gauss.w[6][b] * hh;
            break;
        }
        default: {
            int a = p / qcross, b = p - qcross * (p / qcross);
            sig = c_gauss.x[qcross][a];
            tau = c_gauss.x[qcross][b];
            w = c_gauss.w[qcross][a] * c_gauss.w[qcross][b] * hh;
            break;
        }
    }
    double xx = E.a.x + sig * E.h * E.t.x, xy_ = E.a.y + sig * E.h * E.t.y;
    double yx = F.a.x + tau * F.h * F.t.x, yy = F.a.y + tau * F.h * F.t.y;
    z = make_double2(yx - xx, yy - xy_);
}

// Basis factors for test local index A on E (coordinate sig) and trial local
// index B on F (coordinate tau): b0 = N_A N_B, b1 = N_A N_B', b2 = N_A' N_B,
// b3 = N_A' N_B', with N_0 = 1 - s, N_1 = s, N_0' = -1/h, N_1' = 1/h.
__device__ __forceinline__ void basis4(int A, int B, double sig, double tau, double he, double hf,
                                       double &b0, double &b1, double &b2, double &b3) {
    double na = A ? sig : 1.0 - sig, nb = B ? tau : 1.0 - tau;
    double da = (A ? 1.0 : -1.0) / he, db = (B ? 1.0 : -1.0) / hf;
    b0 = na * nb; b1 = na * db; b2 = da * nb; b3 = da * db;
}

// Accumulate, in this lane, the part of element pair (E,F) assigned to it
// (points lane, lane+32, ...).  fwd: A(test hat on E with local index A,
// trial hat on F with local index B).  If rev != nullptr also the reversed
// entry A(test hat on F / B, trial hat on E / A) from the same point pairs.
__device__ __forceinline__ void pair_accum_lane(const PhysDev &P, int kind, int qcross, const Elem &E,
                                                const Elem &F, int A, int B, int lane, cplx fwd[2][2],
                                                cplx (*rev)[2]) {
    const int np = pair_points(kind, qcross);
    for (int p = lane; p < np; p += 32) {
        double sig, tau, w;
        double2 z;
        pair_point(kind, p, qcross, E, F, sig, tau, z, w);
        double r = sqrt(z.x * z.x + z.y * z.y);
        Hank H = hankels(P, r);
        double b0, b1, b2, b3;
        basis4(A, B, sig, tau, E.h, F.h, b0, b1, b2, b3);
        kernel_accum(P, H, z, r, E.n, F.n, w, b0, b1, b2, b3, fwd);
        if (rev) kernel_accum(P, H, make_double2(-z.x, -z.y), r, F.n, E.n, w, b0, b2, b1, b3, rev);
        if (kind == PK_SELF) {
            // mirror point: (sig, tau) <-> (tau, sig), z -> -z
            basis4(A, B, tau, sig, E.h, F.h, b0, b1, b2, b3);
            kernel_accum(P, H, make_double2(-z.x, -z.y), r, E.n, F.n, w, b0, b1, b2, b3, fwd);
            if (rev) kernel_accum(P, H, z, r, F.n, E.n, w, b0, b2, b1, b3, rev);
        }
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void warp_reduce_block(cplx a[2][2]) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            a[i][j].x = warp_sum(a[i][j].x);
            a[i][j].y = warp_sum(a[i][j].y);
        }
}

// Exact P1 mass entry int phi^s phi^t over the polygon.
__device__ __forceinline__ double mass_entry(const double *__restrict__ xy, int N, int s, int t) {
    int sp = (s == 0) ? N - 1 : s - 1;
    int tp = (t == 0) ? N - 1 : t - 1;
    double m = 0.0;
    // hat s: elements sp (local 1), s (local 0); hat t likewise
    int es[2] = {sp, s}, ls[2] = {1, 0};
    int et[2] = {tp, t}, lt[2] = {1, 0};
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
            if (es[a] == et[b]) {
                int e = es[a], e1 = (e + 1 == N) ? 0 : e + 1;
                double dx = xy[2 * e1] - xy[2 * e], dy = xy[2 * e1 + 1] - xy[2 * e + 1];
                double h = sqrt(dx * dx + dy * dy);
                m += (ls[a] == lt[b]) ? h / 3.0 : h / 6.0;
            }
    return m;
}

// Warp-cooperative Galerkin entry of the boundary matrix between test hat s
// and trial hat t (same polygon), including I_0/2.  If rev != nullptr the
// entry (t, s) is produced too from the same quadrature points.  Result is
// valid in every lane.
__device__ __forceinline__ void hat_pair_same(const PhysDev &P, const double *__restrict__ xy, int N, int s,
                                              int t, int lane, cplx out[2][2], cplx (*rev)[2]) {
    cplx f[2][2], r[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) { f[i][j] = mkc(0, 0); r[i][j] = mkc(0, 0); }
    const int sp = (s == 0) ? N - 1 : s - 1;
    const int tp = (t == 0) ? N - 1 : t - 1;
    for (int a = 0; a < 2; ++a) {
        const int ie = a == 0 ? sp : s, A = a == 0 ? 1 : 0;
        const Elem E = load_elem(xy, N, ie);
        for (int b = 0; b < 2; ++b) {
            const int jf = b == 0 ? tp : t, B = b == 0 ? 1 : 0;
            const Elem F = load_elem(xy, N, jf);
            const int kind = pair_kind(E, F, ie, jf, N);
            pair_accum_lane(P, kind, 0, E, F, A, B, lane, f, rev ? r : nullptr);
        }
    }
    warp_reduce_block(f);
    if (rev) warp_reduce_block(r);
    const double m = 0.5 * mass_entry(xy, N, s, t);
    f[0][0].x += m; f[1][1].x += m;
    r[0][0].x += m; r[1][1].x += m;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            out[i][j] = f[i][j];
            if (rev) rev[i][j] = r[i][j];
        }
}

// Warp-cooperative entry between test hat s on polygon X and trial hat t on
// polygon Y (fixed q x q rule, no mass).  With rev: also the entry of test
// hat t on Y against trial hat s on X.
__device__ __forceinline__ void hat_pair_cross(const PhysDev &P, const double *__restrict__ X, int NX, int s,
                                               const double *__restrict__ Y, int NY, int t, int q, int lane,
                                               cplx out[2][2], cplx (*rev)[2]) {
    cplx f[2][2], r[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) { f[i][j] = mkc(0, 0); r[i][j] = mkc(0, 0); }
    const int sp = (s == 0) ? NX - 1 : s - 1;
    const int tp = (t == 0) ? NY - 1 : t - 1;
    for (int a = 0; a < 2; ++a) {
        const Elem E = load_elem(X, NX, a == 0 ? sp : s);
        for (int b = 0; b < 2; ++b) {
            const Elem F = load_elem(Y, NY, b == 0 ? tp : t);
            pair_accum_lane(P, PK_CROSS, q, E, F, a == 0 ? 1 : 0, b == 0 ? 1 : 0, lane, f, rev ? r : nullptr);
        }
    }
    warp_reduce_block(f);
    if (rev) warp_reduce_block(r);
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            out[i][j] = f[i][j];
            if (rev) rev[i][j] = r[i][j];
        }
}

}  // namespace fdsk
