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
// with d_k d_p F = (i/4) [(2Q - P) zh_k zh_p - Q delta_kp],
// P = kT^2 H0(kT r) - kL^2 H0(kL r), Q = kT^2 E(kT r) - kL^2 E(kL r),
// E(z) = (z H1(z) + 2i/pi)/z^2.
//
// Quadrature rule per element pair (x on element e, y on element f):
//   self      (u, v) split of the unit square, u = w^5, 20 Gauss nodes in w,
//             4 in v; both triangles (u and -u) at every node -> principal value
//   adjacent  Duffy split at the shared vertex, xi = w^4, 16 x 8 nodes
//   near      midpoint distance < 2.5 max(h): halve both elements, 8x8 per sub-pair
//   mid       < 6 max(h): 8x8;   far: < 12 max(h): 6x6;   far2: 4x4;
//   far3      >= 24 max(h) with k_T max(h) <= 0.02: 3x3
//   cross     (proxy polygon vs boundary): fixed q x q (the build uses q = 2).
//
// Work is organised in tiles of at most TILE test hats x TILE trial hats:
// the hats' supporting elements are deduplicated (consecutive hats share an
// element), every element-pair integral is evaluated once for all four P1
// basis combinations and, optionally, for the transposed entry from the same
// quadrature points, then scattered into the tile's entries in shared memory.
#pragma once

#include "common.cuh"

namespace fdsk {

#ifndef FDS_TILE_THREADS
#define FDS_TILE_THREADS 128
#endif

constexpr int TILE = 15;        // 15 consecutive hats span 16 elements: 256 element pairs

// Quadrature points evaluated (point pairs x orientations), counted when
// d_count_points is set; read back by the timing registry.
static __device__ unsigned long long d_quad_points;
static __device__ int d_count_points;
constexpr int TILE_EL = 2 * TILE;      // worst case: no shared elements

// ---------------------------------------------------------------- rules
// Gauss–Legendre nodes/weights on [0,1] copied into shared memory at the
// start of a kernel (divergent indices would serialise __constant__ reads).
struct Rules {
    double x3[3], w3[3], x4[4], w4[4], x6[6], w6[6], x8[8], w8[8], x16[16], w16[16], x20[20], w20[20];
    double xq[8], wq[8];
    int q;
};

__device__ __forceinline__ void load_rules(Rules &R, int qcross) {
    for (int i = threadIdx.x; i < 20; i += blockDim.x) {
        if (i < 3) { R.x3[i] = c_gauss.x[3][i]; R.w3[i] = c_gauss.w[3][i]; }
        if (i < 4) { R.x4[i] = c_gauss.x[4][i]; R.w4[i] = c_gauss.w[4][i]; }
        if (i < 6) { R.x6[i] = c_gauss.x[6][i]; R.w6[i] = c_gauss.w[6][i]; }
        if (i < 8) { R.x8[i] = c_gauss.x[8][i]; R.w8[i] = c_gauss.w[8][i]; }
        if (i < 16) { R.x16[i] = c_gauss.x[16][i]; R.w16[i] = c_gauss.w[16][i]; }
        R.x20[i] = c_gauss.x[20][i];
        R.w20[i] = c_gauss.w[20][i];
        if (qcross > 0 && i < qcross) { R.xq[i] = c_gauss.x[qcross][i]; R.wq[i] = c_gauss.w[qcross][i]; }
    }
    if (threadIdx.x == 0) R.q = qcross;
}

// ---------------------------------------------------------------- Bessel
// H0^(1)(z), H1^(1)(z) and E(z) = (z H1(z) + 2i/pi)/z^2.  For z < 2 from the
// ascending series (Abramowitz & Stegun 9.1.10, 9.1.11, 9.1.13) as
// polynomials in q = -z^2/4 with tabulated coefficients (Horner):
//   J0 = sum q^m/(m!)^2,  J1/z = (1/2) sum q^m/(m!(m+1)!),
//   Y0 = (2/pi) [ (ln(z/2) + g) J0 - sum_{m>=1} H_m q^m/(m!)^2 ],
//   Im E = (2/pi) ln(z/2) J1/z - (1/(2 pi)) sum (2 (H_m - g) + 1/(m+1)) q^m/(m!(m+1)!),
//   Y1 = z Im E - 2/(pi z).
// 14 terms reach 1e-16 for z < 2, 8 for z < 0.63, 6 for z < 0.2, 4 for
// z < 0.02 and 3 for z < 0.002 (the tails are below 1e-17 of the leading
// terms).  For z >= 2 from CUDA's
// j0/y0/j1/y1.
struct Hk {
    cplx h0, h1, e;
};

// Coefficients are read from __constant__ memory: every lane reads the same
// address, so the reads are broadcasts and need no registers.
template <int M>
__device__ __forceinline__ void series4(const Rules &G, double q, double &J0, double &Su, double &SH, double &Sp) {
    (void)G;
    J0 = c_gauss.sa[M - 1];
    Su = c_gauss.sb[M - 1];
    SH = c_gauss.sh[M - 1];
    Sp = c_gauss.sp[M - 1];
#pragma unroll
    for (int m = M - 2; m >= 0; --m) {
        J0 = fma(J0, q, c_gauss.sa[m]);
        Su = fma(Su, q, c_gauss.sb[m]);
        SH = fma(SH, q, c_gauss.sh[m]);
        Sp = fma(Sp, q, c_gauss.sp[m]);
    }
}

__device__ __forceinline__ Hk hankel_k(const Rules &G, double z, double lhalf) {
    Hk H;
    if (z < 2.0) {
        const double g = 0.57721566490153286061;
        const double q = -0.25 * z * z;
        double J0, Su, SH, Sp;
        // terms needed for 1e-17 relative: 3 below z = 0.002, 4 below 0.02,
        // 6 below 0.2, 8 below 0.63
        if (q > -1e-6) series4<3>(G, q, J0, Su, SH, Sp);
        else if (q > -1e-4) series4<4>(G, q, J0, Su, SH, Sp);
        else if (q > -0.01) series4<6>(G, q, J0, Su, SH, Sp);
        else if (q > -0.1) series4<8>(G, q, J0, Su, SH, Sp);
        else series4<SER_TERMS>(G, q, J0, Su, SH, Sp);
        const double j1z = 0.5 * Su;                      // J1(z)/z
        const double Y0 = (2.0 / FDS_PI) * ((lhalf + g) * J0 - SH);
        const double eim = (2.0 / FDS_PI) * lhalf * j1z - Sp * (0.5 / FDS_PI);
        H.h0 = mkc(J0, Y0);
        H.e = mkc(j1z, eim);
        H.h1 = mkc(z * j1z, z * eim - (2.0 / FDS_PI) / z);
    } else {
        const double a0 = j0(z), b0 = y0(z), a1 = j1(z), b1 = y1(z);
        const double iz2 = 1.0 / (z * z);
        H.h0 = mkc(a0, b0);
        H.h1 = mkc(a1, b1);
        H.e = mkc(z * a1 * iz2, (z * b1 + 2.0 / FDS_PI) * iz2);
    }
    return H;
}

// ---------------------------------------------------------------- radial part
// Quantities of the kernel that depend on r only (shared by both entry
// orientations of a point pair).
struct Radial {
    cplx gT, gL;       // g_T, g_L
    cplx gTp, gLp;     // g_T', g_L'  (d/dr)
    cplx a, b;         // d_k d_p F = a zh_k zh_p - b delta_kp
};

__device__ __forceinline__ Radial radial(const PhysDev &P, const Rules &G, double r) {
    // ln r enters the series branch only (z < 2; k_L < k_T)
    const double lr = (P.kL * r < 2.0) ? log(r) : 0.0;
    const Hk T = hankel_k(G, P.kT * r, P.lhalfT + lr);
    const Hk L = hankel_k(G, P.kL * r, P.lhalfL + lr);
    Radial R;
    // g = (i/4) H0 ; g' = -(i/4) k H1
    R.gT = mkc(-0.25 * T.h0.y, 0.25 * T.h0.x);
    R.gL = mkc(-0.25 * L.h0.y, 0.25 * L.h0.x);
    R.gTp = mkc(0.25 * P.kT * T.h1.y, -0.25 * P.kT * T.h1.x);
    R.gLp = mkc(0.25 * P.kL * L.h1.y, -0.25 * P.kL * L.h1.x);
    const double kT2 = P.kT * P.kT, kL2 = P.kL * P.kL;
    const cplx Pf = mkc(kT2 * T.h0.x - kL2 * L.h0.x, kT2 * T.h0.y - kL2 * L.h0.y);
    const cplx Qf = mkc(kT2 * T.e.x - kL2 * L.e.x, kT2 * T.e.y - kL2 * L.e.y);
    // a = (i/4)(2Q - P), b = (i/4) Q
    R.a = mkc(-0.25 * (2.0 * Qf.y - Pf.y), 0.25 * (2.0 * Qf.x - Pf.x));
    R.b = mkc(-0.25 * Qf.y, 0.25 * Qf.x);
    return R;
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

enum PairKind {
    PK_SELF = 0, PK_ADJ_NEXT = 1, PK_ADJ_PREV = 2, PK_NEAR = 3, PK_MID = 4, PK_FAR = 5, PK_FAR2 = 6, PK_CROSS = 7,
    PK_FAR3 = 8, PK_SKIP = 9    // PK_SKIP: a pair a diagonal tile leaves out
};
constexpr int PK_N = 10;

__device__ __forceinline__ int pair_kind(const Elem &E, const Elem &F, int ie, int jf, int N, double kT) {
    if (ie == jf) return PK_SELF;
    int in = (ie + 1 == N) ? 0 : ie + 1;
    int jn = (jf + 1 == N) ? 0 : jf + 1;
    if (jf == in) return PK_ADJ_NEXT;
    if (ie == jn) return PK_ADJ_PREV;
    double mx = E.a.x + 0.5 * E.h * E.t.x - (F.a.x + 0.5 * F.h * F.t.x);
    double my = E.a.y + 0.5 * E.h * E.t.y - (F.a.y + 0.5 * F.h * F.t.y);
    // midpoint distance d against multiples of L, compared as squares
    const double d2 = mx * mx + my * my;
    const double L = fmax(E.h, F.h), L2 = L * L;
    if (d2 >= 576.0 * L2 && kT * L <= 0.02) return PK_FAR3;   // d >= 24 L
    if (d2 >= 144.0 * L2) return PK_FAR2;                      // d >= 12 L
    if (d2 >= 36.0 * L2) return PK_FAR;                        // d >= 6 L
    if (d2 >= 6.25 * L2) return PK_MID;                        // d >= 2.5 L
    return PK_NEAR;
}

__device__ __forceinline__ bool cheap_kind(int kind) { return kind >= PK_MID; }

__device__ __forceinline__ int pair_points(int kind, int qcross) {
    switch (kind) {
        case PK_SELF: return 20 * 4;          // each node evaluates the +u and -u points
        case PK_ADJ_NEXT:
        case PK_ADJ_PREV: return 2 * 16 * 8;
        case PK_NEAR: return 4 * 64;
        case PK_MID: return 64;
        case PK_FAR: return 36;
        case PK_FAR2: return 16;
        case PK_FAR3: return 9;
        default: return qcross * qcross;
    }
}

// One quadrature point of the element-pair rule: local coordinates
// (sig on E, tau on F), relative vector z = y - x and weight (incl. h_e h_f).
// For PK_SELF the point also has the mirror (sig, tau) <-> (tau, sig), z -> -z.
__device__ __forceinline__ void pair_point(const Rules &G, int kind, int p, const Elem &E, const Elem &F,
                                           double &sig, double &tau, double2 &z, double &w) {
    const double hh = E.h * F.h;
    switch (kind) {
        case PK_SELF: {
            const int a = p >> 2, b = p & 3;
            const double wv = G.x20[a];
            const double w2 = wv * wv, w4 = w2 * w2;
            const double u = w4 * wv;
            const double du = G.w20[a] * 5.0 * w4;
            const double v = (1.0 - u) * G.x4[b];
            w = du * (1.0 - u) * G.w4[b] * hh;
            sig = v;
            tau = v + u;
            z = make_double2(u * E.h * E.t.x, u * E.h * E.t.y);
            return;
        }
        case PK_ADJ_NEXT:
        case PK_ADJ_PREV: {
            const int tri = p >> 7, rem = p & 127;
            const int a = rem >> 3, b = rem & 7;
            const double wx = G.x16[a];
            const double wx2 = wx * wx;
            const double xi = wx2 * wx2;
            const double dxi = G.w16[a] * 4.0 * wx2 * wx;
            const double eta = G.x8[b];
            const double al = tri == 0 ? xi : xi * eta;
            const double be = tri == 0 ? xi * eta : xi;
            w = dxi * G.w8[b] * xi * hh;
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
            const int sub = p >> 6, rem = p & 63;
            const int a = rem >> 3, b = rem & 7;
            sig = 0.5 * (sub >> 1) + 0.5 * G.x8[a];
            tau = 0.5 * (sub & 1) + 0.5 * G.x8[b];
            w = 0.25 * G.w8[a] * G.w8[b] * hh;
            break;
        }
        case PK_MID: {
            const int a = p >> 3, b = p & 7;
            sig = G.x8[a];
            tau = G.x8[b];
            w = G.w8[a] * G.w8[b] * hh;
            break;
        }
        case PK_FAR: {
            const int a = p / 6, b = p - 6 * (p / 6);
            sig = G.x6[a];
            tau = G.x6[b];
            w = G.w6[a] * G.w6[b] * hh;
            break;
        }
        case PK_FAR2: {
            const int a = p >> 2, b = p & 3;
            sig = G.x4[a];
            tau = G.x4[b];
            w = G.w4[a] * G.w4[b] * hh;
            break;
        }
        case PK_FAR3: {
            const int a = p / 3, b = p - 3 * (p / 3);
            sig = G.x3[a];
            tau = G.x3[b];
            w = G.w3[a] * G.w3[b] * hh;
            break;
        }
        default: {
            const int q = G.q;
            const int a = p / q, b = p - q * (p / q);
            sig = G.xq[a];
            tau = G.xq[b];
            w = G.wq[a] * G.wq[b] * hh;
            break;
        }
    }
    const double xx = E.a.x + sig * E.h * E.t.x, xy_ = E.a.y + sig * E.h * E.t.y;
    const double yx = F.a.x + tau * F.h * F.t.x, yy = F.a.y + tau * F.h * F.t.y;
    z = make_double2(yx - xx, yy - xy_);
}

// ---------------------------------------------------------------- accumulation
// Element-pair accumulator, flat so that every index is a compile-time
// constant (keeps it in registers): v[fidx(A,B,i,j)] is the integral for the
// test hat with local index A on E against the trial hat with local index B on
// F (component block i, j); v[ridx(B,A,i,j)] the transposed entry (test hat B
// on F, trial hat A on E) from the same points.
struct PairAcc {
    double v[32];
};
#define FIDX(A, B, i, j) (((((A)*2 + (B)) * 4) + (i)*2 + (j)) * 2)
#define RIDX(B, A, i, j) (32 + ((((B)*2 + (A)) * 4) + (i)*2 + (j)) * 2)

__device__ __forceinline__ void acc_zero(PairAcc &S) {
#pragma unroll
    for (int k = 0; k < 32; ++k) S.v[k] = 0.0;
}

// Per-point quantities shared by both orientations of a point pair.
struct PointShared {
    Radial R;
    double zx, zy;          // unit vector zh = z / r (forward orientation)
    cplx AgL, AgT;          // alpha rho w^2 g_L, alpha rho w^2 g_T
    cplx MgTp, MgLp;        // -2 mu alpha g_T', -2 mu alpha g_L'
    cplx k3_00, k3_11, k3_01;   // K3 = 2 mu alpha (2 delta g_T + c (a zp zp^T - b I))
    cplx e1[2][2];          // even part of K1: -(2 eps_ji g_T + c (a zp_j zh_i - b eps_ji))
};

__device__ __forceinline__ void point_shared(const PhysDev &P, const Rules &G, double2 z, PointShared &Q) {
    const double r = sqrt(z.x * z.x + z.y * z.y);
    const double ir = 1.0 / r;
    Q.zx = z.x * ir;
    Q.zy = z.y * ir;
    Q.R = radial(P, G, r);
    Q.AgL = cmul(P.alpha_rw2, Q.R.gL);
    Q.AgT = cmul(P.alpha_rw2, Q.R.gT);
    Q.MgTp = cmul(P.alpha_m2mu, Q.R.gTp);
    Q.MgLp = cmul(P.alpha_m2mu, Q.R.gLp);
    const double zp0 = Q.zy, zp1 = -Q.zx;
    const cplx ca = cscale(Q.R.a, P.c2);
    const cplx A2 = cscale(P.alpha_m2mu, -1.0);                      // 2 mu alpha
    const cplx k3d = csub(cscale(Q.R.gT, 2.0), cscale(Q.R.b, P.c2));
    Q.k3_00 = cmul(A2, cadd(cscale(ca, zp0 * zp0), k3d));
    Q.k3_11 = cmul(A2, cadd(cscale(ca, zp1 * zp1), k3d));
    Q.k3_01 = cmul(A2, cscale(ca, zp0 * zp1));
    // e1_ij = -c a zp_j zh_i + eps_ji (c b - 2 g_T); eps_01 = 1, eps_10 = -1
    const cplx cb2 = csub(cscale(Q.R.b, P.c2), cscale(Q.R.gT, 2.0));
    const double zh[2] = {Q.zx, Q.zy}, zp[2] = {zp0, zp1};
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            cplx v = cscale(ca, -zp[j] * zh[i]);
            if (j == 0 && i == 1) v = cadd(v, cb2);
            if (j == 1 && i == 0) v = csub(v, cb2);
            Q.e1[i][j] = v;
        }
}

// K0, K1, K2 of D + alpha N for one orientation: test normal nx, trial normal
// ny, direction zh scaled by sgn (+1 forward, -1 transposed):
//   K0_ij = P_i n^y_j + Q_i t^y_j,  P_i = g_L' zh_i + alpha rho w^2 g_L n^x_i,
//                                  Q_i = g_T' zp_i + alpha rho w^2 g_T t^x_i
//   K1_ij = e1_ij + t^x_i X_j + n^x_i Y_j,  X_j = -2 mu alpha g_T' zh_j,
//                                          Y_j = 2 mu alpha g_L' zp_j
//   K2_ij = -(n^y_j Y_i + t^y_j X_i)
__device__ __forceinline__ void blocks_orient(const PointShared &Q, double sgn, double2 nx, double2 ny,
                                              cplx k0[2][2], cplx k1[2][2], cplx k2[2][2]) {
    const double zh[2] = {sgn * Q.zx, sgn * Q.zy}, zp[2] = {sgn * Q.zy, -sgn * Q.zx};
    const double nxv[2] = {nx.x, nx.y}, txv[2] = {nx.y, -nx.x};
    const double nyv[2] = {ny.x, ny.y}, tyv[2] = {ny.y, -ny.x};
    cplx Pv[2], Qv[2], X[2], Y[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        Pv[i] = cadd(cscale(Q.R.gLp, zh[i]), cscale(Q.AgL, nxv[i]));
        Qv[i] = cadd(cscale(Q.R.gTp, zp[i]), cscale(Q.AgT, txv[i]));
        X[i] = cscale(Q.MgTp, zh[i]);
        Y[i] = cscale(Q.MgLp, -zp[i]);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            k0[i][j] = cadd(cscale(Pv[i], nyv[j]), cscale(Qv[i], tyv[j]));
            k1[i][j] = cadd(Q.e1[i][j], cadd(cscale(X[j], txv[i]), cscale(Y[j], nxv[i])));
            k2[i][j] = cneg(cadd(cscale(Y[i], nyv[j]), cscale(X[i], tyv[j])));
        }
}

// acc[T][U] += sum over the four kernel blocks with weights
//   b0 = nt[T] ns[U], b1 = nt[T] ds[U], b2 = dt[T] ns[U], b3 = dt[T] ds[U]
// factored as u_U = ns[U] k0 + ds[U] k1, v_U = ns[U] k2 + ds[U] k3,
// acc[T][U] += nt[T] u_U + dt[T] v_U.
template <bool TRANSPOSED, int BASE, int NV>
__device__ __forceinline__ void accum_orient(double (&acc)[NV], const cplx k0[2][2], const cplx k1[2][2],
                                             const cplx k2[2][2], const PointShared &Q, const double nt[2],
                                             const double dt[2], const double ns[2], const double ds[2], int mt,
                                             int ms) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const cplx k3 = (i == j) ? (i == 0 ? Q.k3_00 : Q.k3_11) : Q.k3_01;
            // ns = (1 - ns[1], ns[1]) and ds = (-ds[1], ds[1]): the U = 0 terms
            // are the U = 1 ones subtracted from k0 and k2
            const cplx u1 = cadd(cscale(k0[i][j], ns[1]), cscale(k1[i][j], ds[1]));
            const cplx v1 = cadd(cscale(k2[i][j], ns[1]), cscale(k3, ds[1]));
#pragma unroll
            for (int U = 0; U < 2; ++U) {
                if (!(ms & (1 << U))) continue;
                const cplx u = U ? u1 : csub(k0[i][j], u1);
                const cplx v = U ? v1 : csub(k2[i][j], v1);
#pragma unroll
                for (int T = 0; T < 2; ++T) {
                    if (!(mt & (1 << T))) continue;
                    // forward: FIDX(A = T, B = U); transposed: RIDX(B = T, A = U)
                    const int q = (TRANSPOSED ? RIDX(T, U, i, j) : FIDX(T, U, i, j)) - BASE;
                    acc[q] = fma(nt[T], u.x, fma(dt[T], v.x, acc[q]));
                    acc[q + 1] = fma(nt[T], u.y, fma(dt[T], v.y, acc[q + 1]));
                }
            }
        }
}

// Add one point (local coords sig, tau; relative z; weight w) to the forward
// (dir 0) or the transposed (dir 1) entries.  maskA/maskB: local basis
// indices used on E / F; ihE, ihF = 1/h of E, F.
__device__ __forceinline__ void acc_point(const PhysDev &P, const Rules &G, const Elem &E, const Elem &F, double ihE,
                                          double ihF, double sig, double tau, double2 z, double w, int dir, int maskA,
                                          int maskB, PairAcc &S) {
    PointShared Q;
    point_shared(P, G, z, Q);
    cplx k0[2][2], k1[2][2], k2[2][2];
    if (dir == 0) {
        blocks_orient(Q, 1.0, E.n, F.n, k0, k1, k2);
        const double nt[2] = {w * (1.0 - sig), w * sig}, dt[2] = {-w * ihE, w * ihE};
        const double ns[2] = {1.0 - tau, tau}, ds[2] = {-ihF, ihF};
        accum_orient<false, 0>(S.v, k0, k1, k2, Q, nt, dt, ns, ds, maskA, maskB);
    } else {
        blocks_orient(Q, -1.0, F.n, E.n, k0, k1, k2);
        const double nt[2] = {w * (1.0 - tau), w * tau}, dt[2] = {-w * ihF, w * ihF};
        const double ns[2] = {1.0 - sig, sig}, ds[2] = {-ihE, ihE};
        accum_orient<true, 32>(S.v, k0, k1, k2, Q, nt, dt, ns, ds, maskB, maskA);
    }
}

// Both orientations from one evaluation of the radial functions: v[0..31] =
// forward entries (index FIDX), v[32..63] = transposed entries (RIDX).
struct PairAcc2 {
    double v[64];
};

__device__ __forceinline__ void acc_point2(const PhysDev &P, const Rules &G, const Elem &E, const Elem &F, double ihE,
                                           double ihF, double sig, double tau, double2 z, double w, int maskA,
                                           int maskB, PairAcc2 &S) {
    PointShared Q;
    point_shared(P, G, z, Q);
    {
        cplx k0[2][2], k1[2][2], k2[2][2];
        blocks_orient(Q, 1.0, E.n, F.n, k0, k1, k2);
        const double nt[2] = {w * (1.0 - sig), w * sig}, dt[2] = {-w * ihE, w * ihE};
        const double ns[2] = {1.0 - tau, tau}, ds[2] = {-ihF, ihF};
        accum_orient<false, 0>(S.v, k0, k1, k2, Q, nt, dt, ns, ds, maskA, maskB);
    }
    {
        // transposed: test point on F (normal F.n), trial on E, z -> -z
        cplx k0[2][2], k1[2][2], k2[2][2];
        blocks_orient(Q, -1.0, F.n, E.n, k0, k1, k2);
        const double nt[2] = {w * (1.0 - tau), w * tau}, dt[2] = {-w * ihF, w * ihF};
        const double ns[2] = {1.0 - sig, sig}, ds[2] = {-ihE, ihE};
        accum_orient<true, 0>(S.v, k0, k1, k2, Q, nt, dt, ns, ds, maskB, maskA);
    }
}

__device__ __forceinline__ void acc_pair2(const PhysDev &P, const Rules &G, int kind, const Elem &E, const Elem &F,
                                          int p0, int stride, int maskA, int maskB, PairAcc2 &S) {
    const int np = pair_points(kind, G.q);
    const double ihE = 1.0 / E.h, ihF = 1.0 / F.h;
    for (int p = p0; p < np; p += stride) {
        double sig, tau, w;
        double2 z;
        pair_point(G, kind, p, E, F, sig, tau, z, w);
        acc_point2(P, G, E, F, ihE, ihF, sig, tau, z, w, maskA, maskB, S);
        if (kind == PK_SELF) acc_point2(P, G, E, F, ihE, ihF, tau, sig, make_double2(-z.x, -z.y), w, maskA, maskB, S);
    }
}

// All points p = p0, p0 + stride, ... of element pair (E, F) under rule
// `kind`, for the forward (dir 0) or transposed (dir 1) entries.
__device__ __forceinline__ void acc_pair(const PhysDev &P, const Rules &G, int kind, const Elem &E, const Elem &F,
                                         int p0, int stride, int dir, int maskA, int maskB, PairAcc &S) {
    const int np = pair_points(kind, G.q);
    const double ihE = 1.0 / E.h, ihF = 1.0 / F.h;
    for (int p = p0; p < np; p += stride) {
        double sig, tau, w;
        double2 z;
        pair_point(G, kind, p, E, F, sig, tau, z, w);
        acc_point(P, G, E, F, ihE, ihF, sig, tau, z, w, dir, maskA, maskB, S);
        if (kind == PK_SELF) acc_point(P, G, E, F, ihE, ihF, tau, sig, make_double2(-z.x, -z.y), w, dir, maskA, maskB, S);
    }
}

// ---------------------------------------------------------------- tiles
// A tile side: up to TILE hats on one closed polygon; its deduplicated
// elements with, for each, the tile positions of the hat that uses it as local
// node 0 (hat = element index) and as local node 1 (hat = element index + 1).
struct TileSide {
    int nh;
    int hats[TILE];
    int alias[TILE];    // first position holding the same hat (lists may repeat a hat)
    int ne;
    int el[TILE_EL];
    int pos[TILE_EL][2];
};

// Build the element list of a tile side (single thread).
__device__ __forceinline__ void tile_side_build(TileSide &T, int N) {
    T.ne = 0;
    for (int k = 0; k < T.nh; ++k) {
        const int s = T.hats[k];
        T.alias[k] = k;
        for (int q = 0; q < k; ++q)
            if (T.hats[q] == s) { T.alias[k] = q; break; }
        if (T.alias[k] != k) continue;
        const int e1 = (s == 0) ? N - 1 : s - 1;   // local node 1 of element s-1
        const int e0 = s;                          // local node 0 of element s
        for (int which = 0; which < 2; ++which) {
            const int e = which ? e1 : e0, A = which ? 1 : 0;
            int slot = -1;
            for (int q = 0; q < T.ne; ++q)
                if (T.el[q] == e) { slot = q; break; }
            if (slot < 0) {
                slot = T.ne++;
                T.el[slot] = e;
                T.pos[slot][0] = -1;
                T.pos[slot][1] = -1;
            }
            T.pos[slot][A] = k;
        }
    }
}

// Shared-memory state of one tile evaluation.
struct TileSmem {
    Rules G;
    TileSide R, C;
    Elem eR[TILE_EL], eC[TILE_EL];        // geometry of the tile's elements
    // the tile's element pairs grouped by rule: cheap rules first (costliest
    // first), then the singular ones; pk[q] = rule of pair q
    unsigned short plist[TILE_EL * TILE_EL];
    unsigned char pk[TILE_EL * TILE_EL];
    int kcount[PK_N], kstart[PK_N], ncheap, ncostly;
    double ef[TILE][TILE][2][2][2];   // forward entries  [row][col][i][j][re/im]
    double er[TILE][TILE][2][2][2];   // transposed entries [col][row][i][j][re/im]
};

__device__ __forceinline__ void tile_zero(TileSmem &S) {
    double *a = &S.ef[0][0][0][0][0], *b = &S.er[0][0][0][0][0];
    for (int k = threadIdx.x; k < TILE * TILE * 8; k += blockDim.x) { a[k] = 0.0; b[k] = 0.0; }
}

// Scatter one element pair's accumulator (forward, dir 0, or transposed,
// dir 1) into the tile entries: value k is added by lane k % nlanes
// (nlanes = 1 or 32).
__device__ __forceinline__ void tile_scatter(TileSmem &S, int re, int ce, const PairAcc &A, int dir, int lane,
                                             int nlanes) {
    const int pr0 = S.R.pos[re][0], pr1 = S.R.pos[re][1];
    const int pc0 = S.C.pos[ce][0], pc1 = S.C.pos[ce][1];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        if (nlanes != 1 && k != lane) continue;
        const int x = k >> 4, y = (k >> 3) & 1, i = (k >> 2) & 1, j = (k >> 1) & 1, ri = k & 1;
        if (dir == 0) {
            // test hat local x on the row element, trial local y on the column element
            const int pr = x ? pr1 : pr0, pc = y ? pc1 : pc0;
            if (pr < 0 || pc < 0) continue;
            atomicAdd(&S.ef[pr][pc][i][j][ri], A.v[k]);
        } else {
            // test hat local x on the column element, trial local y on the row element
            const int pc = x ? pc1 : pc0, pr = y ? pr1 : pr0;
            if (pr < 0 || pc < 0) continue;
            atomicAdd(&S.er[pc][pr][i][j][ri], A.v[k]);
        }
    }
}

__device__ __forceinline__ void tile_scatter2(TileSmem &S, int re, int ce, const PairAcc2 &A, int lane,
                                              int nlanes) {
    const int pr0 = S.R.pos[re][0], pr1 = S.R.pos[re][1];
    const int pc0 = S.C.pos[ce][0], pc1 = S.C.pos[ce][1];
#pragma unroll
    for (int k = 0; k < 64; ++k) {
        if (nlanes != 1 && (k & 31) != lane) continue;
        const int rem = k & 31;
        const int x = rem >> 4, y = (rem >> 3) & 1, i = (rem >> 2) & 1, j = (rem >> 1) & 1, ri = rem & 1;
        if (k < 32) {
            const int pr = x ? pr1 : pr0, pc = y ? pc1 : pc0;
            if (pr < 0 || pc < 0) continue;
            atomicAdd(&S.ef[pr][pc][i][j][ri], A.v[k]);
        } else {
            const int pc = x ? pc1 : pc0, pr = y ? pr1 : pr0;
            if (pr < 0 || pc < 0) continue;
            atomicAdd(&S.er[pc][pr][i][j][ri], A.v[k]);
        }
    }
}

// Warp reduce-scatter of NV values (NV = 32 or 64): afterwards lane L holds
// in v[0] the warp sum of index L and (NV = 64) in v[32] that of index L + 32.
// Five halving steps (16, 8, 4, 2, 1 values per set of 32): 31 additions and
// shuffles per set instead of 160 for a full reduction of every value.
template <int NV>
__device__ __forceinline__ void warp_reduce_scatter(double (&v)[NV], int lane) {
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int o = 16 >> s;
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int set = 0; set < NV / 32; ++set)
#pragma unroll
            for (int i = 0; i < (16 >> s); ++i) {
                const double a = v[set * 32 + i], b = v[set * 32 + i + (16 >> s)];
                const double keep = up ? b : a, send = up ? a : b;
                v[set * 32 + i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
    }
}


// Add one value of a pair's accumulator to the tile entries: k in 0..31
// forward (dir 0) or transposed (dir 1); for the dual accumulator k in 0..63
// (k >= 32 transposed).
__device__ __forceinline__ void tile_add_one(TileSmem &S, int re, int ce, int k, int dir, double val) {
    const int pr0 = S.R.pos[re][0], pr1 = S.R.pos[re][1];
    const int pc0 = S.C.pos[ce][0], pc1 = S.C.pos[ce][1];
    const int rem = k & 31;
    const int x = rem >> 4, y = (rem >> 3) & 1, i = (rem >> 2) & 1, j = (rem >> 1) & 1, ri = rem & 1;
    if (dir == 0 && k < 32) {
        const int pr = x ? pr1 : pr0, pc = y ? pc1 : pc0;
        if (pr >= 0 && pc >= 0) atomicAdd(&S.ef[pr][pc][i][j][ri], val);
    } else {
        const int pc = x ? pc1 : pc0, pr = y ? pr1 : pr0;
        if (pr >= 0 && pc >= 0) atomicAdd(&S.er[pc][pr][i][j][ri], val);
    }
}


// Evaluate all element pairs of a tile into S.ef / S.er.
//   same  : both sides on the same polygon X (singular-aware rule set);
//           otherwise rows on X, columns on Y with the cross rule S.G.q.
//   dual  : also accumulate the transposed entries.
//   diag  : rows and columns are the same hat list; only element pairs with
//           row element index <= column element index are evaluated, the
//           transposed contributions of pairs re < ce are folded in, and self
//           pairs are taken once.
// Cheap rules run one element pair per thread, costly ones one per warp.
static __device__ void tile_eval(const PhysDev &P, TileSmem &S, const double *__restrict__ X, int NX,
                          const double *__restrict__ Y, int NY, bool same, bool dual, bool diag) {
    const int npairs = S.R.ne * S.C.ne;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    // element geometry once per tile
    for (int k = threadIdx.x; k < S.R.ne + S.C.ne; k += blockDim.x) {
        if (k < S.R.ne) {
            S.eR[k] = load_elem(X, NX, S.R.el[k]);
        } else {
            const int c = k - S.R.ne;
            S.eC[c] = load_elem(same ? X : Y, same ? NX : NY, S.C.el[c]);
        }
    }
    __syncthreads();
    // classify the pairs and group them by rule (counting sort), so that the
    // threads of a warp integrate pairs with the same number of points
    for (int k = threadIdx.x; k < PK_N; k += blockDim.x) S.kcount[k] = 0;
    __syncthreads();
    for (int q = threadIdx.x; q < npairs; q += blockDim.x) {
        const int re = q / S.C.ne, ce = q - re * S.C.ne;
        const int ie = S.R.el[re], jf = S.C.el[ce];
        int kind = PK_SKIP;
        if (!(diag && ie > jf)) kind = same ? pair_kind(S.eR[re], S.eC[ce], ie, jf, NX, P.kT) : PK_CROSS;
        S.pk[q] = (unsigned char)kind;
        atomicAdd(&S.kcount[kind], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // order: mid, far, far2, far3, cross (cheap, costliest first), then self, adjacent, near
        const int ord[PK_N] = {PK_MID, PK_FAR, PK_FAR2, PK_FAR3, PK_CROSS, PK_SELF, PK_ADJ_NEXT, PK_ADJ_PREV,
                               PK_NEAR, PK_SKIP};
        int pos = 0;
        for (int o = 0; o < PK_N; ++o) {
            S.kstart[ord[o]] = pos;
            pos += S.kcount[ord[o]];
            if (o == 4) S.ncheap = pos;
            if (o == 8) S.ncostly = pos - S.ncheap;
            S.kcount[ord[o]] = 0;
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < npairs; q += blockDim.x) {
        const int kind = S.pk[q];
        S.plist[S.kstart[kind] + atomicAdd(&S.kcount[kind], 1)] = (unsigned short)q;
    }
    __syncthreads();
    // pass 1: cheap pairs, one per thread
    for (int idx = threadIdx.x; idx < S.ncheap; idx += blockDim.x) {
        const int q = S.plist[idx];
        const int re = q / S.C.ne, ce = q - re * S.C.ne;
        const Elem E = S.eR[re];
        const Elem F = S.eC[ce];
        const int kind = S.pk[q];
        const int mA = (S.R.pos[re][0] >= 0 ? 1 : 0) | (S.R.pos[re][1] >= 0 ? 2 : 0);
        const int mB = (S.C.pos[ce][0] >= 0 ? 1 : 0) | (S.C.pos[ce][1] >= 0 ? 2 : 0);
        if (dual || diag) {
            PairAcc2 A;
#pragma unroll
            for (int k = 0; k < 64; ++k) A.v[k] = 0.0;
            acc_pair2(P, S.G, kind, E, F, 0, 1, mA, mB, A);
            tile_scatter2(S, re, ce, A, 0, 1);
            if (d_count_points) atomicAdd(&d_quad_points, 2ull * pair_points(kind, S.G.q) * (kind == PK_SELF ? 2 : 1));
        } else {
            PairAcc A;
            acc_zero(A);
            acc_pair(P, S.G, kind, E, F, 0, 1, 0, mA, mB, A);
            tile_scatter(S, re, ce, A, 0, 0, 1);
            if (d_count_points) atomicAdd(&d_quad_points, 1ull * pair_points(kind, S.G.q) * (kind == PK_SELF ? 2 : 1));
        }
    }
    // pass 2: singular / near-singular pairs, one per warp
    for (int idx = warp; idx < S.ncostly; idx += nw) {
        const int q = S.plist[S.ncheap + idx];
        const int re = q / S.C.ne, ce = q - re * S.C.ne;
        const int ie = S.R.el[re], jf = S.C.el[ce];
        const Elem E = S.eR[re];
        const Elem F = S.eC[ce];
        const int kind = S.pk[q];
        const int mA = (S.R.pos[re][0] >= 0 ? 1 : 0) | (S.R.pos[re][1] >= 0 ? 2 : 0);
        const int mB = (S.C.pos[ce][0] >= 0 ? 1 : 0) | (S.C.pos[ce][1] >= 0 ? 2 : 0);
        // a self pair in a diagonal tile: its transposed entries are forward entries too
        const bool d = diag ? (ie != jf) : dual;
        if (d) {
            PairAcc2 A;
#pragma unroll
            for (int k = 0; k < 64; ++k) A.v[k] = 0.0;
            acc_pair2(P, S.G, kind, E, F, lane, 32, mA, mB, A);
            warp_reduce_scatter<64>(A.v, lane);
            tile_add_one(S, re, ce, lane, 0, A.v[0]);
            tile_add_one(S, re, ce, lane + 32, 0, A.v[32]);
            if (d_count_points && lane == 0)
                atomicAdd(&d_quad_points, 2ull * pair_points(kind, S.G.q) * (kind == PK_SELF ? 2 : 1));
        } else {
            PairAcc A;
            acc_zero(A);
            acc_pair(P, S.G, kind, E, F, lane, 32, 0, mA, mB, A);
            warp_reduce_scatter<32>(A.v, lane);
            tile_add_one(S, re, ce, lane, 0, A.v[0]);
            if (d_count_points && lane == 0)
                atomicAdd(&d_quad_points, 1ull * pair_points(kind, S.G.q) * (kind == PK_SELF ? 2 : 1));
        }
    }
}

// Fold the transposed entries of a diagonal tile into the forward ones.
__device__ __forceinline__ void tile_fold(TileSmem &S) {
    double *a = &S.ef[0][0][0][0][0];
    const double *b = &S.er[0][0][0][0][0];
    for (int k = threadIdx.x; k < TILE * TILE * 8; k += blockDim.x) a[k] += b[k];
}

// Exact P1 mass entry int phi^s phi^t over the polygon.
__device__ __forceinline__ double mass_entry(const double *__restrict__ xy, int N, int s, int t) {
    int sp = (s == 0) ? N - 1 : s - 1;
    int tp = (t == 0) ? N - 1 : t - 1;
    double m = 0.0;
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

// Entry (row item r, column item c) of the forward / transposed tile;
// repeated hats read the first occurrence.
__device__ __forceinline__ cplx tile_f(const TileSmem &S, int r, int c, int i, int j) {
    r = S.R.alias[r];
    c = S.C.alias[c];
    return mkc(S.ef[r][c][i][j][0], S.ef[r][c][i][j][1]);
}
__device__ __forceinline__ cplx tile_r(const TileSmem &S, int c, int r, int i, int j) {
    r = S.R.alias[r];
    c = S.C.alias[c];
    return mkc(S.er[c][r][i][j][0], S.er[c][r][i][j][1]);
}

}  // namespace fdsk
