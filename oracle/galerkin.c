/*
 * ORACLE — test infrastructure only.  Plain, slow FP64 CPU restatement of the
 * Galerkin P1 Burton–Miller boundary element matrix of arXiv 2411.18026
 * ("Linearly scalable fast direct solver based on proxy surface method for
 * two-dimensional elastic wave scattering by cavity").  Only tests/,
 * __graft_entry__.smoke() and bench.py's cpu_baseline leg may load this
 * library; the product path never does.  It shares no code with the CUDA path.
 *
 * What it computes
 *   A_pq = D + I_0/2 + alpha N  between P1 hat functions (Sec. 4, eq. (Aijpq)
 *   and the block definitions just before it), the right-hand side
 *   f = int psi (u^I + alpha T u^I)  (Sec. 4, eq. (gal)), and, for the proxy
 *   matrices of Sec. 7 (eq. (mv) and the M^U definition), entries between hats
 *   on an auxiliary polygon and hats on the boundary; and the displacement
 *   off the boundary from the boundary solution by the integral
 *   representation of Sec. 3, eq. (integ_rep).
 *
 * Kernel (Sec. 3, eq. (funda)): G = (1/mu) g_T I + (1/(rho w^2)) grad grad
 * (g_T - g_L) with g_k = (i/4) H0^(1)(k r).  The double-layer kernel
 * T^{n_y} G and the hypersingular kernel T^{n_x} T^{n_y} G are used in the
 * regularised Galerkin form obtained by moving every tangential (Gunter)
 * derivative onto the P1 test/trial functions (the 2D version of the
 * regularisation cited in Sec. 4).  With z = y - x, t = (n_2, -n_1),
 * eps = [[0,1],[-1,0]], c = 2/k_T^2, F = g_T - g_L:
 *   <psi, D phi>_ij = int int psi phi [n^y_j d_i g_L + t^y_j eps_iq d_q g_T]
 *                   - psi phi' [2 eps_ji g_T + c eps_jp d_p d_i F]
 *   <psi, N phi>_ij = int int psi phi rho w^2 (n^x_i n^y_j g_L + t^x_i t^y_j g_T)
 *                   - 2 mu psi phi' [t^x_i d_j g_T - n^x_i eps_jk d_k g_L]
 *                   - 2 mu psi' phi [n^y_j eps_ik d_k g_L - t^y_j d_i g_T]
 *                   + 2 mu psi' phi' [2 delta_ij g_T + c eps_ik eps_jp d_k d_p F]
 * (prime = derivative along the counter-clockwise arclength).  The tests pin
 * these forms against direct quadrature of T^{n_y}G and T^{n_x}T^{n_y}G on
 * separated element pairs.
 *
 * Quadrature definition (the same definition is restated independently on
 * the GPU):  element pairs are SELF, ADJACENT (shared vertex), NEAR
 * (midpoint distance < 2.5 max(h)), MID (< 6 max(h)), FAR (< 12 max(h)),
 * FAR2, or FAR3 (>= 24 max(h) on a fine mesh: k_T max(h) <= 0.02).  FAR3: 3x3
 * Gauss; FAR2: 4x4; FAR: 6x6; MID: 8x8; NEAR: both elements halved, 8x8 on
 * each of the 4 sub-pairs;
 * ADJACENT: Duffy split at the shared vertex, radial variable xi = w^4 with 16
 * Gauss points in w, 8 in the angular variable; SELF: (u = tau - sigma,
 * v) coordinates with u = w^5, 20 Gauss points in w and 4 in v, the two
 * triangles paired so the principal value of the odd (Cauchy) parts is
 * taken.  Proxy pairs use a fixed q x q Gauss rule (the solver uses q = 2).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

typedef struct {
    double lam, mu, rho, omega;
    double alpha_re, alpha_im;
} orc_phys;

typedef struct {
    double kT, kL, lam, mu, rho, omega;
    cplx alpha;
} phys_t;

static phys_t make_phys(const orc_phys *p)
{
    phys_t q;
    q.lam = p->lam; q.mu = p->mu; q.rho = p->rho; q.omega = p->omega;
    /* c_L = sqrt((lam+2mu)/rho), c_T = sqrt(mu/rho), k = omega/c  (Sec. 2) */
    q.kL = p->omega / sqrt((p->lam + 2.0 * p->mu) / p->rho);
    q.kT = p->omega / sqrt(p->mu / p->rho);
    q.alpha = p->alpha_re + I * p->alpha_im;
    return q;
}

/* ---------------------------------------------------------------- Gauss */
/* Gauss–Legendre nodes/weights on [0,1] by Newton iteration on P_n. */
#define MAXQ 32
typedef struct { int n; double x[MAXQ], w[MAXQ]; } rule_t;

static void gauss01(int n, rule_t *r)
{
    r->n = n;
    for (int i = 0; i < n; i++) {
        double x = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            if (n == 1) { p1 = x; p0 = 1.0; }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
        }
        r->x[i] = 0.5 * (1.0 - x);
        r->w[i] = 1.0 / ((1.0 - x * x) * dp * dp);   /* 2/((1-x^2)P'^2) * 1/2 */
    }
}

/* ---------------------------------------------------------------- Bessel */
/* H0^(1), H1^(1) of a real positive argument from libm's j0/j1/y0/y1. */
static void hankel01(double x, cplx *H0, cplx *H1)
{
    *H0 = j0(x) + I * y0(x);
    *H1 = j1(x) + I * y1(x);
}

/* Ehat(z) = (z H1^(1)(z) + 2i/pi) / z^2.  For z < 1 from the ascending series
 * of J_1 and Y_1 (Abramowitz & Stegun 9.1.10 and 9.1.11, n = 1):
 *   J1(z)/z = sum_m (-1)^m (z/2)^{2m} / (2 m! (m+1)!)
 *   z Y1(z) + 2/pi = (2/pi) z ln(z/2) J1(z)
 *                    - (z^2/(2 pi)) sum_m (psi(m+1)+psi(m+2)) (-z^2/4)^m / (m!(m+1)!)
 * so no cancellation of the 1/z poles occurs when two such terms with different
 * wavenumbers are subtracted. */
static cplx ehat(double z)
{
    if (z >= 1.0) {
        cplx H0, H1;
        hankel01(z, &H0, &H1);
        return (z * H1 + 2.0 * I / M_PI) / (z * z);
    }
    const double gam = 0.57721566490153286061;
    double q = -0.25 * z * z;
    double term = 1.0;          /* (-z^2/4)^m / (m!(m+1)!) */
    double j1z = 0.0, s = 0.0;
    double psi1 = -gam, psi2 = 1.0 - gam;  /* psi(m+1), psi(m+2) */
    for (int m = 0; m < 30; m++) {
        j1z += 0.5 * term;
        s += (psi1 + psi2) * term;
        if (fabs(term) < 1e-18) break;
        psi1 += 1.0 / (m + 1);
        psi2 += 1.0 / (m + 2);
        term *= q / ((m + 1.0) * (m + 2.0));
    }
    /* j1z = J1(z)/z */
    double re = j1z;
    double im = (2.0 / M_PI) * log(0.5 * z) * j1z - s / (2.0 * M_PI);
    return re + I * im;
}

/* ---------------------------------------------------------------- kernel */
/* Kernel blocks at relative position z = y - x (x: test point with normal nx,
 * y: trial point with normal ny).  K[0]: multiplies psi phi, K[1]: psi phi',
 * K[2]: psi' phi, K[3]: psi' phi'.  Combined operator D + alpha N. */
static void kernel_blocks(const phys_t *P, const double z[2], const double nx[2],
                          const double ny[2], cplx K[4][2][2])
{
    const double r = hypot(z[0], z[1]);
    const double zh[2] = { z[0] / r, z[1] / r };
    const double tx[2] = { nx[1], -nx[0] };
    const double ty[2] = { ny[1], -ny[0] };
    const double eps[2][2] = { { 0.0, 1.0 }, { -1.0, 0.0 } };
    const double del[2][2] = { { 1.0, 0.0 }, { 0.0, 1.0 } };
    const double kT = P->kT, kL = P->kL, mu = P->mu;
    const double rw2 = P->rho * P->omega * P->omega;
    const double c = 2.0 / (kT * kT);
    cplx H0T, H1T, H0L, H1L;
    hankel01(kT * r, &H0T, &H1T);
    hankel01(kL * r, &H0L, &H1L);
    const cplx gT = 0.25 * I * H0T, gL = 0.25 * I * H0L;
    const cplx gTp = -0.25 * I * kT * H1T, gLp = -0.25 * I * kL * H1L;
    cplx dgT[2], dgL[2];
    for (int a = 0; a < 2; a++) { dgT[a] = gTp * zh[a]; dgL[a] = gLp * zh[a]; }
    /* d_k d_p F = -(i/4) Pf zh zh + (i/4) Qf (2 zh zh - delta),
     * Pf = kT^2 H0(kT r) - kL^2 H0(kL r),
     * Qf = (kT H1(kT r) - kL H1(kL r))/r = kT^2 Ehat(kT r) - kL^2 Ehat(kL r). */
    const cplx Pf = kT * kT * H0T - kL * kL * H0L;
    const cplx Qf = kT * kT * ehat(kT * r) - kL * kL * ehat(kL * r);
    cplx HF[2][2];
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++)
            HF[a][b] = -0.25 * I * Pf * zh[a] * zh[b]
                       + 0.25 * I * Qf * (2.0 * zh[a] * zh[b] - del[a][b]);
    const cplx al = P->alpha;
    for (int i = 0; i < 2; i++) {
        for (int j = 0; j < 2; j++) {
            /* D parts */
            cplx epsdgT_i = 0.0;                 /* eps_iq d_q g_T */
            for (int q = 0; q < 2; q++) epsdgT_i += eps[i][q] * dgT[q];
            cplx D0 = ny[j] * dgL[i] + ty[j] * epsdgT_i;
            cplx epsH = 0.0;                     /* eps_jp d_p d_i F */
            for (int p = 0; p < 2; p++) epsH += eps[j][p] * HF[p][i];
            cplx D1 = -(2.0 * eps[j][i] * gT + c * epsH);
            /* N parts */
            cplx epsdgL_j = 0.0, epsdgL_i = 0.0;
            for (int k = 0; k < 2; k++) { epsdgL_j += eps[j][k] * dgL[k]; epsdgL_i += eps[i][k] * dgL[k]; }
            cplx N0 = rw2 * (nx[i] * ny[j] * gL + tx[i] * ty[j] * gT);
            cplx N1 = -2.0 * mu * (tx[i] * dgT[j] - nx[i] * epsdgL_j);
            cplx N2 = -2.0 * mu * (ny[j] * epsdgL_i - ty[j] * dgT[i]);
            cplx ee = 0.0;
            for (int k = 0; k < 2; k++)
                for (int p = 0; p < 2; p++) ee += eps[i][k] * eps[j][p] * HF[k][p];
            cplx N3 = 2.0 * mu * (2.0 * del[i][j] * gT + c * ee);
            K[0][i][j] = D0 + al * N0;
            K[1][i][j] = D1 + al * N1;
            K[2][i][j] = al * N2;
            K[3][i][j] = al * N3;
        }
    }
}

/* ---------------------------------------------------------------- elements */
typedef struct { double a[2], b[2], t[2], n[2], h; } elem_t;

static void make_elem(const double *xy, int N, int e, elem_t *E)
{
    int e1 = (e + 1) % N;
    E->a[0] = xy[2 * e]; E->a[1] = xy[2 * e + 1];
    E->b[0] = xy[2 * e1]; E->b[1] = xy[2 * e1 + 1];
    double dx = E->b[0] - E->a[0], dy = E->b[1] - E->a[1];
    E->h = hypot(dx, dy);
    E->t[0] = dx / E->h; E->t[1] = dy / E->h;
    /* normal = tangent rotated by +90 degrees: for counter-clockwise nodes it
     * points into the cavity, the direction Sec. 2 prescribes. */
    E->n[0] = -E->t[1]; E->n[1] = E->t[0];
}

/* out[A][B][i][j] += w * (basis products x kernel blocks)
 * sigma: test local coordinate on e, tau: trial local coordinate on f. */
static void accumulate(const phys_t *P, const elem_t *e, const elem_t *f,
                       double sig, double tau, const double z[2], double w,
                       cplx out[2][2][2][2])
{
    cplx K[4][2][2];
    kernel_blocks(P, z, e->n, f->n, K);
    const double Na[2] = { 1.0 - sig, sig }, dNa[2] = { -1.0 / e->h, 1.0 / e->h };
    const double Nb[2] = { 1.0 - tau, tau }, dNb[2] = { -1.0 / f->h, 1.0 / f->h };
    for (int A = 0; A < 2; A++)
        for (int B = 0; B < 2; B++) {
            const double b0 = Na[A] * Nb[B], b1 = Na[A] * dNb[B];
            const double b2 = dNa[A] * Nb[B], b3 = dNa[A] * dNb[B];
            for (int i = 0; i < 2; i++)
                for (int j = 0; j < 2; j++)
                    out[A][B][i][j] += w * (b0 * K[0][i][j] + b1 * K[1][i][j]
                                            + b2 * K[2][i][j] + b3 * K[3][i][j]);
        }
}

/* Plain tensor Gauss rule over sub-intervals [s0,s1] of e and [t0,t1] of f. */
static void pair_gauss(const phys_t *P, const elem_t *e, const elem_t *f,
                       double s0, double s1, double t0, double t1, int q,
                       cplx out[2][2][2][2])
{
    rule_t g; gauss01(q, &g);
    for (int a = 0; a < q; a++) {
        double sig = s0 + (s1 - s0) * g.x[a];
        double x[2] = { e->a[0] + sig * e->h * e->t[0], e->a[1] + sig * e->h * e->t[1] };
        for (int b = 0; b < q; b++) {
            double tau = t0 + (t1 - t0) * g.x[b];
            double y[2] = { f->a[0] + tau * f->h * f->t[0], f->a[1] + tau * f->h * f->t[1] };
            double z[2] = { y[0] - x[0], y[1] - x[1] };
            double w = g.w[a] * g.w[b] * (s1 - s0) * (t1 - t0) * e->h * f->h;
            accumulate(P, e, f, sig, tau, z, w, out);
        }
    }
}

/* SELF pair: integral over the unit square written as
 *   int_0^1 du int_0^{1-u} [F(v, v+u) + F(v+u, v)] dv,
 * u = w^5.  The relative vector z = +-u h t is formed directly. */
static void pair_self(const phys_t *P, const elem_t *e, cplx out[2][2][2][2])
{
    rule_t gw, gv; gauss01(20, &gw); gauss01(4, &gv);
    const double p = 5.0;
    for (int a = 0; a < gw.n; a++) {
        double wv = gw.x[a];
        double u = pow(wv, p);
        double du = gw.w[a] * p * pow(wv, p - 1.0);
        for (int b = 0; b < gv.n; b++) {
            double v = (1.0 - u) * gv.x[b];
            double wt = du * (1.0 - u) * gv.w[b] * e->h * e->h;
            double z1[2] = { u * e->h * e->t[0], u * e->h * e->t[1] };
            double z2[2] = { -z1[0], -z1[1] };
            accumulate(P, e, e, v, v + u, z1, wt, out);
            accumulate(P, e, e, v + u, v, z2, wt, out);
        }
    }
}

/* ADJACENT pair sharing one vertex.  next = 1: e's end is f's start;
 * next = 0: e's start is f's end.  alpha, beta = distances (fractions of h)
 * from the shared vertex; Duffy triangles alpha >= beta and beta > alpha with
 * radial variable xi = w^4. */
static void pair_adjacent(const phys_t *P, const elem_t *e, const elem_t *f, int next,
                          cplx out[2][2][2][2])
{
    rule_t gw, ge; gauss01(16, &gw); gauss01(8, &ge);
    const double p = 4.0;
    for (int tri = 0; tri < 2; tri++)
        for (int a = 0; a < gw.n; a++) {
            double xi = pow(gw.x[a], p);
            double dxi = gw.w[a] * p * pow(gw.x[a], p - 1.0);
            for (int b = 0; b < ge.n; b++) {
                double eta = ge.x[b];
                double al = tri == 0 ? xi : xi * eta;
                double be = tri == 0 ? xi * eta : xi;
                double w = dxi * ge.w[b] * xi * e->h * f->h;
                double sig, tau, z[2];
                if (next) {
                    sig = 1.0 - al; tau = be;
                    z[0] = be * f->h * f->t[0] + al * e->h * e->t[0];
                    z[1] = be * f->h * f->t[1] + al * e->h * e->t[1];
                } else {
                    sig = al; tau = 1.0 - be;
                    z[0] = -be * f->h * f->t[0] - al * e->h * e->t[0];
                    z[1] = -be * f->h * f->t[1] - al * e->h * e->t[1];
                }
                accumulate(P, e, f, sig, tau, z, w, out);
            }
        }
}

/* Element-pair integral for two elements of the same closed polygon. */
static void pair_integral(const phys_t *P, const double *xy, int N, int ie, int jf,
                          cplx out[2][2][2][2])
{
    elem_t e, f;
    make_elem(xy, N, ie, &e);
    make_elem(xy, N, jf, &f);
    memset(out, 0, sizeof(cplx) * 16);
    if (ie == jf) { pair_self(P, &e, out); return; }
    if (jf == (ie + 1) % N) { pair_adjacent(P, &e, &f, 1, out); return; }
    if (ie == (jf + 1) % N) { pair_adjacent(P, &e, &f, 0, out); return; }
    double me[2] = { 0.5 * (e.a[0] + e.b[0]), 0.5 * (e.a[1] + e.b[1]) };
    double mf[2] = { 0.5 * (f.a[0] + f.b[0]), 0.5 * (f.a[1] + f.b[1]) };
    double d = hypot(me[0] - mf[0], me[1] - mf[1]);
    double L = e.h > f.h ? e.h : f.h;
    if (d >= 24.0 * L && P->kT * L <= 0.02) { pair_gauss(P, &e, &f, 0, 1, 0, 1, 3, out); return; }
    if (d >= 12.0 * L) { pair_gauss(P, &e, &f, 0, 1, 0, 1, 4, out); return; }
    if (d >= 6.0 * L) { pair_gauss(P, &e, &f, 0, 1, 0, 1, 6, out); return; }
    if (d >= 2.5 * L) { pair_gauss(P, &e, &f, 0, 1, 0, 1, 8, out); return; }
    for (int s = 0; s < 2; s++)
        for (int t = 0; t < 2; t++)
            pair_gauss(P, &e, &f, 0.5 * s, 0.5 * s + 0.5, 0.5 * t, 0.5 * t + 0.5, 8, out);
}

/* Hat s lives on element s-1 (as its local node 1) and element s (local node 0). */
static void hat_elems(int s, int N, int el[2], int loc[2])
{
    el[0] = (s - 1 + N) % N; loc[0] = 1;
    el[1] = s;               loc[1] = 0;
}

/* P1 mass matrix entry int phi^s phi^t ds on the polygon (exact). */
static double mass_entry(const double *xy, int N, int s, int t)
{
    double m = 0.0;
    int es[2], ls[2], et[2], lt[2];
    hat_elems(s, N, es, ls);
    hat_elems(t, N, et, lt);
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++)
            if (es[a] == et[b]) {
                elem_t E; make_elem(xy, N, es[a], &E);
                m += (ls[a] == lt[b]) ? E.h / 3.0 : E.h / 6.0;
            }
    return m;
}

/*
 * Matrix block A(rows, cols) of the Galerkin system (Sec. 4): rows = test hat
 * indices, cols = trial hat indices on the same closed polygon xy[2N] (nodes
 * counter-clockwise).  out is row-major (2 nr) x (2 nc), complex, with the
 * component-blocked layout of eq. (discre_x): row r + i*nr is component i+1 of
 * hat rows[r]; column c + j*nc is component j+1 of hat cols[c].
 * Entry = D + I_0/2 + alpha N.
 */
void orc_entries(const orc_phys *pp, const double *xy, int N,
                 const int *rows, int nr, const int *cols, int nc, double *out_ri)
{
    phys_t P = make_phys(pp);
    cplx *out = (cplx *)out_ri;
    const long ld = 2L * nc;
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (int r = 0; r < nr; r++)
        for (int c = 0; c < nc; c++) {
            int s = rows[r], t = cols[c];
            int es[2], ls[2], et[2], lt[2];
            hat_elems(s, N, es, ls);
            hat_elems(t, N, et, lt);
            cplx acc[2][2] = { { 0 } };
            for (int a = 0; a < 2; a++)
                for (int b = 0; b < 2; b++) {
                    cplx I4[2][2][2][2];
                    pair_integral(&P, xy, N, es[a], et[b], I4);
                    for (int i = 0; i < 2; i++)
                        for (int j = 0; j < 2; j++) acc[i][j] += I4[ls[a]][lt[b]][i][j];
                }
            double m = mass_entry(xy, N, s, t);
            acc[0][0] += 0.5 * m;
            acc[1][1] += 0.5 * m;
            for (int i = 0; i < 2; i++)
                for (int j = 0; j < 2; j++)
                    out[(r + (long)i * nr) * ld + c + (long)j * nc] = acc[i][j];
        }
}

/*
 * Entries between hats on two different closed polygons with a fixed q x q
 * Gauss rule on every element pair (no singular pairs can occur): test hats
 * rows[] on polygon X (NX nodes), trial hats cols[] on polygon Y (NY nodes).
 * Used for the proxy interaction matrices M^V (X = proxy polygon, Y = boundary)
 * and M^U (X = boundary, Y = proxy polygon) of Sec. 7.  No mass term.
 */
void orc_cross_entries(const orc_phys *pp, const double *X, int NX, const int *rows, int nr,
                       const double *Y, int NY, const int *cols, int nc, int q, double *out_ri)
{
    phys_t P = make_phys(pp);
    cplx *out = (cplx *)out_ri;
    const long ld = 2L * nc;
#pragma omp parallel for schedule(dynamic, 4) collapse(2)
    for (int r = 0; r < nr; r++)
        for (int c = 0; c < nc; c++) {
            int es[2], ls[2], et[2], lt[2];
            hat_elems(rows[r], NX, es, ls);
            hat_elems(cols[c], NY, et, lt);
            cplx acc[2][2] = { { 0 } };
            for (int a = 0; a < 2; a++)
                for (int b = 0; b < 2; b++) {
                    elem_t e, f;
                    make_elem(X, NX, es[a], &e);
                    make_elem(Y, NY, et[b], &f);
                    cplx I4[2][2][2][2];
                    memset(I4, 0, sizeof(I4));
                    pair_gauss(&P, &e, &f, 0, 1, 0, 1, q, I4);
                    for (int i = 0; i < 2; i++)
                        for (int j = 0; j < 2; j++) acc[i][j] += I4[ls[a]][lt[b]][i][j];
                }
            for (int i = 0; i < 2; i++)
                for (int j = 0; j < 2; j++)
                    out[(r + (long)i * nr) * ld + c + (long)j * nc] = acc[i][j];
        }
}

/*
 * Galerkin load vector f_i^s = int psi^s (u^I_i + alpha T^{n_x}_ij u^I_j) ds
 * (Sec. 4) for a plane wave of direction d = (cos th, sin th):
 *   kind 0 (P):  u^I = d exp(i k_L d.x)
 *   kind 1 (SV): u^I = d_perp exp(i k_T d.x), d_perp = (-d_2, d_1)
 * out[2N] complex: component 1 at hats 0..N-1, then component 2.
 * 8-point Gauss on each element.
 */
void orc_rhs(const orc_phys *pp, const double *xy, int N, int kind, double th, double *out_ri)
{
    phys_t P = make_phys(pp);
    cplx *out = (cplx *)out_ri;
    rule_t g; gauss01(8, &g);
    const double d[2] = { cos(th), sin(th) };
    const double dp[2] = { -d[1], d[0] };
    for (int s = 0; s < 2 * N; s++) out[s] = 0.0;
    for (int e = 0; e < N; e++) {
        elem_t E; make_elem(xy, N, e, &E);
        for (int a = 0; a < g.n; a++) {
            double sig = g.x[a];
            double x[2] = { E.a[0] + sig * E.h * E.t[0], E.a[1] + sig * E.h * E.t[1] };
            const double *n = E.n;
            cplx u[2], tr[2];
            if (kind == 0) {
                cplx ph = cexp(I * P.kL * (d[0] * x[0] + d[1] * x[1]));
                double nd = n[0] * d[0] + n[1] * d[1];
                for (int i = 0; i < 2; i++) {
                    u[i] = d[i] * ph;
                    tr[i] = I * P.kL * ph * (P.lam * n[i] + 2.0 * P.mu * nd * d[i]);
                }
            } else {
                cplx ph = cexp(I * P.kT * (d[0] * x[0] + d[1] * x[1]));
                double nd = n[0] * d[0] + n[1] * d[1];
                double ndp = n[0] * dp[0] + n[1] * dp[1];
                for (int i = 0; i < 2; i++) {
                    u[i] = dp[i] * ph;
                    tr[i] = I * P.kT * P.mu * ph * (nd * dp[i] + ndp * d[i]);
                }
            }
            double Nl[2] = { 1.0 - sig, sig };
            int nodes[2] = { e, (e + 1) % N };
            for (int A = 0; A < 2; A++)
                for (int i = 0; i < 2; i++)
                    out[nodes[A] + (long)i * N] += g.w[a] * E.h * Nl[A] * (u[i] + P.alpha * tr[i]);
        }
    }
}

/*
 * Displacement at points x off the boundary from the boundary solution u
 * (Sec. 3, eq. (integ_rep)), for a traction-free cavity:
 *   u_i(x) = u^I_i(x) - int_Gamma K_ij(x, y) u_j(y) ds(y),
 *   K_ij = T^{n_y}_{jk} G_ik = lam n_j d_k G_ik + mu (n_q d_q G_ij + n_k d_j G_ik),
 * the derivatives taken in y, with z = y - x:
 *   G_ik(z) = i/(4 mu) [H0(k_T r) delta_ik + k_T^-2 d_i d_k (H0(k_T r) - H0(k_L r))].
 * For a radial f(r) with D_m = (r^-1 d/dr)^m f:  d_a f = z_a D_1,
 *   d_a d_b d_c f = (delta_ab z_c + delta_ac z_b + delta_bc z_a) D_2 + z_a z_b z_c D_3,
 * and for f = H0(k r), D_m = (-k/r)^m H_m(k r).  u is linear on each element
 * (P1 nodal values, component 1 at nodes 0..N-1 then component 2), 8-point
 * Gauss per element.  u^I: the plane wave of orc_rhs (kind, th).
 * u: 2N complex; pts: 2 npts doubles; out: 2 npts complex (component 1 at the
 * points, then component 2).
 */
static void hankel0123(double x, cplx H[4])
{
    hankel01(x, &H[0], &H[1]);
    H[2] = (2.0 / x) * H[1] - H[0];
    H[3] = (4.0 / x) * H[2] - H[1];
}

void orc_field(const orc_phys *pp, const double *xy, int N, const double *u_ri, int kind, double th,
               const double *pts, int npts, double *out_ri)
{
    phys_t P = make_phys(pp);
    const cplx *u = (const cplx *)u_ri;
    cplx *out = (cplx *)out_ri;
    rule_t g; gauss01(8, &g);
    const double d[2] = { cos(th), sin(th) };
    const double dp[2] = { -d[1], d[0] };
    const double del[2][2] = { { 1.0, 0.0 }, { 0.0, 1.0 } };
    const cplx a = I / (4.0 * P.mu);
    for (int p = 0; p < npts; p++) {
        const double x[2] = { pts[2 * p], pts[2 * p + 1] };
        cplx acc[2] = { 0.0, 0.0 };
        for (int e = 0; e < N; e++) {
            elem_t E; make_elem(xy, N, e, &E);
            const int e1 = (e + 1) % N;
            for (int q = 0; q < g.n; q++) {
                const double sig = g.x[q];
                const double z[2] = { E.a[0] + sig * E.h * E.t[0] - x[0], E.a[1] + sig * E.h * E.t[1] - x[1] };
                const double r = hypot(z[0], z[1]);
                cplx HT[4], HL[4];
                hankel0123(P.kT * r, HT);
                hankel0123(P.kL * r, HL);
                cplx DT[4], DL[4];
                for (int m = 0; m < 4; m++) {
                    DT[m] = cpow(-P.kT / r, m) * HT[m];
                    DL[m] = cpow(-P.kL / r, m) * HL[m];
                }
                /* G1[i][k][c] = d_c G_ik */
                cplx G1[2][2][2];
                for (int i = 0; i < 2; i++)
                    for (int k = 0; k < 2; k++)
                        for (int c = 0; c < 2; c++) {
                            const double t3 = del[i][k] * z[c] + del[i][c] * z[k] + del[k][c] * z[i];
                            const cplx d3 = t3 * (DT[2] - DL[2]) + z[i] * z[k] * z[c] * (DT[3] - DL[3]);
                            G1[i][k][c] = a * (del[i][k] * z[c] * DT[1] + d3 / (P.kT * P.kT));
                        }
                const double *n = E.n;
                cplx uy[2];
                for (int j = 0; j < 2; j++) uy[j] = (1.0 - sig) * u[e + (long)j * N] + sig * u[e1 + (long)j * N];
                const double w = g.w[q] * E.h;
                for (int i = 0; i < 2; i++) {
                    const cplx div = G1[i][0][0] + G1[i][1][1];
                    for (int j = 0; j < 2; j++) {
                        const cplx K = P.lam * n[j] * div + P.mu * (n[0] * G1[i][j][0] + n[1] * G1[i][j][1])
                                       + P.mu * (n[0] * G1[i][0][j] + n[1] * G1[i][1][j]);
                        acc[i] += w * K * uy[j];
                    }
                }
            }
        }
        cplx uI[2];
        if (kind == 0) {
            const cplx ph = cexp(I * P.kL * (d[0] * x[0] + d[1] * x[1]));
            uI[0] = d[0] * ph;
            uI[1] = d[1] * ph;
        } else {
            const cplx ph = cexp(I * P.kT * (d[0] * x[0] + d[1] * x[1]));
            uI[0] = dp[0] * ph;
            uI[1] = dp[1] * ph;
        }
        out[p] = uI[0] - acc[0];
        out[p + (long)npts] = uI[1] - acc[1];
    }
}

/* Kernel blocks at one point pair (exported for the tests' direct-kernel pins). */
void orc_kernel_blocks(const orc_phys *pp, const double *z, const double *nx, const double *ny,
                       double *out_ri)
{
    phys_t P = make_phys(pp);
    cplx K[4][2][2];
    kernel_blocks(&P, z, nx, ny, K);
    memcpy(out_ri, K, sizeof(K));
}

/* Ehat exported for the Bessel pins. */
void orc_ehat(double z, double *out_ri)
{
    cplx e = ehat(z);
    out_ri[0] = creal(e); out_ri[1] = cimag(e);
}

/* Element-pair integral exported for quadrature-convergence pins. */
void orc_pair(const orc_phys *pp, const double *xy, int N, int ie, int jf, double *out_ri)
{
    phys_t P = make_phys(pp);
    cplx I4[2][2][2][2];
    pair_integral(&P, xy, N, ie, jf, I4);
    memcpy(out_ri, I4, sizeof(I4));
}
