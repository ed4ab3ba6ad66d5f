/*
 * dwf_oracle.c -- plain FP64 CPU oracle (test infrastructure only; see dwf_oracle.h).
 *
 * Follows Chiu, Hsieh, Mao, Ogawa, "GPU-Based Conjugate Gradient Solver for Lattice
 * QCD with Domain-Wall Fermions" (Lattice 2010), Sec. 2:
 *   Eq. 1   the 5D operator D(mq) with weights omega_s, sigma_s
 *   Eq. 2   the Wilson operator D_w with the -m0 term
 *   Eq. 3-4 the chiral hopping matrix L = P+ L+ + P- L-
 *   Eq. 7-9 X, Y, M5, S1, S2
 *   Eq. 10-11 the LDU form and the Schur complement C
 *   Eq. 12  the hopping blocks D_w^{OE}, D_w^{EO}
 *   Algorithm 1 conjugate gradient
 * Everything is written out directly: full 4x4 spin matrices, dense Ns x Ns matrices,
 * Gauss-Jordan inversion.  No blocking, fusion or reordering.
 */
#include "dwf_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define DIM 4

/* ------------------------------------------------------------ geometry */

static int dims_ok(const int d[4]) {
    for (int mu = 0; mu < 4; ++mu)
        if (d[mu] < 2 || (d[mu] & 1)) return 0;
    return 1;
}
static long vol(const int d[4]) { return (long)d[0] * d[1] * d[2] * d[3]; }
static void coords_of(const int d[4], long site, int c[4]) {
    for (int mu = 0; mu < 4; ++mu) { c[mu] = (int)(site % d[mu]); site /= d[mu]; }
}
static long site_of(const int d[4], const int c[4]) {
    return c[0] + (long)d[0] * (c[1] + (long)d[1] * (c[2] + (long)d[2] * c[3]));
}
static int parity_of(const int d[4], long site) {
    int c[4]; coords_of(d, site, c);
    return (c[0] + c[1] + c[2] + c[3]) & 1;
}
/* neighbour x + dir*mu_hat with periodic wrap */
static long neighbour(const int d[4], long site, int mu, int dir) {
    int c[4]; coords_of(d, site, c);
    c[mu] = (c[mu] + dir + d[mu]) % d[mu];
    return site_of(d, c);
}

/* ------------------------------------------------------------ gamma matrices */

static cplx G[5][4][4];
static int g_ready = 0;

static void matmul4(cplx a[4][4], cplx b[4][4], cplx out[4][4]) {
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cplx s = 0;
            for (int k = 0; k < 4; ++k) s += a[i][k] * b[k][j];
            out[i][j] = s;
        }
}

static void init_gamma(void) {
    if (g_ready) return;
    cplx sig[3][2][2] = {
        {{0, 1}, {1, 0}},
        {{0, -I}, {I, 0}},
        {{1, 0}, {0, -1}},
    };
    memset(G, 0, sizeof(G));
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                G[k][i][2 + j] = -I * sig[k][i][j];
                G[k][2 + i][j] = I * sig[k][i][j];
            }
    for (int i = 0; i < 2; ++i) { G[3][i][2 + i] = 1; G[3][2 + i][i] = 1; }
    cplx t1[4][4], t2[4][4];
    matmul4(G[0], G[1], t1);
    matmul4(t1, G[2], t2);
    matmul4(t2, G[3], G[4]);
    g_ready = 1;
}

int or_gamma(int mu, double *out32) {
    if (mu < 0 || mu > 4 || !out32) return -1;
    init_gamma();
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            out32[2 * (4 * i + j)] = creal(G[mu][i][j]);
            out32[2 * (4 * i + j) + 1] = cimag(G[mu][i][j]);
        }
    return 0;
}

/* ------------------------------------------------------------ spin x colour blocks */

/* pointer to the 12 complex components (spin, colour) of (site, s) */
static cplx *spinor_at(double *v, int Ns, long site, int s) {
    return (cplx *)v + ((size_t)site * Ns + s) * 12;
}
static const cplx *cspinor_at(const double *v, int Ns, long site, int s) {
    return (const cplx *)v + ((size_t)site * Ns + s) * 12;
}
static const cplx *link_at(const double *U, long site, int mu) {
    return (const cplx *)U + ((size_t)site * 4 + mu) * 9;
}

/* acc += coef * (S (x) V) psi, S a 4x4 spin matrix, V a 3x3 colour matrix
 * (dagger_v != 0 uses V^dagger). */
static void add_block(cplx acc[12], cplx coef, cplx S[4][4], const cplx *V, int dagger_v,
                      const cplx psi[12]) {
    cplx w[4][3];
    for (int beta = 0; beta < 4; ++beta)
        for (int a = 0; a < 3; ++a) {
            cplx s = 0;
            for (int b = 0; b < 3; ++b) {
                cplx vab = dagger_v ? conj(V[3 * b + a]) : V[3 * a + b];
                s += vab * psi[3 * beta + b];
            }
            w[beta][a] = s;
        }
    for (int alpha = 0; alpha < 4; ++alpha)
        for (int a = 0; a < 3; ++a) {
            cplx s = 0;
            for (int beta = 0; beta < 4; ++beta) s += S[alpha][beta] * w[beta][a];
            acc[3 * alpha + a] += coef * s;
        }
}

/* (1 + sgn*gamma_mu), and its conjugate transpose */
static void one_pm_gamma(int mu, int sgn, cplx out[4][4]) {
    init_gamma();
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) out[i][j] = (i == j ? 1.0 : 0.0) + sgn * G[mu][i][j];
}
static void dagger4(cplx in[4][4], cplx out[4][4]) {
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) out[i][j] = conj(in[j][i]);
}

/* ------------------------------------------------------------ Eq. 2 and Eq. 12 */

/* hopping sum of Eq. 2 / Eq. 12 at one site and slice:
 * -1/2 sum_mu [ (1-g_mu) U_mu(x) psi(x+mu) + (1+g_mu) U_mu(x-mu)^dag psi(x-mu) ] */
static void hop_site(const int d[4], int Ns, const double *U, long x, int s, const double *in,
                     cplx acc[12]) {
    for (int mu = 0; mu < 4; ++mu) {
        cplx Sm[4][4], Sp[4][4];
        one_pm_gamma(mu, -1, Sm);
        one_pm_gamma(mu, +1, Sp);
        long xf = neighbour(d, x, mu, +1);
        long xb = neighbour(d, x, mu, -1);
        add_block(acc, -0.5, Sm, link_at(U, x, mu), 0, cspinor_at(in, Ns, xf, s));
        add_block(acc, -0.5, Sp, link_at(U, xb, mu), 1, cspinor_at(in, Ns, xb, s));
    }
}

int or_dw(const int dims[4], int Ns, const double *U, double m0, const double *in, double *out) {
    if (!dims_ok(dims) || Ns < 1 || !U || !in || !out || in == out) return -1;
    long V = vol(dims);
    for (long x = 0; x < V; ++x)
        for (int s = 0; s < Ns; ++s) {
            cplx acc[12];
            const cplx *p = cspinor_at(in, Ns, x, s);
            for (int i = 0; i < 12; ++i) acc[i] = (DIM - m0) * p[i];
            hop_site(dims, Ns, U, x, s, in, acc);
            memcpy(spinor_at(out, Ns, x, s), acc, sizeof(acc));
        }
    return 0;
}

int or_hop(const int dims[4], int Ns, const double *U, int p, const double *in, double *out) {
    if (!dims_ok(dims) || Ns < 1 || (p != 0 && p != 1) || !U || !in || !out || in == out)
        return -1;
    long V = vol(dims);
    for (long x = 0; x < V; ++x)
        for (int s = 0; s < Ns; ++s) {
            cplx acc[12] = {0};
            if (parity_of(dims, x) == p) hop_site(dims, Ns, U, x, s, in, acc);
            memcpy(spinor_at(out, Ns, x, s), acc, sizeof(acc));
        }
    return 0;
}

int or_hop_dag(const int dims[4], int Ns, const double *U, int p, const double *in, double *out) {
    if (!dims_ok(dims) || Ns < 1 || (p != 0 && p != 1) || !U || !in || !out || in == out)
        return -1;
    long V = vol(dims);
    memset(out, 0, sizeof(double) * 24 * (size_t)Ns * V);
    /* scatter: every block B_{x,x'} of the row x (parity p) contributes B^dag in(x) to x' */
    for (long x = 0; x < V; ++x) {
        if (parity_of(dims, x) != p) continue;
        for (int mu = 0; mu < 4; ++mu) {
            cplx Sm[4][4], Sp[4][4], SmD[4][4], SpD[4][4];
            one_pm_gamma(mu, -1, Sm);
            one_pm_gamma(mu, +1, Sp);
            dagger4(Sm, SmD);
            dagger4(Sp, SpD);
            long xf = neighbour(dims, x, mu, +1);
            long xb = neighbour(dims, x, mu, -1);
            for (int s = 0; s < Ns; ++s) {
                const cplx *src = cspinor_at(in, Ns, x, s);
                /* forward block -1/2 (1-g) U_mu(x) sits at column x+mu: adjoint uses U_mu(x)^dag */
                add_block(spinor_at(out, Ns, xf, s), -0.5, SmD, link_at(U, x, mu), 1, src);
                /* backward block -1/2 (1+g) U_mu(x-mu)^dag at column x-mu: adjoint uses U_mu(x-mu) */
                add_block(spinor_at(out, Ns, xb, s), -0.5, SpD, link_at(U, xb, mu), 0, src);
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------ fifth dimension, Eq. 3-9 */

int or_lmat(int Ns, double m0, double mq, double *Lp, double *Lm) {
    if (Ns < 1 || !Lp || !Lm || m0 == 0.0) return -1;
    memset(Lp, 0, sizeof(double) * Ns * Ns);
    /* Eq. 4 with 1-based s: (L+)_{s,s-1} = 1 for 1 < s <= Ns; (L+)_{1,Ns} = -mq/(2 m0) */
    for (int s = 1; s <= Ns; ++s) {
        if (s > 1) Lp[(s - 1) * Ns + (s - 2)] += 1.0;
        else Lp[(s - 1) * Ns + (Ns - 1)] += -mq / (2.0 * m0);
    }
    for (int i = 0; i < Ns; ++i)
        for (int j = 0; j < Ns; ++j) Lm[i * Ns + j] = Lp[j * Ns + i];
    return 0;
}

/* Gauss-Jordan inversion with partial pivoting (n <= 64) */
static int invert(int n, const double *A, double *Ainv) {
    double *a = (double *)malloc(sizeof(double) * n * 2 * n);
    if (!a) return -1;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < 2 * n; ++j)
            a[i * 2 * n + j] = j < n ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(a[r * 2 * n + col]) > fabs(a[piv * 2 * n + col])) piv = r;
        if (a[piv * 2 * n + col] == 0.0) { free(a); return -1; }
        if (piv != col)
            for (int j = 0; j < 2 * n; ++j) {
                double t = a[col * 2 * n + j];
                a[col * 2 * n + j] = a[piv * 2 * n + j];
                a[piv * 2 * n + j] = t;
            }
        double inv = 1.0 / a[col * 2 * n + col];
        for (int j = 0; j < 2 * n; ++j) a[col * 2 * n + j] *= inv;
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double f = a[r * 2 * n + col];
            if (f != 0.0)
                for (int j = 0; j < 2 * n; ++j) a[r * 2 * n + j] -= f * a[col * 2 * n + j];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Ainv[i * n + j] = a[i * 2 * n + n + j];
    free(a);
    return 0;
}

static void matmul(int n, const double *A, const double *B, double *C) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0;
            for (int k = 0; k < n; ++k) s += A[i * n + k] * B[k * n + j];
            C[i * n + j] = s;
        }
}

/* M5 = [ (d-m0) + w^{-1/2} (1-L)(1+cL)^{-1} w^{-1/2} ]^{-1} for one chirality (Eq. 8) */
static int m5_one(int Ns, double m0, const double *omega, const double *sigma, const double *L,
                  double *M5) {
    size_t sz = sizeof(double) * Ns * Ns;
    double *A = malloc(sz), *Ai = malloc(sz), *B = malloc(sz), *T = malloc(sz), *oneL = malloc(sz);
    int rc = -1;
    if (!A || !Ai || !B || !T || !oneL) goto done;
    for (int i = 0; i < Ns; ++i)
        for (int j = 0; j < Ns; ++j) {
            double c_i = sigma[i] / omega[i];
            A[i * Ns + j] = (i == j ? 1.0 : 0.0) + c_i * L[i * Ns + j]; /* 1 + cL */
            oneL[i * Ns + j] = (i == j ? 1.0 : 0.0) - L[i * Ns + j];   /* 1 - L */
        }
    if (invert(Ns, A, Ai)) goto done;
    matmul(Ns, oneL, Ai, B); /* (1-L)(1+cL)^{-1} */
    for (int i = 0; i < Ns; ++i)
        for (int j = 0; j < Ns; ++j)
            T[i * Ns + j] = (i == j ? (DIM - m0) : 0.0) + B[i * Ns + j] / sqrt(omega[i] * omega[j]);
    if (invert(Ns, T, M5)) goto done;
    rc = 0;
done:
    free(A); free(Ai); free(B); free(T); free(oneL);
    return rc;
}

static int weights_ok(int Ns, const double *omega, const double *sigma) {
    if (Ns < 1 || Ns > 64 || !omega || !sigma) return 0;
    for (int s = 0; s < Ns; ++s)
        if (!(omega[s] > 0.0)) return 0;
    return 1;
}

int or_m5(int Ns, double m0, double mq, const double *omega, const double *sigma, double *M5p,
          double *M5m) {
    if (!weights_ok(Ns, omega, sigma) || !M5p || !M5m || m0 == 0.0) return -1;
    size_t sz = sizeof(double) * Ns * Ns;
    double *Lp = malloc(sz), *Lm = malloc(sz);
    int rc = -1;
    if (Lp && Lm && or_lmat(Ns, m0, mq, Lp, Lm) == 0 && m5_one(Ns, m0, omega, sigma, Lp, M5p) == 0 &&
        m5_one(Ns, m0, omega, sigma, Lm, M5m) == 0)
        rc = 0;
    free(Lp); free(Lm);
    return rc;
}

int or_s1s2(int Ns, double m0, double mq, const double *omega, const double *sigma, double *S1p,
            double *S1m, double *S2p, double *S2m) {
    if (!weights_ok(Ns, omega, sigma) || !S1p || !S1m || !S2p || !S2m || m0 == 0.0) return -1;
    size_t sz = sizeof(double) * Ns * Ns;
    double *Lp = malloc(sz), *Lm = malloc(sz), *M5 = malloc(sz), *Y = malloc(sz), *Yi = malloc(sz);
    int rc = -1;
    if (!Lp || !Lm || !M5 || !Y || !Yi) goto done;
    if (or_lmat(Ns, m0, mq, Lp, Lm)) goto done;
    for (int chi = 0; chi < 2; ++chi) {
        const double *L = chi == 0 ? Lp : Lm;
        double *S1 = chi == 0 ? S1p : S1m;
        double *S2 = chi == 0 ? S2p : S2m;
        if (m5_one(Ns, m0, omega, sigma, L, M5)) goto done;
        /* S1 = M5 omega^{-1/2} (Eq. 9) */
        for (int i = 0; i < Ns; ++i)
            for (int j = 0; j < Ns; ++j) S1[i * Ns + j] = M5[i * Ns + j] / sqrt(omega[j]);
        /* Y = omega (1 + cL) (Eq. 7), S2 = Y^{-1} sqrt(omega) (Eq. 9) */
        for (int i = 0; i < Ns; ++i)
            for (int j = 0; j < Ns; ++j)
                Y[i * Ns + j] = omega[i] * ((i == j ? 1.0 : 0.0) + sigma[i] / omega[i] * L[i * Ns + j]);
        if (invert(Ns, Y, Yi)) goto done;
        for (int i = 0; i < Ns; ++i)
            for (int j = 0; j < Ns; ++j) S2[i * Ns + j] = Yi[i * Ns + j] * sqrt(omega[j]);
    }
    rc = 0;
done:
    free(Lp); free(Lm); free(M5); free(Y); free(Yi);
    return rc;
}

int or_apply_s(const int dims[4], int Ns, const double *Mp, const double *Mm, int transpose,
               int parity, const double *in, double *out) {
    if (!dims_ok(dims) || Ns < 1 || !Mp || !Mm || !in || !out || in == out) return -1;
    long V = vol(dims);
    for (long x = 0; x < V; ++x) {
        int keep = parity < 0 || parity_of(dims, x) == parity;
        for (int s = 0; s < Ns; ++s) {
            cplx *o = spinor_at(out, Ns, x, s);
            for (int spin = 0; spin < 4; ++spin) {
                const double *M = spin < 2 ? Mp : Mm; /* P+ = spins 0,1; P- = spins 2,3 */
                for (int a = 0; a < 3; ++a) {
                    cplx acc = 0;
                    if (keep)
                        for (int t = 0; t < Ns; ++t) {
                            double m = transpose ? M[t * Ns + s] : M[s * Ns + t];
                            acc += m * cspinor_at(in, Ns, x, t)[3 * spin + a];
                        }
                    o[3 * spin + a] = acc;
                }
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------ Eq. 1 */

int or_dfull(const int dims[4], int Ns, const double *U, double m0, double mq,
             const double *omega, const double *sigma, const double *in, double *out) {
    if (!dims_ok(dims) || !weights_ok(Ns, omega, sigma) || !U || !in || !out || in == out ||
        m0 == 0.0)
        return -1;
    long V = vol(dims);
    size_t n = 24 * (size_t)Ns * V;
    double *Lp = malloc(sizeof(double) * Ns * Ns), *Lm = malloc(sizeof(double) * Ns * Ns);
    double *Lpsi = malloc(sizeof(double) * n), *Dpsi = malloc(sizeof(double) * n),
           *DLpsi = malloc(sizeof(double) * n);
    int rc = -1;
    if (!Lp || !Lm || !Lpsi || !Dpsi || !DLpsi) goto done;
    if (or_lmat(Ns, m0, mq, Lp, Lm)) goto done;
    /* L psi with L = P+ L+ + P- L- (Eq. 3) */
    if (or_apply_s(dims, Ns, Lp, Lm, 0, -1, in, Lpsi)) goto done;
    if (or_dw(dims, Ns, U, m0, in, Dpsi)) goto done;
    if (or_dw(dims, Ns, U, m0, Lpsi, DLpsi)) goto done;
    /* Eq. 1: [(omega_s D_w + 1) delta_ss' + (sigma_s D_w - 1) L_ss'] psi_s' */
    for (long x = 0; x < V; ++x)
        for (int s = 0; s < Ns; ++s) {
            size_t o = 24 * ((size_t)x * Ns + s);
            for (int c = 0; c < 24; ++c)
                out[o + c] = omega[s] * Dpsi[o + c] + in[o + c] + sigma[s] * DLpsi[o + c] - Lpsi[o + c];
        }
    rc = 0;
done:
    free(Lp); free(Lm); free(Lpsi); free(Dpsi); free(DLpsi);
    return rc;
}

/* ------------------------------------------------------------ Eq. 11 */

static void parity_mask(const int dims[4], int Ns, int p, double *v) {
    long V = vol(dims);
    for (long x = 0; x < V; ++x)
        if (parity_of(dims, x) != p) memset(v + 24 * (size_t)Ns * x, 0, sizeof(double) * 24 * Ns);
}

int or_c(const int dims[4], int Ns, const double *U, const double *M5p, const double *M5m, int p,
         const double *in, double *out) {
    if (!dims_ok(dims) || Ns < 1 || (p != 0 && p != 1) || !in || !out || in == out) return -1;
    size_t n = 24 * (size_t)Ns * vol(dims);
    double *a = malloc(sizeof(double) * n), *b = malloc(sizeof(double) * n);
    double *v = malloc(sizeof(double) * n);
    int rc = -1;
    if (!a || !b || !v) goto done;
    memcpy(v, in, sizeof(double) * n);
    parity_mask(dims, Ns, p, v);
    if (or_hop(dims, Ns, U, 1 - p, v, a)) goto done;          /* D^{1-p,p} v */
    if (or_apply_s(dims, Ns, M5p, M5m, 0, 1 - p, a, b)) goto done; /* M5 . */
    if (or_hop(dims, Ns, U, p, b, a)) goto done;              /* D^{p,1-p} . */
    if (or_apply_s(dims, Ns, M5p, M5m, 0, p, a, b)) goto done;     /* M5 . */
    for (size_t i = 0; i < n; ++i) out[i] = v[i] - b[i];
    rc = 0;
done:
    free(a); free(b); free(v);
    return rc;
}

int or_cdag(const int dims[4], int Ns, const double *U, const double *M5p, const double *M5m, int p,
            const double *in, double *out) {
    if (!dims_ok(dims) || Ns < 1 || (p != 0 && p != 1) || !in || !out || in == out) return -1;
    size_t n = 24 * (size_t)Ns * vol(dims);
    double *a = malloc(sizeof(double) * n), *b = malloc(sizeof(double) * n);
    double *v = malloc(sizeof(double) * n);
    int rc = -1;
    if (!a || !b || !v) goto done;
    memcpy(v, in, sizeof(double) * n);
    parity_mask(dims, Ns, p, v);
    /* (M5 D^{p,1-p} M5 D^{1-p,p})^dag = (D^{1-p,p})^dag M5^T (D^{p,1-p})^dag M5^T */
    if (or_apply_s(dims, Ns, M5p, M5m, 1, p, v, a)) goto done;
    if (or_hop_dag(dims, Ns, U, p, a, b)) goto done;          /* lands on 1-p */
    if (or_apply_s(dims, Ns, M5p, M5m, 1, 1 - p, b, a)) goto done;
    if (or_hop_dag(dims, Ns, U, 1 - p, a, b)) goto done;      /* lands on p */
    for (size_t i = 0; i < n; ++i) out[i] = v[i] - b[i];
    rc = 0;
done:
    free(a); free(b); free(v);
    return rc;
}

int or_ccdag(const int dims[4], int Ns, const double *U, const double *M5p, const double *M5m,
             int p, const double *in, double *out) {
    if (!dims_ok(dims) || Ns < 1) return -1;
    size_t n = 24 * (size_t)Ns * vol(dims);
    double *t = malloc(sizeof(double) * n);
    if (!t) return -1;
    int rc = or_cdag(dims, Ns, U, M5p, M5m, p, in, t);
    if (!rc) rc = or_c(dims, Ns, U, M5p, M5m, p, t, out);
    free(t);
    return rc;
}

/* ------------------------------------------------------------ Algorithm 1 */

int or_dot(long nreal, const double *a, const double *b, double *re, double *im) {
    if (nreal < 0 || (nreal & 1) || !a || !b) return -1;
    const cplx *ca = (const cplx *)a, *cb = (const cplx *)b;
    cplx s = 0;
    for (long i = 0; i < nreal / 2; ++i) s += conj(ca[i]) * cb[i];
    if (re) *re = creal(s);
    if (im) *im = cimag(s);
    return 0;
}

static double norm2(size_t n, const double *a) {
    double s = 0;
    for (size_t i = 0; i < n; ++i) s += a[i] * a[i];
    return s;
}

int or_cg(const int dims[4], int Ns, const double *U, const double *M5p, const double *M5m, int p,
          const double *b, double *x, double tol, int maxiter, int *iters, double *relres) {
    if (!dims_ok(dims) || Ns < 1 || (p != 0 && p != 1) || !b || !x || maxiter < 0) return -1;
    size_t n = 24 * (size_t)Ns * vol(dims);
    double *r = malloc(sizeof(double) * n), *pv = malloc(sizeof(double) * n),
           *Ap = malloc(sizeof(double) * n);
    int rc = -1, k = 0;
    if (!r || !pv || !Ap) goto done;
    parity_mask(dims, Ns, p, x);
    /* r0 = b - A x0, p0 = r0 */
    if (or_ccdag(dims, Ns, U, M5p, M5m, p, x, Ap)) goto done;
    for (size_t i = 0; i < n; ++i) r[i] = b[i] - Ap[i];
    parity_mask(dims, Ns, p, r);
    memcpy(pv, r, sizeof(double) * n);
    double rr = norm2(n, r);
    double bb = norm2(n, b);
    while (sqrt(rr) > tol * sqrt(bb) && k < maxiter) {
        if (or_ccdag(dims, Ns, U, M5p, M5m, p, pv, Ap)) goto done;
        double pAp, im;
        or_dot((long)n, pv, Ap, &pAp, &im);
        double alpha = rr / pAp;
        for (size_t i = 0; i < n; ++i) r[i] -= alpha * Ap[i];
        double rr_new = norm2(n, r);
        double beta = rr_new / rr;
        for (size_t i = 0; i < n; ++i) x[i] += alpha * pv[i];
        for (size_t i = 0; i < n; ++i) pv[i] = r[i] + beta * pv[i];
        rr = rr_new;
        ++k;
    }
    if (iters) *iters = k;
    if (relres) {
        if (or_ccdag(dims, Ns, U, M5p, M5m, p, x, Ap)) goto done;
        for (size_t i = 0; i < n; ++i) r[i] = b[i] - Ap[i];
        parity_mask(dims, Ns, p, r);
        *relres = sqrt(norm2(n, r) / bb);
    }
    rc = 0;
done:
    free(r); free(pv); free(Ap);
    return rc;
}

/* ------------------------------------------------------------ Eq. 10 */

int or_solve_full(const int dims[4], int Ns, const double *U, double m0, double mq,
                  const double *omega, const double *sigma, int p, const double *eta, double *psi,
                  double tol, int maxiter, int *iters, double *relres) {
    if (!dims_ok(dims) || !weights_ok(Ns, omega, sigma) || (p != 0 && p != 1) || !U || !eta ||
        !psi || m0 == 0.0)
        return -1;
    size_t n = 24 * (size_t)Ns * vol(dims);
    size_t mm = sizeof(double) * Ns * Ns;
    double *M5p = malloc(mm), *M5m = malloc(mm), *S1p = malloc(mm), *S1m = malloc(mm),
           *S2p = malloc(mm), *S2m = malloc(mm);
    double *etap = malloc(sizeof(double) * n), *b = malloc(sizeof(double) * n),
           *t1 = malloc(sizeof(double) * n), *t2 = malloc(sizeof(double) * n),
           *y = calloc(n, sizeof(double)), *phi = malloc(sizeof(double) * n);
    int rc = -1;
    if (!M5p || !M5m || !S1p || !S1m || !S2p || !S2m || !etap || !b || !t1 || !t2 || !y || !phi)
        goto done;
    if (or_m5(Ns, m0, mq, omega, sigma, M5p, M5m)) goto done;
    if (or_s1s2(Ns, m0, mq, omega, sigma, S1p, S1m, S2p, S2m)) goto done;
    /* eta' = S1 eta */
    if (or_apply_s(dims, Ns, S1p, S1m, 0, -1, eta, etap)) goto done;
    /* b = eta'_p - M5 D^{p,1-p} eta'_{1-p} */
    memcpy(t2, etap, sizeof(double) * n);
    parity_mask(dims, Ns, 1 - p, t2);
    if (or_hop(dims, Ns, U, p, t2, t1)) goto done;
    if (or_apply_s(dims, Ns, M5p, M5m, 0, p, t1, t2)) goto done;
    for (size_t i = 0; i < n; ++i) b[i] = etap[i] - t2[i];
    parity_mask(dims, Ns, p, b);
    /* C C^dag y = b */
    if (or_cg(dims, Ns, U, M5p, M5m, p, b, y, tol, maxiter, iters, relres)) goto done;
    /* phi_p = C^dag y */
    if (or_cdag(dims, Ns, U, M5p, M5m, p, y, phi)) goto done;
    /* phi_{1-p} = eta'_{1-p} - M5 D^{1-p,p} phi_p */
    if (or_hop(dims, Ns, U, 1 - p, phi, t1)) goto done;
    if (or_apply_s(dims, Ns, M5p, M5m, 0, 1 - p, t1, t2)) goto done;
    {
        long V = vol(dims);
        for (long x = 0; x < V; ++x) {
            if (parity_of(dims, x) == p) continue;
            size_t o = 24 * (size_t)Ns * x;
            for (size_t c = 0; c < 24 * (size_t)Ns; ++c) phi[o + c] = etap[o + c] - t2[o + c];
        }
    }
    /* psi = S2 phi */
    if (or_apply_s(dims, Ns, S2p, S2m, 0, -1, phi, psi)) goto done;
    rc = 0;
done:
    free(M5p); free(M5m); free(S1p); free(S1m); free(S2p); free(S2m);
    free(etap); free(b); free(t1); free(t2); free(y); free(phi);
    return rc;
}
