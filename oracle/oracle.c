/*
 * FP64 CPU oracle for leading-order event reweighting  --  TEST INFRASTRUCTURE.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline/reference
 * arm may load this library.  The product path (the CUDA library) shares no
 * code, header, table or constant with it and never calls it.
 *
 * What it computes (arXiv:2312.07440, Sec. 2):
 *   - per event the tree-level squared matrix element |M|^2, averaged over
 *     initial spins and colours and summed over final ones (Sec. 2.1, the
 *     |M|^2 factor of Eq. 1);
 *   - the reweighting ratio r = |M'|^2/|M|^2 and new weight W' = r W
 *     (Sec. 2.2, Eq. 3), the validity condition |M|^2 != 0 (Sec. 2.2);
 *   - the cross section sigma = sum_k W_k (Sec. 2.1, Eq. 2) is summed exactly
 *     by the Python wrapper (math.fsum).
 *
 * How (plain and slow, by design):
 *   - Dirac matrices are explicit 4x4 complex matrices in the chiral basis,
 *     gamma5 = i g0 g1 g2 g3 formed by matrix products;
 *   - external spinors from u^s(p) = (sqrt(p.sigma) xi, sqrt(p.sigmabar) xi),
 *     v^s(p) = (sqrt(p.sigma) eta, -sqrt(p.sigmabar) eta) with the 2x2 matrix
 *     square roots written out (Peskin & Schroeder, Sec. 3.3);
 *   - gluon polarisations as explicit transverse vectors;
 *   - QCD amplitudes (g g -> t tbar + n g) as colour-ordered partial
 *     amplitudes A_sigma, one Berends-Giele recursion per ordering sigma
 *     (Berends & Giele, Nucl. Phys. B306 (1988) 759), with colour-ordered
 *     3- and 4-gluon vertices derived from the Feynman rules of Peskin &
 *     Schroeder Ch. 16 (D_mu = d_mu - i g A^a t^a);
 *   - |M|^2 = sum_hel sum_{sigma,tau} A_sigma^* C_{sigma tau} A_tau with
 *     C_{sigma tau} = sum_colours (t^sigma)^*_{ij} (t^tau)_{ij}, formed by
 *     brute force from the 8 Gell-Mann matrices;
 *   - e+ e- -> mu+ mu- from explicit photon and Z currents, Z propagator in
 *     unitary gauge with a fixed width;
 *   - e+ e- -> n photons (pure QED, massless electrons) as the sum over the
 *     n! orders in which the photons attach to the electron line, one 4x4
 *     matrix chain per order (the n! Feynman diagrams written out);
 *   - two further independent evaluations used only as pins: spin sums by
 *     traces with (pslash + m) projectors, and full-colour amplitudes from the
 *     colour-dressed (f^{abc}, t^a) Feynman rules.
 *
 * Readings where the paper is silent (it prints no amplitude formulas):
 *   - |M|^2 normalisation: 1/4 spin average, 1/64 colour average for g g,
 *     1/n! for n identical outgoing gluons or photons;
 *   - e+ e- -> 5 photons: massless electrons, coupling e = sqrt(4 pi alpha)
 *     with alpha = 1/alpha_em_inv (the "electroweak coupling" the paper's
 *     benchmark varies);
 *   - EW inputs (alpha, G_F, M_Z) with M_W, s_W derived per parameter set;
 *   - top width 0 in every top propagator (all are off shell);
 *   - a top-mass change moves the event onto the new mass shell by a common
 *     rescaling of the outgoing 3-momenta at fixed partonic energy; events
 *     with no solution are outside the new phase space and get |M'|^2 = 0.
 *
 * Parity pins: every function here is pinned by tests/test_oracle_*.py
 * against closed forms, invariances and independent evaluations.
 */
#define _GNU_SOURCE
#include <stdlib.h>
#include <string.h>
#include <tgmath.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* The arithmetic type.  The default build is FP64.  The same source compiled
   with -DORACLE_EXTENDED (real = long double: 64-bit significand on x86-64,
   113-bit IEEE quadruple on AArch64) evaluates the identical formulas with
   far less rounding; it exports only the batch entry points (oracle_me,
   oracle_reshuffle, oracle_reweight), whose event data stay float64 at the
   interface.  <tgmath.h> picks the maths function of the argument's type. */
#ifdef ORACLE_EXTENDED
typedef long double real;
typedef long double complex cx;
#define OR_PI 3.141592653589793238462643383279502884L
#else
typedef double real;
typedef double complex cx;
#define OR_PI M_PI
#endif

#define OR_EE_MUMU 0
#define OR_GG_TT 1
#define OR_GG_TTG 2
#define OR_GG_TTGG 3
#define OR_EE_5A 4  /* e- e+ -> 5 photons (the paper's own process, Table 1) */
#define MAXG 4      /* max gluons on the quark line */
#define MAXK 24     /* 4! colour orderings */
#define MAXN 7      /* max external particles */
#define MAXA 5      /* max photons on the electron line */

/* model parameters, same field order as the product's rw_params */
typedef struct {
    real alpha_s, m_t, w_t, yt_scale, alpha_em_inv, G_F, m_Z, w_Z;
} or_params;

/* ------------------------------------------------------------------------ */
/* Minkowski space and Dirac algebra                                         */
/* ------------------------------------------------------------------------ */
static const real GMETRIC[4] = {1.0, -1.0, -1.0, -1.0};
static cx GAMMA[4][4][4]; /* GAMMA[mu][row][col], upper index mu */
static cx GAMMA5[4][4];
static cx IDENT4[4][4];
static int dirac_ready = 0;

static void mat4_mul(cx A[4][4], cx B[4][4], cx C[4][4]) {
    cx T[4][4];
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            cx s = 0;
            for (int k = 0; k < 4; k++) s += A[i][k] * B[k][j];
            T[i][j] = s;
        }
    memcpy(C, T, sizeof(T));
}

static void dirac_init(void) {
    if (dirac_ready) return;
    /* Pauli matrices sigma^0 = 1, sigma^k */
    cx sig[4][2][2] = {{{1, 0}, {0, 1}}, {{0, 1}, {1, 0}}, {{0, -I}, {I, 0}}, {{1, 0}, {0, -1}}};
    memset(GAMMA, 0, sizeof(GAMMA));
    /* chiral basis: gamma^mu = [[0, sigma^mu], [sigmabar^mu, 0]],
       sigma^mu = (1, sigma^k), sigmabar^mu = (1, -sigma^k) */
    for (int mu = 0; mu < 4; mu++)
        for (int i = 0; i < 2; i++)
            for (int j = 0; j < 2; j++) {
                GAMMA[mu][i][2 + j] = sig[mu][i][j];
                GAMMA[mu][2 + i][j] = (mu == 0 ? 1.0 : -1.0) * sig[mu][i][j];
            }
    cx T[4][4];
    mat4_mul(GAMMA[0], GAMMA[1], T);
    mat4_mul(T, GAMMA[2], T);
    mat4_mul(T, GAMMA[3], T);
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            GAMMA5[i][j] = I * T[i][j];
            IDENT4[i][j] = (i == j);
        }
    dirac_ready = 1;
}

/* a.b with the (+,-,-,-) metric, no complex conjugation */
static cx mdot(const cx a[4], const cx b[4]) {
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}
static real rdot(const real a[4], const real b[4]) {
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}

/* S = gamma^mu a_mu */
static void slash(const cx a[4], cx S[4][4]) {
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            cx s = 0;
            for (int mu = 0; mu < 4; mu++) s += GMETRIC[mu] * a[mu] * GAMMA[mu][i][j];
            S[i][j] = s;
        }
}
static void rslash(const real a[4], cx S[4][4]) {
    cx c[4] = {a[0], a[1], a[2], a[3]};
    slash(c, S);
}
static void matvec(cx M[4][4], const cx x[4], cx y[4]) {
    cx t[4];
    for (int i = 0; i < 4; i++) {
        cx s = 0;
        for (int j = 0; j < 4; j++) s += M[i][j] * x[j];
        t[i] = s;
    }
    memcpy(y, t, sizeof(t));
}
/* row spinor times column spinor */
static cx rowcol(const cx r[4], const cx c[4]) {
    cx s = 0;
    for (int i = 0; i < 4; i++) s += r[i] * c[i];
    return s;
}
/* bar(psi) = psi^dagger gamma^0 (row vector) */
static void dirac_bar(const cx psi[4], cx out[4]) {
    for (int j = 0; j < 4; j++) {
        cx s = 0;
        for (int i = 0; i < 4; i++) s += conj(psi[i]) * GAMMA[0][i][j];
        out[j] = s;
    }
}
/* bar(Gamma) = gamma^0 Gamma^dagger gamma^0 */
static void mat_bar(cx G[4][4], cx out[4][4]) {
    cx D[4][4];
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) D[i][j] = conj(G[j][i]);
    mat4_mul(GAMMA[0], D, D);
    mat4_mul(D, GAMMA[0], out);
}
static cx trace4(cx A[4][4]) { return A[0][0] + A[1][1] + A[2][2] + A[3][3]; }

/* ------------------------------------------------------------------------ */
/* External wavefunctions                                                    */
/* ------------------------------------------------------------------------ */

/* sqrt of the 2x2 positive semi-definite Hermitian matrix
   A = p^0 + sgn * pvec.sigma  (sgn = -1: p.sigma, +1: p.sigmabar),
   sqrt(A) = (A + sqrt(det A) 1)/sqrt(tr A + 2 sqrt(det A)), det A = m^2. */
static void sqrt_psig(const real p[4], real m, int sgn, cx R[2][2]) {
    cx A[2][2];
    A[0][0] = p[0] + sgn * p[3];
    A[1][1] = p[0] - sgn * p[3];
    A[0][1] = sgn * (p[1] - I * p[2]);
    A[1][0] = sgn * (p[1] + I * p[2]);
    real sd = fabs(m);
    real nrm = sqrt(2.0 * p[0] + 2.0 * sd);
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++) R[i][j] = (A[i][j] + (i == j ? sd : 0.0)) / nrm;
}

/* two-component basis spinor: basis 0 -> spin along z (s=0 up, s=1 down);
   basis 1 -> helicity eigenstates along pvec (s=0: +1/2, s=1: -1/2). */
static void two_spinor(const real p[4], int basis, int s, cx chi[2]) {
    if (basis == 0) {
        chi[0] = (s == 0);
        chi[1] = (s == 1);
        return;
    }
    real pp = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
    real ct = pp > 0 ? p[3] / pp : 1.0;
    real c2 = sqrt(fmax(0.0, 0.5 * (1.0 + ct))), s2 = sqrt(fmax(0.0, 0.5 * (1.0 - ct)));
    real pt = hypot(p[1], p[2]);
    cx eph = pt > 0 ? (p[1] + I * p[2]) / pt : 1.0;
    if (s == 0) { /* chi_+ */
        chi[0] = c2;
        chi[1] = eph * s2;
    } else { /* chi_- */
        chi[0] = -conj(eph) * s2;
        chi[1] = c2;
    }
}

static void spinor_u(const real p[4], real m, int basis, int s, cx u[4]) {
    cx R[2][2], L[2][2], xi[2];
    two_spinor(p, basis, s, xi);
    sqrt_psig(p, m, -1, L); /* sqrt(p.sigma) */
    sqrt_psig(p, m, +1, R); /* sqrt(p.sigmabar) */
    for (int i = 0; i < 2; i++) {
        u[i] = L[i][0] * xi[0] + L[i][1] * xi[1];
        u[2 + i] = R[i][0] * xi[0] + R[i][1] * xi[1];
    }
}

/* v: helicity label s=0 (+1/2) uses eta = chi_-, s=1 uses chi_+ */
static void spinor_v(const real p[4], real m, int basis, int s, cx v[4]) {
    cx R[2][2], L[2][2], eta[2];
    two_spinor(p, basis, basis == 1 ? 1 - s : s, eta);
    sqrt_psig(p, m, -1, L);
    sqrt_psig(p, m, +1, R);
    for (int i = 0; i < 2; i++) {
        v[i] = L[i][0] * eta[0] + L[i][1] * eta[1];
        v[2 + i] = -(R[i][0] * eta[0] + R[i][1] * eta[1]);
    }
}

/* transverse polarisation for momentum k: basis 0 linear (s=0: e1, s=1: e2),
   basis 1 helicity eps(lambda) = (-lambda e1 - i e2)/sqrt2, s=0 -> +1. */
static void polvec(const real k[4], int basis, int s, cx eps[4]) {
    real kk = sqrt(k[1] * k[1] + k[2] * k[2] + k[3] * k[3]);
    real ct = kk > 0 ? k[3] / kk : 1.0;
    real st = sqrt(fmax(0.0, 1.0 - ct * ct));
    real pt = hypot(k[1], k[2]);
    real cp = pt > 0 ? k[1] / pt : 1.0, sp = pt > 0 ? k[2] / pt : 0.0;
    real e1[4] = {0.0, ct * cp, ct * sp, -st};
    real e2[4] = {0.0, -sp, cp, 0.0};
    for (int mu = 0; mu < 4; mu++) {
        if (basis == 0)
            eps[mu] = s == 0 ? e1[mu] : e2[mu];
        else {
            real lam = s == 0 ? 1.0 : -1.0;
            eps[mu] = (-lam * e1[mu] - I * e2[mu]) / sqrt((real)2);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* SU(3)                                                                     */
/* ------------------------------------------------------------------------ */
static cx TGEN[8][3][3]; /* t^a = lambda^a / 2 */
static real FSTRUCT[8][8][8];
static real CMAT[MAXG + 1][MAXK][MAXK];
static int PERM[MAXG + 1][MAXK][MAXG];
static int NPERM[MAXG + 1];
static int su3_ready = 0;

static void mat3_mul(cx A[3][3], cx B[3][3], cx C[3][3]) {
    cx T[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cx s = 0;
            for (int k = 0; k < 3; k++) s += A[i][k] * B[k][j];
            T[i][j] = s;
        }
    memcpy(C, T, sizeof(T));
}

/* next lexicographic permutation; returns 0 after the last one */
static int next_perm(int *a, int n) {
    int i = n - 2;
    while (i >= 0 && a[i] > a[i + 1]) i--;
    if (i < 0) return 0;
    int j = n - 1;
    while (a[j] < a[i]) j--;
    int t = a[i]; a[i] = a[j]; a[j] = t;
    for (int l = i + 1, r = n - 1; l < r; l++, r--) { t = a[l]; a[l] = a[r]; a[r] = t; }
    return 1;
}

static void su3_init(void) {
    if (su3_ready) return;
#ifdef ORACLE_EXTENDED
    const real s3 = 1 / sqrt((real)3);
#else
    static const real s3 = 0.57735026918962576451; /* 1/sqrt(3) */
#endif
    cx lam[8][3][3];
    memset(lam, 0, sizeof(lam));
    lam[0][0][1] = 1; lam[0][1][0] = 1;
    lam[1][0][1] = -I; lam[1][1][0] = I;
    lam[2][0][0] = 1; lam[2][1][1] = -1;
    lam[3][0][2] = 1; lam[3][2][0] = 1;
    lam[4][0][2] = -I; lam[4][2][0] = I;
    lam[5][1][2] = 1; lam[5][2][1] = 1;
    lam[6][1][2] = -I; lam[6][2][1] = I;
    lam[7][0][0] = s3; lam[7][1][1] = s3; lam[7][2][2] = -2 * s3;
    for (int a = 0; a < 8; a++)
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) TGEN[a][i][j] = 0.5 * lam[a][i][j];
    /* f^{abc} = -2 i Tr(t^a [t^b, t^c]) */
    for (int a = 0; a < 8; a++)
        for (int b = 0; b < 8; b++)
            for (int c = 0; c < 8; c++) {
                cx X[3][3], Y[3][3];
                mat3_mul(TGEN[b], TGEN[c], X);
                mat3_mul(TGEN[c], TGEN[b], Y);
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++) X[i][j] -= Y[i][j];
                mat3_mul(TGEN[a], X, X);
                cx tr = X[0][0] + X[1][1] + X[2][2];
                FSTRUCT[a][b][c] = creal(-2.0 * I * tr);
            }
    /* orderings (lexicographic) and brute-force colour matrices */
    for (int n = 1; n <= MAXG; n++) {
        int a[MAXG];
        for (int i = 0; i < n; i++) a[i] = i;
        int k = 0;
        do {
            for (int i = 0; i < n; i++) PERM[n][k][i] = a[i];
            k++;
        } while (next_perm(a, n));
        NPERM[n] = k;
        static cx S[MAXK][3][3];
        real acc[MAXK][MAXK];
        memset(acc, 0, sizeof(acc));
        int ncol = 1;
        for (int i = 0; i < n; i++) ncol *= 8;
        for (int idx = 0; idx < ncol; idx++) {
            int adj[MAXG], t = idx;
            for (int i = 0; i < n; i++) { adj[i] = t % 8; t /= 8; }
            for (int s = 0; s < k; s++) {
                cx P[3][3];
                memcpy(P, TGEN[adj[PERM[n][s][0]]], sizeof(P));
                for (int i = 1; i < n; i++) mat3_mul(P, TGEN[adj[PERM[n][s][i]]], P);
                memcpy(S[s], P, sizeof(P));
            }
            for (int s = 0; s < k; s++)
                for (int u = 0; u < k; u++) {
                    cx z = 0;
                    for (int i = 0; i < 3; i++)
                        for (int j = 0; j < 3; j++) z += conj(S[s][i][j]) * S[u][i][j];
                    acc[s][u] += creal(z);
                }
        }
        for (int s = 0; s < k; s++)
            for (int u = 0; u < k; u++) CMAT[n][s][u] = acc[s][u];
    }
    su3_ready = 1;
}

static void init_all(void) {
    dirac_init();
    su3_init();
}

/* ------------------------------------------------------------------------ */
/* Colour-ordered vertices (all momenta incoming)                            */
/* ------------------------------------------------------------------------ */
/* 3-gluon: V3(J1,P1;J2,P2)^mu = -J1^mu (2P1+P2).J2 + (J1.J2)(P1-P2)^mu
                               + J2^mu (2P2+P1).J1                           */
static void vertex3(const cx J1[4], const real P1[4], const cx J2[4], const real P2[4], cx out[4]) {
    cx a[4], b[4];
    for (int mu = 0; mu < 4; mu++) {
        a[mu] = 2.0 * P1[mu] + P2[mu];
        b[mu] = 2.0 * P2[mu] + P1[mu];
    }
    cx aJ2 = mdot(a, J2), bJ1 = mdot(b, J1), J12 = mdot(J1, J2);
    for (int mu = 0; mu < 4; mu++) out[mu] = -J1[mu] * aJ2 + J12 * (P1[mu] - P2[mu]) + J2[mu] * bJ1;
}
/* 4-gluon: V4(J1,J2,J3)^mu = 2 J2^mu (J1.J3) - J1^mu (J2.J3) - J3^mu (J1.J2) */
static void vertex4(const cx J1[4], const cx J2[4], const cx J3[4], cx out[4]) {
    cx d13 = mdot(J1, J3), d23 = mdot(J2, J3), d12 = mdot(J1, J2);
    for (int mu = 0; mu < 4; mu++) out[mu] = 2.0 * J2[mu] * d13 - J1[mu] * d23 - J3[mu] * d12;
}

/*
 * Colour-ordered partial amplitude A(sigma) for t(p3) tbar(p4) + n gluons,
 * defined by M_{ij} = sum_sigma (t^{a_sigma1} ... t^{a_sigman})_{ij} A(sigma)
 * (i: top colour, j: antitop colour).  k[g]: incoming momentum of gluon g,
 * eps[g]: its polarisation (already conjugated if outgoing), ubar: top row
 * spinor, v: antitop spinor, p4: antitop momentum.
 */
static cx amp_ordered(int n, const int *sig, real k[][4], cx eps[][4], const real p4[4], const cx ubar[4],
                      const cx v[4], real m, real g) {
    cx J[MAXG][MAXG][4];
    real K[MAXG][MAXG][4];
    cx psi[MAXG + 1][4];
    for (int len = 1; len <= n; len++)
        for (int a = 0; a + len - 1 < n; a++) {
            int b = a + len - 1;
            for (int mu = 0; mu < 4; mu++) {
                real s = 0;
                for (int i = a; i <= b; i++) s += k[sig[i]][mu];
                K[a][b][mu] = s;
            }
            if (len == 1) {
                for (int mu = 0; mu < 4; mu++) J[a][a][mu] = eps[sig[a]][mu];
                continue;
            }
            cx acc[4] = {0, 0, 0, 0}, t[4];
            for (int c = a; c < b; c++) {
                vertex3(J[a][c], K[a][c], J[c + 1][b], K[c + 1][b], t);
                for (int mu = 0; mu < 4; mu++) acc[mu] += -g * t[mu];
            }
            for (int c = a; c < b; c++)
                for (int d = c + 1; d < b; d++) {
                    vertex4(J[a][c], J[c + 1][d], J[d + 1][b], t);
                    for (int mu = 0; mu < 4; mu++) acc[mu] += g * g * t[mu];
                }
            real K2 = rdot(K[a][b], K[a][b]);
            for (int mu = 0; mu < 4; mu++) J[a][b][mu] = acc[mu] / K2;
        }
    memcpy(psi[n], v, sizeof(cx) * 4);
    for (int a = n - 1; a >= 0; a--) {
        real q[4];
        for (int mu = 0; mu < 4; mu++) q[mu] = K[a][n - 1][mu] - p4[mu];
        cx acc[4] = {0, 0, 0, 0}, t[4], S[4][4];
        for (int c = a; c < n; c++) {
            slash(J[a][c], S);
            matvec(S, psi[c + 1], t);
            for (int i = 0; i < 4; i++) acc[i] += t[i];
        }
        cx P[4][4];
        rslash(q, P);
        for (int i = 0; i < 4; i++) P[i][i] += m;
        matvec(P, acc, t);
        real den = rdot(q, q) - m * m;
        for (int i = 0; i < 4; i++) psi[a][i] = -g * t[i] / den;
    }
    cx A = 0, t[4], S[4][4];
    for (int c = 0; c < n; c++) {
        slash(J[0][c], S);
        matvec(S, psi[c + 1], t);
        A += rowcol(ubar, t);
    }
    return g * A;
}

/* Same recursion with the spinors amputated: Gamma(sigma) is the 4x4 matrix
   with A(sigma) = ubar Gamma(sigma) v (used by the trace evaluation). */
static void amp_ordered_matrix(int n, const int *sig, real k[][4], cx eps[][4], const real p4[4], real m,
                               real g, cx Gam[4][4]) {
    cx J[MAXG][MAXG][4];
    real K[MAXG][MAXG][4];
    cx Psi[MAXG + 1][4][4];
    for (int len = 1; len <= n; len++)
        for (int a = 0; a + len - 1 < n; a++) {
            int b = a + len - 1;
            for (int mu = 0; mu < 4; mu++) {
                real s = 0;
                for (int i = a; i <= b; i++) s += k[sig[i]][mu];
                K[a][b][mu] = s;
            }
            if (len == 1) {
                for (int mu = 0; mu < 4; mu++) J[a][a][mu] = eps[sig[a]][mu];
                continue;
            }
            cx acc[4] = {0, 0, 0, 0}, t[4];
            for (int c = a; c < b; c++) {
                vertex3(J[a][c], K[a][c], J[c + 1][b], K[c + 1][b], t);
                for (int mu = 0; mu < 4; mu++) acc[mu] += -g * t[mu];
            }
            for (int c = a; c < b; c++)
                for (int d = c + 1; d < b; d++) {
                    vertex4(J[a][c], J[c + 1][d], J[d + 1][b], t);
                    for (int mu = 0; mu < 4; mu++) acc[mu] += g * g * t[mu];
                }
            real K2 = rdot(K[a][b], K[a][b]);
            for (int mu = 0; mu < 4; mu++) J[a][b][mu] = acc[mu] / K2;
        }
    memcpy(Psi[n], IDENT4, sizeof(IDENT4));
    for (int a = n - 1; a >= 0; a--) {
        real q[4];
        for (int mu = 0; mu < 4; mu++) q[mu] = K[a][n - 1][mu] - p4[mu];
        cx acc[4][4], S[4][4], T[4][4];
        memset(acc, 0, sizeof(acc));
        for (int c = a; c < n; c++) {
            slash(J[a][c], S);
            mat4_mul(S, Psi[c + 1], T);
            for (int i = 0; i < 4; i++)
                for (int j = 0; j < 4; j++) acc[i][j] += T[i][j];
        }
        cx P[4][4];
        rslash(q, P);
        for (int i = 0; i < 4; i++) P[i][i] += m;
        mat4_mul(P, acc, T);
        real den = rdot(q, q) - m * m;
        for (int i = 0; i < 4; i++)
            for (int j = 0; j < 4; j++) Psi[a][i][j] = -g * T[i][j] / den;
    }
    memset(Gam, 0, sizeof(cx) * 16);
    for (int c = 0; c < n; c++) {
        cx S[4][4], T[4][4];
        slash(J[0][c], S);
        mat4_mul(S, Psi[c + 1], T);
        for (int i = 0; i < 4; i++)
            for (int j = 0; j < 4; j++) Gam[i][j] += g * T[i][j];
    }
}

/* ------------------------------------------------------------------------ */
/* Processes                                                                 */
/* ------------------------------------------------------------------------ */
static int n_external(int process) {
    switch (process) {
    case OR_EE_MUMU: return 4;
    case OR_GG_TT: return 4;
    case OR_GG_TTG: return 5;
    case OR_GG_TTGG: return 6;
    case OR_EE_5A: return 7;
    }
    return -1;
}
static int is_qcd(int process) { return process >= OR_GG_TT && process <= OR_GG_TTGG; }
static int n_gluons(int process) { return is_qcd(process) ? n_external(process) - 2 : 0; }

/* gluon g of the quark line -> particle index: g0 = 0, g1 = 1, g2.. = 4.. */
static int gluon_particle(int g) { return g < 2 ? g : g + 2; }
static int factorial(int n) { return n <= 1 ? 1 : n * factorial(n - 1); }

/* electroweak couplings from (alpha^-1, G_F, M_Z) */
typedef struct { real e, gL, gR, MZ, WZ; } ew_coup;
static ew_coup ew_couplings(const or_params *par) {
    ew_coup c;
    real alpha = 1.0 / par->alpha_em_inv;
    real MZ = par->m_Z;
    real MW2 = 0.5 * MZ * MZ + sqrt(0.25 * MZ * MZ * MZ * MZ - OR_PI * alpha * MZ * MZ / (sqrt((real)2) * par->G_F));
    real sw2 = 1.0 - MW2 / (MZ * MZ);
    real sw = sqrt(sw2), cw = sqrt(1.0 - sw2);
    c.e = sqrt(4.0 * OR_PI * alpha);
    real Q = -1.0, T3 = -0.5;
    c.gL = c.e * (T3 - Q * sw2) / (sw * cw);
    c.gR = -c.e * Q * sw2 / (sw * cw);
    c.MZ = MZ;
    c.WZ = par->w_Z;
    return c;
}

/* Gamma^mu for the photon (e Q gamma^mu) and the Z (gamma^mu (gL PL + gR PR)) */
static void ew_vertex(const ew_coup *c, int boson, cx G[4][4][4]) {
    cx PL[4][4], PR[4][4];
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            PL[i][j] = 0.5 * (IDENT4[i][j] - GAMMA5[i][j]);
            PR[i][j] = 0.5 * (IDENT4[i][j] + GAMMA5[i][j]);
        }
    for (int mu = 0; mu < 4; mu++) {
        if (boson == 0) {
            for (int i = 0; i < 4; i++)
                for (int j = 0; j < 4; j++) G[mu][i][j] = c->e * (-1.0) * GAMMA[mu][i][j];
        } else {
            cx C[4][4];
            for (int i = 0; i < 4; i++)
                for (int j = 0; j < 4; j++) C[i][j] = c->gL * PL[i][j] + c->gR * PR[i][j];
            mat4_mul(GAMMA[mu], C, G[mu]);
        }
    }
}

/* boson propagator numerator/denominator contracted: sum_{mu,nu} a^mu P_{mu nu} b^nu */
static cx ew_contract(const ew_coup *c, int boson, const cx a[4], const cx b[4], const real kk[4]) {
    real s = rdot(kk, kk);
    if (boson == 0) return mdot(a, b) / s;
    cx ka = 0, kb = 0;
    cx kc[4] = {kk[0], kk[1], kk[2], kk[3]};
    ka = mdot(kc, a);
    kb = mdot(kc, b);
    cx D = s - c->MZ * c->MZ + I * c->MZ * c->WZ;
    return (mdot(a, b) - ka * kb / (c->MZ * c->MZ)) / D;
}

/* e-(p0) e+(p1) -> mu-(p2) mu+(p3) */
static real me_ee_mumu(real p[][4], const or_params *par) {
    ew_coup c = ew_couplings(par);
    cx G[2][4][4][4];
    ew_vertex(&c, 0, G[0]);
    ew_vertex(&c, 1, G[1]);
    real kk[4];
    for (int mu = 0; mu < 4; mu++) kk[mu] = p[0][mu] + p[1][mu];
    real sum = 0;
    for (int h = 0; h < 16; h++) {
        int s0 = h & 1, s1 = (h >> 1) & 1, s2 = (h >> 2) & 1, s3 = (h >> 3) & 1;
        cx u1[4], v2[4], vb2[4], u3[4], ub3[4], v4[4];
        spinor_u(p[0], 0.0, 0, s0, u1);
        spinor_v(p[1], 0.0, 0, s1, v2);
        dirac_bar(v2, vb2);
        spinor_u(p[2], 0.0, 0, s2, u3);
        dirac_bar(u3, ub3);
        spinor_v(p[3], 0.0, 0, s3, v4);
        cx M = 0;
        for (int V = 0; V < 2; V++) {
            cx jin[4], jout[4], t[4];
            for (int mu = 0; mu < 4; mu++) {
                matvec(G[V][mu], u1, t);
                jin[mu] = rowcol(vb2, t);
                matvec(G[V][mu], v4, t);
                jout[mu] = rowcol(ub3, t);
            }
            M += ew_contract(&c, V, jout, jin, kk);
        }
        sum += creal(M * conj(M));
    }
    return 0.25 * sum;
}

/* incoming momenta and default polarisations of the gluons on the quark line */
static void gluon_kin(int process, real p[][4], real k[][4]) {
    int n = n_gluons(process);
    for (int g = 0; g < n; g++) {
        int ip = gluon_particle(g);
        real sgn = ip < 2 ? 1.0 : -1.0;
        for (int mu = 0; mu < 4; mu++) k[g][mu] = sgn * p[ip][mu];
    }
}

static real me_gg_tt_ng(int process, real p[][4], const or_params *par) {
    int n = n_gluons(process), N = n_external(process);
    int K = NPERM[n];
    real g = sqrt(4.0 * OR_PI * par->alpha_s), m = par->m_t;
    real k[MAXG][4];
    gluon_kin(process, p, k);
    real sum = 0;
    for (int h = 0; h < (1 << N); h++) {
        cx eps[MAXG][4], u3[4], ub3[4], v4[4];
        for (int gg = 0; gg < n; gg++) {
            int ip = gluon_particle(gg);
            polvec(p[ip], 0, (h >> ip) & 1, eps[gg]);
            if (ip >= 2)
                for (int mu = 0; mu < 4; mu++) eps[gg][mu] = conj(eps[gg][mu]);
        }
        spinor_u(p[2], m, 0, (h >> 2) & 1, u3);
        dirac_bar(u3, ub3);
        spinor_v(p[3], m, 0, (h >> 3) & 1, v4);
        cx A[MAXK];
        for (int s = 0; s < K; s++) A[s] = amp_ordered(n, PERM[n][s], k, eps, p[3], ub3, v4, m, g);
        real cs = 0;
        for (int s = 0; s < K; s++)
            for (int t = 0; t < K; t++) cs += CMAT[n][s][t] * creal(conj(A[s]) * A[t]);
        sum += cs;
    }
    return sum / (4.0 * 64.0 * factorial(n - 2));
}

/*
 * e-(p0) e+(p1) -> photons k_1..k_n (particles 2..n+1), massless electrons,
 * pure QED.  For one helicity configuration (basis as in spinor_u/polvec;
 * hel[0] e-, hel[1] e+, hel[2..] photons):
 *   A = e^n sum_{orders s} vbar(p1) eps*_{s_n}slash S(q_{n-1}) ...
 *       eps*_{s_2}slash S(q_1) eps*_{s_1}slash u(p0),
 *   q_j = p0 - k_{s_1} - ... - k_{s_j},  S(q) = qslash / q^2,
 * the n! tree diagrams with the photons attached to the electron line in
 * every order (common factors of i and the vertex sign dropped: every
 * diagram carries the same ones).
 */
static cx amp_ee_photons(int n, real p[][4], int basis, const int *hel, real e, const cx *eps_in) {
    cx u[4], v[4], vb[4], E[MAXA][4][4];
    spinor_u(p[0], 0.0, basis, hel[0], u);
    spinor_v(p[1], 0.0, basis, hel[1], v);
    dirac_bar(v, vb);
    for (int i = 0; i < n; i++) {
        cx eps[4];
        if (eps_in) { /* explicit (already conjugated) polarisation vectors */
            memcpy(eps, eps_in + 4 * i, sizeof(eps));
        } else {
            polvec(p[2 + i], basis, hel[2 + i], eps);
            for (int mu = 0; mu < 4; mu++) eps[mu] = conj(eps[mu]);
        }
        slash(eps, E[i]);
    }
    int order[MAXA];
    for (int i = 0; i < n; i++) order[i] = i;
    cx A = 0;
    do {
        cx psi[4], t[4];
        real q[4];
        memcpy(psi, u, sizeof(psi));
        memcpy(q, p[0], sizeof(q));
        for (int j = 0; j < n; j++) {
            matvec(E[order[j]], psi, t);
            if (j == n - 1) {
                memcpy(psi, t, sizeof(psi));
                break;
            }
            for (int mu = 0; mu < 4; mu++) q[mu] -= p[2 + order[j]][mu];
            cx Q[4][4];
            rslash(q, Q);
            matvec(Q, t, psi);
            real q2 = rdot(q, q);
            for (int a = 0; a < 4; a++) psi[a] /= q2;
        }
        A += rowcol(vb, psi);
    } while (next_perm(order, n));
    return pow(e, n) * A;
}

/* spin-averaged |M|^2 of e- e+ -> n photons (1/4, 1/n!) */
static real me_ee_photons(int n, real p[][4], const or_params *par) {
    real e = sqrt(4.0 * OR_PI / par->alpha_em_inv);
    real sum = 0;
    int hel[MAXA + 2];
    for (int h = 0; h < (1 << (n + 2)); h++) {
        for (int i = 0; i < n + 2; i++) hel[i] = (h >> i) & 1;
        cx A = amp_ee_photons(n, p, 0, hel, e, NULL);
        sum += creal(A * conj(A));
    }
    return sum / (4.0 * factorial(n));
}

static real me_event(int process, real p[][4], const or_params *par) {
    if (process == OR_EE_MUMU) return me_ee_mumu(p, par);
    if (process == OR_EE_5A) return me_ee_photons(5, p, par);
    return me_gg_tt_ng(process, p, par);
}

/* ------------------------------------------------------------------------ */
/* Mass-shell reshuffle (a top-mass change moves the event)                  */
/* ------------------------------------------------------------------------ */
/* Outgoing particles 2..N-1 keep their directions; their 3-momenta are scaled
   by xi with sum_i sqrt(m_i'^2 + xi^2 |p_i|^2) = sum_i E_i (the partonic
   energy in the centre-of-mass frame).  Returns 0 on success, 1 if the new
   masses do not fit (the event is outside the new phase space). */
static int reshuffle(int N, const real *mnew, real pin[][4], real pout[][4]) {
    real etot = 0, msum = 0, p2[MAXN];
    for (int i = 2; i < N; i++) {
        etot += pin[i][0];
        msum += mnew[i];
        p2[i] = pin[i][1] * pin[i][1] + pin[i][2] * pin[i][2] + pin[i][3] * pin[i][3];
    }
    for (int i = 0; i < N; i++)
        for (int mu = 0; mu < 4; mu++) pout[i][mu] = pin[i][mu];
    if (!(msum < etot)) return 1;
    real xi = 1.0;
    for (int it = 0; it < 200; it++) {
        real f = -etot, df = 0;
        for (int i = 2; i < N; i++) {
            real e = sqrt(mnew[i] * mnew[i] + xi * xi * p2[i]);
            f += e;
            df += xi * p2[i] / e;
        }
        real step = f / df;
        if (xi - step <= 0) step = 0.5 * xi;
        xi -= step;
        if (fabs(step) <= 1e-15 * xi) break;
    }
    for (int i = 2; i < N; i++) {
        for (int mu = 1; mu < 4; mu++) pout[i][mu] = xi * pin[i][mu];
        pout[i][0] = sqrt(mnew[i] * mnew[i] + xi * xi * p2[i]);
    }
    return 0;
}

static void new_masses(int process, const or_params *par, real *m) {
    int N = n_external(process);
    for (int i = 0; i < N; i++) m[i] = 0;
    if (is_qcd(process)) m[2] = m[3] = par->m_t;
}

/* the event data stay float64 at the interface in either build */
static void load_event(int N, long E, const double *mom, long e, real p[][4]) {
    for (int i = 0; i < N; i++)
        for (int mu = 0; mu < 4; mu++) p[i][mu] = mom[((long)i * 4 + mu) * E + e];
}

/* parameter vector (alpha_s, m_t, w_t, yt_scale, alpha_em_inv, G_F, m_Z, w_Z) */
static or_params load_params(const double *v) {
    or_params q;
    q.alpha_s = v[0];
    q.m_t = v[1];
    q.w_t = v[2];
    q.yt_scale = v[3];
    q.alpha_em_inv = v[4];
    q.G_F = v[5];
    q.m_Z = v[6];
    q.w_Z = v[7];
    return q;
}

/* ------------------------------------------------------------------------ */
/* Exported API                                                              */
/* ------------------------------------------------------------------------ */
int oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

void oracle_init(void) { init_all(); }

/* |M|^2 per event; mom: SoA [N][4][E] */
int oracle_me(int process, const double *par, long E, const double *mom, double *me_out) {
    if (n_external(process) < 0) return -1;
    init_all();
    int N = n_external(process);
    const or_params pp = load_params(par);
#pragma omp parallel for schedule(dynamic, 16)
    for (long e = 0; e < E; e++) {
        real p[MAXN][4];
        load_event(N, E, mom, e, p);
        me_out[e] = (double)me_event(process, p, &pp);
    }
    return 0;
}

/* mass-shell reshuffle of a batch (for tests); status[e] = 0/1 */
int oracle_reshuffle(int process, const double *par_new, long E, const double *mom, double *mom_out, int *status) {
    if (n_external(process) < 0) return -1;
    int N = n_external(process);
    real m[MAXN];
    const or_params pn = load_params(par_new);
    new_masses(process, &pn, m);
#pragma omp parallel for schedule(static)
    for (long e = 0; e < E; e++) {
        real p[MAXN][4], q[MAXN][4];
        load_event(N, E, mom, e, p);
        status[e] = reshuffle(N, m, p, q);
        for (int i = 0; i < N; i++)
            for (int mu = 0; mu < 4; mu++) mom_out[((long)i * 4 + mu) * E + e] = (double)q[i][mu];
    }
    return 0;
}

/*
 * The reweighting steps of Sec. 3.2 for one event batch: |M|^2 under the
 * original parameters, then for each of the P parameter points |M'|^2,
 * r = |M'|^2/|M|^2 and W' = r W (Eq. 3).  Events with |M|^2 == 0 or
 * non-finite violate the validity condition: r = W' = 0 and they are counted
 * in n_bad.  me0[E], me_pts[P][E], ratio[P][E], wnew[P][E] may be NULL.
 */
int oracle_reweight(int process, const double *par0, int P, const double *pars, long E, const double *mom,
                    const double *w, double *me0, double *me_pts, double *ratio, double *wnew, long *n_bad) {
    if (n_external(process) < 0 || P < 0) return -1;
    init_all();
    int N = n_external(process);
    const or_params p0v = load_params(par0);
    const or_params *p0 = &p0v;
    or_params *pt = (or_params *)malloc(sizeof(or_params) * (P > 0 ? P : 1));
    if (!pt) return -1;
    for (int j = 0; j < P; j++) pt[j] = load_params(pars + 8 * (long)j);
    long bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : bad)
    for (long e = 0; e < E; e++) {
        real p[MAXN][4], q[MAXN][4];
        load_event(N, E, mom, e, p);
        real m0 = me_event(process, p, p0);
        int ok = isfinite(m0) && m0 != 0.0;
        if (!ok) bad++;
        if (me0) me0[e] = (double)m0;
        for (int j = 0; j < P; j++) {
            real m1;
            if (is_qcd(process) && pt[j].m_t != p0->m_t) {
                real mn[MAXN];
                new_masses(process, &pt[j], mn);
                m1 = reshuffle(N, mn, p, q) ? 0.0 : me_event(process, q, &pt[j]);
            } else {
                m1 = me_event(process, p, &pt[j]);
            }
            real r = ok ? m1 / m0 : 0.0;
            if (me_pts) me_pts[(long)j * E + e] = (double)m1;
            if (ratio) ratio[(long)j * E + e] = (double)r;
            if (wnew) wnew[(long)j * E + e] = ok ? (double)(r * w[e]) : 0.0;
        }
    }
    free(pt);
    if (n_bad) *n_bad = bad;
    return 0;
}

/* Everything below is used by the pin tests only and exists in the FP64
   build alone. */
#ifndef ORACLE_EXTENDED

/* colour matrix C[K][K] for n gluons (orderings in lexicographic order) */
int oracle_colour_matrix(int n, real *C, int *perms) {
    if (n < 1 || n > MAXG) return -1;
    init_all();
    int K = NPERM[n];
    for (int s = 0; s < K; s++) {
        for (int t = 0; t < K; t++) C[s * K + t] = CMAT[n][s][t];
        if (perms)
            for (int i = 0; i < n; i++) perms[s * n + i] = PERM[n][s][i];
    }
    return K;
}

/* the generators t^a (8x3x3 complex) and f^{abc} (8x8x8) */
void oracle_su3(cx *t, real *f) {
    init_all();
    if (t) memcpy(t, TGEN, sizeof(TGEN));
    if (f) memcpy(f, FSTRUCT, sizeof(FSTRUCT));
}

/* the Dirac matrices gamma^mu (4x4x4) and gamma5 */
void oracle_dirac(cx *g, cx *g5) {
    init_all();
    if (g) memcpy(g, GAMMA, sizeof(GAMMA));
    if (g5) memcpy(g5, GAMMA5, sizeof(GAMMA5));
}

/*
 * External wavefunctions of one event (AoS p[N][4]) for a QCD process:
 * ext[i][4] complex: gluons -> eps (incoming) or eps^* (outgoing), top -> ubar
 * (row), antitop -> v.  basis 0: z-spin / linear, 1: helicity.  hel[i] in {0,1}.
 */
int oracle_external(int process, const real *p, real m, int basis, const int *hel, cx *ext) {
    if (!is_qcd(process)) return -1;
    init_all();
    int N = n_external(process);
    real pp[MAXN][4];
    memcpy(pp, p, sizeof(real) * 4 * N);
    for (int i = 0; i < N; i++) {
        cx *o = ext + 4 * i;
        if (i == 2) {
            cx u[4];
            spinor_u(pp[2], m, basis, hel[2], u);
            dirac_bar(u, o);
        } else if (i == 3) {
            spinor_v(pp[3], m, basis, hel[3], o);
        } else {
            polvec(pp[i], basis, hel[i], o);
            if (i >= 2)
                for (int mu = 0; mu < 4; mu++) o[mu] = conj(o[mu]);
        }
    }
    return 0;
}

/* raw spinors for tests: kind 0 = u, 1 = v; basis, s as above */
void oracle_spinor(int kind, const real *p, real m, int basis, int s, cx *out) {
    init_all();
    if (kind == 0)
        spinor_u(p, m, basis, s, out);
    else
        spinor_v(p, m, basis, s, out);
}
void oracle_polvec(const real *k, int basis, int s, cx *out) { polvec(k, basis, s, out); }

/* all partial amplitudes A[K] for explicit external wavefunctions ext[N][4] */
int oracle_partial_amps(int process, const real *p, real m, real alpha_s, const cx *ext, cx *A) {
    if (!is_qcd(process)) return -1;
    init_all();
    int n = n_gluons(process), N = n_external(process);
    real pp[MAXN][4], k[MAXG][4];
    memcpy(pp, p, sizeof(real) * 4 * N);
    gluon_kin(process, pp, k);
    cx eps[MAXG][4];
    for (int gg = 0; gg < n; gg++) memcpy(eps[gg], ext + 4 * gluon_particle(gg), sizeof(cx) * 4);
    real g = sqrt(4.0 * OR_PI * alpha_s);
    for (int s = 0; s < NPERM[n]; s++) A[s] = amp_ordered(n, PERM[n][s], k, eps, pp[3], ext + 8, ext + 12, m, g);
    return NPERM[n];
}

/*
 * Spin sums by traces (pin): |M|^2 without external spinors.
 *  g g -> t tbar (+g..): sum over linear gluon polarisations of
 *    sum_{s,t} C_st Tr[(p3slash + m) Gamma_t (p4slash - m) bar(Gamma_s)];
 *  e+ e- -> mu+ mu-: Tr[p3 G^mu p4 bar(G'^nu)] Tr[p1 G^a p0 bar(G'^b)] P_{mu a} P'^*_{nu b}.
 */
real oracle_me_traces(int process, const real *par, const real *p_aos) {
    init_all();
    int N = n_external(process);
    if (N < 0 || process == OR_EE_5A) return NAN;
    const or_params *pp = (const or_params *)par;
    real p[MAXN][4];
    memcpy(p, p_aos, sizeof(real) * 4 * N);
    if (process == OR_EE_MUMU) {
        ew_coup c = ew_couplings(pp);
        cx G[2][4][4][4], Gb[2][4][4][4];
        ew_vertex(&c, 0, G[0]);
        ew_vertex(&c, 1, G[1]);
        for (int V = 0; V < 2; V++)
            for (int mu = 0; mu < 4; mu++) mat_bar(G[V][mu], Gb[V][mu]);
        cx S0[4][4], S1[4][4], S2[4][4], S3[4][4];
        rslash(p[0], S0);
        rslash(p[1], S1);
        rslash(p[2], S2);
        rslash(p[3], S3);
        real kk[4];
        for (int mu = 0; mu < 4; mu++) kk[mu] = p[0][mu] + p[1][mu];
        real s = rdot(kk, kk);
        cx D[2] = {s, s - c.MZ * c.MZ + I * c.MZ * c.WZ};
        real klow[4];
        for (int mu = 0; mu < 4; mu++) klow[mu] = GMETRIC[mu] * kk[mu];
        real total = 0;
        for (int V = 0; V < 2; V++)
            for (int W = 0; W < 2; W++) {
                cx T1[4][4], T2[4][4];
                for (int mu = 0; mu < 4; mu++)
                    for (int nu = 0; nu < 4; nu++) {
                        cx X[4][4];
                        mat4_mul(S2, G[V][mu], X);
                        mat4_mul(X, S3, X);
                        mat4_mul(X, Gb[W][nu], X);
                        T1[mu][nu] = trace4(X);
                        mat4_mul(S1, G[V][mu], X);
                        mat4_mul(X, S0, X);
                        mat4_mul(X, Gb[W][nu], X);
                        T2[mu][nu] = trace4(X);
                    }
                /* propagator tensors with lower indices */
                cx P[4][4], Q[4][4];
                for (int mu = 0; mu < 4; mu++)
                    for (int a = 0; a < 4; a++) {
                        real gm = (mu == a) ? GMETRIC[mu] : 0.0;
                        P[mu][a] = (V == 0 ? gm : gm - klow[mu] * klow[a] / (c.MZ * c.MZ)) / D[V];
                        Q[mu][a] = conj((W == 0 ? gm : gm - klow[mu] * klow[a] / (c.MZ * c.MZ)) / D[W]);
                    }
                cx acc = 0;
                for (int mu = 0; mu < 4; mu++)
                    for (int nu = 0; nu < 4; nu++)
                        for (int a = 0; a < 4; a++)
                            for (int b = 0; b < 4; b++) acc += T1[mu][nu] * T2[a][b] * P[mu][a] * Q[nu][b];
                total += creal(acc);
            }
        return 0.25 * total;
    }
    int n = n_gluons(process);
    int K = NPERM[n];
    real g = sqrt(4.0 * OR_PI * pp->alpha_s), m = pp->m_t;
    real k[MAXG][4];
    gluon_kin(process, p, k);
    cx P3[4][4], P4[4][4];
    rslash(p[2], P3);
    rslash(p[3], P4);
    for (int i = 0; i < 4; i++) {
        P3[i][i] += m;
        P4[i][i] -= m;
    }
    real total = 0;
    for (int h = 0; h < (1 << n); h++) {
        cx eps[MAXG][4];
        for (int gg = 0; gg < n; gg++) {
            int ip = gluon_particle(gg);
            polvec(p[ip], 0, (h >> gg) & 1, eps[gg]);
        }
        cx Gam[MAXK][4][4], Gb[MAXK][4][4];
        for (int s = 0; s < K; s++) {
            amp_ordered_matrix(n, PERM[n][s], k, eps, p[3], m, g, Gam[s]);
            mat_bar(Gam[s], Gb[s]);
        }
        for (int s = 0; s < K; s++)
            for (int t = 0; t < K; t++) {
                cx X[4][4];
                mat4_mul(P3, Gam[t], X);
                mat4_mul(X, P4, X);
                mat4_mul(X, Gb[s], X);
                total += CMAT[n][s][t] * creal(trace4(X));
            }
    }
    return total / (4.0 * 64.0 * factorial(n - 2));
}

/*
 * Full-colour amplitude from the colour-dressed Feynman rules (pin for the
 * colour-ordered decomposition): returns M_{ij} (3x3, top colour i, antitop
 * colour j) for adjoint colours adj[g] of the gluons and wavefunctions ext.
 *   quark-gluon vertex   i g gamma^mu t^a
 *   3-gluon vertex       g f^{abc}[g^{mu nu}(k-p)^rho + g^{nu rho}(p-q)^mu + g^{rho mu}(q-k)^nu]
 *   4-gluon vertex       -i g^2 [f^{abe}f^{cde}(g^{mu rho}g^{nu sigma} - g^{mu sigma}g^{nu rho}) + (b<->c perms)]
 *   propagators          -i g_{mu nu}/k^2,  i(qslash + m)/(q^2 - m^2)
 */
int oracle_full_colour_amp(int process, const real *p_aos, real m, real alpha_s, const cx *ext, const int *adj,
                           cx *Mout) {
    if (!is_qcd(process)) return -1;
    init_all();
    int n = n_gluons(process), N = n_external(process);
    real p[MAXN][4], k[MAXG][4];
    memcpy(p, p_aos, sizeof(real) * 4 * N);
    gluon_kin(process, p, k);
    real g = sqrt(4.0 * OR_PI * alpha_s);
    int full = (1 << n) - 1;
    static cx J[1 << MAXG][8][4];
    static int nz[1 << MAXG][8]; /* J[S][a] not exactly zero */
    real KS[1 << MAXG][4];
    memset(J, 0, sizeof(J));
    memset(nz, 0, sizeof(nz));
    for (int S = 1; S <= full; S++) {
        for (int mu = 0; mu < 4; mu++) {
            real s = 0;
            for (int i = 0; i < n; i++)
                if (S >> i & 1) s += k[i][mu];
            KS[S][mu] = s;
        }
    }
    for (int S = 1; S <= full; S++) {
        int pc = __builtin_popcount(S);
        if (pc == 1) {
            int i = __builtin_ctz(S);
            for (int mu = 0; mu < 4; mu++) J[S][adj[i]][mu] = ext[4 * gluon_particle(i) + mu];
            nz[S][adj[i]] = 1;
            continue;
        }
        real K2 = rdot(KS[S], KS[S]);
        int low = S & -S;
        /* 3-vertex: unordered pairs {S1, S2}, S1 contains the lowest bit */
        for (int S1 = (S - 1) & S; S1 > 0; S1 = (S1 - 1) & S) {
            if (!(S1 & low)) continue;
            int S2 = S ^ S1;
            if (!S2) continue;
            for (int b = 0; b < 8; b++)
                for (int c = 0; c < 8; c++) {
                    if (!nz[S1][b] || !nz[S2][c]) continue; /* exact zeros */
                    cx t[4];
                    vertex3(J[S1][b], KS[S1], J[S2][c], KS[S2], t);
                    for (int a = 0; a < 8; a++) {
                        real f = FSTRUCT[a][b][c];
                        if (f == 0.0) continue;
                        for (int mu = 0; mu < 4; mu++) J[S][a][mu] += (-I / K2) * g * f * t[mu];
                    }
                }
        }
        /* 4-vertex: unordered triples */
        for (int S1 = (S - 1) & S; S1 > 0; S1 = (S1 - 1) & S) {
            if (!(S1 & low)) continue;
            int R = S ^ S1;
            if (!R) continue;
            int low2 = R & -R;
            for (int S2 = R; S2 > 0; S2 = (S2 - 1) & R) {
                if (!(S2 & low2)) continue;
                int S3 = R ^ S2;
                if (!S3) continue;
                for (int b = 0; b < 8; b++)
                    for (int c = 0; c < 8; c++)
                        for (int d = 0; d < 8; d++) {
                            if (!nz[S1][b] || !nz[S2][c] || !nz[S3][d]) continue; /* exact zeros */
                            const cx *J1 = J[S1][b], *J2 = J[S2][c], *J3 = J[S3][d];
                            cx d12 = mdot(J1, J2), d13 = mdot(J1, J3), d23 = mdot(J2, J3);
                            cx T1[4], T2[4], T3[4];
                            for (int mu = 0; mu < 4; mu++) {
                                T1[mu] = J2[mu] * d13 - J3[mu] * d12;
                                T2[mu] = J1[mu] * d23 - J3[mu] * d12;
                                T3[mu] = J1[mu] * d23 - J2[mu] * d13;
                            }
                            for (int a = 0; a < 8; a++) {
                                real c1 = 0, c2 = 0, c3 = 0;
                                for (int e = 0; e < 8; e++) {
                                    c1 += FSTRUCT[a][b][e] * FSTRUCT[c][d][e];
                                    c2 += FSTRUCT[a][c][e] * FSTRUCT[b][d][e];
                                    c3 += FSTRUCT[a][d][e] * FSTRUCT[b][c][e];
                                }
                                if (c1 == 0 && c2 == 0 && c3 == 0) continue;
                                for (int mu = 0; mu < 4; mu++)
                                    J[S][a][mu] += (-I / K2) * (-I * g * g) * (c1 * T1[mu] + c2 * T2[mu] + c3 * T3[mu]);
                            }
                        }
            }
        }
        for (int a = 0; a < 8; a++)
            for (int mu = 0; mu < 4; mu++)
                if (J[S][a][mu] != 0) nz[S][a] = 1;
    }
    /* fermion line from the antitop end: psi[S][i][j][4] */
    static cx psi[1 << MAXG][3][3][4];
    memset(psi, 0, sizeof(psi));
    for (int i = 0; i < 3; i++)
        for (int d = 0; d < 4; d++) psi[0][i][i][d] = ext[12 + d];
    for (int S = 1; S <= full; S++) {
        if (S == full) break;
        real q[4];
        for (int mu = 0; mu < 4; mu++) q[mu] = KS[S][mu] - p[3][mu];
        cx P[4][4];
        rslash(q, P);
        for (int i = 0; i < 4; i++) P[i][i] += m;
        real den = rdot(q, q) - m * m;
        cx acc[3][3][4];
        memset(acc, 0, sizeof(acc));
        for (int S1 = S; S1 > 0; S1 = (S1 - 1) & S) {
            int S2 = S ^ S1;
            for (int a = 0; a < 8; a++) {
                if (!nz[S1][a]) continue; /* exact zeros */
                cx Sl[4][4];
                slash(J[S1][a], Sl);
                for (int i = 0; i < 3; i++)
                    for (int kk = 0; kk < 3; kk++) {
                        cx tik = TGEN[a][i][kk];
                        if (tik == 0) continue;
                        for (int j = 0; j < 3; j++) {
                            cx t[4];
                            matvec(Sl, psi[S2][kk][j], t);
                            for (int d = 0; d < 4; d++) acc[i][j][d] += (I * g) * tik * t[d];
                        }
                    }
            }
        }
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                cx t[4];
                matvec(P, acc[i][j], t);
                for (int d = 0; d < 4; d++) psi[S][i][j][d] = I * t[d] / den;
            }
    }
    /* i M_ij = sum_{S1} ubar (i g gamma.J^a(S1) t^a) psi(full \ S1) */
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) Mout[3 * i + j] = 0;
    for (int S1 = full; S1 > 0; S1 = (S1 - 1) & full) {
        int S2 = full ^ S1;
        for (int a = 0; a < 8; a++) {
            if (!nz[S1][a]) continue; /* exact zeros */
            cx Sl[4][4];
            slash(J[S1][a], Sl);
            for (int i = 0; i < 3; i++)
                for (int kk = 0; kk < 3; kk++) {
                    cx tik = TGEN[a][i][kk];
                    if (tik == 0) continue;
                    for (int j = 0; j < 3; j++) {
                        cx t[4];
                        matvec(Sl, psi[S2][kk][j], t);
                        Mout[3 * i + j] += g * tik * rowcol(ext + 8, t);
                    }
                }
        }
    }
    return 0;
}

/*
 * e- e+ -> n photons (n = 1..5) for one event (AoS p[n+2][4]): the helicity
 * amplitude for hel[n+2] in `basis` (0: z-spin / linear, 1: helicity) into
 * *amp -- with the photon polarisations eps_in[n][4] (used as given, i.e.
 * already conjugated) instead when eps_in is not NULL -- and the
 * spin-averaged |M|^2 (1/4, 1/n!) as the return value.
 */
real oracle_ee_photons(int n, const real *par, const real *p_aos, int basis, const int *hel, cx *amp,
                         const cx *eps_in) {
    if (n < 1 || n > MAXA) return NAN;
    init_all();
    real p[MAXN][4];
    memcpy(p, p_aos, sizeof(real) * 4 * (n + 2));
    const or_params *pp = (const or_params *)par;
    if (amp && hel) *amp = amp_ee_photons(n, p, basis, hel, sqrt(4.0 * OR_PI / pp->alpha_em_inv), eps_in);
    return me_ee_photons(n, p, pp);
}

#endif /* ORACLE_EXTENDED */
