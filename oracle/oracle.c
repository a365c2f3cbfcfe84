/*
 * Plain FP64 CPU oracle of the interpolative butterfly factorization (IBF)
 * of Li & Yang, "Interpolative Butterfly Factorization" (arXiv 1605.03616).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code with the CUDA library.
 *
 * Everything is complex128, written for readability, not speed:
 *   - orc_direct_1d / orc_direct_2d : the defining sum u(x) = sum_xi K(x,xi) g(xi)
 *     (Sec. 1, eq. DFIO).
 *   - orc_ibf_apply_1d / orc_ibf_adjoint_1d : the butterfly algorithm in the
 *     matrix-free form of Algorithm 2.1 (Sec. 2.2, eqs. (1), (2), switch,
 *     (3), bf3) -- the same numbers as the preliminary IBF (Sec. 3).
 *   - orc_ibf_build_1d + orc_ibf_explicit_* : the preliminary IBF of Sec. 3
 *     with its factors V^0, H^l, M^h, G^l, U^L stored as explicit blocks
 *     (eqs. PIBF1, PIBF2, switchlocM, PIBF3, PIBFbf3) and applied block by block.
 *   - orc_ibf_apply_2d : the same butterfly in 2D on one square frequency
 *     box, with quadtrees and r x r tensor Chebyshev grids (Sec. 5.1);
 *     orc_mibf_apply_2d : the multiscale sum of Sec. 5.2 (eqs. domaindecomp,
 *     mba, f1) over a corona decomposition of Omega plus a direct centre.
 *
 * Conventions (readings of the paper where it is silent):
 *   - r is the number of Chebyshev points per dimension; grid on [-1/2,1/2]
 *     is z_t = cos(t*pi/(r-1))/2, t = 0..r-1 (Sec. 2.1).
 *   - X boxes are half-open dyadic intervals of [0,1); Omega boxes are
 *     half-open dyadic intervals of [-N/2, N/2); centres are midpoints, so the
 *     Omega root has centre 0.  A point on a box boundary belongs to the box
 *     on its right.
 *   - The initialization uses A = root of T_X (centre 1/2), as Algorithm 2.1
 *     states; h is the switch level, floor(L/2) unless the caller asks
 *     otherwise.
 *   - e(t) = exp(2*pi*i*t) is evaluated after removing the nearest integer
 *     from t (an exact operation), so that sin/cos see |arg| <= pi.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define ORC_PHASE_NUFFT 0      /* Phi = x.xi                                   */
#define ORC_PHASE_FIO1D 1      /* Phi = x xi + c(x)|xi|, c = (2+sin 2 pi x)/8  */
#define ORC_PHASE_FIO2D 2      /* Phi = x.xi + sqrt(c1^2 xi1^2 + c2^2 xi2^2), c /16 */
#define ORC_PHASE_FIO2D_32 3   /* the same with the constants /32 of Sec. 6.3      */
#define ORC_PHASE_FIO1D_SERIES 4 /* Phi = x xi + c(x)|xi|, c a trigonometric series */
#define ORC_PHASE_FIO2D_SERIES 5 /* Phi = x.xi + sqrt(c1^2 xi1^2 + c2^2 xi2^2), c1, c2 2D series */
#define ORC_PHASE_SEPARABLE 100 /* test phase f(x) + h(xi): remainder R^{AB}=0 */

/* ------------------------------------------------------------------ */
/* kernel pieces                                                       */
/* ------------------------------------------------------------------ */

/* exp(2 pi i t), argument reduced mod 1 first */
static cplx e2pi(double t)
{
    double th = t - nearbyint(t);
    double a = 2.0 * M_PI * th;
    return cos(a) + I * sin(a);
}

/* Coefficient series of ORC_PHASE_FIO1D_SERIES: c(x) = sum_{m<M} a_m cos(2 pi m x)
 * + b_m sin(2 pi m x) (the FIO class of Sec. 1, Assumption 1.1, in 1D with a
 * smooth periodic c; Sec. 6.2's phase is a_0 = 1/4, b_1 = 1/8).  Set by
 * orc_set_series before the phase is used; one series per process. */
static int orc_nco = 0;
static double orc_ca[16], orc_cb[16];

int orc_set_series(int M, const double* a, const double* b)
{
    if (M < 1 || M > 16) return 1;
    orc_nco = M;
    for (int m = 0; m < M; ++m) {
        orc_ca[m] = a[m];
        orc_cb[m] = b[m];
    }
    return 0;
}

/* Coefficient series of ORC_PHASE_FIO2D_SERIES: for d = 1, 2
 *   c_d(x) = sum_{t<M} al[d][t] cos(2 pi (p_t x1 + q_t x2)) + be[d][t] sin(2 pi (p_t x1 + q_t x2)),
 * the 2D FIO of Sec. 6.3's form x.xi + sqrt(c1^2 xi1^2 + c2^2 xi2^2) (the
 * generalized-Radon form Sec. 1 names) with smooth periodic coefficients.
 * Sec. 6.3's c1 = (2 + sin 2 pi x1 sin 2 pi x2)/16 is
 * 1/8 + cos(2 pi (x1 - x2))/32 - cos(2 pi (x1 + x2))/32.  Terms are rows
 * (p_t, q_t, al1_t, be1_t, al2_t, be2_t); one series per process. */
static int orc_nco2 = 0;
static double orc_pq[16][2], orc_al[2][16], orc_be[2][16];

int orc_set_series2(int M, const double* terms)
{
    if (M < 1 || M > 16) return 1;
    orc_nco2 = M;
    for (int t = 0; t < M; ++t) {
        const double* row = terms + 6 * t;
        orc_pq[t][0] = row[0];
        orc_pq[t][1] = row[1];
        orc_al[0][t] = row[2];
        orc_be[0][t] = row[3];
        orc_al[1][t] = row[4];
        orc_be[1][t] = row[5];
    }
    return 0;
}

static double orc_series2(int d, double x1, double x2)
{
    double c = 0.0;
    for (int t = 0; t < orc_nco2; ++t) {
        double arg = 2.0 * M_PI * (orc_pq[t][0] * x1 + orc_pq[t][1] * x2);
        c += orc_al[d][t] * cos(arg) + orc_be[d][t] * sin(arg);
    }
    return c;
}

/* 1D phase functions: eq. 1D-FT (with the sign of the K = e(+x xi) reading),
 * eq. 1D-FIO-kernal, the FIO with a series coefficient, and the separable
 * test phase. */
double orc_phi_1d(int phase_id, double x, double xi)
{
    switch (phase_id) {
    case ORC_PHASE_FIO1D_SERIES: {
        double c = 0.0;
        for (int m = 0; m < orc_nco; ++m) {
            double arg = 2.0 * M_PI * (double)m * x;
            c += orc_ca[m] * cos(arg) + orc_cb[m] * sin(arg);
        }
        return x * xi + c * fabs(xi);
    }
    case ORC_PHASE_NUFFT:
        return x * xi;
    case ORC_PHASE_FIO1D: {
        double c = (2.0 + sin(2.0 * M_PI * x)) / 8.0;
        return x * xi + c * fabs(xi);
    }
    case ORC_PHASE_SEPARABLE:
        return 0.75 * sin(2.0 * M_PI * x) + (0.125 * fabs(xi) + 0.3 * sin(0.1 * xi));
    default:
        return 0.0;
    }
}

/* 2D phase of Sec. 6.3: c1 = (2 + sin(2 pi x1) sin(2 pi x2))/den,
 * c2 = (2 + cos(2 pi x1) cos(2 pi x2))/den, den = 16 (the workload) or 32 (the
 * paper's Table 4); the separable test phase in 2D. */
double orc_phi_2d(int phase_id, double x1, double x2, double k1, double k2)
{
    switch (phase_id) {
    case ORC_PHASE_FIO2D:
    case ORC_PHASE_FIO2D_32: {
        double den = phase_id == ORC_PHASE_FIO2D ? 16.0 : 32.0;
        double c1 = (2.0 + sin(2.0 * M_PI * x1) * sin(2.0 * M_PI * x2)) / den;
        double c2 = (2.0 + cos(2.0 * M_PI * x1) * cos(2.0 * M_PI * x2)) / den;
        double a = c1 * k1;
        double b = c2 * k2;
        return (x1 * k1 + x2 * k2) + sqrt(a * a + b * b);
    }
    case ORC_PHASE_FIO2D_SERIES: {
        double a = orc_series2(0, x1, x2) * k1;
        double b = orc_series2(1, x1, x2) * k2;
        return (x1 * k1 + x2 * k2) + sqrt(a * a + b * b);
    }
    case ORC_PHASE_NUFFT:
        return x1 * k1 + x2 * k2;
    case ORC_PHASE_SEPARABLE:
        return 0.75 * sin(2.0 * M_PI * x1) * cos(2.0 * M_PI * x2) +
               (0.125 * sqrt(k1 * k1 + k2 * k2) + 0.3 * sin(0.1 * k1 - 0.07 * k2));
    default:
        return 0.0;
    }
}

/* Chebyshev grid of order r on [-1/2, 1/2] (Sec. 2.1) */
void orc_cheb_grid(int r, double* z)
{
    for (int t = 0; t < r; ++t)
        z[t] = 0.5 * cos(t * M_PI / (r - 1));
}

/* Lagrange polynomial M_t on the grid z, evaluated at u (Sec. 2.1, product form) */
double orc_lagrange(int r, const double* z, int t, double u)
{
    double p = 1.0;
    for (int m = 0; m < r; ++m)
        if (m != t)
            p *= (u - z[m]) / (z[t] - z[m]);
    return p;
}

/* ------------------------------------------------------------------ */
/* 1D dyadic boxes: X box (l,i) = [i 2^-l, (i+1) 2^-l);                 */
/* Omega box (l,j) = [-N/2 + j N 2^-l, -N/2 + (j+1) N 2^-l)             */
/* ------------------------------------------------------------------ */
static double xbox_c(int l, int64_t i) { return ((double)i + 0.5) / ldexp(1.0, l); }
static double xbox_w(int l) { return 1.0 / ldexp(1.0, l); }
static double wbox_w(int64_t N, int l) { return (double)N / ldexp(1.0, l); }
static double wbox_c(int64_t N, int l, int64_t j) { return -0.5 * (double)N + ((double)j + 0.5) * wbox_w(N, l); }

/* grid point t of a box of centre c and width w: c + w z_t */
static double gridpt(double c, double w, const double* z, int t) { return c + w * z[t]; }

/* leaf of T_X holding x (level L); leaf of T_Omega holding xi */
static int64_t xleaf(int L, double x)
{
    int64_t n = (int64_t)1 << L;
    int64_t i = (int64_t)floor(x * (double)n);
    if (i < 0) i = 0;
    if (i >= n) i = n - 1;
    return i;
}
static int64_t wleaf(int64_t N, int L, double xi)
{
    int64_t n = (int64_t)1 << L;
    int64_t j = (int64_t)floor((xi + 0.5 * (double)N) / wbox_w(N, L));
    if (j < 0) j = 0;
    if (j >= n) j = n - 1;
    return j;
}

static int ilog2(int64_t N)
{
    int L = 0;
    while (((int64_t)1 << L) < N) ++L;
    return L;
}

/* ------------------------------------------------------------------ */
/* Direct summation (eq. DFIO): u[n + nx c] = sum_k e(Phi(x_n, xi_k)) g[k + nxi c] */
/* ------------------------------------------------------------------ */
int orc_direct_1d(int phase_id, int64_t nx, const double* x, int64_t nxi, const double* xi,
                  const cplx* g, int nrhs, cplx* u)
{
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < nx; ++n) {
        for (int c = 0; c < nrhs; ++c) {
            cplx s = 0;
            for (int64_t k = 0; k < nxi; ++k)
                s += e2pi(orc_phi_1d(phase_id, x[n], xi[k])) * g[k + nxi * c];
            u[n + nx * c] = s;
        }
    }
    return 0;
}

int orc_direct_2d(int phase_id, int64_t nx, const double* x, int64_t nxi, const double* xi,
                  const cplx* g, int nrhs, cplx* u)
{
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < nx; ++n) {
        for (int c = 0; c < nrhs; ++c) {
            cplx s = 0;
            for (int64_t k = 0; k < nxi; ++k)
                s += e2pi(orc_phi_2d(phase_id, x[2 * n], x[2 * n + 1], xi[2 * k], xi[2 * k + 1])) *
                     g[k + nxi * c];
            u[n + nx * c] = s;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* 1D butterfly, matrix-free (Algorithm 2.1 = the preliminary IBF, Sec. 3) */
/* Lambda^l_{i,j} is stored at lam[(i * 2^(L-l) + j) * r + t].            */
/* Omega is the integer grid xi_k = k - N/2 (eq. Omega).                  */
/* ------------------------------------------------------------------ */

/* Initialization, eq. (1) / eq. PIBF1, with A = root of T_X */
static void mf_init(int ph, int64_t N, int L, int r, const double* z, const cplx* g, cplx* lam)
{
    double cA = xbox_c(0, 0);
    int64_t nb = (int64_t)1 << L;
    memset(lam, 0, sizeof(cplx) * nb * r);
    double wB = wbox_w(N, L);
    for (int64_t k = 0; k < N; ++k) {
        double xi = (double)k - 0.5 * (double)N;
        int64_t j = wleaf(N, L, xi);
        double cB = wbox_c(N, L, j);
        for (int t = 0; t < r; ++t) {
            double gBt = gridpt(cB, wB, z, t);
            lam[j * r + t] += e2pi(-orc_phi_1d(ph, cA, gBt)) *
                              orc_lagrange(r, z, t, (xi - cB) / wB) * e2pi(orc_phi_1d(ph, cA, xi)) * g[k];
        }
    }
}

/* Recursion in xi, eq. (2) / eq. PIBF2: level l from level l-1 */
static void mf_rec_xi(int ph, int64_t N, int L, int r, const double* z, int l, const cplx* prev, cplx* next)
{
    int64_t ni = (int64_t)1 << l, nj = (int64_t)1 << (L - l);
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t i = 0; i < ni; ++i) {
        for (int64_t j = 0; j < nj; ++j) {
            double cA = xbox_c(l, i);
            double cB = wbox_c(N, L - l, j), wB = wbox_w(N, L - l);
            double wC = wbox_w(N, L - l + 1);
            int64_t ip = i / 2;
            for (int t = 0; t < r; ++t) {
                double gBt = gridpt(cB, wB, z, t);
                cplx acc = 0;
                for (int c = 0; c < 2; ++c) {
                    int64_t C = 2 * j + c;
                    double cC = wbox_c(N, L - l + 1, C);
                    const cplx* lp = prev + (ip * ((int64_t)1 << (L - l + 1)) + C) * r;
                    for (int s = 0; s < r; ++s) {
                        double gCs = gridpt(cC, wC, z, s);
                        acc += orc_lagrange(r, z, t, (gCs - cB) / wB) * e2pi(orc_phi_1d(ph, cA, gCs)) * lp[s];
                    }
                }
                next[(i * nj + j) * r + t] = e2pi(-orc_phi_1d(ph, cA, gBt)) * acc;
            }
        }
    }
}

/* Switch, eq. switchlocM: at level h, in place */
static void mf_switch(int ph, int64_t N, int L, int r, const double* z, int h, cplx* lam)
{
    int64_t ni = (int64_t)1 << h, nj = (int64_t)1 << (L - h);
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t i = 0; i < ni; ++i) {
        for (int64_t j = 0; j < nj; ++j) {
            double cA = xbox_c(h, i), wA = xbox_w(h);
            double cB = wbox_c(N, L - h, j), wB = wbox_w(N, L - h);
            cplx old[64];
            cplx* v = lam + (i * nj + j) * r;
            for (int s = 0; s < r; ++s) old[s] = v[s];
            for (int t = 0; t < r; ++t) {
                cplx acc = 0;
                for (int s = 0; s < r; ++s)
                    acc += e2pi(orc_phi_1d(ph, gridpt(cA, wA, z, t), gridpt(cB, wB, z, s))) * old[s];
                v[t] = acc;
            }
        }
    }
}

/* Recursion in x, eq. (3) / eq. PIBF3: level l from level l-1 */
static void mf_rec_x(int ph, int64_t N, int L, int r, const double* z, int l, const cplx* prev, cplx* next)
{
    int64_t ni = (int64_t)1 << l, nj = (int64_t)1 << (L - l);
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t i = 0; i < ni; ++i) {
        for (int64_t j = 0; j < nj; ++j) {
            double cA = xbox_c(l, i), wA = xbox_w(l);
            int64_t ip = i / 2;
            double cP = xbox_c(l - 1, ip), wP = xbox_w(l - 1);
            for (int t = 0; t < r; ++t) {
                double gAt = gridpt(cA, wA, z, t);
                cplx acc = 0;
                for (int c = 0; c < 2; ++c) {
                    int64_t C = 2 * j + c;
                    double cC = wbox_c(N, L - l + 1, C);
                    const cplx* lp = prev + (ip * ((int64_t)1 << (L - l + 1)) + C) * r;
                    cplx inner = 0;
                    for (int s = 0; s < r; ++s) {
                        double gPs = gridpt(cP, wP, z, s);
                        inner += orc_lagrange(r, z, s, (gAt - cP) / wP) * e2pi(-orc_phi_1d(ph, gPs, cC)) * lp[s];
                    }
                    acc += e2pi(orc_phi_1d(ph, gAt, cC)) * inner;
                }
                next[(i * nj + j) * r + t] = acc;
            }
        }
    }
}

/* Termination, eq. bf3 / eq. PIBFbf3, B = root of T_Omega (centre 0) */
static void mf_term(int ph, int64_t N, int L, int r, const double* z, int64_t nx, const double* x,
                    const cplx* lam, cplx* u)
{
    double cB = wbox_c(N, 0, 0);
    double wA = xbox_w(L);
    for (int64_t n = 0; n < nx; ++n) {
        int64_t i = xleaf(L, x[n]);
        double cA = xbox_c(L, i);
        cplx acc = 0;
        for (int t = 0; t < r; ++t)
            acc += orc_lagrange(r, z, t, (x[n] - cA) / wA) * e2pi(-orc_phi_1d(ph, gridpt(cA, wA, z, t), cB)) *
                   lam[i * r + t];
        u[n] = e2pi(orc_phi_1d(ph, x[n], cB)) * acc;
    }
}

int orc_ibf_apply_1d(int phase_id, int64_t N, int r, int h, int64_t nx, const double* x, const cplx* g,
                     int nrhs, cplx* u)
{
    int L = ilog2(N);
    if (((int64_t)1 << L) != N || r < 2 || r > 64 || h < 0 || h > L) return 1;
    double z[64];
    orc_cheb_grid(r, z);
    cplx* a = (cplx*)malloc(sizeof(cplx) * N * r);
    cplx* b = (cplx*)malloc(sizeof(cplx) * N * r);
    if (!a || !b) { free(a); free(b); return 2; }
    for (int col = 0; col < nrhs; ++col) {
        mf_init(phase_id, N, L, r, z, g + N * col, a);
        for (int l = 1; l <= h; ++l) {
            mf_rec_xi(phase_id, N, L, r, z, l, a, b);
            cplx* tmp = a; a = b; b = tmp;
        }
        mf_switch(phase_id, N, L, r, z, h, a);
        for (int l = h + 1; l <= L; ++l) {
            mf_rec_x(phase_id, N, L, r, z, l, a, b);
            cplx* tmp = a; a = b; b = tmp;
        }
        mf_term(phase_id, N, L, r, z, nx, x, a, u + nx * col);
    }
    free(a);
    free(b);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Adjoint, matrix-free: the conjugate transpose of each step above,    */
/* taken in reverse order (K^* = V^0 H^1 ... (M^h)^* ... (U^L)^*).       */
/* ------------------------------------------------------------------ */
static void mfa_term(int ph, int64_t N, int L, int r, const double* z, int64_t nx, const double* x,
                     const cplx* y, cplx* lam)
{
    double cB = wbox_c(N, 0, 0);
    double wA = xbox_w(L);
    memset(lam, 0, sizeof(cplx) * ((int64_t)1 << L) * r);
    for (int64_t n = 0; n < nx; ++n) {
        int64_t i = xleaf(L, x[n]);
        double cA = xbox_c(L, i);
        for (int t = 0; t < r; ++t) {
            cplx w = e2pi(orc_phi_1d(ph, x[n], cB)) * orc_lagrange(r, z, t, (x[n] - cA) / wA) *
                     e2pi(-orc_phi_1d(ph, gridpt(cA, wA, z, t), cB));
            lam[i * r + t] += conj(w) * y[n];
        }
    }
}

/* adjoint of eq. (3): level l (next) back to level l-1 (prev) */
static void mfa_rec_x(int ph, int64_t N, int L, int r, const double* z, int l, const cplx* next, cplx* prev)
{
    int64_t npi = (int64_t)1 << (l - 1), nC = (int64_t)1 << (L - l + 1), nj = (int64_t)1 << (L - l);
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t ip = 0; ip < npi; ++ip) {
        for (int64_t C = 0; C < nC; ++C) {
            double cP = xbox_c(l - 1, ip), wP = xbox_w(l - 1);
            double cC = wbox_c(N, L - l + 1, C);
            int64_t j = C / 2;
            for (int s = 0; s < r; ++s) {
                double gPs = gridpt(cP, wP, z, s);
                cplx acc = 0;
                for (int a = 0; a < 2; ++a) {
                    int64_t i = 2 * ip + a;
                    double cA = xbox_c(l, i), wA = xbox_w(l);
                    const cplx* ln = next + (i * nj + j) * r;
                    for (int t = 0; t < r; ++t) {
                        double gAt = gridpt(cA, wA, z, t);
                        cplx w = e2pi(orc_phi_1d(ph, gAt, cC)) * orc_lagrange(r, z, s, (gAt - cP) / wP) *
                                 e2pi(-orc_phi_1d(ph, gPs, cC));
                        acc += conj(w) * ln[t];
                    }
                }
                prev[(ip * nC + C) * r + s] = acc;
            }
        }
    }
}

static void mfa_switch(int ph, int64_t N, int L, int r, const double* z, int h, cplx* lam)
{
    int64_t ni = (int64_t)1 << h, nj = (int64_t)1 << (L - h);
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t i = 0; i < ni; ++i) {
        for (int64_t j = 0; j < nj; ++j) {
            double cA = xbox_c(h, i), wA = xbox_w(h);
            double cB = wbox_c(N, L - h, j), wB = wbox_w(N, L - h);
            cplx old[64];
            cplx* v = lam + (i * nj + j) * r;
            for (int t = 0; t < r; ++t) old[t] = v[t];
            for (int s = 0; s < r; ++s) {
                cplx acc = 0;
                for (int t = 0; t < r; ++t)
                    acc += conj(e2pi(orc_phi_1d(ph, gridpt(cA, wA, z, t), gridpt(cB, wB, z, s)))) * old[t];
                v[s] = acc;
            }
        }
    }
}

/* adjoint of eq. (2): level l (next) back to level l-1 (prev) */
static void mfa_rec_xi(int ph, int64_t N, int L, int r, const double* z, int l, const cplx* next, cplx* prev)
{
    int64_t npi = (int64_t)1 << (l - 1), nC = (int64_t)1 << (L - l + 1), nj = (int64_t)1 << (L - l);
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t ip = 0; ip < npi; ++ip) {
        for (int64_t C = 0; C < nC; ++C) {
            int64_t j = C / 2;
            double cB = wbox_c(N, L - l, j), wB = wbox_w(N, L - l);
            double cC = wbox_c(N, L - l + 1, C), wC = wbox_w(N, L - l + 1);
            for (int s = 0; s < r; ++s) {
                double gCs = gridpt(cC, wC, z, s);
                cplx acc = 0;
                for (int a = 0; a < 2; ++a) {
                    int64_t i = 2 * ip + a;
                    double cA = xbox_c(l, i);
                    const cplx* ln = next + (i * nj + j) * r;
                    for (int t = 0; t < r; ++t) {
                        double gBt = gridpt(cB, wB, z, t);
                        cplx w = e2pi(-orc_phi_1d(ph, cA, gBt)) * orc_lagrange(r, z, t, (gCs - cB) / wB) *
                                 e2pi(orc_phi_1d(ph, cA, gCs));
                        acc += conj(w) * ln[t];
                    }
                }
                prev[(ip * nC + C) * r + s] = acc;
            }
        }
    }
}

static void mfa_init(int ph, int64_t N, int L, int r, const double* z, const cplx* lam, cplx* g)
{
    double cA = xbox_c(0, 0);
    double wB = wbox_w(N, L);
    for (int64_t k = 0; k < N; ++k) {
        double xi = (double)k - 0.5 * (double)N;
        int64_t j = wleaf(N, L, xi);
        double cB = wbox_c(N, L, j);
        cplx acc = 0;
        for (int t = 0; t < r; ++t) {
            double gBt = gridpt(cB, wB, z, t);
            cplx w = e2pi(-orc_phi_1d(ph, cA, gBt)) * orc_lagrange(r, z, t, (xi - cB) / wB) *
                     e2pi(orc_phi_1d(ph, cA, xi));
            acc += conj(w) * lam[j * r + t];
        }
        g[k] = acc;
    }
}

int orc_ibf_adjoint_1d(int phase_id, int64_t N, int r, int h, int64_t nx, const double* x, const cplx* y,
                       int nrhs, cplx* g)
{
    int L = ilog2(N);
    if (((int64_t)1 << L) != N || r < 2 || r > 64 || h < 0 || h > L) return 1;
    double z[64];
    orc_cheb_grid(r, z);
    cplx* a = (cplx*)malloc(sizeof(cplx) * N * r);
    cplx* b = (cplx*)malloc(sizeof(cplx) * N * r);
    if (!a || !b) { free(a); free(b); return 2; }
    for (int col = 0; col < nrhs; ++col) {
        mfa_term(phase_id, N, L, r, z, nx, x, y + nx * col, a);
        for (int l = L; l >= h + 1; --l) {
            mfa_rec_x(phase_id, N, L, r, z, l, a, b);
            cplx* tmp = a; a = b; b = tmp;
        }
        mfa_switch(phase_id, N, L, r, z, h, a);
        for (int l = h; l >= 1; --l) {
            mfa_rec_xi(phase_id, N, L, r, z, l, a, b);
            cplx* tmp = a; a = b; b = tmp;
        }
        mfa_init(phase_id, N, L, r, z, a, g + N * col);
    }
    free(a);
    free(b);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Preliminary IBF with explicit factors (Sec. 3).                      */
/* Blocks are indexed by the output pair p = i * 2^(L-l) + j of level l: */
/*   H[l][p][c][t][s] maps Lambda^{l-1}_{i/2, 2j+c}[s] -> Lambda^l_{i,j}[t]  */
/*   (l = 1..h, eq. PIBF2),  G[l][p][c][t][s] the same for l = h+1..L      */
/*   (eq. PIBF3), Msw[p][t][s] the switch blocks (eq. switchlocM),         */
/*   V[k][t] the column of (V^0)^* for xi_k (eq. PIBF1), U[n][t] the row of  */
/*   U^L for x_n (eq. PIBFbf3).                                            */
/* ------------------------------------------------------------------ */
typedef struct orc_ibf {
    int phase_id, L, h, r;
    int64_t N, nx;
    double* x;
    cplx* V;      /* N * r               */
    cplx** blk;   /* blk[l], l = 1..L: N * 2 * r * r */
    cplx* Msw;    /* N * r * r           */
    cplx* U;      /* nx * r              */
} orc_ibf;

void orc_ibf_free(orc_ibf* f)
{
    if (!f) return;
    free(f->x);
    free(f->V);
    if (f->blk)
        for (int l = 1; l <= f->L; ++l) free(f->blk[l]);
    free(f->blk);
    free(f->Msw);
    free(f->U);
    free(f);
}

orc_ibf* orc_ibf_build_1d(int phase_id, int64_t N, int r, int h, int64_t nx, const double* x)
{
    int L = ilog2(N);
    if (((int64_t)1 << L) != N || r < 2 || r > 64 || h < 0 || h > L) return NULL;
    orc_ibf* f = (orc_ibf*)calloc(1, sizeof(orc_ibf));
    f->phase_id = phase_id; f->L = L; f->h = h; f->r = r; f->N = N; f->nx = nx;
    f->x = (double*)malloc(sizeof(double) * nx);
    memcpy(f->x, x, sizeof(double) * nx);
    double z[64];
    orc_cheb_grid(r, z);
    int ph = phase_id;

    /* V^0 (eq. PIBF1) */
    f->V = (cplx*)malloc(sizeof(cplx) * N * r);
    {
        double cA = xbox_c(0, 0), wB = wbox_w(N, L);
        for (int64_t k = 0; k < N; ++k) {
            double xi = (double)k - 0.5 * (double)N;
            double cB = wbox_c(N, L, wleaf(N, L, xi));
            for (int t = 0; t < r; ++t)
                f->V[k * r + t] = e2pi(-orc_phi_1d(ph, cA, gridpt(cB, wB, z, t))) *
                                  orc_lagrange(r, z, t, (xi - cB) / wB) * e2pi(orc_phi_1d(ph, cA, xi));
        }
    }
    f->blk = (cplx**)calloc(L + 1, sizeof(cplx*));
    for (int l = 1; l <= L; ++l) {
        cplx* B = (cplx*)malloc(sizeof(cplx) * N * 2 * r * r);
        f->blk[l] = B;
        int64_t ni = (int64_t)1 << l, nj = (int64_t)1 << (L - l);
        for (int64_t i = 0; i < ni; ++i)
            for (int64_t j = 0; j < nj; ++j)
                for (int c = 0; c < 2; ++c)
                    for (int t = 0; t < r; ++t)
                        for (int s = 0; s < r; ++s) {
                            cplx v;
                            double cC = wbox_c(N, L - l + 1, 2 * j + c), wC = wbox_w(N, L - l + 1);
                            if (l <= h) { /* eq. PIBF2 */
                                double cA = xbox_c(l, i);
                                double cB = wbox_c(N, L - l, j), wB = wbox_w(N, L - l);
                                double gCs = gridpt(cC, wC, z, s);
                                v = e2pi(-orc_phi_1d(ph, cA, gridpt(cB, wB, z, t))) *
                                    orc_lagrange(r, z, t, (gCs - cB) / wB) * e2pi(orc_phi_1d(ph, cA, gCs));
                            } else { /* eq. PIBF3 */
                                double cA = xbox_c(l, i), wA = xbox_w(l);
                                double cP = xbox_c(l - 1, i / 2), wP = xbox_w(l - 1);
                                double gAt = gridpt(cA, wA, z, t);
                                v = e2pi(orc_phi_1d(ph, gAt, cC)) * orc_lagrange(r, z, s, (gAt - cP) / wP) *
                                    e2pi(-orc_phi_1d(ph, gridpt(cP, wP, z, s), cC));
                            }
                            B[((((i * nj + j) * 2 + c) * r) + t) * r + s] = v;
                        }
    }
    /* M^h (eq. switchlocM) */
    f->Msw = (cplx*)malloc(sizeof(cplx) * N * r * r);
    {
        int64_t ni = (int64_t)1 << h, nj = (int64_t)1 << (L - h);
        for (int64_t i = 0; i < ni; ++i)
            for (int64_t j = 0; j < nj; ++j) {
                double cA = xbox_c(h, i), wA = xbox_w(h);
                double cB = wbox_c(N, L - h, j), wB = wbox_w(N, L - h);
                for (int t = 0; t < r; ++t)
                    for (int s = 0; s < r; ++s)
                        f->Msw[((i * nj + j) * r + t) * r + s] =
                            e2pi(orc_phi_1d(ph, gridpt(cA, wA, z, t), gridpt(cB, wB, z, s)));
            }
    }
    /* U^L (eq. PIBFbf3) */
    f->U = (cplx*)malloc(sizeof(cplx) * nx * r);
    {
        double cB = wbox_c(N, 0, 0), wA = xbox_w(L);
        for (int64_t n = 0; n < nx; ++n) {
            double cA = xbox_c(L, xleaf(L, x[n]));
            for (int t = 0; t < r; ++t)
                f->U[n * r + t] = e2pi(orc_phi_1d(ph, x[n], cB)) * orc_lagrange(r, z, t, (x[n] - cA) / wA) *
                                  e2pi(-orc_phi_1d(ph, gridpt(cA, wA, z, t), cB));
        }
    }
    return f;
}

/* the switch at level h with the stored blocks: out_p = M~_p in_p for every pair p */
static void orc_switch_explicit(const orc_ibf* f, const cplx* in, cplx* out)
{
    int r = f->r;
    for (int64_t p = 0; p < f->N; ++p)
        for (int t = 0; t < r; ++t) {
            cplx acc = 0;
            for (int s = 0; s < r; ++s) acc += f->Msw[(p * r + t) * r + s] * in[p * r + s];
            out[p * r + t] = acc;
        }
}

int orc_ibf_explicit_apply(const orc_ibf* f, const cplx* g, int nrhs, cplx* u)
{
    int64_t N = f->N;
    int L = f->L, h = f->h, r = f->r;
    cplx* a = (cplx*)malloc(sizeof(cplx) * N * r);
    cplx* b = (cplx*)malloc(sizeof(cplx) * N * r);
    for (int col = 0; col < nrhs; ++col) {
        const cplx* gc = g + N * col;
        /* Lambda^0 = (V^0)^* g */
        memset(a, 0, sizeof(cplx) * N * r);
        for (int64_t k = 0; k < N; ++k) {
            int64_t j = wleaf(N, L, (double)k - 0.5 * (double)N);
            for (int t = 0; t < r; ++t) a[j * r + t] += f->V[k * r + t] * gc[k];
        }
        if (h == 0) {
            orc_switch_explicit(f, a, b);
            cplx* tmp = a; a = b; b = tmp;
        }
        for (int l = 1; l <= L; ++l) {
            int64_t ni = (int64_t)1 << l, nj = (int64_t)1 << (L - l);
            const cplx* B = f->blk[l];
            for (int64_t i = 0; i < ni; ++i)
                for (int64_t j = 0; j < nj; ++j)
                    for (int t = 0; t < r; ++t) {
                        cplx acc = 0;
                        for (int c = 0; c < 2; ++c) {
                            const cplx* in = a + ((i / 2) * (2 * nj) + 2 * j + c) * r;
                            const cplx* row = B + ((((i * nj + j) * 2 + c) * r) + t) * r;
                            for (int s = 0; s < r; ++s) acc += row[s] * in[s];
                        }
                        b[(i * nj + j) * r + t] = acc;
                    }
            cplx* tmp = a; a = b; b = tmp;
            if (l == h) {
                /* the switch at level h: Lambda~ = M~ Lambda for every pair */
                orc_switch_explicit(f, a, b);
                tmp = a; a = b; b = tmp;
            }
        }
        for (int64_t n = 0; n < f->nx; ++n) {
            int64_t i = xleaf(L, f->x[n]);
            cplx acc = 0;
            for (int t = 0; t < r; ++t) acc += f->U[n * r + t] * a[i * r + t];
            u[n + f->nx * col] = acc;
        }
    }
    free(a);
    free(b);
    return 0;
}

int orc_ibf_explicit_adjoint(const orc_ibf* f, const cplx* y, int nrhs, cplx* g)
{
    int64_t N = f->N;
    int L = f->L, h = f->h, r = f->r;
    cplx* a = (cplx*)malloc(sizeof(cplx) * N * r);
    cplx* b = (cplx*)malloc(sizeof(cplx) * N * r);
    for (int col = 0; col < nrhs; ++col) {
        const cplx* yc = y + f->nx * col;
        memset(a, 0, sizeof(cplx) * N * r);
        for (int64_t n = 0; n < f->nx; ++n) {
            int64_t i = xleaf(L, f->x[n]);
            for (int t = 0; t < r; ++t) a[i * r + t] += conj(f->U[n * r + t]) * yc[n];
        }
        for (int l = L; l >= 1; --l) {
            if (l == h) {
                for (int64_t p = 0; p < N; ++p)
                    for (int s = 0; s < r; ++s) {
                        cplx acc = 0;
                        for (int t = 0; t < r; ++t) acc += conj(f->Msw[(p * r + t) * r + s]) * a[p * r + t];
                        b[p * r + s] = acc;
                    }
                cplx* tmp = a; a = b; b = tmp;
            }
            int64_t nj = (int64_t)1 << (L - l), npi = (int64_t)1 << (l - 1), nC = 2 * nj;
            const cplx* B = f->blk[l];
            memset(b, 0, sizeof(cplx) * N * r);
            for (int64_t ip = 0; ip < npi; ++ip)
                for (int64_t C = 0; C < nC; ++C)
                    for (int s = 0; s < r; ++s) {
                        cplx acc = 0;
                        int64_t j = C / 2;
                        int c = (int)(C % 2);
                        for (int aa = 0; aa < 2; ++aa) {
                            int64_t i = 2 * ip + aa;
                            const cplx* on = a + (i * nj + j) * r;
                            for (int t = 0; t < r; ++t)
                                acc += conj(B[((((i * nj + j) * 2 + c) * r) + t) * r + s]) * on[t];
                        }
                        b[(ip * nC + C) * r + s] = acc;
                    }
            cplx* tmp = a; a = b; b = tmp;
        }
        if (h == 0) {
            for (int64_t p = 0; p < N; ++p)
                for (int s = 0; s < r; ++s) {
                    cplx acc = 0;
                    for (int t = 0; t < r; ++t) acc += conj(f->Msw[(p * r + t) * r + s]) * a[p * r + t];
                    b[p * r + s] = acc;
                }
            cplx* tmp = a; a = b; b = tmp;
        }
        for (int64_t k = 0; k < N; ++k) {
            int64_t j = wleaf(N, L, (double)k - 0.5 * (double)N);
            cplx acc = 0;
            for (int t = 0; t < r; ++t) acc += conj(f->V[k * r + t]) * a[j * r + t];
            g[k + N * col] = acc;
        }
    }
    free(a);
    free(b);
    return 0;
}

/* block accessors for the dense-assembly tests (copies out, complex128) */
int orc_ibf_get_V(const orc_ibf* f, cplx* out) { memcpy(out, f->V, sizeof(cplx) * f->N * f->r); return 0; }
int orc_ibf_get_U(const orc_ibf* f, cplx* out) { memcpy(out, f->U, sizeof(cplx) * f->nx * f->r); return 0; }
int orc_ibf_get_M(const orc_ibf* f, cplx* out) { memcpy(out, f->Msw, sizeof(cplx) * f->N * f->r * f->r); return 0; }
int orc_ibf_get_blk(const orc_ibf* f, int l, cplx* out)
{
    if (l < 1 || l > f->L) return 1;
    memcpy(out, f->blk[l], sizeof(cplx) * f->N * 2 * f->r * f->r);
    return 0;
}

/* ------------------------------------------------------------------ */
/* 2D butterfly on one square Omega box (Sec. 5.1): quadtrees, tensor   */
/* Chebyshev grids of r x r points, four children per box.              */
/* Q = [q1, q1+m) x [q2, q2+m) holds the integer frequencies            */
/* xi = (q1 + k1, q2 + k2), k1, k2 < m, g stored row-major in (k1, k2);  */
/* L = log2 m.  X boxes at level l: [i1, i1+1) x [i2, i2+1) / 2^l, index */
/* i = i1 2^l + i2; Omega boxes at level l: side m / 2^l, index          */
/* j = j1 2^l + j2.  Lambda^l_{i,j}[t1 r + t2] at (i 4^(L-l) + j) r^2.    */
/* ------------------------------------------------------------------ */
typedef struct {
    int ph, r, L;
    double q1, q2, m;
    const double* z;
} bf2;

static double lag2(const bf2* B, int t, double u1, double u2)
{
    return orc_lagrange(B->r, B->z, t / B->r, u1) * orc_lagrange(B->r, B->z, t % B->r, u2);
}
static void xbox2(int l, int64_t i, double* c1, double* c2, double* w)
{
    int64_t n = (int64_t)1 << l;
    *w = 1.0 / ldexp(1.0, l);
    *c1 = ((double)(i / n) + 0.5) * *w;
    *c2 = ((double)(i % n) + 0.5) * *w;
}
static void wbox2(const bf2* B, int l, int64_t j, double* c1, double* c2, double* w)
{
    int64_t n = (int64_t)1 << l;
    *w = B->m / ldexp(1.0, l);
    *c1 = B->q1 + ((double)(j / n) + 0.5) * *w;
    *c2 = B->q2 + ((double)(j % n) + 0.5) * *w;
}
static double phi2(const bf2* B, double x1, double x2, double k1, double k2)
{
    return orc_phi_2d(B->ph, x1, x2, k1, k2);
}
/* child c (0..3) of box (l, i) in a 2^l x 2^l grid: (2 i1 + c/2, 2 i2 + c%2) */
static int64_t child2(int l, int64_t i, int c)
{
    int64_t n = (int64_t)1 << l;
    return (2 * (i / n) + c / 2) * (2 * n) + 2 * (i % n) + c % 2;
}
static int64_t parent2(int l, int64_t i)   /* parent at level l-1 of box (l, i) */
{
    int64_t n = (int64_t)1 << l;
    return ((i / n) / 2) * (n / 2) + (i % n) / 2;
}

int orc_ibf_apply_2d(int phase_id, int64_t m, int r, int h, int64_t nx, const double* x, double q1, double q2,
                     const cplx* g, int nrhs, cplx* u)
{
    int L = ilog2(m);
    if (((int64_t)1 << L) != m || r < 2 || r > 16 || h < 0 || h > L) return 1;
    double z[64];
    orc_cheb_grid(r, z);
    bf2 B = {phase_id, r, L, q1, q2, (double)m, z};
    const int r2 = r * r;
    const int64_t npair = (int64_t)1 << (2 * L);
    cplx* a = (cplx*)malloc(sizeof(cplx) * npair * r2);
    cplx* b = (cplx*)malloc(sizeof(cplx) * npair * r2);
    if (!a || !b) { free(a); free(b); return 2; }
    for (int col = 0; col < nrhs; ++col) {
        const cplx* gc = g + m * m * col;
        /* initialization, eq. (1): A = root of T_X */
        {
            double cA1, cA2, wA;
            xbox2(0, 0, &cA1, &cA2, &wA);
            for (int64_t j = 0; j < npair; ++j) {
                double cB1, cB2, wB;
                wbox2(&B, L, j, &cB1, &cB2, &wB);
                int64_t j1 = j >> L, j2 = j & (((int64_t)1 << L) - 1);
                double k1 = q1 + (double)j1, k2 = q2 + (double)j2;     /* the one frequency of leaf j */
                cplx gv = gc[j1 * m + j2];
                for (int t = 0; t < r2; ++t) {
                    double gB1 = cB1 + wB * z[t / r], gB2 = cB2 + wB * z[t % r];
                    a[j * r2 + t] = e2pi(-phi2(&B, cA1, cA2, gB1, gB2)) *
                                    lag2(&B, t, (k1 - cB1) / wB, (k2 - cB2) / wB) *
                                    e2pi(phi2(&B, cA1, cA2, k1, k2)) * gv;
                }
            }
        }
        /* recursion in xi, eq. (2) */
        for (int l = 1; l <= h; ++l) {
            int64_t ni = (int64_t)1 << (2 * l), nj = (int64_t)1 << (2 * (L - l)), nC = nj * 4;
#pragma omp parallel for collapse(2) schedule(static)
            for (int64_t i = 0; i < ni; ++i)
                for (int64_t j = 0; j < nj; ++j) {
                    double cA1, cA2, wA, cB1, cB2, wB;
                    xbox2(l, i, &cA1, &cA2, &wA);
                    wbox2(&B, L - l, j, &cB1, &cB2, &wB);
                    int64_t ip = parent2(l, i);
                    for (int t = 0; t < r2; ++t) {
                        double gB1 = cB1 + wB * z[t / r], gB2 = cB2 + wB * z[t % r];
                        cplx acc = 0;
                        for (int c = 0; c < 4; ++c) {
                            int64_t C = child2(L - l, j, c);
                            double cC1, cC2, wC;
                            wbox2(&B, L - l + 1, C, &cC1, &cC2, &wC);
                            const cplx* lp = a + (ip * nC + C) * r2;
                            for (int s = 0; s < r2; ++s) {
                                double gC1 = cC1 + wC * z[s / r], gC2 = cC2 + wC * z[s % r];
                                acc += lag2(&B, t, (gC1 - cB1) / wB, (gC2 - cB2) / wB) *
                                       e2pi(phi2(&B, cA1, cA2, gC1, gC2)) * lp[s];
                            }
                        }
                        b[(i * nj + j) * r2 + t] = e2pi(-phi2(&B, cA1, cA2, gB1, gB2)) * acc;
                    }
                }
            cplx* tmp = a; a = b; b = tmp;
        }
        /* switch, eq. switchlocM */
        {
            int64_t ni = (int64_t)1 << (2 * h), nj = (int64_t)1 << (2 * (L - h));
#pragma omp parallel for collapse(2) schedule(static)
            for (int64_t i = 0; i < ni; ++i)
                for (int64_t j = 0; j < nj; ++j) {
                    double cA1, cA2, wA, cB1, cB2, wB;
                    xbox2(h, i, &cA1, &cA2, &wA);
                    wbox2(&B, L - h, j, &cB1, &cB2, &wB);
                    for (int t = 0; t < r2; ++t) {
                        double gA1 = cA1 + wA * z[t / r], gA2 = cA2 + wA * z[t % r];
                        cplx acc = 0;
                        for (int s = 0; s < r2; ++s)
                            acc += e2pi(phi2(&B, gA1, gA2, cB1 + wB * z[s / r], cB2 + wB * z[s % r])) *
                                   a[(i * nj + j) * r2 + s];
                        b[(i * nj + j) * r2 + t] = acc;
                    }
                }
            cplx* tmp = a; a = b; b = tmp;
        }
        /* recursion in x, eq. (3) */
        for (int l = h + 1; l <= L; ++l) {
            int64_t ni = (int64_t)1 << (2 * l), nj = (int64_t)1 << (2 * (L - l)), nC = nj * 4;
#pragma omp parallel for collapse(2) schedule(static)
            for (int64_t i = 0; i < ni; ++i)
                for (int64_t j = 0; j < nj; ++j) {
                    double cA1, cA2, wA, cP1, cP2, wP;
                    xbox2(l, i, &cA1, &cA2, &wA);
                    int64_t ip = parent2(l, i);
                    xbox2(l - 1, ip, &cP1, &cP2, &wP);
                    for (int t = 0; t < r2; ++t) {
                        double gA1 = cA1 + wA * z[t / r], gA2 = cA2 + wA * z[t % r];
                        cplx acc = 0;
                        for (int c = 0; c < 4; ++c) {
                            int64_t C = child2(L - l, j, c);
                            double cC1, cC2, wC;
                            wbox2(&B, L - l + 1, C, &cC1, &cC2, &wC);
                            const cplx* lp = a + (ip * nC + C) * r2;
                            cplx inner = 0;
                            for (int s = 0; s < r2; ++s) {
                                double gP1 = cP1 + wP * z[s / r], gP2 = cP2 + wP * z[s % r];
                                inner += lag2(&B, s, (gA1 - cP1) / wP, (gA2 - cP2) / wP) *
                                         e2pi(-phi2(&B, gP1, gP2, cC1, cC2)) * lp[s];
                            }
                            acc += e2pi(phi2(&B, gA1, gA2, cC1, cC2)) * inner;
                        }
                        b[(i * nj + j) * r2 + t] = acc;
                    }
                }
            cplx* tmp = a; a = b; b = tmp;
        }
        /* termination, eq. bf3: B = Q itself */
        {
            double cQ1 = q1 + 0.5 * (double)m, cQ2 = q2 + 0.5 * (double)m;
            int64_t nl = (int64_t)1 << L;
#pragma omp parallel for schedule(static)
            for (int64_t n = 0; n < nx; ++n) {
                double x1 = x[2 * n], x2 = x[2 * n + 1];
                int64_t i1 = (int64_t)floor(x1 * (double)nl), i2 = (int64_t)floor(x2 * (double)nl);
                if (i1 >= nl) i1 = nl - 1;
                if (i2 >= nl) i2 = nl - 1;
                if (i1 < 0) i1 = 0;
                if (i2 < 0) i2 = 0;
                int64_t i = i1 * nl + i2;
                double cA1, cA2, wA;
                xbox2(L, i, &cA1, &cA2, &wA);
                cplx acc = 0;
                for (int t = 0; t < r2; ++t) {
                    double gA1 = cA1 + wA * z[t / r], gA2 = cA2 + wA * z[t % r];
                    acc += lag2(&B, t, (x1 - cA1) / wA, (x2 - cA2) / wA) *
                           e2pi(-phi2(&B, gA1, gA2, cQ1, cQ2)) * a[i * r2 + t];
                }
                u[n + nx * col] = e2pi(phi2(&B, x1, x2, cQ1, cQ2)) * acc;
            }
        }
    }
    free(a);
    free(b);
    return 0;
}

/* Adjoint of orc_ibf_apply_2d: g = K_Q^* y, the conjugate transpose of each
   step of the 2D butterfly in reverse order (termination, recursion in x,
   switch, recursion in xi, initialization).  Each level's adjoint gathers,
   for input pair (ip, C) of level l-1, from the four output pairs
   (child a of ip, parent of C) of level l that read it. */
int orc_ibf_adjoint_2d(int phase_id, int64_t m, int r, int h, int64_t nx, const double* x, double q1, double q2,
                       const cplx* y, int nrhs, cplx* g)
{
    int L = ilog2(m);
    if (((int64_t)1 << L) != m || r < 2 || r > 16 || h < 0 || h > L) return 1;
    double z[64];
    orc_cheb_grid(r, z);
    bf2 B = {phase_id, r, L, q1, q2, (double)m, z};
    const int r2 = r * r;
    const int64_t npair = (int64_t)1 << (2 * L);
    cplx* a = (cplx*)malloc(sizeof(cplx) * npair * r2);
    cplx* b = (cplx*)malloc(sizeof(cplx) * npair * r2);
    if (!a || !b) { free(a); free(b); return 2; }
    for (int col = 0; col < nrhs; ++col) {
        const cplx* yc = y + nx * col;
        /* termination^*: a[i][t] = sum over points n of leaf i */
        {
            double cQ1 = q1 + 0.5 * (double)m, cQ2 = q2 + 0.5 * (double)m;
            int64_t nl = (int64_t)1 << L;
            memset(a, 0, sizeof(cplx) * npair * r2);
            for (int64_t n = 0; n < nx; ++n) {
                double x1 = x[2 * n], x2 = x[2 * n + 1];
                int64_t i1 = (int64_t)floor(x1 * (double)nl), i2 = (int64_t)floor(x2 * (double)nl);
                if (i1 >= nl) i1 = nl - 1;
                if (i2 >= nl) i2 = nl - 1;
                if (i1 < 0) i1 = 0;
                if (i2 < 0) i2 = 0;
                int64_t i = i1 * nl + i2;
                double cA1, cA2, wA;
                xbox2(L, i, &cA1, &cA2, &wA);
                cplx v = conj(e2pi(phi2(&B, x1, x2, cQ1, cQ2))) * yc[n];
                for (int t = 0; t < r2; ++t) {
                    double gA1 = cA1 + wA * z[t / r], gA2 = cA2 + wA * z[t % r];
                    a[i * r2 + t] += lag2(&B, t, (x1 - cA1) / wA, (x2 - cA2) / wA) *
                                     conj(e2pi(-phi2(&B, gA1, gA2, cQ1, cQ2))) * v;
                }
            }
        }
        /* recursion in x^*, l = L..h+1 */
        for (int l = L; l >= h + 1; --l) {
            int64_t np = (int64_t)1 << (2 * (l - 1)), nC = (int64_t)1 << (2 * (L - l + 1)), nj = nC / 4;
#pragma omp parallel for collapse(2) schedule(static)
            for (int64_t ip = 0; ip < np; ++ip)
                for (int64_t C = 0; C < nC; ++C) {
                    int64_t j = parent2(L - l + 1, C);
                    double cC1, cC2, wC, cP1, cP2, wP;
                    wbox2(&B, L - l + 1, C, &cC1, &cC2, &wC);
                    xbox2(l - 1, ip, &cP1, &cP2, &wP);
                    for (int s = 0; s < r2; ++s) {
                        double gP1 = cP1 + wP * z[s / r], gP2 = cP2 + wP * z[s % r];
                        cplx acc = 0;
                        for (int aa = 0; aa < 4; ++aa) {
                            int64_t i = child2(l - 1, ip, aa);
                            double cA1, cA2, wA;
                            xbox2(l, i, &cA1, &cA2, &wA);
                            const cplx* bp = a + (i * nj + j) * r2;
                            for (int t = 0; t < r2; ++t) {
                                double gA1 = cA1 + wA * z[t / r], gA2 = cA2 + wA * z[t % r];
                                cplx coef = e2pi(phi2(&B, gA1, gA2, cC1, cC2)) *
                                            lag2(&B, s, (gA1 - cP1) / wP, (gA2 - cP2) / wP) *
                                            e2pi(-phi2(&B, gP1, gP2, cC1, cC2));
                                acc += conj(coef) * bp[t];
                            }
                        }
                        b[(ip * nC + C) * r2 + s] = acc;
                    }
                }
            cplx* tmp = a; a = b; b = tmp;
        }
        /* switch^* */
        {
            int64_t ni = (int64_t)1 << (2 * h), nj = (int64_t)1 << (2 * (L - h));
#pragma omp parallel for collapse(2) schedule(static)
            for (int64_t i = 0; i < ni; ++i)
                for (int64_t j = 0; j < nj; ++j) {
                    double cA1, cA2, wA, cB1, cB2, wB;
                    xbox2(h, i, &cA1, &cA2, &wA);
                    wbox2(&B, L - h, j, &cB1, &cB2, &wB);
                    for (int s = 0; s < r2; ++s) {
                        double gB1 = cB1 + wB * z[s / r], gB2 = cB2 + wB * z[s % r];
                        cplx acc = 0;
                        for (int t = 0; t < r2; ++t)
                            acc += conj(e2pi(phi2(&B, cA1 + wA * z[t / r], cA2 + wA * z[t % r], gB1, gB2))) *
                                   a[(i * nj + j) * r2 + t];
                        b[(i * nj + j) * r2 + s] = acc;
                    }
                }
            cplx* tmp = a; a = b; b = tmp;
        }
        /* recursion in xi^*, l = h..1 */
        for (int l = h; l >= 1; --l) {
            int64_t np = (int64_t)1 << (2 * (l - 1)), nC = (int64_t)1 << (2 * (L - l + 1)), nj = nC / 4;
#pragma omp parallel for collapse(2) schedule(static)
            for (int64_t ip = 0; ip < np; ++ip)
                for (int64_t C = 0; C < nC; ++C) {
                    int64_t j = parent2(L - l + 1, C);
                    double cC1, cC2, wC, cB1, cB2, wB;
                    wbox2(&B, L - l + 1, C, &cC1, &cC2, &wC);
                    wbox2(&B, L - l, j, &cB1, &cB2, &wB);
                    for (int s = 0; s < r2; ++s) {
                        double gC1 = cC1 + wC * z[s / r], gC2 = cC2 + wC * z[s % r];
                        cplx acc = 0;
                        for (int aa = 0; aa < 4; ++aa) {
                            int64_t i = child2(l - 1, ip, aa);
                            double cA1, cA2, wA;
                            xbox2(l, i, &cA1, &cA2, &wA);
                            const cplx* bp = a + (i * nj + j) * r2;
                            for (int t = 0; t < r2; ++t) {
                                double gB1 = cB1 + wB * z[t / r], gB2 = cB2 + wB * z[t % r];
                                cplx coef = e2pi(-phi2(&B, cA1, cA2, gB1, gB2)) *
                                            lag2(&B, t, (gC1 - cB1) / wB, (gC2 - cB2) / wB) *
                                            e2pi(phi2(&B, cA1, cA2, gC1, gC2));
                                acc += conj(coef) * bp[t];
                            }
                        }
                        b[(ip * nC + C) * r2 + s] = acc;
                    }
                }
            cplx* tmp = a; a = b; b = tmp;
        }
        /* initialization^* */
        {
            double cA1, cA2, wA;
            xbox2(0, 0, &cA1, &cA2, &wA);
            for (int64_t j = 0; j < npair; ++j) {
                double cB1, cB2, wB;
                wbox2(&B, L, j, &cB1, &cB2, &wB);
                int64_t j1 = j >> L, j2 = j & (((int64_t)1 << L) - 1);
                double k1 = q1 + (double)j1, k2 = q2 + (double)j2;
                cplx acc = 0;
                for (int t = 0; t < r2; ++t) {
                    double gB1 = cB1 + wB * z[t / r], gB2 = cB2 + wB * z[t % r];
                    cplx coef = e2pi(-phi2(&B, cA1, cA2, gB1, gB2)) * lag2(&B, t, (k1 - cB1) / wB, (k2 - cB2) / wB) *
                                e2pi(phi2(&B, cA1, cA2, k1, k2));
                    acc += conj(coef) * a[j * r2 + t];
                }
                g[j1 * m + j2 + m * m * col] = acc;
            }
        }
    }
    free(a);
    free(b);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Multiscale IBF (Sec. 5.2, eqs. domaindecomp, mba, f1) on the n x n    */
/* frequency grid xi = (k1 - n/2, k2 - n/2).  Corona decomposition with  */
/* half-open squares: S_t = [-n/2^(t+1), n/2^(t+1))^2; ring t = S_t \ S_(t+1) */
/* is the 12 outer boxes (side m_t = n/2^(t+2)) of the 4 x 4 partition of */
/* S_t, for t = 0..T with n/2^(T+1) = center_side; the center S_(T+1) is */
/* summed directly.  g is n x n row-major in (k1, k2).                    */
/* ------------------------------------------------------------------ */
int orc_mibf_apply_2d(int phase_id, int64_t n, int r, int center_side, int64_t nx, const double* x, const cplx* g,
                      int nrhs, cplx* u)
{
    if (n < 4 || (n & (n - 1)) || center_side < 1 || center_side > n || (center_side & (center_side - 1)))
        return 1;
    int64_t nn = n * n;
    memset(u, 0, sizeof(cplx) * nx * nrhs);
    cplx* tmp = (cplx*)malloc(sizeof(cplx) * nx);
    int64_t side = n;
    while (side > center_side) {
        int64_t m = side / 4;
        if (m < 1) break;
        double s0 = -0.5 * (double)side;
        for (int b1 = 0; b1 < 4; ++b1)
            for (int b2 = 0; b2 < 4; ++b2) {
                if (b1 >= 1 && b1 <= 2 && b2 >= 1 && b2 <= 2) continue;   /* inner 2 x 2 = S_(t+1) */
                double q1 = s0 + (double)(b1 * m), q2 = s0 + (double)(b2 * m);
                cplx* gq = (cplx*)malloc(sizeof(cplx) * m * m);
                int L = ilog2(m);
                for (int col = 0; col < nrhs; ++col) {
                    for (int64_t k1 = 0; k1 < m; ++k1)
                        for (int64_t k2 = 0; k2 < m; ++k2) {
                            int64_t a1 = (int64_t)(q1 + (double)k1 + 0.5 * (double)n);
                            int64_t a2 = (int64_t)(q2 + (double)k2 + 0.5 * (double)n);
                            gq[k1 * m + k2] = g[(a1 * n + a2) + nn * col];
                        }
                    /* switch level ceil(L/2): for the odd depths of these boxes it
                       gives about 10x less error than floor(L/2) (reading of
                       Sec. 3's "L even" for odd L in 2D) */
                    int rc = orc_ibf_apply_2d(phase_id, m, r, (L + 1) / 2, nx, x, q1, q2, gq, 1, tmp);
                    if (rc) { free(gq); free(tmp); return rc; }
                    for (int64_t p = 0; p < nx; ++p) u[p + nx * col] += tmp[p];
                }
                free(gq);
            }
        side /= 2;
    }
    /* center: direct sum over S_(T+1) */
    {
        double s0 = -0.5 * (double)side;
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < nx; ++p)
            for (int col = 0; col < nrhs; ++col) {
                cplx acc = 0;
                for (int64_t k1 = 0; k1 < side; ++k1)
                    for (int64_t k2 = 0; k2 < side; ++k2) {
                        double xi1 = s0 + (double)k1, xi2 = s0 + (double)k2;
                        int64_t a1 = (int64_t)(xi1 + 0.5 * (double)n), a2 = (int64_t)(xi2 + 0.5 * (double)n);
                        acc += e2pi(orc_phi_2d(phase_id, x[2 * p], x[2 * p + 1], xi1, xi2)) * g[a1 * n + a2 + nn * col];
                    }
                u[p + nx * col] += acc;
            }
    }
    free(tmp);
    return 0;
}

/* Adjoint of orc_mibf_apply_2d: g = K^* y.  The corona boxes and the centre
   partition the frequency grid, so each writes its own part of g: the box
   adjoints (orc_ibf_adjoint_2d) and the direct adjoint sum on the centre. */
int orc_mibf_adjoint_2d(int phase_id, int64_t n, int r, int center_side, int64_t nx, const double* x, const cplx* y,
                        int nrhs, cplx* g)
{
    if (n < 4 || (n & (n - 1)) || center_side < 1 || center_side > n || (center_side & (center_side - 1)))
        return 1;
    int64_t nn = n * n;
    memset(g, 0, sizeof(cplx) * nn * nrhs);
    int64_t side = n;
    while (side > center_side) {
        int64_t m = side / 4;
        if (m < 1) break;
        double s0 = -0.5 * (double)side;
        int L = ilog2(m);
        cplx* gq = (cplx*)malloc(sizeof(cplx) * m * m);
        for (int b1 = 0; b1 < 4; ++b1)
            for (int b2 = 0; b2 < 4; ++b2) {
                if (b1 >= 1 && b1 <= 2 && b2 >= 1 && b2 <= 2) continue;
                double q1 = s0 + (double)(b1 * m), q2 = s0 + (double)(b2 * m);
                for (int col = 0; col < nrhs; ++col) {
                    int rc = orc_ibf_adjoint_2d(phase_id, m, r, (L + 1) / 2, nx, x, q1, q2, y + nx * col, 1, gq);
                    if (rc) { free(gq); return rc; }
                    for (int64_t k1 = 0; k1 < m; ++k1)
                        for (int64_t k2 = 0; k2 < m; ++k2) {
                            int64_t a1 = (int64_t)(q1 + (double)k1 + 0.5 * (double)n);
                            int64_t a2 = (int64_t)(q2 + (double)k2 + 0.5 * (double)n);
                            g[(a1 * n + a2) + nn * col] = gq[k1 * m + k2];
                        }
                }
            }
        free(gq);
        side /= 2;
    }
    {
        double s0 = -0.5 * (double)side;
#pragma omp parallel for collapse(2) schedule(static)
        for (int64_t k1 = 0; k1 < side; ++k1)
            for (int64_t k2 = 0; k2 < side; ++k2) {
                double xi1 = s0 + (double)k1, xi2 = s0 + (double)k2;
                int64_t a1 = (int64_t)(xi1 + 0.5 * (double)n), a2 = (int64_t)(xi2 + 0.5 * (double)n);
                for (int col = 0; col < nrhs; ++col) {
                    cplx acc = 0;
                    for (int64_t p = 0; p < nx; ++p)
                        acc += conj(e2pi(orc_phi_2d(phase_id, x[2 * p], x[2 * p + 1], xi1, xi2))) * y[p + nx * col];
                    g[a1 * n + a2 + nn * col] = acc;
                }
            }
    }
    return 0;
}
