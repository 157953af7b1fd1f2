/*
 * FP64 CPU oracle for SAFR (Singular value-based Atmospheric tomography with
 * Fourier domain Regularization), arXiv 2510.19542.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU path computes.  Only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or constant with the CUDA library, and includes none of it.
 *
 * Every routine follows one passage of the paper:
 *   - cone coefficients c_l ......................... Section 2
 *   - tomography operator (A_g phi)(r) .............. Section 2, Eq. (defAperonly)
 *   - A_jk, w^(beta)_{jk,l}, tau_{l,T}, omega ....... Section 3.1
 *   - Tikhonov filter g(s) = s/(s^2+alpha) .......... Section 3.1
 *   - b_{jk,lg} coefficients ........................ Section 3.2 / Algorithm 2
 *   - DFT2 / IDFT2 (unnormalised / 1/M^2) ........... Section 3.2
 *   - shifted index n(j) ............................ Section 3.2
 *   - hard real-time apply .......................... Algorithm 1
 *   - split tomography (LGS + TTS, results added) ... Section 3.3, Algorithm 3
 *   - removeTT (planar component of LGS wavefronts) . Section 3.3, Algorithm 3
 *   - learned filter phi/sigma (MLP factor) ......... Section 3.1 (general filter g)
 *   - Philox4x32-10 and the training frames ......... Salmon et al. (SC 2011); Section 2
 *   - POLC, psi + A(a) with bilinear layers ......... Algorithm 3 line 2, Eq. (defAperonly)
 *   - integrator ..................................... Algorithm 3 line 5
 *
 * Readings where the paper is silent or assumes odd M (all even-M grids):
 *   - Nyquist: the symmetric truncation keeps |n| <= M/2-1, so B is zero on the
 *     row j = M/2 and the column k = M/2 (the paper's M = 2m+1 has no such bin).
 *   - V is indexed V_{l,r} (R_alpha = V g(Sigma^T) U^H, Section 3.1); Algorithm 2
 *     prints the transpose.
 *   - Mixed LGS+NGS: LGS-group layers live on the pitch c_l*delta grid; for the
 *     metric output they are bilinearly resampled (periodic wrap) onto the pitch
 *     delta grid and then added to the NGS-group layers.
 *   - removeTT: least-squares plane a + b x + c y over the pupil-mask pixels,
 *     subtract b x + c y inside the mask (piston kept).
 *
 * Build: gcc -O2 -fopenmp -std=c11 -shared -fPIC oracle.c -o liboracle.so -lm
 * OpenMP only runs independent outer iterations in parallel; every sum is
 * taken in the same order whatever the thread count.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static const double PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------------- */
/* DFT2 / IDFT2 (Section 3.2): direct separable sums.                         */
/* The twiddle exp(-2 pi i t / M) is taken from a table indexed by the exact   */
/* integer residue t = (j*p) mod M.                                           */
/* ------------------------------------------------------------------------- */
static cplx *twiddle_table(int M, int inverse)
{
    cplx *w = (cplx *)malloc(sizeof(cplx) * (size_t)M);
    for (int t = 0; t < M; ++t) {
        double a = 2.0 * PI * (double)t / (double)M;
        w[t] = cos(a) + (inverse ? 1.0 : -1.0) * I * sin(a);
    }
    return w;
}

/* Y = DFT2(X) (inverse = 0) or IDFT2(X) (inverse = 1), X, Y [M][M] row-major,
 * first index p <-> j, second index q <-> k.  X and Y may not alias. */
int oracle_dft2(int M, const cplx *X, cplx *Y, int inverse)
{
    if (M <= 0 || !X || !Y) return -1;
    cplx *w = twiddle_table(M, inverse);
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)M * M);
    /* sum over q for every (p, k) */
#pragma omp parallel for schedule(static)
    for (int p = 0; p < M; ++p)
        for (int k = 0; k < M; ++k) {
            cplx s = 0;
            for (int q = 0; q < M; ++q)
                s += X[(size_t)p * M + q] * w[((long)k * q) % M];
            tmp[(size_t)p * M + k] = s;
        }
    /* sum over p for every (j, k) */
    double scale = inverse ? 1.0 / ((double)M * (double)M) : 1.0;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < M; ++j)
        for (int k = 0; k < M; ++k) {
            cplx s = 0;
            for (int p = 0; p < M; ++p)
                s += tmp[(size_t)p * M + k] * w[((long)j * p) % M];
            Y[(size_t)j * M + k] = s * scale;
        }
    free(tmp);
    free(w);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* One-sided (Hestenes) Jacobi SVD of a complex m x n matrix A (row-major).    */
/* Returns U [m][n], S [n], V [n][n] with A = U diag(S) V^H.  Columns of A are */
/* rotated pairwise until every pair is orthogonal to relative 1e-15; the     */
/* column norms are then the singular values.  Columns whose norm is zero     */
/* give S = 0 and a zero column of U.  No LAPACK.                             */
/* ------------------------------------------------------------------------- */
int oracle_svd(int m, int n, const cplx *A, cplx *U, double *S, cplx *V)
{
    if (m <= 0 || n <= 0) return -1;
    cplx *W = (cplx *)malloc(sizeof(cplx) * (size_t)m * n);
    memcpy(W, A, sizeof(cplx) * (size_t)m * n);
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) V[a * n + b] = (a == b) ? 1.0 : 0.0;

    /* Pairs are rotated until |w_i^H w_j| <= 1e-15 ||w_i|| ||w_j||.  A column
     * whose squared norm has fallen below 1e-30 ||A||_F^2 is rounding residue of
     * a rank-deficient A (more columns than rows) and is not rotated further. */
    const double tol = 1e-15;
    double frob = 0;
    for (int i = 0; i < m * n; ++i) frob += creal(A[i]) * creal(A[i]) + cimag(A[i]) * cimag(A[i]);
    const double floor_sq = 1e-30 * frob;
    int sweep;
    for (sweep = 0; sweep < 100; ++sweep) {
        int rotated = 0;
        for (int i = 0; i < n - 1; ++i)
            for (int j = i + 1; j < n; ++j) {
                double ai = 0, aj = 0;
                cplx gij = 0; /* w_i^H w_j */
                for (int r = 0; r < m; ++r) {
                    cplx wi = W[r * n + i], wj = W[r * n + j];
                    ai += creal(wi) * creal(wi) + cimag(wi) * cimag(wi);
                    aj += creal(wj) * creal(wj) + cimag(wj) * cimag(wj);
                    gij += conj(wi) * wj;
                }
                double ag = cabs(gij);
                if (ai <= floor_sq || aj <= floor_sq || ag <= tol * sqrt(ai * aj)) continue;
                rotated = 1;
                cplx ph = gij / ag; /* e^{i phi} */
                double zeta = (aj - ai) / (2.0 * ag);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                /* w_j'' = w_j e^{-i phi}; then a real plane rotation */
                for (int r = 0; r < m; ++r) {
                    cplx wi = W[r * n + i], wj = W[r * n + j] * conj(ph);
                    W[r * n + i] = c * wi - s * wj;
                    W[r * n + j] = s * wi + c * wj;
                }
                for (int r = 0; r < n; ++r) {
                    cplx vi = V[r * n + i], vj = V[r * n + j] * conj(ph);
                    V[r * n + i] = c * vi - s * vj;
                    V[r * n + j] = s * vi + c * vj;
                }
            }
        if (!rotated) break;
    }
    for (int i = 0; i < n; ++i) {
        double nrm = 0;
        for (int r = 0; r < m; ++r) nrm += creal(W[r * n + i]) * creal(W[r * n + i]) +
                                           cimag(W[r * n + i]) * cimag(W[r * n + i]);
        nrm = sqrt(nrm);
        S[i] = nrm;
        for (int r = 0; r < m; ++r) U[r * n + i] = nrm > 0 ? W[r * n + i] / nrm : 0.0;
    }
    free(W);
    return sweep;
}

/* ------------------------------------------------------------------------- */
/* Geometry (Section 2)                                                       */
/* ------------------------------------------------------------------------- */

/* c_l = 1 (NGS) or 1 - h_l / h_LGS (LGS). */
void oracle_cone(int L, const double *h, double h_lgs, int lgs, double *c)
{
    for (int l = 0; l < L; ++l) c[l] = lgs ? 1.0 - h[l] / h_lgs : 1.0;
}

/* shifted index n(j) of Section 3.2 for even M with the Nyquist bin
 * j = M/2 kept apart (the caller zeroes it). */
static int shifted_index(int j, int M) { return j < M / 2 ? j : j - M; }

/* ------------------------------------------------------------------------- */
/* Algorithm 2: b_{n,lg} for one star group, every frequency of the full       */
/* M x M spectrum.  B is [M][M][L][G] (j, k, l, g), complex.                  */
/*                                                                             */
/*   A_n[g][l] = s_l(n) exp(i omega n.(alpha_g h_l) / c_l),  omega = pi / T     */
/*   s_l(n)    = gamma_l^{1/2} / c_l * (1 + tau_l |n|^2)^{-beta/2}              */
/*   tau_l     = pi^2 / (c_l T)^2                                               */
/*   B_n[l][g] = s_l(n) sum_r V_{l r} g(sigma_r) conj(U_{g r}),                 */
/*   g(s)      = s / (s^2 + alpha)                                              */
/*                                                                             */
/* A_n = (2T) w^(beta)_{n,l}(alpha_g h_l) with w^(beta) and w of Section 3.1.   */
/* ------------------------------------------------------------------------- */
int oracle_group_B(int M, double T, int L, const double *h, const double *c,
                   const double *gamma, int G, const double *ax, const double *ay,
                   double alpha, double beta, cplx *B)
{
    if (M <= 0 || M % 2 || L <= 0 || G <= 0) return -1;
    const double omega = PI / T;
#pragma omp parallel for schedule(dynamic, 16)
    for (long f = 0; f < (long)M * M; ++f) {
        int j = (int)(f / M), k = (int)(f % M);
        cplx *Bf = B + (size_t)f * L * G;
        if (j == M / 2 || k == M / 2) { /* Nyquist row / column */
            for (int i = 0; i < L * G; ++i) Bf[i] = 0;
            continue;
        }
        double nx = shifted_index(j, M), ny = shifted_index(k, M);
        double *s = (double *)malloc(sizeof(double) * L);
        int R = G < L ? G : L; /* number of singular values */
        cplx *A = (cplx *)malloc(sizeof(cplx) * (size_t)G * L);
        cplx *AH = (cplx *)malloc(sizeof(cplx) * (size_t)G * L);
        cplx *Ux = (cplx *)malloc(sizeof(cplx) * (size_t)G * L);
        cplx *Vx = (cplx *)malloc(sizeof(cplx) * (size_t)L * L);
        cplx *U = (cplx *)malloc(sizeof(cplx) * (size_t)G * R); /* [G][R] */
        cplx *V = (cplx *)malloc(sizeof(cplx) * (size_t)L * R); /* [L][R] */
        double *S = (double *)malloc(sizeof(double) * L);
        for (int l = 0; l < L; ++l) {
            double tau = PI * PI / ((c[l] * T) * (c[l] * T));
            s[l] = sqrt(gamma[l]) / c[l] * pow(1.0 + tau * (nx * nx + ny * ny), -beta / 2.0);
        }
        for (int g = 0; g < G; ++g)
            for (int l = 0; l < L; ++l) {
                double arg = omega * (nx * ax[g] * h[l] + ny * ay[g] * h[l]) / c[l];
                A[g * L + l] = s[l] * (cos(arg) + I * sin(arg));
            }
        /* A = U Sigma V^H.  One-sided Jacobi runs on the orientation with no more
         * columns than rows: on A itself when G >= L, else on A^H = V Sigma U^H. */
        if (G >= L) {
            oracle_svd(G, L, A, Ux, S, Vx);
            for (int g = 0; g < G; ++g) for (int r = 0; r < R; ++r) U[g * R + r] = Ux[g * L + r];
            for (int l = 0; l < L; ++l) for (int r = 0; r < R; ++r) V[l * R + r] = Vx[l * L + r];
        } else {
            for (int g = 0; g < G; ++g) for (int l = 0; l < L; ++l) AH[l * G + g] = conj(A[g * L + l]);
            oracle_svd(L, G, AH, Ux, S, Vx); /* Ux [L][G], Vx [G][G] */
            for (int g = 0; g < G; ++g) for (int r = 0; r < R; ++r) U[g * R + r] = Vx[g * G + r];
            for (int l = 0; l < L; ++l) for (int r = 0; r < R; ++r) V[l * R + r] = Ux[l * G + r];
        }
        for (int l = 0; l < L; ++l)
            for (int g = 0; g < G; ++g) {
                cplx acc = 0;
                for (int r = 0; r < R; ++r) {
                    if (S[r] == 0.0) continue;
                    double filt = S[r] / (S[r] * S[r] + alpha); /* g_alpha(sigma_r) */
                    acc += V[l * R + r] * filt * conj(U[g * R + r]);
                }
                Bf[l * G + g] = s[l] * acc;
            }
        free(s); free(A); free(AH); free(Ux); free(Vx); free(U); free(V); free(S);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* removeTT (Algorithm 3): least-squares plane over the pupil mask.            */
/* psi [P][P] is modified in place: psi -= b x + c y on mask pixels.           */
/* x_a = (a - (P-1)/2) delta along the first index, y likewise along the      */
/* second.  Returns the fitted (a, b, c) in abc if abc != NULL.               */
/* ------------------------------------------------------------------------- */
int oracle_remove_tt(int P, double delta, const unsigned char *mask, double *psi, double *abc)
{
    double N[3][3] = {{0}}, r[3] = {0};
    for (int a = 0; a < P; ++a)
        for (int b = 0; b < P; ++b) {
            if (!mask[a * P + b]) continue;
            double x = (a - (P - 1) / 2.0) * delta, y = (b - (P - 1) / 2.0) * delta;
            double phi[3] = {1.0, x, y};
            for (int u = 0; u < 3; ++u) {
                r[u] += phi[u] * psi[a * P + b];
                for (int v = 0; v < 3; ++v) N[u][v] += phi[u] * phi[v];
            }
        }
    /* Gaussian elimination with partial pivoting on the 3x3 normal equations */
    double Mx[3][4];
    for (int u = 0; u < 3; ++u) {
        for (int v = 0; v < 3; ++v) Mx[u][v] = N[u][v];
        Mx[u][3] = r[u];
    }
    for (int col = 0; col < 3; ++col) {
        int piv = col;
        for (int u = col + 1; u < 3; ++u)
            if (fabs(Mx[u][col]) > fabs(Mx[piv][col])) piv = u;
        if (Mx[piv][col] == 0.0) return -1;
        if (piv != col)
            for (int v = 0; v < 4; ++v) { double t = Mx[col][v]; Mx[col][v] = Mx[piv][v]; Mx[piv][v] = t; }
        for (int u = col + 1; u < 3; ++u) {
            double f = Mx[u][col] / Mx[col][col];
            for (int v = col; v < 4; ++v) Mx[u][v] -= f * Mx[col][v];
        }
    }
    double sol[3];
    for (int u = 2; u >= 0; --u) {
        double acc = Mx[u][3];
        for (int v = u + 1; v < 3; ++v) acc -= Mx[u][v] * sol[v];
        sol[u] = acc / Mx[u][u];
    }
    for (int a = 0; a < P; ++a)
        for (int b = 0; b < P; ++b) {
            if (!mask[a * P + b]) continue;
            double x = (a - (P - 1) / 2.0) * delta, y = (b - (P - 1) / 2.0) * delta;
            psi[a * P + b] -= sol[1] * x + sol[2] * y;
        }
    if (abc) { abc[0] = sol[0]; abc[1] = sol[1]; abc[2] = sol[2]; }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Metric-grid resample of a layer sampled at pitch c*delta (Section 3.2 grid  */
/* x^l_p = c_l x_p): the metric sample x_p sits at fractional layer index      */
/* u = M/2 + (p - M/2)/c.  Bilinear interpolation, periodic wrap mod M.        */
/* ------------------------------------------------------------------------- */
void oracle_resample(int M, double c, const double *src, double *dst)
{
    for (int p = 0; p < M; ++p) {
        double u = M / 2.0 + (p - M / 2.0) / c;
        double fu0 = floor(u), fu = u - fu0;
        long i0 = (long)fu0;
        int ia = (int)(((i0 % M) + M) % M), ib = (int)((((i0 + 1) % M) + M) % M);
        for (int q = 0; q < M; ++q) {
            double v = M / 2.0 + (q - M / 2.0) / c;
            double fv0 = floor(v), fv = v - fv0;
            long j0 = (long)fv0;
            int ja = (int)(((j0 % M) + M) % M), jb = (int)((((j0 + 1) % M) + M) % M);
            dst[p * M + q] = (1 - fu) * (1 - fv) * src[ia * M + ja] + fu * (1 - fv) * src[ib * M + ja] +
                             (1 - fu) * fv * src[ia * M + jb] + fu * fv * src[ib * M + jb];
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Plan: geometry, the star groups and their B (Algorithm 2), then the per-    */
/* frame reconstruction (Algorithm 1 per group, Algorithm 3 line 4 sum).       */
/* ------------------------------------------------------------------------- */
typedef struct {
    int M, P, L, G, output_metric, remove_tt, mixed;
    double delta, T;
    double *h, *gamma;
    int ngroups;
    int grp_kind[2];   /* 1 = LGS, 0 = NGS */
    int grp_G[2];
    int *grp_star[2];  /* star indices (input order) */
    double *grp_c[2];  /* c_l per group */
    cplx *grp_B[2];    /* [M][M][L][Gg] */
    unsigned char *mask; /* [P][P] pupil mask */
} oracle_plan;

void oracle_plan_free(oracle_plan *pl)
{
    if (!pl) return;
    free(pl->h); free(pl->gamma); free(pl->mask);
    for (int i = 0; i < 2; ++i) { free(pl->grp_star[i]); free(pl->grp_c[i]); free(pl->grp_B[i]); }
    free(pl);
}

/* Pupil mask: annulus of outer diameter D and inner diameter obstruction*D,
 * pixel centres at ((a-(P-1)/2) delta, (b-(P-1)/2) delta).  D <= 0 means the
 * full P x P square. */
void oracle_pupil_mask(int P, double delta, double D, double obstruction, unsigned char *mask)
{
    double ro = D / 2.0, ri = obstruction * D / 2.0;
    for (int a = 0; a < P; ++a)
        for (int b = 0; b < P; ++b) {
            double x = (a - (P - 1) / 2.0) * delta, y = (b - (P - 1) / 2.0) * delta;
            double r2 = x * x + y * y;
            mask[a * P + b] = (D <= 0.0) ? 1 : (r2 <= ro * ro && r2 >= ri * ri);
        }
}

oracle_plan *oracle_plan_new(int M, int P, double delta, double D, double obstruction,
                             int L, const double *h, const double *cn2,
                             int G, const double *ax, const double *ay, const int *kind,
                             double h_lgs, double alpha, double alpha_tt, double beta,
                             int output_metric, int remove_tt)
{
    if (M <= 0 || M % 2 || P <= 0 || P > M || L <= 0 || G <= 0) return NULL;
    oracle_plan *pl = (oracle_plan *)calloc(1, sizeof(oracle_plan));
    pl->M = M; pl->P = P; pl->L = L; pl->G = G;
    pl->delta = delta; pl->T = M * delta / 2.0;
    pl->h = (double *)malloc(sizeof(double) * L);
    pl->gamma = (double *)malloc(sizeof(double) * L);
    double sum = 0;
    for (int l = 0; l < L; ++l) sum += cn2[l];
    for (int l = 0; l < L; ++l) { pl->h[l] = h[l]; pl->gamma[l] = cn2[l] / sum; }
    int nl = 0, nn = 0;
    for (int g = 0; g < G; ++g) {
        if (kind[g]) ++nl;
        else ++nn;
    }
    pl->mixed = nl > 0 && nn > 0;
    pl->output_metric = output_metric;
    pl->remove_tt = remove_tt && pl->mixed;
    pl->mask = (unsigned char *)malloc((size_t)P * P);
    oracle_pupil_mask(P, delta, D, obstruction, pl->mask);
    /* LGS group first, then NGS (Section 3.3) */
    int kinds[2] = {1, 0};
    for (int i = 0; i < 2; ++i) {
        int cnt = kinds[i] ? nl : nn;
        if (!cnt) continue;
        int gi = pl->ngroups++;
        pl->grp_kind[gi] = kinds[i];
        pl->grp_G[gi] = cnt;
        pl->grp_star[gi] = (int *)malloc(sizeof(int) * cnt);
        double *gx = (double *)malloc(sizeof(double) * cnt), *gy = (double *)malloc(sizeof(double) * cnt);
        int t = 0;
        for (int g = 0; g < G; ++g)
            if (kind[g] == kinds[i]) { pl->grp_star[gi][t] = g; gx[t] = ax[g]; gy[t] = ay[g]; ++t; }
        pl->grp_c[gi] = (double *)malloc(sizeof(double) * L);
        oracle_cone(L, h, h_lgs, kinds[i], pl->grp_c[gi]);
        pl->grp_B[gi] = (cplx *)malloc(sizeof(cplx) * (size_t)M * M * L * cnt);
        /* the TTS group of a mixed plan takes alpha_TT (Algorithm 3, line 4) */
        double a = (pl->mixed && !kinds[i]) ? alpha_tt : alpha;
        oracle_group_B(M, pl->T, L, h, pl->grp_c[gi], pl->gamma, cnt, gx, gy, a, beta, pl->grp_B[gi]);
        free(gx); free(gy);
    }
    return pl;
}

int oracle_plan_ngroups(const oracle_plan *pl) { return pl->ngroups; }

/* copy one group's B [M][M][L][Gg], its star list and its c_l */
int oracle_plan_group(const oracle_plan *pl, int gi, int *kind, int *Gg, int *stars, double *c, cplx *B)
{
    if (gi < 0 || gi >= pl->ngroups) return -1;
    if (kind) *kind = pl->grp_kind[gi];
    if (Gg) *Gg = pl->grp_G[gi];
    if (stars) memcpy(stars, pl->grp_star[gi], sizeof(int) * pl->grp_G[gi]);
    if (c) memcpy(c, pl->grp_c[gi], sizeof(double) * pl->L);
    if (B) memcpy(B, pl->grp_B[gi], sizeof(cplx) * (size_t)pl->M * pl->M * pl->L * pl->grp_G[gi]);
    return 0;
}

/* Spectra b_l(n) of every group (Algorithm 1 lines 1-6): zero-pad, removeTT
 * on LGS wavefronts of a mixed plan, DFT2 per star, apply B.
 * spec: [ngroups][L][M][M] complex. */
static void plan_spectra(const oracle_plan *pl, const double *wavefronts, cplx *spec)
{
    int M = pl->M, P = pl->P, L = pl->L, G = pl->G, o = (M - P) / 2;
    cplx *d = (cplx *)malloc(sizeof(cplx) * (size_t)G * M * M);
    cplx *pad = (cplx *)malloc(sizeof(cplx) * (size_t)M * M);
    double *psi = (double *)malloc(sizeof(double) * (size_t)P * P);
    for (int g = 0; g < G; ++g) {
        memcpy(psi, wavefronts + (size_t)g * P * P, sizeof(double) * P * P);
        int is_lgs = 0;
        for (int gi = 0; gi < pl->ngroups; ++gi)
            for (int t = 0; t < pl->grp_G[gi]; ++t)
                if (pl->grp_star[gi][t] == g && pl->grp_kind[gi]) is_lgs = 1;
        if (pl->remove_tt && is_lgs) oracle_remove_tt(P, pl->delta, pl->mask, psi, NULL);
        for (size_t i = 0; i < (size_t)M * M; ++i) pad[i] = 0;
        for (int a = 0; a < P; ++a)
            for (int b = 0; b < P; ++b) pad[(size_t)(a + o) * M + (b + o)] = psi[a * P + b];
        oracle_dft2(M, pad, d + (size_t)g * M * M, 0);
    }
    for (int gi = 0; gi < pl->ngroups; ++gi) {
        int Gg = pl->grp_G[gi];
        const cplx *B = pl->grp_B[gi];
        cplx *out = spec + (size_t)gi * L * M * M;
#pragma omp parallel for schedule(static)
        for (long f = 0; f < (long)M * M; ++f)
            for (int l = 0; l < L; ++l) {
                cplx acc = 0;
                for (int t = 0; t < Gg; ++t)
                    acc += B[((size_t)f * L + l) * Gg + t] * d[(size_t)pl->grp_star[gi][t] * M * M + f];
                out[(size_t)l * M * M + f] = acc;
            }
    }
    free(d); free(pad); free(psi);
}

/* Full reconstruction.  wavefronts [G][P][P], layers [L][M][M].
 * imag_max (optional) receives max |Im IDFT2| over all groups and layers. */
int oracle_plan_reconstruct(const oracle_plan *pl, const double *wavefronts, double *layers, double *imag_max)
{
    int M = pl->M, L = pl->L;
    cplx *spec = (cplx *)malloc(sizeof(cplx) * (size_t)pl->ngroups * L * M * M);
    cplx *phi = (cplx *)malloc(sizeof(cplx) * (size_t)M * M);
    double *re = (double *)malloc(sizeof(double) * (size_t)M * M);
    double *rs = (double *)malloc(sizeof(double) * (size_t)M * M);
    double im = 0;
    plan_spectra(pl, wavefronts, spec);
    memset(layers, 0, sizeof(double) * (size_t)L * M * M);
    for (int gi = 0; gi < pl->ngroups; ++gi)
        for (int l = 0; l < L; ++l) {
            oracle_dft2(M, spec + ((size_t)gi * L + l) * M * M, phi, 1); /* Algorithm 1 line 8 */
            for (size_t i = 0; i < (size_t)M * M; ++i) {
                re[i] = creal(phi[i]);
                if (fabs(cimag(phi[i])) > im) im = fabs(cimag(phi[i]));
            }
            const double *src = re;
            if (pl->grp_kind[gi] && pl->output_metric) {
                oracle_resample(M, pl->grp_c[gi][l], re, rs);
                src = rs;
            }
            for (size_t i = 0; i < (size_t)M * M; ++i) layers[(size_t)l * M * M + i] += src[i];
        }
    if (imag_max) *imag_max = im;
    free(spec); free(phi); free(re); free(rs);
    return 0;
}

/* Sampled reconstruction: layer values at n (l, p, q) triples only.  Each value
 * is the IDFT2 sum at that point (and, for a resampled LGS layer, at its four
 * bilinear neighbours), so a full-size frame can be checked point by point. */
int oracle_plan_reconstruct_samples(const oracle_plan *pl, const double *wavefronts, int n,
                                    const int *lpq, double *out)
{
    int M = pl->M, L = pl->L;
    cplx *spec = (cplx *)malloc(sizeof(cplx) * (size_t)pl->ngroups * L * M * M);
    plan_spectra(pl, wavefronts, spec);
    cplx *w = twiddle_table(M, 1);
#pragma omp parallel for schedule(dynamic, 1)
    for (int s = 0; s < n; ++s) {
        int l = lpq[3 * s], p = lpq[3 * s + 1], q = lpq[3 * s + 2];
        double total = 0;
        for (int gi = 0; gi < pl->ngroups; ++gi) {
            const cplx *b = spec + ((size_t)gi * L + l) * M * M;
            int resample = pl->grp_kind[gi] && pl->output_metric;
            int np = resample ? 2 : 1;
            int rows[2], cols[2];
            double wr[2], wc[2];
            if (resample) {
                double c = pl->grp_c[gi][l];
                double u = M / 2.0 + (p - M / 2.0) / c, v = M / 2.0 + (q - M / 2.0) / c;
                double fu0 = floor(u), fv0 = floor(v);
                long i0 = (long)fu0, j0 = (long)fv0;
                rows[0] = (int)(((i0 % M) + M) % M); rows[1] = (int)((((i0 + 1) % M) + M) % M);
                cols[0] = (int)(((j0 % M) + M) % M); cols[1] = (int)((((j0 + 1) % M) + M) % M);
                wr[0] = 1 - (u - fu0); wr[1] = u - fu0; wc[0] = 1 - (v - fv0); wc[1] = v - fv0;
            } else {
                rows[0] = p; cols[0] = q; wr[0] = 1; wc[0] = 1;
            }
            for (int a = 0; a < np; ++a)
                for (int bb = 0; bb < np; ++bb) {
                    int pp = rows[a], qq = cols[bb];
                    cplx acc = 0;
                    for (int j = 0; j < M; ++j)
                        for (int k = 0; k < M; ++k)
                            acc += b[(size_t)j * M + k] * w[((long)j * pp + (long)k * qq) % M];
                    total += wr[a] * wc[bb] * creal(acc) / ((double)M * (double)M);
                }
        }
        out[s] = total;
    }
    free(w); free(spec);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Learned spectral filter.  Section 3.1 writes the regularised inverse as     */
/* R(A) = V g(Sigma^T) U^H for a regularising filter g of the singular values. */
/* Here g(sigma_r) = phi / sigma_r with phi in (0, 1) from an MLP of the point */
/* x = (|n| / (M/2), h_l / 20 km, (log10 sigma_r + 4) / 4, noise / 0.05), and */
/* the factor may differ per layer l:                                          */
/*   B_n[l][g] = s_l(n) sum_r V_{l r} (phi_{l r} / sigma_r) conj(U_{g r}).      */
/* MLP: 4 -> 64 -> 64 -> 64 -> 1, GELU(z) = z (1 + erf(z / sqrt 2)) / 2 after  */
/* each hidden layer, logistic output; parameters W0[64][4] b0[64] W1[64][64]  */
/* b1[64] W2[64][64] b2[64] W3[64] b3, rows = outputs.                         */
/* A singular value sigma_r <= 1e-13 sigma_max is a numerical zero (the rank of */
/* A_n): its direction is dropped, since phi / sigma_r, unlike the Tikhonov    */
/* factor, does not vanish as sigma_r -> 0.                                    */
/* ------------------------------------------------------------------------- */
#define MLP_H 64

static double gelu_erf(double z) { return 0.5 * z * (1.0 + erf(z / sqrt(2.0))); }

double oracle_mlp_phi(const double *p, const double *x)
{
    const double *W0 = p, *b0 = W0 + MLP_H * 4, *W1 = b0 + MLP_H, *b1 = W1 + MLP_H * MLP_H;
    const double *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H, *W3 = b2 + MLP_H, *b3 = W3 + MLP_H;
    double h1[MLP_H], h2[MLP_H], h3[MLP_H];
    for (int i = 0; i < MLP_H; ++i) {
        double z = b0[i];
        for (int q = 0; q < 4; ++q) z += W0[i * 4 + q] * x[q];
        h1[i] = gelu_erf(z);
    }
    for (int i = 0; i < MLP_H; ++i) {
        double z = b1[i];
        for (int q = 0; q < MLP_H; ++q) z += W1[i * MLP_H + q] * h1[q];
        h2[i] = gelu_erf(z);
    }
    for (int i = 0; i < MLP_H; ++i) {
        double z = b2[i];
        for (int q = 0; q < MLP_H; ++q) z += W2[i * MLP_H + q] * h2[q];
        h3[i] = gelu_erf(z);
    }
    double o = b3[0];
    for (int q = 0; q < MLP_H; ++q) o += W3[q] * h3[q];
    return 1.0 / (1.0 + exp(-o));
}

int oracle_group_B_learned(int M, double T, int L, const double *h, const double *c, const double *gamma, int G,
                           const double *ax, const double *ay, double beta, const double *params,
                           double noise_level, cplx *B)
{
    if (M <= 0 || M % 2 || L <= 0 || G <= 0) return -1;
    const double omega = PI / T;
#pragma omp parallel for schedule(dynamic, 16)
    for (long f = 0; f < (long)M * M; ++f) {
        int j = (int)(f / M), k = (int)(f % M);
        cplx *Bf = B + (size_t)f * L * G;
        for (int i = 0; i < L * G; ++i) Bf[i] = 0;
        if (j == M / 2 || k == M / 2) continue; /* Nyquist row / column */
        double nx = shifted_index(j, M), ny = shifted_index(k, M);
        int R = G < L ? G : L;
        double *s = (double *)malloc(sizeof(double) * L);
        cplx *A = (cplx *)malloc(sizeof(cplx) * (size_t)G * L);
        cplx *AH = (cplx *)malloc(sizeof(cplx) * (size_t)G * L);
        cplx *Ux = (cplx *)malloc(sizeof(cplx) * (size_t)G * L);
        cplx *Vx = (cplx *)malloc(sizeof(cplx) * (size_t)L * L);
        cplx *U = (cplx *)malloc(sizeof(cplx) * (size_t)G * R);
        cplx *V = (cplx *)malloc(sizeof(cplx) * (size_t)L * R);
        double *S = (double *)malloc(sizeof(double) * L);
        for (int l = 0; l < L; ++l) {
            double tau = PI * PI / ((c[l] * T) * (c[l] * T));
            s[l] = sqrt(gamma[l]) / c[l] * pow(1.0 + tau * (nx * nx + ny * ny), -beta / 2.0);
        }
        for (int g = 0; g < G; ++g)
            for (int l = 0; l < L; ++l) {
                double arg = omega * (nx * ax[g] * h[l] + ny * ay[g] * h[l]) / c[l];
                A[g * L + l] = s[l] * (cos(arg) + I * sin(arg));
            }
        if (G >= L) {
            oracle_svd(G, L, A, Ux, S, Vx);
            for (int g = 0; g < G; ++g) for (int r = 0; r < R; ++r) U[g * R + r] = Ux[g * L + r];
            for (int l = 0; l < L; ++l) for (int r = 0; r < R; ++r) V[l * R + r] = Vx[l * L + r];
        } else {
            for (int g = 0; g < G; ++g) for (int l = 0; l < L; ++l) AH[l * G + g] = conj(A[g * L + l]);
            oracle_svd(L, G, AH, Ux, S, Vx);
            for (int g = 0; g < G; ++g) for (int r = 0; r < R; ++r) U[g * R + r] = Vx[g * G + r];
            for (int l = 0; l < L; ++l) for (int r = 0; r < R; ++r) V[l * R + r] = Ux[l * G + r];
        }
        double smax = 0;
        for (int r = 0; r < R; ++r) smax = S[r] > smax ? S[r] : smax;
        const double nabs = sqrt(nx * nx + ny * ny);
        for (int l = 0; l < L; ++l)
            for (int r = 0; r < R; ++r) {
                if (!(S[r] > 1e-13 * smax)) continue;
                double x[4] = {nabs / (0.5 * M), h[l] / 20e3, (log10(S[r] > 1e-12 ? S[r] : 1e-12) + 4.0) / 4.0,
                               noise_level / 0.05};
                double w = oracle_mlp_phi(params, x) / S[r];
                for (int g = 0; g < G; ++g) Bf[l * G + g] += s[l] * V[l * R + r] * w * conj(U[g * R + r]);
            }
        free(s); free(A); free(AH); free(Ux); free(Vx); free(U); free(V); free(S);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as    */
/* easy as 1, 2, 3", SC 2011): ten rounds; each round multiplies counter words */
/* 0 and 2 by 0xD2511F53 and 0xCD9E8D57 (64-bit products), and the new words   */
/* are (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the   */
/* key is bumped by (0x9E3779B9, 0xBB67AE85) between rounds.                   */
/* ------------------------------------------------------------------------- */
void oracle_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out)
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3], k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0, n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1, n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Two standard normals by Box-Muller from the first two output words of    */
/* counter (a, b, c, e): u = (word + 1/2) 2^-32 in (0, 1).                  */
static void normal_pair(uint32_t a, uint32_t b, uint32_t c, uint32_t e, uint32_t k0, uint32_t k1, double *z0,
                        double *z1)
{
    uint32_t ctr[4] = {a, b, c, e}, key[2] = {k0, k1}, o[4];
    oracle_philox4x32_10(ctr, key, o);
    double u1 = ((double)o[0] + 0.5) / 4294967296.0, u2 = ((double)o[1] + 0.5) / 4294967296.0;
    double rad = sqrt(-2.0 * log(u1));
    *z0 = rad * cos(2.0 * PI * u2);
    *z1 = rad * sin(2.0 * PI * u2);
}

/* ------------------------------------------------------------------------- */
/* Training frames of the learned filter: the layered model of Section 2     */
/* seen through the aperture.                                                 */
/*   phi_l(n): the DFT of layer l over its own M x M grid (pitch c_l delta,   */
/*     period 2 c_l T), complex normal with E|phi_l(n)|^2 =                   */
/*     M^4 (1/2) PSD_l(|n| / (2 c_l T)) / (2 c_l T)^2,                        */
/*     PSD_l(f) = 0.023 (r0 gamma_l^{-3/5})^{-5/3} (f^2 + L0^-2)^{-11/6}       */
/*     (von Karman; half the power per complex coefficient of a real screen; */
/*     zero at n = 0 and on the Nyquist row and column);                     */
/*   phi_l(-n) = conj(phi_l(n)), so each layer is real;                      */
/*   c_g(n) = sum_l exp(i omega n.(alpha_g h_l) / c_l) phi_l(n);               */
/*   psi_g = IDFT2(c_g) on the pupil (P x P at offset (M-P)/2, annulus mask   */
/*     of diameter D when D > 0), zero elsewhere, plus white noise of std     */
/*     noise x RMS of the masked noise-free psi_g on the pupil pixels;        */
/*   d_g = DFT2(psi_g).                                                      */
/* Random numbers: Philox4x32-10 and Box-Muller.  Frame F draws phi_l(j, k),  */
/* k < M/2, from counter (F, k M + j, l, 0), the row k = 0 taking j > M/2 as  */
/* the conjugate of M - j, and the noise at grid pixel (p, q) of star g from  */
/* the first normal of counter (F, p M + q, g, 1).                            */
/* ------------------------------------------------------------------------- */
typedef struct {
    int M, L, G, P;
    double T, D, obstruction, noise;
    const double *h, *c, *ax, *ay;
    uint32_t k0, k1;
    double *var;          /* [M/2][M][L] */
    unsigned char *mask;  /* [M][M] */
} frame_model;

static int frame_model_init(frame_model *fm, int M, double T, int L, const double *h, const double *c,
                            const double *gamma, int G, const double *ax, const double *ay, int P, double D,
                            double obstruction, double r0, double L0, double noise, uint32_t k0, uint32_t k1)
{
    if (M <= 0 || M % 2 || L <= 0 || G <= 0 || P <= 0 || P > M) return -1;
    const int Mh = M / 2;
    fm->M = M; fm->L = L; fm->G = G; fm->P = P; fm->T = T; fm->D = D; fm->obstruction = obstruction;
    fm->noise = noise; fm->h = h; fm->c = c; fm->ax = ax; fm->ay = ay; fm->k0 = k0; fm->k1 = k1;
    fm->var = (double *)malloc(sizeof(double) * (size_t)Mh * M * L);
    fm->mask = (unsigned char *)calloc((size_t)M * M, 1);
    for (int k = 0; k < Mh; ++k)
        for (int j = 0; j < M; ++j)
            for (int l = 0; l < L; ++l) {
                double v = 0;
                if (j != M / 2 && !(j == 0 && k == 0)) {
                    double nx = shifted_index(j, M), ny = k, per = 2.0 * c[l] * T;
                    double f2 = (nx * nx + ny * ny) / (per * per);
                    double r0l = r0 * pow(gamma[l], -3.0 / 5.0);
                    double psd = 0.023 * pow(r0l, -5.0 / 3.0) * pow(f2 + 1.0 / (L0 * L0), -11.0 / 6.0);
                    v = pow((double)M, 4) * 0.5 * psd / (per * per);
                }
                fm->var[((size_t)k * M + j) * L + l] = v;
            }
    unsigned char *pm = (unsigned char *)malloc((size_t)P * P);
    if (D > 0) oracle_pupil_mask(P, 2.0 * T / M, D, obstruction, pm);
    else memset(pm, 1, (size_t)P * P);
    const int o = (M - P) / 2;
    for (int a = 0; a < P; ++a)
        for (int b = 0; b < P; ++b) fm->mask[(size_t)(o + a) * M + o + b] = pm[(size_t)a * P + b];
    free(pm);
    return 0;
}

static void frame_model_free(frame_model *fm)
{
    free(fm->var);
    free(fm->mask);
}

/* phi [M/2][M][L] (stored half, k < M/2) and d [G][M][M] of frame F. */
static void frame_draw(const frame_model *fm, uint32_t F, cplx *phi, cplx *d)
{
    const int M = fm->M, Mh = M / 2, L = fm->L, G = fm->G;
    const double omega = PI / fm->T;
    for (int k = 0; k < Mh; ++k)
        for (int j = 0; j < M; ++j)
            for (int l = 0; l < L; ++l) {
                int flip = k == 0 && j > M / 2;
                int jj = flip ? M - j : j;
                double z0, z1, sd = sqrt(0.5 * fm->var[((size_t)k * M + jj) * L + l]);
                normal_pair(F, (uint32_t)(k * M + jj), (uint32_t)l, 0u, fm->k0, fm->k1, &z0, &z1);
                phi[((size_t)k * M + j) * L + l] = sd * z0 + I * (flip ? -sd * z1 : sd * z1);
            }
    cplx *cs = (cplx *)malloc(sizeof(cplx) * (size_t)M * M);
    cplx *ps = (cplx *)malloc(sizeof(cplx) * (size_t)M * M);
    for (int g = 0; g < G; ++g) {
        for (int j = 0; j < M; ++j)
            for (int k = 0; k < M; ++k) {
                cplx v = 0;
                if (j != M / 2 && k != M / 2) {
                    /* phi at n or, for k > M/2, the conjugate of phi at -n */
                    int neg = k > M / 2;
                    int js = neg ? (M - j) % M : j, ks = neg ? M - k : k;
                    double nx = shifted_index(j, M), ny = shifted_index(k, M);
                    for (int l = 0; l < L; ++l) {
                        cplx p = phi[((size_t)ks * M + js) * L + l];
                        if (neg) p = conj(p);
                        double arg = omega * (nx * fm->ax[g] * fm->h[l] + ny * fm->ay[g] * fm->h[l]) / fm->c[l];
                        v += (cos(arg) + I * sin(arg)) * p;
                    }
                }
                cs[(size_t)j * M + k] = v;
            }
        oracle_dft2(M, cs, ps, 1);
        double s2 = 0;
        int cnt = 0;
        for (int i = 0; i < M * M; ++i) {
            double v = fm->mask[i] ? creal(ps[i]) : 0.0;
            ps[i] = v;
            if (fm->mask[i]) {
                s2 += v * v;
                ++cnt;
            }
        }
        double sigma = cnt ? fm->noise * sqrt(s2 / cnt) : 0.0;
        if (sigma > 0)
            for (int i = 0; i < M * M; ++i)
                if (fm->mask[i]) {
                    double z0, z1;
                    normal_pair(F, (uint32_t)i, (uint32_t)g, 1u, fm->k0, fm->k1, &z0, &z1);
                    ps[i] += sigma * z0;
                }
        oracle_dft2(M, ps, d + (size_t)g * M * M, 0);
    }
    free(cs);
    free(ps);
}

int oracle_filter_frame(int M, double T, int L, const double *h, const double *c, const double *gamma, int G,
                        const double *ax, const double *ay, int P, double D, double obstruction, double r0,
                        double L0, double noise_level, uint32_t k0, uint32_t k1, uint32_t F, cplx *phi, cplx *d)
{
    frame_model fm;
    if (frame_model_init(&fm, M, T, L, h, c, gamma, G, ax, ay, P, D, obstruction, r0, L0, noise_level, k0, k1))
        return -1;
    frame_draw(&fm, F, phi, d);
    frame_model_free(&fm);
    return 0;
}

/* loss = sum_frames sum_n w_n sum_l |sum_g B_n[l][g] d_g(n) - phi_l(n)|^2 and       */
/* energy = sum_frames sum_n w_n sum_l |phi_l(n)|^2 over the stored frequencies      */
/* (k < M/2, j != M/2; w_n = 1 on the row k = 0, which holds both n and -n, else 2). */
/* B is [M][M][L][G] over (j, k) as oracle_group_B gives it.  Frames                 */
/* (frame0 + i) mod nwrap, i < nframes.                                              */
int oracle_filter_frames_loss(int M, double T, int L, const double *h, const double *c, const double *gamma,
                              int G, const double *ax, const double *ay, const cplx *B, int P, double D,
                              double obstruction, double r0, double L0, double noise_level, uint32_t k0,
                              uint32_t k1, uint32_t frame0, uint32_t nwrap, int nframes, double *loss,
                              double *energy)
{
    if (nwrap == 0 || nframes < 0) return -1;
    frame_model fm;
    if (frame_model_init(&fm, M, T, L, h, c, gamma, G, ax, ay, P, D, obstruction, r0, L0, noise_level, k0, k1))
        return -1;
    const int Mh = M / 2;
    double *fl = (double *)calloc((size_t)(nframes > 0 ? nframes : 1), sizeof(double));
    double *fe = (double *)calloc((size_t)(nframes > 0 ? nframes : 1), sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int fr = 0; fr < nframes; ++fr) {
        uint32_t F = (uint32_t)((frame0 + (uint32_t)fr) % nwrap);
        cplx *phi = (cplx *)malloc(sizeof(cplx) * (size_t)Mh * M * L);
        cplx *d = (cplx *)malloc(sizeof(cplx) * (size_t)G * M * M);
        frame_draw(&fm, F, phi, d);
        double tl = 0, te = 0;
        for (int k = 0; k < Mh; ++k)
            for (int j = 0; j < M; ++j) {
                if (j == M / 2) continue;
                double wn = k == 0 ? 1.0 : 2.0;
                const cplx *Bf = B + ((size_t)j * M + k) * L * G;
                for (int l = 0; l < L; ++l) {
                    cplx rec = 0;
                    for (int g = 0; g < G; ++g) rec += Bf[l * G + g] * d[(size_t)g * M * M + (size_t)j * M + k];
                    cplx p = phi[((size_t)k * M + j) * L + l];
                    cplx e = rec - p;
                    tl += wn * (creal(e) * creal(e) + cimag(e) * cimag(e));
                    te += wn * (creal(p) * creal(p) + cimag(p) * cimag(p));
                }
            }
        fl[fr] = tl;
        fe[fr] = te;
        free(phi);
        free(d);
    }
    double tl = 0, te = 0;
    for (int fr = 0; fr < nframes; ++fr) { /* in frame order */
        tl += fl[fr];
        te += fe[fr];
    }
    frame_model_free(&fm);
    free(fl);
    free(fe);
    *loss = tl;
    *energy = te;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Pseudo open loop control (Algorithm 3, line 2) and the integrator (line 5). */
/* POLC: out_g = mask (psi_g + A_g a), (A_g a)(r) = sum_l a_l(c_l r + alpha_g h_l) */
/* (Eq. defAperonly), at the pupil sample r = delta (o + p - M/2) per axis     */
/* (o = (M - P)/2), the layers a_l known at the output-grid samples: metric    */
/* grid x = delta (u - M/2), native grid x = c_l delta (u - M/2), periodic     */
/* with M samples, interpolated bilinearly between the four neighbours.        */
/* Integrator: a <- (1 - gain) a + gain phi.                                    */
/* ------------------------------------------------------------------------- */
static double bilinear_periodic(const double *a, int M, double u, double v)
{
    double fu = floor(u), fv = floor(v);
    double wu = u - fu, wv = v - fv;
    long i0 = ((long)fu % M + M) % M, j0 = ((long)fv % M + M) % M;
    long i1 = (i0 + 1) % M, j1 = (j0 + 1) % M;
    return (1 - wu) * ((1 - wv) * a[i0 * M + j0] + wv * a[i0 * M + j1]) +
           wu * ((1 - wv) * a[i1 * M + j0] + wv * a[i1 * M + j1]);
}

int oracle_polc(int M, int P, double delta, double D, double obstruction, int L, const double *h, int G,
                const double *ax, const double *ay, const int *kind, double h_lgs, int output_metric,
                const double *psi, const double *a, double *out)
{
    if (M <= 0 || P <= 0 || P > M || L <= 0 || G <= 0) return -1;
    unsigned char *mask = (unsigned char *)malloc((size_t)P * P);
    oracle_pupil_mask(P, delta, D, obstruction, mask);
    const int o = (M - P) / 2;
    double *c = (double *)malloc(sizeof(double) * L);
    for (int g = 0; g < G; ++g) {
        oracle_cone(L, h, h_lgs, kind[g] == 1, c);
        for (int p = 0; p < P; ++p)
            for (int q = 0; q < P; ++q) {
                size_t i = ((size_t)g * P + p) * P + q;
                if (!mask[p * P + q]) {
                    out[i] = 0.0;
                    continue;
                }
                double rx = delta * (o + p - M / 2.0), ry = delta * (o + q - M / 2.0);
                double acc = psi[i];
                for (int l = 0; l < L; ++l) {
                    double X = c[l] * rx + ax[g] * h[l], Y = c[l] * ry + ay[g] * h[l];
                    double pitch = output_metric ? delta : c[l] * delta;
                    acc += bilinear_periodic(a + (size_t)l * M * M, M, M / 2.0 + X / pitch, M / 2.0 + Y / pitch);
                }
                out[i] = acc;
            }
    }
    free(mask);
    free(c);
    return 0;
}

void oracle_integrate(long n, const double *phi, double *a, double gain)
{
    for (long i = 0; i < n; ++i) a[i] = (1.0 - gain) * a[i] + gain * phi[i];
}
