/*
 * fdm_oracle.c -- plain, slow, FP64 CPU oracle for the field-dislocation-mechanics
 * (FDM) layer-case time step of Morin, Brenner & Suquet, "Numerical simulation of
 * model problems in plasticity based on field dislocation mechanics" (arXiv 1911.03225).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  It shares no code, header, table or
 * helper with the CUDA path and never calls it.
 *
 * What it computes, in the paper's order (section 3, "General resolution procedure"):
 *   1. static problem (Sec. 3.1.2, Eq. for sigma-hat, and Sec. 3.2.1 layer reduction):
 *        tau13 = IFFT( K(xi1,xi2) * FFT(U13) ) + sigma_bar13
 *      where K is the layer average of the homogeneous isotropic Green-operator stress
 *      symbol m(xi) over the 3-D cell (derivation in oracle_kernel_table below);
 *   2. celerity v0 = (tau_y cos(U13/beta) - tau13)/eta~ (Sec. 3.2.2, Hamiltonian H),
 *      or a prescribed uniform v0 (Sec. 4.1);
 *   3. time step from the CFL rule |v0| dt/dx = CFL (Sec. 4.2, Sec. 5.2);
 *   4. the Kurganov-Noelle-Petrova central-upwind Hamilton-Jacobi update
 *      (Sec. 3.2.2 Steps 1-4 in 1-D, Sec. 3.2.3 Steps 1-4 in 2-D);
 *   5. macroscopic loading update (Sec. 5.1: zero mean stress, strain ramp).
 *
 * Readings of passages the paper leaves open (each also listed in the design notes):
 *   G1  2-D projection weights: the 1-D projection of Sec. 3.2.2 Step 4 applied in x and
 *       in y (a bilinear interpolation between the four intermediate points); the mixed
 *       a-b+ and a+b- terms therefore carry a minus sign.
 *   G2  2-D interpolant: on the quadrant cell next to the node, the limited row quadratic
 *       plus the limited column quadratic plus the bilinear cross term.
 *   G3  time level: default = midpoint rule (gradient advanced by dt/2 with the local
 *       Hessian of the interpolant); option "literal" evaluates H at t^n as printed.
 *   G4  one-sided speeds are the max/min over all four (phi_x^s, phi_y^t) pairs.
 *   G5  a+ = a- (= 0): the two intermediate points coincide; weights 1/2, 1/2.
 *   G6  dH/dp at grad phi = 0 is 0.
 *   G7  v0 is the node's value from the previous static solve; grad v0 is ignored.
 *   G8  continuous frequencies xi = 2 pi k~/(N dx); even symbols kept at Nyquist, odd
 *       symbols (curl-inverse, spectral derivative) zeroed there; a stress symbol of the
 *       3-D cell odd in one direction is zeroed at that axis's Nyquist index.
 *   G9  layer of nh voxels in a cubic periodic cell of nz voxels.
 *   G10 strain control: sigma_bar13 = 2 mu eps_bar13 - mu (nh/nz) <U13>.
 *
 * Layout: every 2-D field is row-major [n2][n1] (x1 fastest), FP64.
 *
 * Threads: built with OpenMP, the loops over independent rows, columns and nodes (the
 * 2-D transform, the kernel table, the 2-D transport step) are split across threads.
 * Every value is still computed by the same sequence of operations as in one thread, and
 * every sum keeps its serial order, so results do not depend on the thread count
 * (oracle_set_threads; 1 = the plain serial program).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 1;   /* threads of the parallel loops (1 = serial) */

/* Sets the thread count of the parallel loops (n < 1: all available); returns the count
 * in effect, 1 when the library was built without OpenMP. */
int oracle_set_threads(int n)
{
#ifdef _OPENMP
    g_threads = n >= 1 ? n : omp_get_num_procs();
#else
    (void)n;
    g_threads = 1;
#endif
    return g_threads;
}

int oracle_threads(void) { return g_threads; }

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------- */
/* Complex FFT: textbook iterative radix-2 Cooley-Tukey (decimation in time).  */
/* sign = -1 forward, +1 inverse; unnormalised.  n must be a power of two.     */
/* ------------------------------------------------------------------------- */
static int is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

void oracle_fft1d(int n, double *re, double *im, int sign)
{
    /* bit-reversal permutation */
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    /* butterflies */
    for (int len = 2; len <= n; len <<= 1) {
        int half = len >> 1;
        for (int k = 0; k < half; k++) {
            double ang = sign * 2.0 * OR_PI * (double)k / (double)len;
            double wr = cos(ang), wi = sin(ang);
            for (int s = 0; s < n; s += len) {
                int a = s + k, b = s + k + half;
                double xr = re[b] * wr - im[b] * wi;
                double xi = re[b] * wi + im[b] * wr;
                re[b] = re[a] - xr; im[b] = im[a] - xi;
                re[a] = re[a] + xr; im[a] = im[a] + xi;
            }
        }
    }
}

/* 2-D transform of a complex [n2][n1] array: all rows, then all columns. */
void oracle_fft2d(int n1, int n2, double *re, double *im, int sign)
{
#pragma omp parallel for schedule(static) num_threads(g_threads) if (g_threads > 1)
    for (int y = 0; y < n2; y++) oracle_fft1d(n1, re + (size_t)y * n1, im + (size_t)y * n1, sign);
#pragma omp parallel num_threads(g_threads) if (g_threads > 1)
    {
        double *cr = malloc(sizeof(double) * n2), *ci = malloc(sizeof(double) * n2);
#pragma omp for schedule(static)
        for (int x = 0; x < n1; x++) {
            for (int y = 0; y < n2; y++) { cr[y] = re[(size_t)y * n1 + x]; ci[y] = im[(size_t)y * n1 + x]; }
            oracle_fft1d(n2, cr, ci, sign);
            for (int y = 0; y < n2; y++) { re[(size_t)y * n1 + x] = cr[y]; im[(size_t)y * n1 + x] = ci[y]; }
        }
        free(cr); free(ci);
    }
}

/* signed frequency index k~ in (-n/2, n/2]; at Nyquist k~ = +n/2 */
static int signed_index(int k, int n) { return (k <= n / 2) ? k : k - n; }

/* ------------------------------------------------------------------------- */
/* Static problem (Sec. 3.1.2 and Sec. 3.2.1).                                 */
/* ------------------------------------------------------------------------- */

/*
 * Green-operator stress symbol for U^p = U13 e1 (x) e3 in an isotropic medium.
 * From sigma-hat = (C0:Gamma0-hat - I):C0:U^p-hat (Sec. 3.1.2) with
 * Gamma0-hat = [xi (x) (xi.C0.xi)^-1 (x) xi]^(s):  the polarisation stress is
 * s = 2 mu sym(U^p); with n = xi/|xi|,
 *   eps13-hat = U/2 (n1^2 + n3^2) - 2 mu kappa n1^2 n3^2 U,  kappa = (lambda+mu)/(mu(lambda+2mu)),
 *   sigma13-hat = 2 mu (eps13-hat - U/2) = m(n) U,
 *   m(n) = -mu [ n2^2 + 2 n1^2 n3^2 / (1 - nu) ].
 */
double oracle_layer_symbol(double n1, double n2, double n3, double mu, double nu)
{
    return -mu * (n2 * n2 + 2.0 * n1 * n1 * n3 * n3 / (1.0 - nu));
}

/*
 * K(xi1,xi2): layer average (Sec. 3.2.1, tau13 = (1/h) int sigma13 dx3) of the 3-D
 * stress produced by U13(x1,x2) chi(x3), chi = indicator of nh contiguous voxels of a
 * periodic cell nz voxels deep (G9):
 *   tau13-hat(xi1,xi2) = U13-hat * (1/(nz nh)) sum_k3 m(xi1,xi2,xi3) |chi-hat(k3)|^2,
 *   |chi-hat(k3)|^2 = sin^2(pi k3 nh / nz) / sin^2(pi k3 / nz)   (= nh^2 at k3 = 0).
 * The (0,0,0) mode is excluded (it carries the macroscopic stress).  Output [n2][n1].
 */
void oracle_kernel_table(int n1, int n2, int nz, int nh, double mu, double nu, double *K)
{
#pragma omp parallel for schedule(dynamic, 4) num_threads(g_threads) if (g_threads > 1)
    for (int k2 = 0; k2 < n2; k2++) {
        for (int k1 = 0; k1 < n1; k1++) {
            /* frequencies on a cubic-voxel grid (dx cancels in the direction n) */
            double x1 = (double)signed_index(k1, n1) / (double)n1;
            double x2 = (double)signed_index(k2, n2) / (double)n2;
            double acc = 0.0;
            for (int k3 = 0; k3 < nz; k3++) {
                double x3 = (double)signed_index(k3, nz) / (double)nz;
                double r2 = x1 * x1 + x2 * x2 + x3 * x3;
                if (r2 == 0.0) continue;
                double r = sqrt(r2);
                double w;
                if (k3 == 0) {
                    w = (double)nh * (double)nh;
                } else {
                    double sn = sin(OR_PI * (double)k3 * (double)nh / (double)nz);
                    double sd = sin(OR_PI * (double)k3 / (double)nz);
                    w = (sn * sn) / (sd * sd);
                }
                acc += oracle_layer_symbol(x1 / r, x2 / r, x3 / r, mu, nu) * w;
            }
            K[(size_t)k2 * n1 + k1] = acc / ((double)nz * (double)nh);
        }
    }
}

/* tau13 = IFFT2(K * FFT2(U13)) + sigma_bar13 (mean of tau13 = sigma_bar13, Sec. 3.1.2). */
void oracle_static_tau(int n1, int n2, const double *up13, const double *K, double sigma_bar13,
                       double *tau13)
{
    size_t n = (size_t)n1 * n2;
    double *re = malloc(sizeof(double) * n), *im = calloc(n, sizeof(double));
    memcpy(re, up13, sizeof(double) * n);
    oracle_fft2d(n1, n2, re, im, -1);
    for (size_t i = 0; i < n; i++) { re[i] *= K[i]; im[i] *= K[i]; }
    re[0] = sigma_bar13 * (double)n;
    im[0] = 0.0;
    oracle_fft2d(n1, n2, re, im, +1);
    for (size_t i = 0; i < n; i++) tau13[i] = re[i] / (double)n;
    free(re); free(im);
}

/*
 * sigma13 on chosen planes of the 3-D periodic cell (Sec. 3.1.2 static problem on the cell
 * of nz voxels, Sec. 3.2.1 layer): U^p = U13(x1, x2) chi(x3) e1 (x) e3, chi = 1 on the planes
 * x3 = 0 .. nh-1.  The 3-D transform of the layered field is U13-hat(k1, k2) chi-hat(k3),
 * chi-hat(k3) = sum_{j < nh} exp(-2 pi i k3 j / nz); sigma13-hat = m(xi) U^p-hat for xi != 0
 * and the macroscopic stress at xi = 0.  The inverse 3-D transform is evaluated at each
 * requested plane x3: the sum over k3 first, then the inverse 2-D transform.
 * out: [nplanes][n2][n1].
 */
void oracle_stress13_planes(int n1, int n2, int nz, int nh, double mu, double nu, const double *up13,
                            double sigma_bar13, int nplanes, const int *planes, double *out)
{
    size_t n = (size_t)n1 * n2;
    double *ur = malloc(sizeof(double) * n), *ui = calloc(n, sizeof(double));
    double *re = malloc(sizeof(double) * n), *im = malloc(sizeof(double) * n);
    double *cr = malloc(sizeof(double) * nz), *ci = malloc(sizeof(double) * nz);
    memcpy(ur, up13, sizeof(double) * n);
    oracle_fft2d(n1, n2, ur, ui, -1);
    for (int k3 = 0; k3 < nz; k3++) {      /* chi-hat(k3), summed term by term */
        cr[k3] = 0.0;
        ci[k3] = 0.0;
        for (int j = 0; j < nh; j++) {
            double a = -2.0 * OR_PI * (double)k3 * (double)j / (double)nz;
            cr[k3] += cos(a);
            ci[k3] += sin(a);
        }
    }
    for (int ip = 0; ip < nplanes; ip++) {
        int x3 = planes[ip];
        for (int k2 = 0; k2 < n2; k2++) {
            for (int k1 = 0; k1 < n1; k1++) {
                double x1 = (double)signed_index(k1, n1) / (double)n1;
                double x2 = (double)signed_index(k2, n2) / (double)n2;
                double sr = 0.0, si = 0.0;   /* sum over k3 of m chi-hat exp(2 pi i k3 x3 / nz) */
                for (int k3 = 0; k3 < nz; k3++) {
                    double z3 = (double)signed_index(k3, nz) / (double)nz;
                    double r2 = x1 * x1 + x2 * x2 + z3 * z3;
                    if (r2 == 0.0) continue;
                    double r = sqrt(r2);
                    double m = oracle_layer_symbol(x1 / r, x2 / r, z3 / r, mu, nu);
                    double a = 2.0 * OR_PI * (double)k3 * (double)x3 / (double)nz;
                    double er = cos(a), ei = sin(a);
                    sr += m * (cr[k3] * er - ci[k3] * ei);
                    si += m * (cr[k3] * ei + ci[k3] * er);
                }
                size_t i = (size_t)k2 * n1 + k1;
                re[i] = (sr * ur[i] - si * ui[i]) / (double)nz;
                im[i] = (sr * ui[i] + si * ur[i]) / (double)nz;
            }
        }
        re[0] = sigma_bar13 * (double)n;   /* xi = 0: the macroscopic stress */
        im[0] = 0.0;
        oracle_fft2d(n1, n2, re, im, +1);
        for (size_t i = 0; i < n; i++) out[(size_t)ip * n + i] = re[i] / (double)n;
    }
    free(ur); free(ui); free(re); free(im); free(cr); free(ci);
}

/*
 * Every component of the stress of the layered eigen-distortion (Sec. 3.1.2), for the
 * Voigt index comp: 0 = 11, 1 = 22, 2 = 33, 3 = 23, 4 = 13, 5 = 12.  With n = xi/|xi| the
 * Green operator Gamma0-hat = [xi (x) (xi.C0.xi)^-1 (x) xi]^(s) applied to the polarisation
 * C0:U^p-hat = mu U (e1 (x) e3 + e3 (x) e1) gives the strain
 *   eps-hat = sym(h (x) n),   h = (1/mu) (I - n (x) n / (2 (1 - nu))) (C0:U^p-hat) n,
 * because (xi.C0.xi)^-1 = (I - c n (x) n)/(mu |xi|^2) with c = (lambda + mu)/(lambda + 2 mu)
 * = 1/(2 (1 - nu)); the stress is sigma-hat = lambda tr(eps-hat) I + 2 mu (eps-hat - eps^p),
 * eps^p = sym(U^p) (trace free).  Returns sigma-hat_comp / U-hat for U-hat = 1.
 */
static const int voigt_i[6] = {0, 1, 2, 1, 0, 0}, voigt_j[6] = {0, 1, 2, 2, 2, 1};

double oracle_stress_symbol(int comp, double n1, double n2, double n3, double mu, double nu)
{
    const double n[3] = {n1, n2, n3};
    const double lam = 2.0 * mu * nu / (1.0 - 2.0 * nu);
    const double c = 1.0 / (2.0 * (1.0 - nu));
    const double sn[3] = {n3, 0.0, n1};             /* (C0:U^p-hat) n / mu */
    const double ns = n1 * sn[0] + n2 * sn[1] + n3 * sn[2];
    double h[3];
    for (int a = 0; a < 3; a++) h[a] = sn[a] - c * n[a] * ns;
    const int i = voigt_i[comp], j = voigt_j[comp];
    const double tr = h[0] * n[0] + h[1] * n[1] + h[2] * n[2];
    double s = mu * (h[i] * n[j] + h[j] * n[i]);
    if (i == j) s += lam * tr;
    if (comp == 4) s -= mu;                         /* 2 mu eps^p_13 = mu U */
    return s;
}

/*
 * Parity of the component's symbol in (n1, n2, n3): 1 where it is odd in that direction.
 * (h is linear in n3 and n1 through C0:U^p, so 11, 22 and 33 carry n1 n3, 12 carries n2 n3,
 * 23 carries n1 n2, and 13 is even in all three.)  Reading G8 extended: a symbol odd in a
 * direction has no value at that axis's Nyquist index, so the term is dropped there.
 */
static const int stress_odd[6][3] = {{1, 0, 1}, {1, 0, 1}, {1, 0, 1}, {1, 1, 0}, {0, 0, 0}, {0, 1, 1}};

/*
 * One stress component on chosen planes of the 3-D periodic cell (Sec. 3.1.2 on the cell of
 * nz voxels, Sec. 3.2.1 layer on planes 0 .. nh-1): the 3-D transform of U13(x1, x2) chi(x3)
 * multiplied by the component's symbol term by term, then the inverse transform evaluated
 * at each plane, the sum over k3 first.  The xi = 0 term is the macroscopic stress:
 * sigma_bar13 for comp 4, zero otherwise (the loading only prescribes the 13 component and
 * U^p has no other mean part).  out: [nplanes][n2][n1].
 */
void oracle_stress_planes(int n1, int n2, int nz, int nh, double mu, double nu, const double *up13,
                          double sigma_bar13, int comp, int nplanes, const int *planes, double *out)
{
    size_t n = (size_t)n1 * n2;
    const int *odd = stress_odd[comp];
    double *ur = malloc(sizeof(double) * n), *ui = calloc(n, sizeof(double));
    double *re = malloc(sizeof(double) * n), *im = malloc(sizeof(double) * n);
    double *cr = malloc(sizeof(double) * nz), *ci = malloc(sizeof(double) * nz);
    memcpy(ur, up13, sizeof(double) * n);
    oracle_fft2d(n1, n2, ur, ui, -1);
    for (int k3 = 0; k3 < nz; k3++) {      /* chi-hat(k3), summed term by term */
        cr[k3] = 0.0;
        ci[k3] = 0.0;
        for (int j = 0; j < nh; j++) {
            double a = -2.0 * OR_PI * (double)k3 * (double)j / (double)nz;
            cr[k3] += cos(a);
            ci[k3] += sin(a);
        }
    }
    for (int ip = 0; ip < nplanes; ip++) {
        int x3 = planes[ip];
        for (int k2 = 0; k2 < n2; k2++) {
            for (int k1 = 0; k1 < n1; k1++) {
                size_t i = (size_t)k2 * n1 + k1;
                re[i] = 0.0;
                im[i] = 0.0;
                if ((odd[0] && 2 * k1 == n1) || (odd[1] && 2 * k2 == n2)) continue;
                double x1 = (double)signed_index(k1, n1) / (double)n1;
                double x2 = (double)signed_index(k2, n2) / (double)n2;
                double sr = 0.0, si = 0.0;
                for (int k3 = 0; k3 < nz; k3++) {
                    if (odd[2] && 2 * k3 == nz) continue;
                    double z3 = (double)signed_index(k3, nz) / (double)nz;
                    double r2 = x1 * x1 + x2 * x2 + z3 * z3;
                    if (r2 == 0.0) continue;
                    double r = sqrt(r2);
                    double m = oracle_stress_symbol(comp, x1 / r, x2 / r, z3 / r, mu, nu);
                    double a = 2.0 * OR_PI * (double)k3 * (double)x3 / (double)nz;
                    double er = cos(a), ei = sin(a);
                    sr += m * (cr[k3] * er - ci[k3] * ei);
                    si += m * (cr[k3] * ei + ci[k3] * er);
                }
                re[i] = (sr * ur[i] - si * ui[i]) / (double)nz;
                im[i] = (sr * ui[i] + si * ur[i]) / (double)nz;
            }
        }
        re[0] = comp == 4 ? sigma_bar13 * (double)n : 0.0;
        im[0] = 0.0;
        oracle_fft2d(n1, n2, re, im, +1);
        for (size_t i = 0; i < n; i++) out[(size_t)ip * n + i] = re[i] / (double)n;
    }
    free(ur); free(ui); free(re); free(im); free(cr); free(ci);
}

/*
 * Curl inverse (Sec. 3.1.2, U^p-hat = i (alpha-hat x xi)/|xi|^2; Sec. 2.2 Poisson problem):
 * for the layer ansatz alpha = a11 e1(x)e1 + a12 e1(x)e2 (Sec. 3.2.1) the 13 component is
 *   U13-hat = i (a11-hat xi2 - a12-hat xi1) / |xi|^2,   U13-hat(0) = mean_up13 * N.
 * Odd multipliers are zeroed at their Nyquist index (G8).  Returns the relative
 * divergence residual |xi1 a11-hat + xi2 a12-hat| / |alpha-hat| (div alpha = 0, Sec. 2.1)
 * and writes the mean of (a11, a12) to mean_alpha[2] (net Burgers vector / area).
 */
double oracle_curl_inverse(int n1, int n2, double dx, const double *a11, const double *a12,
                           double mean_up13, double *up13, double *mean_alpha)
{
    size_t n = (size_t)n1 * n2;
    double *r11 = malloc(sizeof(double) * n), *i11 = calloc(n, sizeof(double));
    double *r12 = malloc(sizeof(double) * n), *i12 = calloc(n, sizeof(double));
    memcpy(r11, a11, sizeof(double) * n);
    memcpy(r12, a12, sizeof(double) * n);
    oracle_fft2d(n1, n2, r11, i11, -1);
    oracle_fft2d(n1, n2, r12, i12, -1);
    if (mean_alpha) { mean_alpha[0] = r11[0] / (double)n; mean_alpha[1] = r12[0] / (double)n; }
    double num = 0.0, den = 0.0;
    double *pr = malloc(sizeof(double) * n), *pi = malloc(sizeof(double) * n);
    for (int k2 = 0; k2 < n2; k2++) {
        for (int k1 = 0; k1 < n1; k1++) {
            size_t i = (size_t)k2 * n1 + k1;
            double xi1 = 2.0 * OR_PI * signed_index(k1, n1) / (n1 * dx);
            double xi2 = 2.0 * OR_PI * signed_index(k2, n2) / (n2 * dx);
            double o1 = (2 * k1 == n1) ? 0.0 : xi1; /* odd use of xi1 */
            double o2 = (2 * k2 == n2) ? 0.0 : xi2; /* odd use of xi2 */
            double dr = o1 * r11[i] + o2 * r12[i], di = o1 * i11[i] + o2 * i12[i];
            num += dr * dr + di * di;
            den += (o1 * o1 + o2 * o2) * (r11[i] * r11[i] + i11[i] * i11[i] + r12[i] * r12[i] + i12[i] * i12[i]);
            double q = xi1 * xi1 + xi2 * xi2;
            if (q == 0.0) { pr[i] = 0.0; pi[i] = 0.0; continue; }
            /* w = a11 xi2 - a12 xi1 ; U = i w / q */
            double wr = r11[i] * o2 - r12[i] * o1;
            double wi = i11[i] * o2 - i12[i] * o1;
            pr[i] = -wi / q;
            pi[i] = wr / q;
        }
    }
    pr[0] = mean_up13 * (double)n;
    pi[0] = 0.0;
    oracle_fft2d(n1, n2, pr, pi, +1);
    for (size_t i = 0; i < n; i++) up13[i] = pr[i] / (double)n;
    free(r11); free(i11); free(r12); free(i12); free(pr); free(pi);
    return den > 0.0 ? sqrt(num / den) : 0.0;
}

/* alpha11 = -d2 U13, alpha12 = d1 U13 (Sec. 3.2.1), spectral derivatives, odd symbol
 * zeroed at Nyquist (G8). */
void oracle_alpha_from_up(int n1, int n2, double dx, const double *up13, double *a11, double *a12)
{
    size_t n = (size_t)n1 * n2;
    double *re = malloc(sizeof(double) * n), *im = calloc(n, sizeof(double));
    double *br = malloc(sizeof(double) * n), *bi = malloc(sizeof(double) * n);
    memcpy(re, up13, sizeof(double) * n);
    oracle_fft2d(n1, n2, re, im, -1);
    /* a12 = i xi1 U */
    for (int k2 = 0; k2 < n2; k2++)
        for (int k1 = 0; k1 < n1; k1++) {
            size_t i = (size_t)k2 * n1 + k1;
            double xi1 = (2 * k1 == n1) ? 0.0 : 2.0 * OR_PI * signed_index(k1, n1) / (n1 * dx);
            br[i] = -xi1 * im[i];
            bi[i] = xi1 * re[i];
        }
    oracle_fft2d(n1, n2, br, bi, +1);
    for (size_t i = 0; i < n; i++) a12[i] = br[i] / (double)n;
    /* a11 = -i xi2 U */
    for (int k2 = 0; k2 < n2; k2++)
        for (int k1 = 0; k1 < n1; k1++) {
            size_t i = (size_t)k2 * n1 + k1;
            double xi2 = (2 * k2 == n2) ? 0.0 : 2.0 * OR_PI * signed_index(k2, n2) / (n2 * dx);
            br[i] = xi2 * im[i];
            bi[i] = -xi2 * re[i];
        }
    oracle_fft2d(n1, n2, br, bi, +1);
    for (size_t i = 0; i < n; i++) a11[i] = br[i] / (double)n;
    free(re); free(im); free(br); free(bi);
}

/* ------------------------------------------------------------------------- */
/* Transport: Kurganov-Noelle-Petrova central-upwind scheme (Sec. 3.2.2-3.2.3) */
/* ------------------------------------------------------------------------- */

/* minmod of three arguments (Sec. 3.2.2, Step 1) */
static double minmod3(double a, double b, double c)
{
    if (a > 0.0 && b > 0.0 && c > 0.0) return fmin(a, fmin(b, c));
    if (a < 0.0 && b < 0.0 && c < 0.0) return fmax(a, fmax(b, c));
    return 0.0;
}

/* limited second difference (Delta phi)'_{j+1/2} from the four first differences
 * D_{j-1/2}, D_{j+1/2}, D_{j+3/2} (Sec. 3.2.2 Step 1). */
static double limited_second(double theta, double d_m, double d_c, double d_p)
{
    return minmod3(theta * (d_p - d_c), 0.5 * (d_p - d_m), theta * (d_c - d_m));
}

static int wrap(int i, int n) { i %= n; return i < 0 ? i + n : i; }

/*
 * One 1-D KNP step (Sec. 3.2.2, Steps 1-4) for phi_t + v0 |phi_x| = 0 on a periodic
 * row of n nodes, v0 given per node.  time_level: 0 = midpoint (G3), 1 = literal.
 */
void oracle_knp1d_step(int n, double h, double theta, double dt, int time_level,
                       const double *phi, const double *v0, double *out)
{
    for (int j = 0; j < n; j++) {
        double f_m2 = phi[wrap(j - 2, n)], f_m1 = phi[wrap(j - 1, n)], f0 = phi[j];
        double f_p1 = phi[wrap(j + 1, n)], f_p2 = phi[wrap(j + 2, n)];
        double D_m3 = f_m1 - f_m2, D_m1 = f0 - f_m1, D_p1 = f_p1 - f0, D_p3 = f_p2 - f_p1;
        double S_p = limited_second(theta, D_m1, D_p1, D_p3); /* (Delta phi)'_{j+1/2} */
        double S_m = limited_second(theta, D_m3, D_m1, D_p1); /* (Delta phi)'_{j-1/2} */
        /* Step 2: one-sided derivatives and speeds, H'(p) = v0 sign(p) */
        double px_p = D_p1 / h - S_p / (2.0 * h);
        double px_m = D_m1 / h + S_m / (2.0 * h);
        double c = v0[j];
        double hp1 = (px_p > 0.0) ? c : (px_p < 0.0 ? -c : 0.0);
        double hp2 = (px_m > 0.0) ? c : (px_m < 0.0 ? -c : 0.0);
        double ap = fmax(fmax(hp1, hp2), 0.0), am = fmin(fmin(hp1, hp2), 0.0);
        /* Step 3: values at x_{j+-} = x_j + a+- dt */
        double res[2];
        for (int s = 0; s < 2; s++) {
            double d = (s == 0 ? ap : am) * dt;
            double val, der, curv;
            if (s == 0) { /* right cell [x_j, x_{j+1}] */
                val = f0 + D_p1 * d / h + S_p * d * (d - h) / (2.0 * h * h);
                der = D_p1 / h + S_p * (2.0 * d - h) / (2.0 * h * h);
                curv = S_p / (h * h);
            } else {      /* left cell [x_{j-1}, x_j] */
                val = f0 + D_m1 * d / h + S_m * d * (d + h) / (2.0 * h * h);
                der = D_m1 / h + S_m * (2.0 * d + h) / (2.0 * h * h);
                curv = S_m / (h * h);
            }
            if (time_level == 0) {
                double hprime = (der > 0.0) ? c : (der < 0.0 ? -c : 0.0);
                der -= 0.5 * dt * curv * hprime;
            }
            res[s] = val - dt * c * fabs(der);
        }
        /* Step 4: projection */
        double wp, wm;
        if (ap - am > 0.0) { wp = -am / (ap - am); wm = ap / (ap - am); }
        else { wp = 0.5; wm = 0.5; }
        out[j] = wm * res[1] + wp * res[0];
    }
}

/*
 * One 2-D KNP step (Sec. 3.2.3, Steps 1-4) for phi_t + v0 sqrt(phi_x^2 + phi_y^2) = 0,
 * periodic [n2][n1] grid, cell size h in both directions, v0 per node.
 */
void oracle_knp2d_step(int n1, int n2, double h, double theta, double dt, int time_level,
                       const double *phi, const double *v0, double *out)
{
#define P(jj, kk) phi[(size_t)wrap((kk), n2) * n1 + wrap((jj), n1)]
#pragma omp parallel for schedule(static) num_threads(g_threads) if (g_threads > 1)
    for (int k = 0; k < n2; k++) {
        for (int j = 0; j < n1; j++) {
            double f0 = P(j, k);
            /* Step 1, x: first differences and limited second differences along the row */
            double Dx_m3 = P(j - 1, k) - P(j - 2, k), Dx_m1 = f0 - P(j - 1, k);
            double Dx_p1 = P(j + 1, k) - f0, Dx_p3 = P(j + 2, k) - P(j + 1, k);
            double Sx_p = limited_second(theta, Dx_m1, Dx_p1, Dx_p3);
            double Sx_m = limited_second(theta, Dx_m3, Dx_m1, Dx_p1);
            /* Step 1, y: same along the column */
            double Dy_m3 = P(j, k - 1) - P(j, k - 2), Dy_m1 = f0 - P(j, k - 1);
            double Dy_p1 = P(j, k + 1) - f0, Dy_p3 = P(j, k + 2) - P(j, k + 1);
            double Sy_p = limited_second(theta, Dy_m1, Dy_p1, Dy_p3);
            double Sy_m = limited_second(theta, Dy_m3, Dy_m1, Dy_p1);
            /* one-sided derivatives at the node */
            double px[2] = { Dx_p1 / h - Sx_p / (2.0 * h), Dx_m1 / h + Sx_m / (2.0 * h) };
            double qy[2] = { Dy_p1 / h - Sy_p / (2.0 * h), Dy_m1 / h + Sy_m / (2.0 * h) };
            double c = v0[(size_t)k * n1 + j];
            /* Step 2: one-sided speeds over the four (phi_x^s, phi_y^t) pairs (G4, G6) */
            double ap = 0.0, am = 0.0, bp = 0.0, bm = 0.0;
            for (int s = 0; s < 2; s++)
                for (int t = 0; t < 2; t++) {
                    double p = px[s], q = qy[t];
                    double r = sqrt(p * p + q * q);
                    double Hp = (r > 0.0) ? c * p / r : 0.0;
                    double Hq = (r > 0.0) ? c * q / r : 0.0;
                    ap = fmax(ap, Hp); am = fmin(am, Hp);
                    bp = fmax(bp, Hq); bm = fmin(bm, Hq);
                }
            /* Step 3: values at the four intermediate points (G2, G3) */
            double psi[2][2];
            for (int s = 0; s < 2; s++) {
                double dx = (s == 0 ? ap : am) * dt;
                int cx = (s == 0) ? 1 : -1;
                double X, dX, Sx;
                if (s == 0) {
                    X = Dx_p1 * dx / h + Sx_p * dx * (dx - h) / (2.0 * h * h);
                    dX = Dx_p1 / h + Sx_p * (2.0 * dx - h) / (2.0 * h * h);
                    Sx = Sx_p;
                } else {
                    X = Dx_m1 * dx / h + Sx_m * dx * (dx + h) / (2.0 * h * h);
                    dX = Dx_m1 / h + Sx_m * (2.0 * dx + h) / (2.0 * h * h);
                    Sx = Sx_m;
                }
                for (int t = 0; t < 2; t++) {
                    double dy = (t == 0 ? bp : bm) * dt;
                    int cy = (t == 0) ? 1 : -1;
                    double Y, dY, Sy;
                    if (t == 0) {
                        Y = Dy_p1 * dy / h + Sy_p * dy * (dy - h) / (2.0 * h * h);
                        dY = Dy_p1 / h + Sy_p * (2.0 * dy - h) / (2.0 * h * h);
                        Sy = Sy_p;
                    } else {
                        Y = Dy_m1 * dy / h + Sy_m * dy * (dy + h) / (2.0 * h * h);
                        dY = Dy_m1 / h + Sy_m * (2.0 * dy + h) / (2.0 * h * h);
                        Sy = Sy_m;
                    }
                    double cross = (P(j + cx, k + cy) - P(j + cx, k) - P(j, k + cy) + f0) /
                                   ((double)(cx * cy) * h * h);
                    double val = f0 + X + Y + cross * dx * dy;
                    double p = dX + cross * dy;
                    double q = dY + cross * dx;
                    if (time_level == 0) {
                        double r = sqrt(p * p + q * q);
                        double gx = (r > 0.0) ? c * p / r : 0.0;
                        double gy = (r > 0.0) ? c * q / r : 0.0;
                        double hxx = Sx / (h * h), hyy = Sy / (h * h);
                        double np = p - 0.5 * dt * (hxx * gx + cross * gy);
                        double nq = q - 0.5 * dt * (cross * gx + hyy * gy);
                        p = np; q = nq;
                    }
                    psi[s][t] = val - dt * c * sqrt(p * p + q * q);
                }
            }
            /* Step 4: projection, the 1-D weights in x and in y (G1, G5) */
            double wx[2], wy[2];
            if (ap - am > 0.0) { wx[0] = -am / (ap - am); wx[1] = ap / (ap - am); }
            else { wx[0] = 0.5; wx[1] = 0.5; }
            if (bp - bm > 0.0) { wy[0] = -bm / (bp - bm); wy[1] = bp / (bp - bm); }
            else { wy[0] = 0.5; wy[1] = 0.5; }
            out[(size_t)k * n1 + j] = wx[0] * wy[0] * psi[0][0] + wx[0] * wy[1] * psi[0][1] +
                                      wx[1] * wy[0] * psi[1][0] + wx[1] * wy[1] * psi[1][1];
        }
    }
#undef P
}

/* ------------------------------------------------------------------------- */
/* Reductions                                                                  */
/* ------------------------------------------------------------------------- */

/* Neumaier-compensated sum */
double oracle_sum(size_t n, const double *x)
{
    double s = 0.0, c = 0.0;
    for (size_t i = 0; i < n; i++) {
        double t = s + x[i];
        if (fabs(s) >= fabs(x[i])) c += (s - t) + x[i];
        else c += (x[i] - t) + s;
        s = t;
    }
    return s + c;
}

/*
 * Dislocation-density sums of the staggered (forward-difference) Nye components
 * a12 = (U_{j+1,k} - U_{jk})/h, a11 = -(U_{j,k+1} - U_{jk})/h (Sec. 3.2.1), over all nodes:
 * out[0] = sum a12>0, out[1] = sum a12<0, out[2] = sum a11>0, out[3] = sum a11<0,
 * out[4] = sum sqrt(a11^2 + a12^2).   The total Burgers vector per unit length
 * (Sec. 4.2, b = int alpha.n dS) is h^2 (out[0] + out[1]) resp. h^2 (out[2] + out[3]).
 */
void oracle_alpha_sums(int n1, int n2, double h, const double *up13, double *out)
{
    size_t n = (size_t)n1 * n2;
    double *t = malloc(sizeof(double) * n * 5);
    for (int k = 0; k < n2; k++)
        for (int j = 0; j < n1; j++) {
            size_t i = (size_t)k * n1 + j;
            double a12 = (up13[(size_t)k * n1 + wrap(j + 1, n1)] - up13[i]) / h;
            double a11 = -(up13[(size_t)wrap(k + 1, n2) * n1 + j] - up13[i]) / h;
            t[i] = a12 > 0.0 ? a12 : 0.0;
            t[n + i] = a12 < 0.0 ? a12 : 0.0;
            t[2 * n + i] = a11 > 0.0 ? a11 : 0.0;
            t[3 * n + i] = a11 < 0.0 ? a11 : 0.0;
            t[4 * n + i] = sqrt(a11 * a11 + a12 * a12);
        }
    for (int q = 0; q < 5; q++) out[q] = oracle_sum(n, t + q * n);
    free(t);
}

/* ------------------------------------------------------------------------- */
/* Full time step (Sec. 3.1.1: static problem with U^p_n, then transport).     */
/* ------------------------------------------------------------------------- */

/* parameter block, mirrored field by field by the ctypes wrapper */
typedef struct {
    int32_t n1, n2, nz, nh;
    double dx, E, nu;
    int32_t velocity_mode;      /* 0 prescribed uniform v0, 1 stress driven */
    double v0, mobility, tau_y, beta, theta, cfl, dt_max;
    int32_t loading_mode;       /* 0 stress (sigma_bar13), 1 strain ramp per step, 2 zero mean
                                   stress, 3 strain rate in time */
    double sigma_bar13, eps_bar13_0, eps_bar13_rate;
    int32_t time_level;         /* 0 midpoint, 1 literal */
} oracle_params;

/* scalar state carried between steps */
typedef struct {
    int64_t step;
    double t, dt, max_abs_v0, mean_up13, eps_bar13, sigma_bar13;
} oracle_scalars;

static double shear_modulus(const oracle_params *p) { return p->E / (2.0 * (1.0 + p->nu)); }

/* macroscopic stress at step `step`, time t (Sec. 3.1.2 sigma-hat(0); Sec. 5.1 loading
 * paths; G10).  Modes: 0 given stress; 1 strain ramp per step; 2 zero mean stress (the
 * equilibration stage of Sec. 5.1); 3 strain rate in time, eps = eps0 + rate t (Sec. 5.1). */
static void loading(const oracle_params *p, int64_t step, double t, double mean_up13, double *eps, double *sig)
{
    double mu = shear_modulus(p), frac = (double)p->nh / (double)p->nz;
    if (p->loading_mode == 0) {
        *sig = p->sigma_bar13;
        *eps = (p->sigma_bar13 + mu * frac * mean_up13) / (2.0 * mu);
    } else if (p->loading_mode == 1 || p->loading_mode == 3) {
        double x = p->loading_mode == 1 ? (double)step : t;
        *eps = p->eps_bar13_0 + p->eps_bar13_rate * x;
        *sig = 2.0 * mu * (*eps) - mu * frac * mean_up13;
    } else {
        *eps = 0.5 * frac * mean_up13;  /* eps_bar13 = <U13>/2 over the cell (Sec. 5.1) */
        *sig = 0.0;
    }
}

/*
 * Advance `nsteps` steps in place.  K is the table from oracle_kernel_table; tau13 and v0
 * (may be NULL) receive the fields of the last step's static solve.  mfac (may be NULL):
 * per-node mobility factor m(x) >= 0 multiplying the celerity -- a heterogeneous drag
 * eta(x) = eta~ / m(x), with m = 0 inside impenetrable precipitates (Sec. 5.3, Orowan
 * mechanism).  Returns 0, or 1 if a non-finite value appeared.
 */
int oracle_hetero_antiplane(int n1, int n2, const double *mu, const double *up13, int stress_control,
                            double load, double tol, int max_iter, double *sig13, double *sig23, double *res);

/* Static problem of one step: the layer solve with K, or, with a shear-modulus field mu, the
 * heterogeneous antiplane problem (stress control in loading modes 0 and 2, strain control
 * in modes 1 and 3). */
static void static_problem(const oracle_params *p, const double *K, const double *mu, double tol, int max_iter,
                           const double *up13, double eps, double sig, double *tau)
{
    if (!mu) {
        oracle_static_tau(p->n1, p->n2, up13, K, sig, tau);
        return;
    }
    int stress = p->loading_mode == 0 || p->loading_mode == 2;
    oracle_hetero_antiplane(p->n1, p->n2, mu, up13, stress, stress ? sig : eps, tol, max_iter, tau, NULL, NULL);
}

/* oracle_run with, when mu != NULL, the heterogeneous static problem of a shear-modulus
 * field mu (layer filling the cell) in every step, iterated as oracle_hetero_antiplane
 * with tol and max_iter. */
int oracle_run_hetero(const oracle_params *p, const double *K, double *up13, oracle_scalars *st,
                      int nsteps, double *tau_out, double *v0_out, const double *mfac,
                      const double *mu, double tol, int max_iter)
{
    int n1 = p->n1, n2 = p->n2;
    size_t n = (size_t)n1 * n2;
    double *tau = malloc(sizeof(double) * n), *v0 = malloc(sizeof(double) * n);
    double *nxt = malloc(sizeof(double) * n);
    int rc = 0;
    for (int it = 0; it < nsteps; it++) {
        double mean = oracle_sum(n, up13) / (double)n;
        double eps, sig;
        loading(p, st->step, st->t, mean, &eps, &sig);
        /* static problem with the previous plastic distortion (Sec. 3.1.1) */
        static_problem(p, K, mu, tol, max_iter, up13, eps, sig, tau);
        /* celerity (Sec. 3.2.3 Hamiltonian; Sec. 4.1 prescribed) */
        double vmax = 0.0;
        for (size_t i = 0; i < n; i++) {
            double c;
            if (p->velocity_mode == 0) c = p->v0;
            else {
                double fr = (p->tau_y != 0.0) ? p->tau_y * cos(up13[i] / p->beta) : 0.0;
                c = p->mobility * (fr - tau[i]);
            }
            if (mfac) c *= mfac[i];
            v0[i] = c;
            if (fabs(c) > vmax) vmax = fabs(c);
        }
        /* CFL time step (Sec. 5.2: dt adjusted to keep the CFL number) */
        double dt;
        if (vmax > 0.0) {
            dt = p->cfl * p->dx / vmax;
            if (p->dt_max > 0.0 && dt > p->dt_max) dt = p->dt_max;
        } else {
            dt = p->dt_max > 0.0 ? p->dt_max : 0.0;
        }
        oracle_knp2d_step(n1, n2, p->dx, p->theta, dt, p->time_level, up13, v0, nxt);
        memcpy(up13, nxt, sizeof(double) * n);
        st->step += 1;
        st->t += dt;
        st->dt = dt;
        st->max_abs_v0 = vmax;
        st->mean_up13 = oracle_sum(n, up13) / (double)n;
        /* loading state of the new step (used by the next static solve) */
        loading(p, st->step, st->t, st->mean_up13, &eps, &sig);
        st->eps_bar13 = eps;
        st->sigma_bar13 = sig;
        if (!isfinite(dt)) rc = 1;
    }
    if (nsteps == 0) {
        double mean = oracle_sum(n, up13) / (double)n, eps, sig;
        loading(p, st->step, st->t, mean, &eps, &sig);
        static_problem(p, K, mu, tol, max_iter, up13, eps, sig, tau);
        for (size_t i = 0; i < n; i++) {
            double fr = (p->tau_y != 0.0) ? p->tau_y * cos(up13[i] / p->beta) : 0.0;
            v0[i] = (p->velocity_mode == 0) ? p->v0 : p->mobility * (fr - tau[i]);
            if (mfac) v0[i] *= mfac[i];
        }
        st->mean_up13 = mean; st->eps_bar13 = eps; st->sigma_bar13 = sig;
    }
    for (size_t i = 0; i < n; i++) if (!isfinite(up13[i])) { rc = 1; break; }
    if (tau_out) memcpy(tau_out, tau, sizeof(double) * n);
    if (v0_out) memcpy(v0_out, v0, sizeof(double) * n);
    free(tau); free(v0); free(nxt);
    return rc;
}

int oracle_run(const oracle_params *p, const double *K, double *up13, oracle_scalars *st,
               int nsteps, double *tau_out, double *v0_out, const double *mfac)
{
    return oracle_run_hetero(p, K, up13, st, nsteps, tau_out, v0_out, mfac, NULL, 0.0, 0);
}

/*
 * Heterogeneous elasticity (Sec. 3.1.2, heterogeneous medium): static problem for a shear
 * modulus mu(x1, x2) that varies in the plane, with the plastic layer filling the cell
 * (nh = nz).  U^p = U13(x1, x2) e1 (x) e3 then does not vary along x3 and the problem is
 * antiplane shear: u = u3(x1, x2) e3, unknown g = grad u3, stresses
 *   sigma13 = mu (g1 - U13),   sigma23 = mu g2,   equilibrium d1 sigma13 + d2 sigma23 = 0.
 * With a reference medium mu0 the paper's polarisation is tau = (mu - mu0) g - mu (U13, 0) and
 * sigma = mu0 g + tau, and its series expansion of the solution is summed by the fixed-point
 * iteration (each iterate adds the next term of the series)
 *   g <- G - Gamma0 * tau(g),  Gamma0-hat(xi) = xi (x) xi / (mu0 |xi|^2) for xi != 0,
 * with the odd products xi1 xi2 zeroed at the Nyquist indices (G8), g-hat(0) = G.
 * Loading: strain control G = (2 eps_bar13, 0); stress control G = ((sigma_bar13 - <tau1>) /
 * mu0, -<tau2> / mu0), recomputed from each iterate's tau so that <sigma13> = sigma_bar13.
 * mu0 = (min mu + max mu) / 2; g starts at zero.  Stops when
 *   rms(g_new - g) <= tol * max(rms(g_new), rms(U13 - <U13>))
 * or after max_iter iterations (tol = 0: exactly max_iter).  Returns the iterations done;
 * *res receives the last ratio rms(g_new - g) / max(...).  Outputs [n2][n1].
 */
int oracle_hetero_antiplane(int n1, int n2, const double *mu, const double *up13, int stress_control,
                            double load, double tol, int max_iter, double *sig13, double *sig23, double *res)
{
    size_t n = (size_t)n1 * n2;
    double mmin = mu[0], mmax = mu[0];
    for (size_t i = 1; i < n; i++) { if (mu[i] < mmin) mmin = mu[i]; if (mu[i] > mmax) mmax = mu[i]; }
    const double mu0 = 0.5 * (mmin + mmax);
    double *g1 = calloc(n, sizeof(double)), *g2 = calloc(n, sizeof(double));
    double *t1r = malloc(sizeof(double) * n), *t1i = malloc(sizeof(double) * n);
    double *t2r = malloc(sizeof(double) * n), *t2i = malloc(sizeof(double) * n);
    double umean = oracle_sum(n, up13) / (double)n, urms = 0.0;
    for (size_t i = 0; i < n; i++) urms += (up13[i] - umean) * (up13[i] - umean);
    urms = sqrt(urms / (double)n);
    int it = 0;
    double r = 0.0;
    while (it < max_iter) {
        it++;
        for (size_t i = 0; i < n; i++) {
            t1r[i] = (mu[i] - mu0) * g1[i] - mu[i] * up13[i];
            t2r[i] = (mu[i] - mu0) * g2[i];
            t1i[i] = 0.0;
            t2i[i] = 0.0;
        }
        oracle_fft2d(n1, n2, t1r, t1i, -1);
        oracle_fft2d(n1, n2, t2r, t2i, -1);
        double G1, G2;
        if (stress_control) {
            G1 = (load - t1r[0] / (double)n) / mu0;
            G2 = -(t2r[0] / (double)n) / mu0;
        } else {
            G1 = 2.0 * load;
            G2 = 0.0;
        }
        for (int k2 = 0; k2 < n2; k2++) {
            for (int k1 = 0; k1 < n1; k1++) {
                size_t i = (size_t)k2 * n1 + k1;
                if (k1 == 0 && k2 == 0) {
                    t1r[i] = G1 * (double)n; t1i[i] = 0.0;
                    t2r[i] = G2 * (double)n; t2i[i] = 0.0;
                    continue;
                }
                double x1 = 2.0 * OR_PI * (double)signed_index(k1, n1) / (double)n1;
                double x2 = 2.0 * OR_PI * (double)signed_index(k2, n2) / (double)n2;
                double o1 = (2 * k1 == n1) ? 0.0 : x1, o2 = (2 * k2 == n2) ? 0.0 : x2;
                double q = mu0 * (x1 * x1 + x2 * x2);
                double a11 = x1 * x1 / q, a12 = o1 * o2 / q, a22 = x2 * x2 / q;
                double ar = t1r[i], ai = t1i[i], br = t2r[i], bi = t2i[i];
                t1r[i] = -(a11 * ar + a12 * br);
                t1i[i] = -(a11 * ai + a12 * bi);
                t2r[i] = -(a12 * ar + a22 * br);
                t2i[i] = -(a12 * ai + a22 * bi);
            }
        }
        oracle_fft2d(n1, n2, t1r, t1i, +1);
        oracle_fft2d(n1, n2, t2r, t2i, +1);
        double dd = 0.0, gg = 0.0;
        for (size_t i = 0; i < n; i++) {
            double a = t1r[i] / (double)n, b = t2r[i] / (double)n;
            dd += (a - g1[i]) * (a - g1[i]) + (b - g2[i]) * (b - g2[i]);
            gg += a * a + b * b;
            g1[i] = a;
            g2[i] = b;
        }
        double scale = fmax(sqrt(gg / (double)n), urms);
        r = scale > 0.0 ? sqrt(dd / (double)n) / scale : 0.0;
        if (tol > 0.0 && r <= tol) break;
    }
    for (size_t i = 0; i < n; i++) {
        if (sig13) sig13[i] = mu[i] * (g1[i] - up13[i]);
        if (sig23) sig23[i] = mu[i] * g2[i];
    }
    if (res) *res = r;
    free(g1); free(g2); free(t1r); free(t1i); free(t2r); free(t2i);
    return it;
}

/*
 * Heterogeneous elasticity with a plastic layer thinner than the cell (Sec. 3.1.2,
 * heterogeneous medium; the layer of Sec. 3.2.1).  Periodic cell of n1 x n2 x nz cubic
 * voxels; the eigen-distortion U^p = U13(x1, x2) chi(x3) e1 (x) e3, chi = 1 on the planes
 * x3 = 0 .. nh-1, i.e. the eigenstrain eps^p_13 = eps^p_31 = U13 chi / 2.  The medium is
 * isotropic, C(x) = f(x1, x2) C_iso(lambda, mu) with lambda = 2 mu nu / (1 - 2 nu): the
 * modulus field varies in the plane and is uniform through the cell's depth (reading H5).
 * Reference medium C0 = f0 C_iso, f0 = (min f + max f) / 2.  Unknown: the strain eps (3x3,
 * symmetric).  The paper's series expansion is summed by the fixed-point iteration, from
 * eps = 0,
 *   tau = (C - C0) : eps - C : eps^p,
 *   eps-hat(xi) = -Gamma0-hat(xi) : tau-hat(xi) (xi != 0),   eps-hat(0) = E,
 *   Gamma0-hat_ijkl = (delta_ik xi_j xi_l + delta_il xi_j xi_k + delta_jk xi_i xi_l
 *                      + delta_jl xi_i xi_k) / (4 mu0 |xi|^2)
 *                     - (lambda0 + mu0) / (mu0 (lambda0 + 2 mu0)) xi_i xi_j xi_k xi_l / |xi|^4,
 * with every product of frequency components that contains an axis's Nyquist frequency an
 * odd number of times set to zero (reading G8: a real field cannot carry it).  Loading:
 * strain control E = eps_bar13 (e1 (x) e3 + e3 (x) e1); stress control <sigma> = sigma_bar13
 * (e1 (x) e3 + e3 (x) e1), i.e. E = C0^-1 : (Sigma - <tau>) from each iterate's tau.
 * Stops when rms(eps_new - eps) <= tol max(rms(eps_new), rms(eps^p - <eps^p>)) (rms over the
 * cell of the tensor's Frobenius norm) or after max_iter iterations (tol = 0: exactly
 * max_iter).  Outputs the layer average of sigma13 = 2 f mu (eps13 - eps^p13) over the nh
 * planes, tau13[n2][n1], and (may be NULL) sigma13 of every plane, s13_planes[nz][n2][n1].
 * Returns the iterations done; *res (may be NULL) the last ratio.
 */
static double gamma_term(const int *idx, int nidx, const double xi[3], const int nyq[3])
{
    /* product of xi over the listed axes; zero when an axis at its Nyquist frequency occurs
       an odd number of times */
    int count[3] = {0, 0, 0};
    double p = 1.0;
    for (int t = 0; t < nidx; t++) { count[idx[t]]++; p *= xi[idx[t]]; }
    for (int a = 0; a < 3; a++) if (nyq[a] && (count[a] & 1)) return 0.0;
    return p;
}

int oracle_hetero_layer(int n1, int n2, int nz, int nh, double mu, double nu, const double *f, const double *up13,
                        int stress_control, double load, double tol, int max_iter, double *tau13, double *s13_planes,
                        double *res)
{
    const size_t n2d = (size_t)n1 * n2, n = n2d * nz;
    const double lam = 2.0 * mu * nu / (1.0 - 2.0 * nu);
    double flo = f[0], fhi = f[0];
    for (size_t i = 1; i < n2d; i++) { if (f[i] < flo) flo = f[i]; if (f[i] > fhi) fhi = f[i]; }
    const double f0 = 0.5 * (flo + fhi), mu0 = f0 * mu, lam0 = f0 * lam;
    const double cc = (lam0 + mu0) / (mu0 * (lam0 + 2.0 * mu0));
    /* strain components e[c] for c = (i, j) with i <= j: 00 11 22 12 02 01 */
    static const int ci[6] = {0, 1, 2, 1, 0, 0}, cj[6] = {0, 1, 2, 2, 2, 1};
    double *eps = calloc(6 * n, sizeof(double));
    double *re = malloc(sizeof(double) * 6 * n), *im = malloc(sizeof(double) * 6 * n);
    double *zr = malloc(sizeof(double) * nz), *zi = malloc(sizeof(double) * nz);
    /* eigenstrain 13 component and its rms about the mean */
    double pmean = 0.0;
    for (int z = 0; z < nh; z++) for (size_t q = 0; q < n2d; q++) pmean += 0.5 * up13[q];
    pmean /= (double)n;
    double prms = 0.0;
    for (int z = 0; z < nz; z++)
        for (size_t q = 0; q < n2d; q++) {
            double e = (z < nh ? 0.5 * up13[q] : 0.0) - pmean;
            prms += 2.0 * e * e;   /* eps^p_13 and eps^p_31 */
        }
    prms = sqrt(prms / (double)n);
    int it = 0;
    double r = 0.0;
    while (it < max_iter) {
        it++;
        /* polarisation tau = (C - C0) : eps - C : eps^p (isotropic: lambda tr + 2 mu) */
        double tmean[6] = {0, 0, 0, 0, 0, 0};
        for (int z = 0; z < nz; z++)
            for (size_t q = 0; q < n2d; q++) {
                size_t x = (size_t)z * n2d + q;
                double dl = (f[q] - f0) * lam, dm = (f[q] - f0) * mu;
                double tr = eps[0 * n + x] + eps[1 * n + x] + eps[2 * n + x];
                for (int c = 0; c < 6; c++) {
                    double t = 2.0 * dm * eps[c * n + x] + (c < 3 ? dl * tr : 0.0);
                    if (c == 4 && z < nh) t -= 2.0 * f[q] * mu * 0.5 * up13[q];   /* - C : eps^p */
                    re[c * n + x] = t;
                    im[c * n + x] = 0.0;
                    tmean[c] += t;
                }
            }
        for (int c = 0; c < 6; c++) tmean[c] /= (double)n;
        /* macroscopic strain of this iterate */
        double E[6] = {0, 0, 0, 0, 0, 0};
        if (stress_control) {
            /* E = C0^-1 : (Sigma - <tau>), isotropic compliance: e = (s - nu0/(1+nu0) tr s I)/(2 mu0) */
            double S[6];
            for (int c = 0; c < 6; c++) S[c] = (c == 4 ? load : 0.0) - tmean[c];
            double nu0 = lam0 / (2.0 * (lam0 + mu0));
            double trs = S[0] + S[1] + S[2];
            for (int c = 0; c < 6; c++) E[c] = (S[c] - (c < 3 ? nu0 / (1.0 + nu0) * trs : 0.0)) / (2.0 * mu0);
        } else {
            E[4] = load;
        }
        /* 3-D transform of each component: planes, then along x3 */
        for (int c = 0; c < 6; c++) {
            for (int z = 0; z < nz; z++) oracle_fft2d(n1, n2, re + c * n + (size_t)z * n2d, im + c * n + (size_t)z * n2d, -1);
            for (size_t q = 0; q < n2d; q++) {
                for (int z = 0; z < nz; z++) { zr[z] = re[c * n + (size_t)z * n2d + q]; zi[z] = im[c * n + (size_t)z * n2d + q]; }
                oracle_fft1d(nz, zr, zi, -1);
                for (int z = 0; z < nz; z++) { re[c * n + (size_t)z * n2d + q] = zr[z]; im[c * n + (size_t)z * n2d + q] = zi[z]; }
            }
        }
        /* Green operator */
        for (int k3 = 0; k3 < nz; k3++)
            for (int k2 = 0; k2 < n2; k2++)
                for (int k1 = 0; k1 < n1; k1++) {
                    size_t x = (size_t)k3 * n2d + (size_t)k2 * n1 + k1;
                    if (k1 == 0 && k2 == 0 && k3 == 0) {
                        for (int c = 0; c < 6; c++) { re[c * n + x] = E[c] * (double)n; im[c * n + x] = 0.0; }
                        continue;
                    }
                    double xi[3] = {2.0 * OR_PI * signed_index(k1, n1) / n1, 2.0 * OR_PI * signed_index(k2, n2) / n2,
                                    2.0 * OR_PI * signed_index(k3, nz) / nz};
                    int nyq[3] = {2 * k1 == n1, 2 * k2 == n2, 2 * k3 == nz};
                    double q2 = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
                    double tr_[3][3], ti_[3][3];
                    for (int c = 0; c < 6; c++) {
                        tr_[ci[c]][cj[c]] = tr_[cj[c]][ci[c]] = re[c * n + x];
                        ti_[ci[c]][cj[c]] = ti_[cj[c]][ci[c]] = im[c * n + x];
                    }
                    for (int c = 0; c < 6; c++) {
                        int i = ci[c], j = cj[c];
                        double sr = 0.0, si = 0.0;
                        for (int k = 0; k < 3; k++)
                            for (int l = 0; l < 3; l++) {
                                double g = 0.0;
                                int a2[2];
                                if (i == k) { a2[0] = j; a2[1] = l; g += gamma_term(a2, 2, xi, nyq); }
                                if (i == l) { a2[0] = j; a2[1] = k; g += gamma_term(a2, 2, xi, nyq); }
                                if (j == k) { a2[0] = i; a2[1] = l; g += gamma_term(a2, 2, xi, nyq); }
                                if (j == l) { a2[0] = i; a2[1] = k; g += gamma_term(a2, 2, xi, nyq); }
                                g /= 4.0 * mu0 * q2;
                                int a4[4] = {i, j, k, l};
                                g -= cc * gamma_term(a4, 4, xi, nyq) / (q2 * q2);
                                sr += g * tr_[k][l];
                                si += g * ti_[k][l];
                            }
                        re[c * n + x] = -sr;
                        im[c * n + x] = -si;
                    }
                }
        /* back to real space */
        for (int c = 0; c < 6; c++) {
            for (size_t q = 0; q < n2d; q++) {
                for (int z = 0; z < nz; z++) { zr[z] = re[c * n + (size_t)z * n2d + q]; zi[z] = im[c * n + (size_t)z * n2d + q]; }
                oracle_fft1d(nz, zr, zi, +1);
                for (int z = 0; z < nz; z++) { re[c * n + (size_t)z * n2d + q] = zr[z]; im[c * n + (size_t)z * n2d + q] = zi[z]; }
            }
            for (int z = 0; z < nz; z++) oracle_fft2d(n1, n2, re + c * n + (size_t)z * n2d, im + c * n + (size_t)z * n2d, +1);
        }
        double dd = 0.0, ee = 0.0;
        for (int c = 0; c < 6; c++) {
            double w = (c < 3) ? 1.0 : 2.0;   /* off-diagonal components count twice */
            for (size_t x = 0; x < n; x++) {
                double v = re[c * n + x] / (double)n;
                double d = v - eps[c * n + x];
                dd += w * d * d;
                ee += w * v * v;
                eps[c * n + x] = v;
            }
        }
        double scale = fmax(sqrt(ee / (double)n), prms);
        r = scale > 0.0 ? sqrt(dd / (double)n) / scale : 0.0;
        if (tol > 0.0 && r <= tol) break;
    }
    for (size_t q = 0; q < n2d; q++) {
        double acc = 0.0;
        for (int z = 0; z < nz; z++) {
            double s = 2.0 * f[q] * mu * (eps[4 * n + (size_t)z * n2d + q] - (z < nh ? 0.5 * up13[q] : 0.0));
            if (s13_planes) s13_planes[(size_t)z * n2d + q] = s;
            if (z < nh) acc += s;
        }
        if (tau13) tau13[q] = acc / (double)nh;
    }
    if (res) *res = r;
    free(eps); free(re); free(im); free(zr); free(zi);
    return it;
}

/* size check used by the wrapper */
int oracle_valid_size(int n) { return is_pow2(n) && n >= 4; }
