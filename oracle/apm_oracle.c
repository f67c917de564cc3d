/*
 * apm_oracle.c -- oracle for the adaptive particle-mesh (APM) level solve of
 * Passy & Bryan, "An adaptive particle-mesh gravity solver for ENZO"
 * (arXiv:1410.0010).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously-correct FP64
 * CPU statement of what the CUDA path computes.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark load it; the product
 * library never links, includes or calls it, and it includes nothing from the
 * product.  It is compiled with -O2 -ffp-contract=off (no fused multiply-add,
 * no fast-math), so every floating-point operation is rounded exactly as
 * written here.
 *
 * Readings of the paper where it is silent or garbled (each is listed in the
 * design notes of the repository):
 *   R1  G = 1, attractive sign: continuum kernel -4 pi S^2 / k^2 (Sec. 1 Eq. 1-2,
 *       fixed by the closed forms of Sec. 3.3 and Eq. sinewave).
 *   R2  Eq. assignment prints prod sinc^6 for U; that product is U^2 for TSC
 *       (Eq. assignment2 is the alias sum of sinc^6), so U^2 = prod sinc^6.
 *   R3  The root reference force is read with S_0^2 (so the levels telescope);
 *       S-hat uses its Taylor series for eta < 1 (cancellation).
 *   R4  Isolated root: real-space S_0-S_0 pair potential on the doubled grid
 *       (minimum image), transformed, plus the k-space optimal correction
 *       G_opt - (-4 pi S_0^2/k^2) on non-degenerate modes.
 *   R5  Modes where the FD gradient vanishes identically (every kappa_j in
 *       {0, M_j/2}) get G = 0 (decided by integer index).  kappa = 0: periodic
 *       root 0 (mean removed, Sec. 3.4); refined level: the finite limit
 *       -4 pi (a_{l-1}^2 - a_l^2)/30.
 *   R6  Padding 0.65 R a / delta = 4.42 -> B = 5 cells per side of GMF border;
 *       FFT length M = smallest {2,3,5,7}-smooth integer >= N + 4B; the result
 *       is the circular convolution on that M grid (Sec. 2.2).
 *   R7  Isolated root: GMF is exactly N^3; TSC weights outside [0,N) fold into
 *       the boundary cell, in deposit and interpolation alike.
 *   R8  FD gradient: two-point centred difference, D_j = sin(k_j delta)/delta.
 *   R10 Parent carry: potential and acceleration, trilinear interpolation from
 *       parent cell centres in FP64 (Sec. 2.2, last paragraph).
 *   R11 TSC weights in fixed point (the paper fixes the TSC assignment of
 *       Sec. 2, not its arithmetic): the drifted coordinate x + v dt/2 (FP64,
 *       two rounded operations) in root cells is rounded once to
 *       X = rint(x/delta0 2^31), the same for every level, and on a periodic
 *       domain taken modulo the box (N0 2^31); on
 *       level l (2^l cells per root cell) the cell is i = floor(X / 2^(31-l))
 *       and t = (X mod 2^(31-l)) / 2^(31-l) the offset from its lower face;
 *       the three weights of the cells i-1, i, i+1 are (1-t)^2/2,
 *       3/4 - (t-1/2)^2, t^2/2, computed as
 *       exact integers on the scale 2^63 (they sum to 2^63 exactly); the 3-D
 *       weight of the 26 outer cells is the product x, then y, then z, each
 *       product rounded half up to the scale 2^63, and the centre cell's weight
 *       is 2^63 minus theirs (deposit and interpolation weights sum to one
 *       exactly).
 *   R15 Gradient operator (Sec. 2.2 allows a finite difference or the direct
 *       Fourier-space gradient D = -ik): the two-point difference (R8), the
 *       four-point difference D = (8 sin(k delta) - sin(2 k delta))/(6 delta),
 *       or D = k with 0 on an even M's Nyquist mode; the influence function
 *       is built for the operator the accelerations use.  With the four-point
 *       difference the potential window is [-3, N+3) and an isolated root's
 *       M is the smallest even {2,3,5,7}-smooth length >= 2N + 2, so that the
 *       edge cells' stencils read unwrapped offsets; the spectral gradient
 *       transforms -i D_j phi-hat back once per component.
 *   R14 Time evolution (Sec. 3.1, 3.5 without subcycling; the paper names no
 *       integrator): every level advances with one timestep dt; the solve
 *       evaluates accelerations at the half-step drifted positions
 *       x + v dt/2 (Sec. 2), then v' = v + a dt and x' = x + (v + v')/2 dt.
 *   Fixed point: cell masses are int64 with F fractional bits.  With
 *   M = rint(m 2^F), each of the 26 outer cells receives ((|M| wx) wy) wz,
 *   every product (a b + 2^62) >> 63 (sign of M), the centre cell M minus the
 *   other 26, so integer mass is conserved exactly and the sum is independent
 *   of particle order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* status bits returned by the deposit routines */
#define ORC_ST_OVERFLOW 1  /* |m 2^F| >= 2^62: particle skipped */
#define ORC_ST_OUT_OF_BOX 2 /* isolated root: drifted particle outside [0, box) */

static int64_t floor_div(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
    return q;
}

static int64_t mod_pos(int64_t a, int64_t m) {
    int64_t r = a % m;
    return r < 0 ? r + m : r;
}

/* ------------------------------------------------------------------------ */
/* Smoothing function, Sec. 2.2 Eq. S2k: S-hat(eta) = 12/eta^4 (2 - 2cos eta  */
/* - eta sin eta), eta = k a / 2.  For eta < 1 the Taylor series             */
/* 12 sum_{m>=2} (-1)^m (2m-2)/(2m)! eta^(2m-4) (terms m = 2..13) is used,    */
/* because the closed form cancels catastrophically there (reading R3).      */
/* ------------------------------------------------------------------------ */
double orc_shat(double eta) {
    if (eta < 1.0) {
        double sum = 0.0;
        double fact = 24.0; /* (2m)! for m = 2 */
        double pw = 1.0;    /* eta^(2m-4) */
        for (int m = 2; m <= 13; ++m) {
            if (m > 2) {
                fact = fact * (double)(2 * m - 1) * (double)(2 * m);
                pw = pw * (eta * eta);
            }
            double term = ((double)(2 * m - 2) / fact) * pw;
            if (m % 2 == 0) sum += term; else sum -= term;
        }
        return 12.0 * sum;
    }
    double e2 = eta * eta;
    return 12.0 / (e2 * e2) * (2.0 - 2.0 * cos(eta) - eta * sin(eta));
}

/* Closed form only (used by the pin that compares it with the series). */
double orc_shat_closed(double eta) {
    double e2 = eta * eta;
    return 12.0 / (e2 * e2) * (2.0 - 2.0 * cos(eta) - eta * sin(eta));
}

double orc_sinc(double x) { return x == 0.0 ? 1.0 : sin(x) / x; }

/* Potential between two unit-mass S spheres of diameter a (G = 1) at        */
/* separation r, as a function of xi = r/a; psi_a(r) = orc_psi(r/a)/a.        */
/* This is the real-space kernel whose transform is -4 pi S-hat^2 / k^2       */
/* (reading R4); beyond r = a the spheres do not overlap and it is -1/xi.    */
double orc_psi(double xi) {
    if (xi <= 0.5) {
        double x2 = xi * xi, x4 = x2 * x2;
        return -104.0 / 35.0 + 32.0 / 5.0 * x2 - 64.0 / 5.0 * x4 + 32.0 / 5.0 * x4 * xi
               + 256.0 / 35.0 * x4 * x2 - 192.0 / 35.0 * x4 * x2 * xi;
    }
    if (xi <= 1.0) {
        double x2 = xi * xi, x3 = x2 * xi, x4 = x2 * x2;
        return -3.0 / (35.0 * xi) - 64.0 / 35.0 - 32.0 / 5.0 * xi + 128.0 / 5.0 * x2 - 32.0 * x3
               + 64.0 / 5.0 * x4 + 32.0 / 5.0 * x4 * xi - 256.0 / 35.0 * x4 * x2
               + 64.0 / 35.0 * x4 * x3;
    }
    return -1.0 / xi;
}

/* Sum over all Brillouin zones of U^2 = prod_j sinc^6(k_j delta/2), in its  */
/* closed form prod_j (1 - s_j^2 + 2/15 s_j^4), s_j = sin(pi kappa_j / M_j)   */
/* (Sec. 2.2 Eq. assignment2, reading R2).                                    */
double orc_alias_sum(const int64_t kap[3], const int64_t M[3]) {
    double alias = 1.0;
    for (int j = 0; j < 3; ++j) {
        int64_t kc = kap[j];
        if (kc > M[j] / 2) kc -= M[j];
        double s = sin(ORC_PI * (double)kc / (double)M[j]);
        double s2 = s * s;
        alias *= 1.0 - s2 + (2.0 / 15.0) * s2 * s2;
    }
    return alias;
}

/* ------------------------------------------------------------------------ */
/* Gradient operator D_j at the centred mode kc of an M grid (Sec. 2.2: a     */
/* finite difference or the Fourier-space gradient D = -ik; the factor -i is  */
/* common to all and left out here).  grad 0: two-point difference,           */
/* sin(k delta)/delta (reading R8); grad 1: four-point difference             */
/* (8 sin(k delta) - sin(2 k delta))/(6 delta); grad 2: spectral, k itself,   */
/* except 0 on the Nyquist mode kc = M/2 of an even M (reading R15).          */
/* ------------------------------------------------------------------------ */
double orc_grad_d(int grad, int64_t kc, int64_t M, double delta) {
    double th = 2.0 * ORC_PI * (double)kc / (double)M;   /* k delta */
    if (grad == 0) return sin(th) / delta;
    if (grad == 1) return (8.0 * sin(th) - sin(2.0 * th)) / (6.0 * delta);
    if (2 * kc == M) return 0.0;
    return th / delta;
}

/* ------------------------------------------------------------------------ */
/* Optimal influence function, Sec. 2.2 Eq. influence with Eq. brillouin     */
/* truncated to n in [-1,1]^3, Eq. assignment/assignment2 (reading R2),       */
/* Eq. reference (readings R1, R3) and the gradient D of orc_grad_d.          */
/* kap[j] in [0, M_j); it is centred to (-M/2, M/2] before use.              */
/* use_parent = 0: reference force S(a_lev)^2/k^2 (root);                     */
/* use_parent = 1: (S(a_lev)^2 - S(a_par)^2)/k^2 (refined level).            */
/* Returns G-hat in continuum units (potential = G-hat * density).            */
/* ------------------------------------------------------------------------ */
double orc_green_opt(const int64_t kap[3], const int64_t M[3], double delta,
                     double a_lev, double a_par, int use_parent, int grad) {
    double k[3], D[3];
    double alias = orc_alias_sum(kap, M), D2 = 0.0;
    for (int j = 0; j < 3; ++j) {
        int64_t kc = kap[j];
        if (kc > M[j] / 2) kc -= M[j];
        k[j] = 2.0 * ORC_PI * (double)kc / ((double)M[j] * delta);
        D[j] = orc_grad_d(grad, kc, M[j], delta);
        D2 += D[j] * D[j];
    }
    double num = 0.0;
    for (int n0 = -1; n0 <= 1; ++n0)
        for (int n1 = -1; n1 <= 1; ++n1)
            for (int n2 = -1; n2 <= 1; ++n2) {
                int n[3] = {n0, n1, n2};
                double q[3], U2 = 1.0, Dq = 0.0, qq = 0.0;
                for (int j = 0; j < 3; ++j) {
                    q[j] = k[j] + 2.0 * ORC_PI * (double)n[j] / delta;
                    double sc = orc_sinc(q[j] * delta / 2.0);
                    double sc2 = sc * sc;
                    U2 *= sc2 * sc2 * sc2;
                    Dq += D[j] * q[j];
                    qq += q[j] * q[j];
                }
                double qa = sqrt(qq);
                double sl = orc_shat(qa * a_lev / 2.0);
                double F = sl * sl / qq;
                if (use_parent) {
                    double sp = orc_shat(qa * a_par / 2.0);
                    F -= sp * sp / qq;
                }
                num += U2 * Dq * F;
            }
    return -4.0 * ORC_PI * num / (D2 * alias * alias);
}

/* 1 when the gradient vanishes identically at this mode (reading R5): every */
/* kappa_j is 0 or M_j/2, for each of the three operators.                    */
static int degenerate(const int64_t kap[3], const int64_t M[3]) {
    for (int j = 0; j < 3; ++j)
        if (!(kap[j] == 0 || 2 * kap[j] == M[j])) return 0;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Textbook FFT of one line (used instead of the naive sum when the oracle's  */
/* transform mode is 1): recursive decimation-in-time Cooley-Tukey.  A length */
/* n = p m with p its smallest prime factor is split into the p subsequences  */
/* x[r + p j] (j < m), each transformed recursively, and combined as          */
/*   X[k + q m] = sum_r w_n^(r (k + q m)) Y_r[k],  k < m, q < p,             */
/* with w_n = exp(sign 2 pi i / n).  Every root is taken from the table of    */
/* the full line length L (w_n^t = w_L^(t L/n)) at the exact integer index    */
/* (t L/n) mod L.  x: input at stride `stride`; y: output (n values); t:      */
/* scratch (n values).                                                        */
/* ------------------------------------------------------------------------ */
static int64_t smallest_prime_factor(int64_t n) {
    for (int64_t p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

static void fft_rec(const double* xr, const double* xi, int64_t stride, int64_t n, double* yr, double* yi,
                    double* tr, double* ti, int64_t L, const double* wr, const double* wi) {
    if (n == 1) {
        yr[0] = xr[0];
        yi[0] = xi[0];
        return;
    }
    int64_t p = smallest_prime_factor(n), m = n / p;
    /* sub-transforms Y_r into t[r m .. r m + m), with y[r m ..] as their scratch */
    for (int64_t r = 0; r < p; ++r)
        fft_rec(xr + r * stride, xi + r * stride, stride * p, m, tr + r * m, ti + r * m, yr + r * m,
                yi + r * m, L, wr, wi);
    int64_t scale = L / n;
    for (int64_t q = 0; q < p; ++q)
        for (int64_t k = 0; k < m; ++k) {
            int64_t kk = k + q * m;
            double sr = 0.0, si = 0.0;
            for (int64_t r = 0; r < p; ++r) {
                int64_t t = ((r * kk) % n) * scale;   /* exact index of w_n^(r kk) in the L table */
                double ar = tr[r * m + k], ai = ti[r * m + k];
                sr += ar * wr[t] - ai * wi[t];
                si += ar * wi[t] + ai * wr[t];
            }
            yr[kk] = sr;
            yi[kk] = si;
        }
}

/* transform of the oracle's separable 3-D routines: 0 the naive sum (default), */
/* 1 the textbook FFT above; both compute the same unnormalised DFT            */
static int orc_transform_mode = 0;
void orc_set_transform(int mode) { orc_transform_mode = mode; }
int orc_get_transform(void) { return orc_transform_mode; }

/* ------------------------------------------------------------------------ */
/* Separable naive DFT of a complex M0 x M1 x M2 array (x fastest):           */
/* out[kappa] = sum_j in[j] exp(sign 2 pi i kappa j / M), twiddles indexed by */
/* the exact integer (kappa*j) mod M.  No normalisation.  With transform      */
/* mode 1 each line goes through fft_rec instead (same result, O(M log M)).   */
/* ------------------------------------------------------------------------ */
static void dft_axis(double* re, double* im, const int64_t M[3], int axis, int sign) {
    int64_t L = M[axis];
    int64_t stride = 1;
    for (int j = 0; j < axis; ++j) stride *= M[j];
    int64_t total = M[0] * M[1] * M[2];
    int64_t nlines = total / L;
    double* wr = (double*)malloc(sizeof(double) * L);
    double* wi = (double*)malloc(sizeof(double) * L);
    for (int64_t t = 0; t < L; ++t) {
        wr[t] = cos(2.0 * ORC_PI * (double)t / (double)L);
        wi[t] = (double)sign * sin(2.0 * ORC_PI * (double)t / (double)L);
    }
    const int fft = orc_transform_mode == 1;
#pragma omp parallel
    {
        double* lr = (double*)malloc(sizeof(double) * L);
        double* li = (double*)malloc(sizeof(double) * L);
        double* yr = (double*)malloc(sizeof(double) * L);
        double* yi = (double*)malloc(sizeof(double) * L);
        double* sr_ = (double*)malloc(sizeof(double) * L);
        double* si_ = (double*)malloc(sizeof(double) * L);
#pragma omp for schedule(static)
        for (int64_t line = 0; line < nlines; ++line) {
            /* base index of this line: decompose line into the other two axes */
            int64_t lo = line % stride, hi = line / stride;
            int64_t base = lo + hi * stride * L;
            for (int64_t j = 0; j < L; ++j) {
                lr[j] = re[base + j * stride];
                li[j] = im[base + j * stride];
            }
            if (fft) {
                fft_rec(lr, li, 1, L, yr, yi, sr_, si_, L, wr, wi);
                for (int64_t kk = 0; kk < L; ++kk) {
                    re[base + kk * stride] = yr[kk];
                    im[base + kk * stride] = yi[kk];
                }
                continue;
            }
            for (int64_t kk = 0; kk < L; ++kk) {
                double sr = 0.0, si = 0.0;
                for (int64_t j = 0; j < L; ++j) {
                    int64_t t = (kk * j) % L;
                    sr += lr[j] * wr[t] - li[j] * wi[t];
                    si += lr[j] * wi[t] + li[j] * wr[t];
                }
                re[base + kk * stride] = sr;
                im[base + kk * stride] = si;
            }
        }
        free(lr);
        free(li);
        free(yr);
        free(yi);
        free(sr_);
        free(si_);
    }
    free(wr);
    free(wi);
}

void orc_dft3(double* re, double* im, const int64_t M[3], int sign, int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    for (int axis = 0; axis < 3; ++axis) dft_axis(re, im, M, axis, sign);
}

/* ------------------------------------------------------------------------ */
/* Green's-function table on the octant kappa_j in [0, M_j/2] (x fastest),   */
/* in DFT units: potential = IDFT( T * DFT(cell mass) ) / (M0 M1 M2).         */
/* kind 0: refined level (short range, a_par = R a_lev);                      */
/* kind 1: periodic root; kind 2: isolated root on the doubled grid.          */
/* ------------------------------------------------------------------------ */
void orc_green_table(int kind, const int64_t M[3], double delta, double a_lev, double a_par,
                     int correction, int grad, double* T, int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    int64_t H[3] = {M[0] / 2 + 1, M[1] / 2 + 1, M[2] / 2 + 1};
    double vol = (delta * delta) * delta;
    double* gre = NULL;
    double* gim = NULL;
    if (kind == 2) {
        /* reading R4: real-space pair potential at minimum-image offsets */
        int64_t tot = M[0] * M[1] * M[2];
        gre = (double*)calloc((size_t)tot, sizeof(double));
        gim = (double*)calloc((size_t)tot, sizeof(double));
        for (int64_t z = 0; z < M[2]; ++z)
            for (int64_t y = 0; y < M[1]; ++y)
                for (int64_t x = 0; x < M[0]; ++x) {
                    int64_t d[3] = {x, y, z};
                    double r2 = 0.0;
                    for (int j = 0; j < 3; ++j) {
                        int64_t dj = d[j] <= M[j] / 2 ? d[j] : d[j] - M[j];
                        double rj = (double)dj * delta;
                        r2 += rj * rj;
                    }
                    double r = sqrt(r2);
                    gre[x + M[0] * (y + M[1] * z)] = orc_psi(r / a_lev) / a_lev;
                }
        orc_dft3(gre, gim, M, -1, nthreads);
    }
#pragma omp parallel for collapse(2) schedule(dynamic)
    for (int64_t z = 0; z < H[2]; ++z)
        for (int64_t y = 0; y < H[1]; ++y)
            for (int64_t x = 0; x < H[0]; ++x) {
                int64_t kap[3] = {x, y, z};
                int zero = (x == 0 && y == 0 && z == 0);
                int deg = degenerate(kap, M);
                double v = 0.0;
                if (kind == 0) {
                    if (zero)
                        v = -4.0 * ORC_PI * (a_par * a_par - a_lev * a_lev) / 30.0 / vol;
                    else if (!deg)
                        v = orc_green_opt(kap, M, delta, a_lev, a_par, 1, grad) / vol;
                } else if (kind == 1) {
                    if (!zero && !deg) v = orc_green_opt(kap, M, delta, a_lev, 0.0, 0, grad) / vol;
                } else {
                    v = gre[x + M[0] * (y + M[1] * z)];
                    if (correction && !zero && !deg) {
                        double kk = 0.0;
                        for (int j = 0; j < 3; ++j) {
                            double kj = 2.0 * ORC_PI * (double)kap[j] / ((double)M[j] * delta);
                            kk += kj * kj;
                        }
                        double s = orc_shat(sqrt(kk) * a_lev / 2.0);
                        double gcont = -4.0 * ORC_PI * s * s / kk;
                        v += (orc_green_opt(kap, M, delta, a_lev, 0.0, 0, grad) - gcont) / vol;
                    }
                }
                T[x + H[0] * (y + H[1] * z)] = v;
            }
    free(gre);
    free(gim);
}

/* ------------------------------------------------------------------------ */
/* Half-timestep drift, Sec. 2: x' = x + v * half_dt (two rounded ops);       */
/* on a periodic domain x' -= box * floor(x'/box).                            */
/* ------------------------------------------------------------------------ */
double orc_drift(double x, double v, double half_dt, double box, int periodic) {
    double t = v * half_dt;
    double xd = x + t;
    if (periodic) xd = xd - box * floor(xd / box);
    return xd;
}

/* ------------------------------------------------------------------------ */
/* One timestep of the particles with accelerations a evaluated at the        */
/* half-step drifted positions x + v dt/2 (the drift of Sec. 2 that the       */
/* deposit and interpolation apply): v' = v + a dt, then                      */
/* x' = x + ((v + v')/2) dt, i.e. x + v dt + a dt^2/2, second order.  Each    */
/* operation is one IEEE rounding in this order (no contraction), over n      */
/* particles stored as SoA.  Not in the paper: a driver of the time           */
/* evolutions of Sec. 3.1 and 3.5 without subcycling (reading R14).           */
/* ------------------------------------------------------------------------ */
void orc_kick_drift(int64_t n, double* px, double* py, double* pz, double* pvx, double* pvy,
                    double* pvz, const double* acc, double dt) {
    double* pos[3] = {px, py, pz};
    double* vel[3] = {pvx, pvy, pvz};
    for (int64_t p = 0; p < n; ++p)
        for (int j = 0; j < 3; ++j) {
            double v = vel[j][p];
            double a = acc[(int64_t)j * n + p];
            double vn = v + a * dt;
            double vm = (v + vn) * 0.5;
            pos[j][p] = pos[j][p] + vm * dt;
            vel[j][p] = vn;
        }
}

/* Fixed-point position (reading R11): the drifted coordinate in root cells,
 * u0 = x / delta0, rounded to X = rint(u0 2^31).  Every level reads the same X:
 * level l has 2^l cells per root cell, so its cell index and offset are the
 * high and low bits of X with 31 - l fraction bits. */
#define ORC_POS_BITS 31
int64_t orc_position_fixed(double x, double delta0) {
    /* a coordinate 2^31 root cells or more from the origin (or NaN) saturates
     * at -+2^62: far outside every box */
    double t = ldexp(x / delta0, ORC_POS_BITS);
    double lim = ldexp(1.0, 62);
    if (t >= lim) return (int64_t)1 << 62;
    if (!(t > -lim)) return -((int64_t)1 << 62);
    return (int64_t)rint(t);
}

/* The fixed-point position of a drifted coordinate xd = x + v half_dt, made
 * canonical: on a periodic domain X is taken modulo the box (N0 2^31), i.e. the
 * periodic wrap of Sec. 3.4 is applied to the fixed-point position; on an
 * isolated domain a coordinate inside [0, box) that rounds onto the upper face
 * stays in the last root cell. */
static int64_t pos_fixed(double xd, double delta0, double box, int periodic) {
    int64_t X = orc_position_fixed(xd, delta0);
    int64_t span = (int64_t)llround(box / delta0) << ORC_POS_BITS;
    if (periodic) {
        X %= span;
        if (X < 0) X += span;
    } else if (xd >= 0.0 && xd < box && X >= span) {
        X = span - 1;
    }
    return X;
}

/* Fixed-point TSC weights along one axis (Sec. 2, n = 3^3 cells; reading R11)
 * of the fixed-point position X on level `level`.  Returns the cell i holding
 * the particle; w[0], w[1], w[2] (scale 2^63) go to cells i-1, i, i+1. */
int64_t orc_tsc_fixed(int64_t X, int level, uint64_t w[3]) {
    int P = ORC_POS_BITS - level;                        /* fraction bits */
    int64_t i = X >> P;                                  /* floor(X / 2^P) */
    uint64_t f = (uint64_t)(X - (i << P));               /* in [0, 2^P) */
    uint64_t S = (uint64_t)1 << P;
    int up = 62 - 2 * P;                                 /* scale 2^(2P+1) -> 2^63 */
    w[2] = (f * f) << up;                                /* t^2/2            * 2^63 */
    w[0] = ((S - f) * (S - f)) << up;                    /* (1-t)^2/2        * 2^63 */
    w[1] = ((uint64_t)1 << 63) - w[0] - w[2];            /* 3/4 - (t-1/2)^2  * 2^63 */
    return i;
}

/* product of two weights on the scale 2^63, rounded half up */
static uint64_t wmul(uint64_t a, uint64_t b) {
    unsigned __int128 p = (unsigned __int128)a * b + ((unsigned __int128)1 << 62);
    return (uint64_t)(p >> 63);
}

/* TSC weights as doubles (w / 2^63 rounded to double) of a position x on a
 * root grid of cell delta, for the pins */
int64_t orc_tsc_weights(double x, double delta, double w[3]) {
    uint64_t wi[3];
    int64_t i = orc_tsc_fixed(orc_position_fixed(x, delta), 0, wi);
    for (int k = 0; k < 3; ++k) w[k] = ldexp((double)wi[k], -63);
    return i;
}

/* CIC weights with a cloud of one cell (Sec. 2): cells i0, i0+1.              */
int64_t orc_cic_weights(double x, double delta, double w[2]) {
    double u = x / delta - 0.5;
    double fi = floor(u);
    double f = u - fi;
    w[0] = 1.0 - f;
    w[1] = f;
    return (int64_t)fi;
}

/* ------------------------------------------------------------------------ */
/* TSC deposit of particles into one GMF box, Sec. 2 (Eq. n = 3^3, modified   */
/* deposit of grid + parent + siblings: every particle whose cloud touches   */
/* the box contributes).  The box spans global level cells                    */
/* [lo_j, lo_j + G_j).  mode 0: cloud cells outside the box are dropped        */
/* (refined grid); mode 1: folded into [0, G) (isolated root, reading R7);    */
/* mode 2: wrapped modulo G (periodic root).  delta0: root cell; level: the    */
/* grid's level (reading R11).  gmf is accumulated (+=).                      */
/* Returns status bits (ORC_ST_*).                                            */
/* ------------------------------------------------------------------------ */
int orc_deposit(int64_t n, const double* px, const double* py, const double* pz,
                const double* pvx, const double* pvy, const double* pvz, const double* pm,
                double half_dt, double box, int periodic, double delta0, int level,
                const int64_t lo[3], const int64_t G[3], int mode, int F, int64_t* gmf) {
    int status = 0;
    double scale = ldexp(1.0, F);
    double limit = ldexp(1.0, 62);
    for (int64_t p = 0; p < n; ++p) {
        double pos[3] = {px[p], py[p], pz[p]};
        double vel[3] = {pvx[p], pvy[p], pvz[p]};
        uint64_t w[3][3];
        int64_t ic[3];
        int outside = 0;
        for (int j = 0; j < 3; ++j) {
            double xd = orc_drift(pos[j], vel[j], half_dt, box, 0);
            if (!(xd >= 0.0 && xd < box)) outside = 1;
            ic[j] = orc_tsc_fixed(pos_fixed(xd, delta0, box, periodic), level, w[j]);
        }
        double mq = pm[p] * scale;
        if (!(fabs(mq) < limit)) {
            status |= ORC_ST_OVERFLOW;
            continue;
        }
        if (mode == 1 && outside) status |= ORC_ST_OUT_OF_BOX;
        int64_t M = (int64_t)rint(mq);
        uint64_t aM = (uint64_t)(M < 0 ? -M : M);
        /* fixed-point charges; centre cell takes the remainder */
        int64_t q[3][3][3];
        int64_t others = 0;
        for (int c = 0; c < 3; ++c)
            for (int b = 0; b < 3; ++b)
                for (int a = 0; a < 3; ++a) {
                    if (a == 1 && b == 1 && c == 1) continue;
                    int64_t v = (int64_t)wmul(wmul(wmul(aM, w[0][a]), w[1][b]), w[2][c]);
                    q[c][b][a] = M < 0 ? -v : v;
                    others += q[c][b][a];
                }
        q[1][1][1] = M - others;
        for (int c = 0; c < 3; ++c)
            for (int b = 0; b < 3; ++b)
                for (int a = 0; a < 3; ++a) {
                    int64_t g[3] = {ic[0] + a - 1 - lo[0], ic[1] + b - 1 - lo[1], ic[2] + c - 1 - lo[2]};
                    int inside = 1;
                    for (int j = 0; j < 3; ++j) {
                        if (mode == 1) {
                            if (g[j] < 0) g[j] = 0;
                            if (g[j] >= G[j]) g[j] = G[j] - 1;
                        } else if (mode == 2) {
                            g[j] = mod_pos(g[j], G[j]);
                        } else if (g[j] < 0 || g[j] >= G[j]) {
                            inside = 0;
                        }
                    }
                    if (!inside) continue;
                    /* int64 sums are exact and order-independent: use unsigned wrap */
                    int64_t idx = g[0] + G[0] * (g[1] + G[1] * g[2]);
                    gmf[idx] = (int64_t)((uint64_t)gmf[idx] + (uint64_t)q[c][b][a]);
                }
    }
    return status;
}

/* ------------------------------------------------------------------------ */
/* Baryons into the GMF, Sec. 2: interior cells take the grid's own gas;      */
/* border cells take the parent cell's density (the parent's baryons copied   */
/* onto the boundary); mass = rint((rho * delta^3) * 2^F).  G = N + 2B.       */
/* start: global level index of interior cell 0; pstart: parent's, in parent */
/* cells; R: refinement factor.  pgas may be NULL (no baryons in the border). */
/* A border cell whose parent cell lies outside the parent (a child of an     */
/* isolated root reaching past the box) has no baryons: nothing lies outside  */
/* an isolated domain.                                                        */
/* ------------------------------------------------------------------------ */
void orc_gas(const double* gas, const int64_t N[3], int64_t B, const double* pgas,
             const int64_t Np[3], const int64_t pstart[3], const int64_t start[3], int R,
             double delta, int F, int64_t* gmf) {
    double scale = ldexp(1.0, F);
    double vol = (delta * delta) * delta;
    int64_t G[3] = {N[0] + 2 * B, N[1] + 2 * B, N[2] + 2 * B};
    for (int64_t z = 0; z < G[2]; ++z)
        for (int64_t y = 0; y < G[1]; ++y)
            for (int64_t x = 0; x < G[0]; ++x) {
                int64_t c[3] = {x - B, y - B, z - B};
                int interior = 1;
                for (int j = 0; j < 3; ++j)
                    if (c[j] < 0 || c[j] >= N[j]) interior = 0;
                double rho = 0.0;
                if (interior) {
                    if (gas) rho = gas[c[0] + N[0] * (c[1] + N[1] * c[2])];
                } else if (pgas) {
                    int64_t pc[3];
                    int inside = 1;
                    for (int j = 0; j < 3; ++j) {
                        pc[j] = floor_div(start[j] + c[j], R) - pstart[j];
                        if (pc[j] < 0 || pc[j] >= Np[j]) inside = 0;
                    }
                    if (inside) rho = pgas[pc[0] + Np[0] * (pc[1] + Np[1] * pc[2])];
                }
                int64_t q = (int64_t)rint((rho * vol) * scale);
                int64_t idx = x + G[0] * (y + G[1] * z);
                gmf[idx] = (int64_t)((uint64_t)gmf[idx] + (uint64_t)q);
            }
}

/* ------------------------------------------------------------------------ */
/* Potential of one grid, Sec. 2.2 (Eq. PoissonFourier with the table T):     */
/* the GMF box (G cells, cell mass = GMF * 2^-F) placed at M-grid index 0,    */
/* zeros elsewhere; phi = IDFT_M( T * DFT_M(mass) ) / (M0 M1 M2); the output  */
/* window of W cells starts at M-grid index s0 (taken modulo M).              */
/* T is the octant table of orc_green_table (even in every kappa_j).          */
/* ------------------------------------------------------------------------ */
void orc_solve(const int64_t* gmf, const int64_t G[3], int F, const int64_t M[3],
               const int64_t s0[3], const int64_t W[3], const double* T, double* phis,
               int nthreads) {
    int64_t tot = M[0] * M[1] * M[2];
    int64_t H[3] = {M[0] / 2 + 1, M[1] / 2 + 1, M[2] / 2 + 1};
    double* re = (double*)calloc((size_t)tot, sizeof(double));
    double* im = (double*)calloc((size_t)tot, sizeof(double));
    for (int64_t z = 0; z < G[2]; ++z)
        for (int64_t y = 0; y < G[1]; ++y)
            for (int64_t x = 0; x < G[0]; ++x)
                re[x + M[0] * (y + M[1] * z)] = ldexp((double)gmf[x + G[0] * (y + G[1] * z)], -F);
    orc_dft3(re, im, M, -1, nthreads);
    for (int64_t z = 0; z < M[2]; ++z)
        for (int64_t y = 0; y < M[1]; ++y)
            for (int64_t x = 0; x < M[0]; ++x) {
                int64_t fx = x <= M[0] / 2 ? x : M[0] - x;
                int64_t fy = y <= M[1] / 2 ? y : M[1] - y;
                int64_t fz = z <= M[2] / 2 ? z : M[2] - z;
                double t = T[fx + H[0] * (fy + H[1] * fz)];
                int64_t i = x + M[0] * (y + M[1] * z);
                re[i] *= t;
                im[i] *= t;
            }
    orc_dft3(re, im, M, +1, nthreads);
    double norm = 1.0 / ((double)M[0] * (double)M[1] * (double)M[2]);
    for (int64_t z = 0; z < W[2]; ++z)
        for (int64_t y = 0; y < W[1]; ++y)
            for (int64_t x = 0; x < W[0]; ++x) {
                int64_t mx = mod_pos(s0[0] + x, M[0]);
                int64_t my = mod_pos(s0[1] + y, M[1]);
                int64_t mz = mod_pos(s0[2] + z, M[2]);
                phis[x + W[0] * (y + W[1] * z)] = re[mx + M[0] * (my + M[1] * mz)] * norm;
            }
    free(re);
    free(im);
}

/* ------------------------------------------------------------------------ */
/* Spectral gradient (Sec. 2.2, D = -ik; reading R15): phi-hat = T rho-hat as */
/* in orc_solve, and each short-range acceleration component                  */
/* A_j = -d phi / dx_j is the inverse transform of -i D_j phi-hat, D_j = k_j  */
/* (0 on an even M_j's Nyquist mode).  Writes four windows of W cells one     */
/* after the other: phi, A_x, A_y, A_z.                                       */
/* ------------------------------------------------------------------------ */
void orc_solve_spectral(const int64_t* gmf, const int64_t G[3], int F, const int64_t M[3],
                        const int64_t s0[3], const int64_t W[3], const double* T, double delta,
                        double* out, int nthreads) {
    int64_t tot = M[0] * M[1] * M[2];
    int64_t nw = W[0] * W[1] * W[2];
    int64_t H[3] = {M[0] / 2 + 1, M[1] / 2 + 1, M[2] / 2 + 1};
    double* sre = (double*)calloc((size_t)tot, sizeof(double));
    double* sim = (double*)calloc((size_t)tot, sizeof(double));
    double* re = (double*)malloc((size_t)tot * sizeof(double));
    double* im = (double*)malloc((size_t)tot * sizeof(double));
    for (int64_t z = 0; z < G[2]; ++z)
        for (int64_t y = 0; y < G[1]; ++y)
            for (int64_t x = 0; x < G[0]; ++x)
                sre[x + M[0] * (y + M[1] * z)] = ldexp((double)gmf[x + G[0] * (y + G[1] * z)], -F);
    orc_dft3(sre, sim, M, -1, nthreads);
    for (int64_t z = 0; z < M[2]; ++z)
        for (int64_t y = 0; y < M[1]; ++y)
            for (int64_t x = 0; x < M[0]; ++x) {
                int64_t fx = x <= M[0] / 2 ? x : M[0] - x;
                int64_t fy = y <= M[1] / 2 ? y : M[1] - y;
                int64_t fz = z <= M[2] / 2 ? z : M[2] - z;
                double t = T[fx + H[0] * (fy + H[1] * fz)];
                int64_t i = x + M[0] * (y + M[1] * z);
                sre[i] *= t;
                sim[i] *= t;
            }
    double norm = 1.0 / ((double)M[0] * (double)M[1] * (double)M[2]);
    for (int comp = 0; comp < 4; ++comp) {
        for (int64_t z = 0; z < M[2]; ++z)
            for (int64_t y = 0; y < M[1]; ++y)
                for (int64_t x = 0; x < M[0]; ++x) {
                    int64_t i = x + M[0] * (y + M[1] * z);
                    if (comp == 0) {
                        re[i] = sre[i];
                        im[i] = sim[i];
                        continue;
                    }
                    int64_t kap[3] = {x, y, z};
                    int j = comp - 1;
                    int64_t kc = kap[j] > M[j] / 2 ? kap[j] - M[j] : kap[j];
                    double d = orc_grad_d(2, kc, M[j], delta);
                    /* -i d (a + i b) = d b - i d a */
                    re[i] = d * sim[i];
                    im[i] = -d * sre[i];
                }
        orc_dft3(re, im, M, +1, nthreads);
        for (int64_t z = 0; z < W[2]; ++z)
            for (int64_t y = 0; y < W[1]; ++y)
                for (int64_t x = 0; x < W[0]; ++x) {
                    int64_t mx = mod_pos(s0[0] + x, M[0]);
                    int64_t my = mod_pos(s0[1] + y, M[1]);
                    int64_t mz = mod_pos(s0[2] + z, M[2]);
                    out[comp * nw + x + W[0] * (y + W[1] * z)] = re[mx + M[0] * (my + M[1] * mz)] * norm;
                }
    }
    free(sre);
    free(sim);
    free(re);
    free(im);
}

/* ------------------------------------------------------------------------ */
/* Cell-centred acceleration and carry from the parent, Sec. 2.2 (reading R8, */
/* R10, R15): for c in [-1, N]^3                                              */
/*   phi(c)   = phis(c) + I(parent phi)(c)                                    */
/*   acc_j(c) = A_j(c) + I(parent acc_j)(c), where A_j is                     */
/*     grad 0: -(phis(c+e_j) - phis(c-e_j)) / (2 delta)                       */
/*     grad 1: -(8 (phis(c+e_j) - phis(c-e_j))                                */
/*               - (phis(c+2e_j) - phis(c-2e_j))) / (12 delta)                */
/*     grad 2: the spectral component j + 1 of orc_solve_spectral             */
/* phis spans [-h, N+h)^3 (h = 3 for grad 1, else 2; grad 2: four such        */
/* windows), phi and acc (3 SoA components) span [-1, N+1)^3, parent fields   */
/* span the parent's [-1, Np+1)^3.  I is trilinear from the parent cell      */
/* centres.  pphi == NULL: no parent term (root).                             */
/* ------------------------------------------------------------------------ */
void orc_accel(const double* phis, const int64_t N[3], int grad, double delta,
               const int64_t start[3], const double* pphi, const double* pacc, const int64_t Np[3],
               const int64_t pstart[3], int R, double* phi, double* acc) {
    int64_t h = grad == 1 ? 3 : 2;
    int64_t S[3] = {N[0] + 2 * h, N[1] + 2 * h, N[2] + 2 * h};
    int64_t nw = S[0] * S[1] * S[2];
    int64_t E[3] = {N[0] + 2, N[1] + 2, N[2] + 2};
    int64_t Ep[3] = {Np[0] + 2, Np[1] + 2, Np[2] + 2};
    int64_t ncell = E[0] * E[1] * E[2];
    int64_t npc = Ep[0] * Ep[1] * Ep[2];
    for (int64_t z = -1; z <= N[2]; ++z)
        for (int64_t y = -1; y <= N[1]; ++y)
            for (int64_t x = -1; x <= N[0]; ++x) {
                int64_t c[3] = {x, y, z};
#define PHIS(a, b, d) phis[((a) + h) + S[0] * (((b) + h) + S[1] * ((d) + h))]
                double p0 = PHIS(x, y, z);
                double a0, a1, a2;
                if (grad == 0) {
                    a0 = -(PHIS(x + 1, y, z) - PHIS(x - 1, y, z)) / (2.0 * delta);
                    a1 = -(PHIS(x, y + 1, z) - PHIS(x, y - 1, z)) / (2.0 * delta);
                    a2 = -(PHIS(x, y, z + 1) - PHIS(x, y, z - 1)) / (2.0 * delta);
                } else if (grad == 1) {
                    a0 = -(8.0 * (PHIS(x + 1, y, z) - PHIS(x - 1, y, z))
                           - (PHIS(x + 2, y, z) - PHIS(x - 2, y, z))) / (12.0 * delta);
                    a1 = -(8.0 * (PHIS(x, y + 1, z) - PHIS(x, y - 1, z))
                           - (PHIS(x, y + 2, z) - PHIS(x, y - 2, z))) / (12.0 * delta);
                    a2 = -(8.0 * (PHIS(x, y, z + 1) - PHIS(x, y, z - 1))
                           - (PHIS(x, y, z + 2) - PHIS(x, y, z - 2))) / (12.0 * delta);
                } else {
                    a0 = (phis + nw)[(x + h) + S[0] * ((y + h) + S[1] * (z + h))];
                    a1 = (phis + 2 * nw)[(x + h) + S[0] * ((y + h) + S[1] * (z + h))];
                    a2 = (phis + 3 * nw)[(x + h) + S[0] * ((y + h) + S[1] * (z + h))];
                }
#undef PHIS
                if (pphi) {
                    int64_t i0[3];
                    double f[3];
                    for (int j = 0; j < 3; ++j) {
                        double t = ((double)(start[j] + c[j]) + 0.5) / (double)R - 0.5;
                        double fl = floor(t);
                        i0[j] = (int64_t)fl - pstart[j];
                        f[j] = t - fl;
                    }
                    double ip = 0.0, ia[3] = {0.0, 0.0, 0.0};
                    for (int dz = 0; dz < 2; ++dz)
                        for (int dy = 0; dy < 2; ++dy)
                            for (int dx = 0; dx < 2; ++dx) {
                                double w = ((dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]))
                                           * (dz ? f[2] : 1.0 - f[2]);
                                int64_t pi = (i0[0] + dx + 1)
                                             + Ep[0] * ((i0[1] + dy + 1) + Ep[1] * (i0[2] + dz + 1));
                                ip += w * pphi[pi];
                                for (int j = 0; j < 3; ++j) ia[j] += w * pacc[j * npc + pi];
                            }
                    p0 += ip;
                    a0 += ia[0];
                    a1 += ia[1];
                    a2 += ia[2];
                }
                int64_t o = (x + 1) + E[0] * ((y + 1) + E[1] * (z + 1));
                phi[o] = p0;
                acc[o] = a0;
                acc[ncell + o] = a1;
                acc[2 * ncell + o] = a2;
            }
}

/* ------------------------------------------------------------------------ */
/* TSC interpolation of the cell acceleration back to the particles, Sec. 2   */
/* (same 27 weights as the deposit).  Only particles with owner[p] == grid_id */
/* are written.  acc spans [-1, N+1)^3 (3 SoA components); mode 1 folds the   */
/* cloud into [0, N) (isolated root, reading R7), otherwise the ghost ring is */
/* read directly.  out is 3 x n SoA.                                           */
/* ------------------------------------------------------------------------ */
void orc_interp(int64_t n, const double* px, const double* py, const double* pz,
                const double* pvx, const double* pvy, const double* pvz, double half_dt,
                double box, int periodic, double delta0, int level, const int64_t start[3],
                const int64_t N[3], int mode, const double* acc, const int32_t* owner,
                int32_t grid_id, double* out) {
    int64_t E[3] = {N[0] + 2, N[1] + 2, N[2] + 2};
    int64_t ncell = E[0] * E[1] * E[2];
    for (int64_t p = 0; p < n; ++p) {
        if (owner[p] != grid_id) continue;
        double pos[3] = {px[p], py[p], pz[p]};
        double vel[3] = {pvx[p], pvy[p], pvz[p]};
        uint64_t w[3][3];
        int64_t ic[3];
        for (int j = 0; j < 3; ++j) {
            double xd = orc_drift(pos[j], vel[j], half_dt, box, 0);
            ic[j] = orc_tsc_fixed(pos_fixed(xd, delta0, box, periodic), level, w[j]) - start[j];
        }
        /* the 27 weights of the deposit: the centre takes 2^63 minus the other 26,
           so the weights sum to one exactly, as the charges sum to the mass */
        uint64_t wq[3][3][3];
        uint64_t wsum = 0;
        for (int c = 0; c < 3; ++c)
            for (int b = 0; b < 3; ++b)
                for (int aa = 0; aa < 3; ++aa) {
                    if (aa == 1 && b == 1 && c == 1) continue;
                    wq[c][b][aa] = wmul(wmul(w[0][aa], w[1][b]), w[2][c]);
                    wsum += wq[c][b][aa];
                }
        wq[1][1][1] = ((uint64_t)1 << 63) - wsum;
        double a[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < 3; ++c)
            for (int b = 0; b < 3; ++b)
                for (int aa = 0; aa < 3; ++aa) {
                    int64_t g[3] = {ic[0] + aa - 1, ic[1] + b - 1, ic[2] + c - 1};
                    if (mode == 1)
                        for (int j = 0; j < 3; ++j) {
                            if (g[j] < 0) g[j] = 0;
                            if (g[j] >= N[j]) g[j] = N[j] - 1;
                        }
                    double wt = ldexp((double)wq[c][b][aa], -63);
                    int64_t idx = (g[0] + 1) + E[0] * ((g[1] + 1) + E[1] * (g[2] + 1));
                    for (int j = 0; j < 3; ++j) a[j] += wt * acc[j * ncell + idx];
                }
        out[p] = a[0];
        out[n + p] = a[1];
        out[2 * n + p] = a[2];
    }
}

/* Global level-cell index of a drifted position, the cell the TSC cloud is    */
/* centred on (used to find the finest grid that holds each particle).        */
void orc_cells(int64_t n, const double* px, const double* py, const double* pz,
               const double* pvx, const double* pvy, const double* pvz, double half_dt,
               double box, int periodic, double delta0, int level, int64_t* cells /* 3 x n */) {
    for (int64_t p = 0; p < n; ++p) {
        double pos[3] = {px[p], py[p], pz[p]};
        double vel[3] = {pvx[p], pvy[p], pvz[p]};
        for (int j = 0; j < 3; ++j) {
            double xd = orc_drift(pos[j], vel[j], half_dt, box, 0);
            uint64_t w[3];
            cells[j * n + p] = orc_tsc_fixed(pos_fixed(xd, delta0, box, periodic), level, w);
        }
    }
}
