/*
 * lmoracle.c -- plain, slow, FP64 CPU oracle for the factored
 * Levenberg-Marquardt LNCC registration iteration of
 *   R. Jena, P. Chaudhari, J. C. Gee, "Factored Levenberg-Marquardt for
 *   Diffeomorphic Image Registration: An efficient optimizer for FireANTs".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may call this library.  The CUDA product
 * path never links, loads or calls it, and this file shares no code, header,
 * table or constant with the CUDA path.
 *
 * Everything is written in the most direct form of its definition: box sums
 * are literal k^3 window sums, trilinear sampling is the literal 8-corner
 * weighted sum, and every intermediate is a full FP64 volume.  No blocking,
 * fusion or reordering.
 *
 * Layout: a scalar volume is [nz][ny][nx] with x fastest; a vector field is
 * three such volumes back to back (component 0 = x, 1 = y, 2 = z), in voxel
 * units.  A displacement u(p) names the sample point q = p + u(p) in voxel
 * index coordinates.
 *
 * Readings of points the paper leaves open (each marked "reading" below) are
 * the ones fixed for this project; they are conventions shared with the CUDA
 * path, not facts printed in the paper.
 *
 * Pins (tests/test_oracle_*.py): FD gradients, brute-force and library
 * filters, explicit 3x3 solves (Appendix A, Eq. tilen), identity
 * invariants, scripted loss traces for the damping/rejection rules,
 * translation recovery.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stddef.h>

typedef struct {
    int    win;          /* LNCC box side k (odd) */
    double eps_nr;       /* LNCC numerator stabiliser */
    double eps_dr;       /* LNCC denominator stabiliser */
    double sigma_grad;   /* Gaussian sigma for the gradient (0 = off) */
    double sigma_warp;   /* Gaussian sigma for the composed warp (0 = off) */
    double step;         /* epsilon of the compositive update, voxels */
    double lambda0;      /* initial damping */
    double mu_inc;       /* damping increase factor mu+ */
    double mu_dec;       /* damping decrease factor mu- */
    double lambda_max;   /* damping cap (may be +inf) */
    int    reject;       /* 1 = rejection rule on */
    double tau;          /* rejection tolerance ratio */
    int    max_retries;  /* retries after a rejection */
    int    tile;         /* curvature tile side k (1 = Eq. tile1) */
    int    loss;         /* OR_LNCC or OR_MSE */
    int    method;       /* OR_LM or OR_DEMONS */
    double alpha;        /* Demons damping weight, lambda_x = alpha^2 r_x^2 */
    int    bins;         /* MI: histogram bins B per image */
} or_params;

#define OR_LNCC   0
#define OR_MSE    1
#define OR_MI     2
#define OR_LM     0
#define OR_DEMONS 1

#define OR_ACCEPT  0
#define OR_RETRY   1
#define OR_DISCARD 2

static size_t vox(int nx, int ny, int nz) { return (size_t)nx * ny * nz; }
static size_t at(int nx, int ny, int x, int y, int z)
{
    return ((size_t)z * ny + y) * nx + x;
}

/* Image value with zero outside [0, n-1] (reading: zero padding, the paper
 * never states the boundary rule of its resampler). */
static double img_zero(const double *X, int nx, int ny, int nz,
                       double x, double y, double z)
{
    if (!(x >= 0 && y >= 0 && z >= 0 && x <= nx - 1 && y <= ny - 1 &&
          z <= nz - 1))
        return 0.0; /* also catches NaN coordinates */
    return X[at(nx, ny, (int)x, (int)y, (int)z)];
}

/* Field value with the index clamped to [0, n-1] (reading: a displacement
 * field is extended at the border, not zeroed). */
static double fld_clamp(const double *X, int nx, int ny, int nz,
                        double x, double y, double z)
{
    if (!(x >= 0)) x = 0; /* also maps NaN to the first voxel */
    if (!(y >= 0)) y = 0;
    if (!(z >= 0)) z = 0;
    if (x > nx - 1) x = nx - 1;
    if (y > ny - 1) y = ny - 1;
    if (z > nz - 1) z = nz - 1;
    return X[at(nx, ny, (int)x, (int)y, (int)z)];
}

/* ------------------------------------------------------------------ */
/* Step (a): trilinear resampling J(p) = M(p + u(p)) and dJ/du.        */
/* Section 2.1 (the warp resamples the image at displaced points).     */
/* Cell split from the displacement: c = p + floor(u), f = u - floor(u) */
/* (reading: the split is taken on u itself, not on p + u).            */
/* ------------------------------------------------------------------ */
void or_sample(int nx, int ny, int nz, const double *M, const double *u,
               double *J, double *dJ)
{
    size_t V = vox(nx, ny, nz);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t p = at(nx, ny, x, y, z);
                double d[3] = {u[p], u[V + p], u[2 * V + p]};
                double c[3], f[3];
                const double pos[3] = {x, y, z};
                for (int i = 0; i < 3; ++i) {
                    double fl = floor(d[i]);
                    c[i] = pos[i] + fl;
                    f[i] = d[i] - fl;
                }
                double val = 0, gx = 0, gy = 0, gz = 0;
                for (int sz = 0; sz < 2; ++sz)
                    for (int sy = 0; sy < 2; ++sy)
                        for (int sx = 0; sx < 2; ++sx) {
                            double m = img_zero(M, nx, ny, nz, c[0] + sx,
                                                c[1] + sy, c[2] + sz);
                            double wx = sx ? f[0] : 1 - f[0];
                            double wy = sy ? f[1] : 1 - f[1];
                            double wz = sz ? f[2] : 1 - f[2];
                            val += wx * wy * wz * m;
                            gx += (sx ? 1.0 : -1.0) * wy * wz * m;
                            gy += (sy ? 1.0 : -1.0) * wx * wz * m;
                            gz += (sz ? 1.0 : -1.0) * wx * wy * m;
                        }
                J[p] = val;
                if (dJ) {
                    dJ[p] = gx;
                    dJ[V + p] = gy;
                    dJ[2 * V + p] = gz;
                }
            }
}

/* ------------------------------------------------------------------ */
/* Box mean: S_X(p) = k^-3 * sum over the k^3 window of X, X = 0       */
/* outside the volume, fixed divisor k^3 (reading for LNCC's local     */
/* statistics; the paper names LNCC but prints no formula).            */
/* ------------------------------------------------------------------ */
void or_box(int nx, int ny, int nz, int k, const double *X, double *S)
{
    int w = (k - 1) / 2;
    double inv = 1.0 / ((double)k * k * k);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double s = 0;
                for (int oz = -w; oz <= w; ++oz)
                    for (int oy = -w; oy <= w; ++oy)
                        for (int ox = -w; ox <= w; ++ox) {
                            int xx = x + ox, yy = y + oy, zz = z + oz;
                            if (xx < 0 || yy < 0 || zz < 0 || xx >= nx ||
                                yy >= ny || zz >= nz)
                                continue;
                            s += X[at(nx, ny, xx, yy, zz)];
                        }
                S[at(nx, ny, x, y, z)] = s * inv;
            }
}

/* ------------------------------------------------------------------ */
/* Step (b), forward and coefficients of the backward pass.            */
/* Squared local correlation per voxel (reading of LNCC, Section 2.2): */
/*   A = S_FJ - mF mJ, B = max(S_FF - mF^2, 0), C = max(S_JJ - mJ^2, 0) */
/*   cc = (A^2 + eps_nr) / (B C + eps_dr)                              */
/* and the partial derivatives of cc with respect to the three J-side  */
/* window means:                                                       */
/*   a = d cc / d S_FJ, b = d cc / d S_JJ, c = d cc / d S_J.           */
/* Reading: the clamps only guard against rounding (an exact window    */
/* variance is never negative), so C's derivative is taken as 1, its   */
/* value on C >= 0; b = -(A^2 + eps_nr) B / D^2 everywhere.  A slope of */
/* 0 on the clamped side would let rounding decide a jump of b in      */
/* windows where J is constant.                                        */
/* ------------------------------------------------------------------ */
void or_lncc_terms(int nx, int ny, int nz, int k, double eps_nr,
                   double eps_dr, const double *F, const double *J,
                   double *cc, double *a, double *b, double *c)
{
    size_t V = vox(nx, ny, nz);
    double *FF = malloc(V * sizeof(double)), *JJ = malloc(V * sizeof(double));
    double *FJ = malloc(V * sizeof(double));
    double *sF = malloc(V * sizeof(double)), *sJ = malloc(V * sizeof(double));
    double *sFF = malloc(V * sizeof(double)), *sJJ = malloc(V * sizeof(double));
    double *sFJ = malloc(V * sizeof(double));
    for (size_t p = 0; p < V; ++p) {
        FF[p] = F[p] * F[p];
        JJ[p] = J[p] * J[p];
        FJ[p] = F[p] * J[p];
    }
    or_box(nx, ny, nz, k, F, sF);
    or_box(nx, ny, nz, k, J, sJ);
    or_box(nx, ny, nz, k, FF, sFF);
    or_box(nx, ny, nz, k, JJ, sJJ);
    or_box(nx, ny, nz, k, FJ, sFJ);
    for (size_t p = 0; p < V; ++p) {
        double mF = sF[p], mJ = sJ[p];
        double A = sFJ[p] - mF * mJ;
        double Braw = sFF[p] - mF * mF;
        double Craw = sJJ[p] - mJ * mJ;
        double B = Braw > 0 ? Braw : 0;
        double C = Craw > 0 ? Craw : 0;
        double N = A * A + eps_nr;
        double D = B * C + eps_dr;
        double ccv = N / D;
        double av = 2.0 * A / D;
        double bv = -N * B / (D * D);
        double cv = -av * mF - 2.0 * bv * mJ;
        if (cc) cc[p] = ccv;
        if (a) a[p] = av;
        if (b) b[p] = bv;
        if (c) c[p] = cv;
    }
    free(FF); free(JJ); free(FJ); free(sF); free(sJ); free(sFF); free(sJJ);
    free(sFJ);
}

/* ------------------------------------------------------------------ */
/* Gaussian taps: t_j proportional to exp(-j^2 / (2 sigma^2)) for      */
/* |j| <= R = ceil(3 sigma), normalised to sum 1; sigma = 0 gives the  */
/* single tap 1 (reading: radius and normalisation are not stated).    */
/* Returns R; taps[0..2R] hold t_{-R..R}.  taps must hold 2R+1 values. */
/* ------------------------------------------------------------------ */
int or_gauss_radius(double sigma)
{
    if (!(sigma > 0)) return 0;
    return (int)ceil(3.0 * sigma);
}

int or_gauss_taps(double sigma, double *taps)
{
    int R = or_gauss_radius(sigma);
    if (R == 0) {
        taps[0] = 1.0;
        return 0;
    }
    double s = 0;
    for (int j = -R; j <= R; ++j) {
        taps[j + R] = exp(-(double)j * j / (2.0 * sigma * sigma));
        s += taps[j + R];
    }
    for (int j = 0; j <= 2 * R; ++j) taps[j] /= s;
    return R;
}

/* One 1-D convolution along axis (0 = x, 1 = y, 2 = z).  clamp = 0: zero
 * padding; clamp = 1: the index is clamped to the volume (edge replicated). */
static void conv1d(int nx, int ny, int nz, int axis, int R, const double *t,
                   int clamp, const double *X, double *Y)
{
    int n[3] = {nx, ny, nz};
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int p[3] = {x, y, z};
                double s = 0;
                for (int j = -R; j <= R; ++j) {
                    int q[3] = {x, y, z};
                    q[axis] = p[axis] + j;
                    if (q[axis] < 0 || q[axis] >= n[axis]) {
                        if (!clamp) continue;
                        q[axis] = q[axis] < 0 ? 0 : n[axis] - 1;
                    }
                    s += t[j + R] * X[at(nx, ny, q[0], q[1], q[2])];
                }
                Y[at(nx, ny, x, y, z)] = s;
            }
}

/* Separable Gaussian smoothing of one scalar volume (x, then y, then z),
 * zero padding (gradients, images) or edge clamping (displacement fields). */
static void smooth_mode(int nx, int ny, int nz, double sigma, int clamp,
                        const double *X, double *Y)
{
    size_t V = vox(nx, ny, nz);
    int R = or_gauss_radius(sigma);
    if (R == 0) {
        memcpy(Y, X, V * sizeof(double));
        return;
    }
    double *t = malloc((2 * R + 1) * sizeof(double));
    or_gauss_taps(sigma, t);
    double *T1 = malloc(V * sizeof(double)), *T2 = malloc(V * sizeof(double));
    conv1d(nx, ny, nz, 0, R, t, clamp, X, T1);
    conv1d(nx, ny, nz, 1, R, t, clamp, T1, T2);
    conv1d(nx, ny, nz, 2, R, t, clamp, T2, Y);
    free(t); free(T1); free(T2);
}

void or_smooth(int nx, int ny, int nz, double sigma, const double *X,
               double *Y)
{
    smooth_mode(nx, ny, nz, sigma, 0, X, Y);
}

void or_smooth_field(int nx, int ny, int nz, double sigma, const double *X,
                     double *Y)
{
    smooth_mode(nx, ny, nz, sigma, 1, X, Y);
}

/* ------------------------------------------------------------------ */
/* Mutual information with Parzen windows (Section 2.2: the squared-loss */
/* form (log2 B - MI)^2, B bins).  Readings (the paper names only the    */
/* Parzen windowing and B):                                              */
/*   - both images map to [0, 1] through the joint range [lo, hi] of F,   */
/*     M and 0 (0 is the resampler's padding value);                     */
/*   - a value v sits at bin coordinate t = 1 + (B - 3) (v - lo)/(hi - lo)*/
/*     and spreads over the four bins floor(t) - 1 .. floor(t) + 2 with  */
/*     cubic B-spline weights beta3(t - i), which sum to one;            */
/*   - p_ij = V^-1 sum_x a_i(F(x)) b_j(J(x)), with the fixed and moving   */
/*     marginals p_i = sum_j p_ij, q_j = sum_i p_ij;                      */
/*   - MI = sum_ij p_ij log2(p_ij / (p_i q_j)) (0 log 0 = 0), in bits, so */
/*     0 <= MI <= log2 B.                                                */
/* dMI/dJ(x) = V^-1 dt/dv sum_ij a_i(F(x)) b_j'(J(x)) log2(p_ij / q_j)     */
/* (the marginal of F does not depend on J; the terms of the derivative  */
/* of the logs cancel because sum_ij dp_ij = sum_j dq_j).                */
/* ------------------------------------------------------------------ */
static double bspline3(double x)
{
    double a = fabs(x);
    if (a < 1.0) return 2.0 / 3.0 - a * a + 0.5 * a * a * a;
    if (a < 2.0) {
        double b = 2.0 - a;
        return b * b * b / 6.0;
    }
    return 0.0;
}

static double bspline3_deriv(double x)
{
    double a = fabs(x), s = x < 0 ? -1.0 : 1.0;
    if (a < 1.0) return s * (-2.0 * a + 1.5 * a * a);
    if (a < 2.0) {
        double b = 2.0 - a;
        return -s * 0.5 * b * b;
    }
    return 0.0;
}

void or_mi_range(int nx, int ny, int nz, const double *F, const double *M,
                 double *lo, double *hi)
{
    size_t V = vox(nx, ny, nz);
    double a = 0.0, b = 0.0;
    for (size_t p = 0; p < V; ++p) {
        if (F[p] < a) a = F[p];
        if (F[p] > b) b = F[p];
        if (M[p] < a) a = M[p];
        if (M[p] > b) b = M[p];
    }
    if (!(b > a)) b = a + 1.0;   /* constant images: any width */
    *lo = a;
    *hi = b;
}

/* MI of (F, J) and dMI/dJ per voxel (dmi, may be NULL). */
void or_mi(int nx, int ny, int nz, int B, double lo, double hi,
           const double *F, const double *J, double *mi_out, double *dmi)
{
    size_t V = vox(nx, ny, nz);
    double sc = (B - 3) / (hi - lo);
    double *pj = calloc((size_t)B * B, sizeof(double));
    for (size_t p = 0; p < V; ++p) {
        double tf = 1.0 + sc * (F[p] - lo), tm = 1.0 + sc * (J[p] - lo);
        for (int i = 0; i < B; ++i) {
            double a = bspline3(tf - i);
            if (a == 0.0) continue;
            for (int j = 0; j < B; ++j) pj[i * B + j] += a * bspline3(tm - j);
        }
    }
    for (int e = 0; e < B * B; ++e) pj[e] /= (double)V;
    double *pf = calloc(B, sizeof(double)), *qm = calloc(B, sizeof(double));
    for (int i = 0; i < B; ++i)
        for (int j = 0; j < B; ++j) {
            pf[i] += pj[i * B + j];
            qm[j] += pj[i * B + j];
        }
    double mi = 0.0;
    for (int i = 0; i < B; ++i)
        for (int j = 0; j < B; ++j) {
            double v = pj[i * B + j];
            if (v > 0) mi += v * log2(v / (pf[i] * qm[j]));
        }
    *mi_out = mi;
    if (dmi) {
        for (size_t p = 0; p < V; ++p) {
            double tf = 1.0 + sc * (F[p] - lo), tm = 1.0 + sc * (J[p] - lo);
            double s = 0.0;
            for (int i = 0; i < B; ++i) {
                double a = bspline3(tf - i);
                if (a == 0.0) continue;
                for (int j = 0; j < B; ++j) {
                    double v = pj[i * B + j];
                    if (v > 0)
                        s += a * bspline3_deriv(tm - j) * log2(v / qm[j]);
                }
            }
            dmi[p] = s * sc / (double)V;
        }
    }
    free(pj);
    free(pf);
    free(qm);
}

/* ------------------------------------------------------------------ */
/* Steps (a)-(c): one evaluation of the loss and its smoothed gradient. */
/*   L = r = 1 - LNCC, LNCC = V^-1 sum_p cc(p)  (Section 2.2, (1-LNCC)  */
/*   is the residual of the squared-loss form; reading: the rules of    */
/*   Eq. lambda-update / Eq. rejection compare r).                     */
/*   dL/dJ(y) = -V^-1 [F(y) Box(a)(y) + 2 J(y) Box(b)(y) + Box(c)(y)]   */
/*   g_raw = dL/dJ * dJ/du, g = G_sigma_grad * g_raw (per component).   */
/*   gmax = max_p |g(p)|_2.                                            */
/* Optional outputs (NULL to skip): dLdJ[V], graw[3V], g[3V], ccmap[V]. */
/* ------------------------------------------------------------------ */
void or_eval(int nx, int ny, int nz, const double *F, const double *M,
             const double *u, const or_params *P, double *L_out,
             double *dLdJ, double *graw, double *g, double *gmax_out,
             double *ccmap)
{
    size_t V = vox(nx, ny, nz);
    double *J = malloc(V * sizeof(double));
    double *dJ = malloc(3 * V * sizeof(double));
    double *cc = malloc(V * sizeof(double));
    double *a = malloc(V * sizeof(double)), *b = malloc(V * sizeof(double));
    double *c = malloc(V * sizeof(double));
    double *Ba = malloc(V * sizeof(double)), *Bb = malloc(V * sizeof(double));
    double *Bc = malloc(V * sizeof(double));
    double *gr = malloc(3 * V * sizeof(double));

    or_sample(nx, ny, nz, M, u, J, dJ);
    double L;
    if (P->loss == OR_MI) {
        /* Section 2.2, MI: r = L = log2(B) - MI (the residual of the
         * squared-loss form), dL/dJ = -dMI/dJ; cc receives 0. */
        double lo, hi, mi;
        or_mi_range(nx, ny, nz, F, M, &lo, &hi);
        or_mi(nx, ny, nz, P->bins, lo, hi, F, J, &mi, a);
        L = log2((double)P->bins) - mi;
        for (size_t p = 0; p < V; ++p) {
            double dl = -a[p];
            if (dLdJ) dLdJ[p] = dl;
            for (int i = 0; i < 3; ++i) gr[i * V + p] = dl * dJ[i * V + p];
            cc[p] = 0.0;
        }
    } else if (P->loss == OR_MSE) {
        /* Section 2.2, MSE: L = r = V^-1 sum_p (F(p) - J(p))^2 (already a
         * squared loss; reading: r is the loss value, as for LNCC), and
         * dL/dJ(p) = -2 (F(p) - J(p)) / V.  cc receives (F - J)^2. */
        double sum = 0;
        for (size_t p = 0; p < V; ++p) {
            double d = F[p] - J[p];
            cc[p] = d * d;
            sum += d * d;
        }
        L = sum / (double)V;
        for (size_t p = 0; p < V; ++p) {
            double dl = -2.0 * (F[p] - J[p]) / (double)V;
            if (dLdJ) dLdJ[p] = dl;
            for (int i = 0; i < 3; ++i) gr[i * V + p] = dl * dJ[i * V + p];
        }
    } else {
        or_lncc_terms(nx, ny, nz, P->win, P->eps_nr, P->eps_dr, F, J, cc, a, b,
                      c);
        double sum = 0;
        for (size_t p = 0; p < V; ++p) sum += cc[p];
        L = 1.0 - sum / (double)V;
        or_box(nx, ny, nz, P->win, a, Ba);
        or_box(nx, ny, nz, P->win, b, Bb);
        or_box(nx, ny, nz, P->win, c, Bc);
        for (size_t p = 0; p < V; ++p) {
            double dl = -(F[p] * Ba[p] + 2.0 * J[p] * Bb[p] + Bc[p]) / (double)V;
            if (dLdJ) dLdJ[p] = dl;
            for (int i = 0; i < 3; ++i) gr[i * V + p] = dl * dJ[i * V + p];
        }
    }
    if (graw) memcpy(graw, gr, 3 * V * sizeof(double));

    double gm = 0;
    if (g || gmax_out) {
        double *gs = g ? g : malloc(3 * V * sizeof(double));
        for (int i = 0; i < 3; ++i)
            or_smooth(nx, ny, nz, P->sigma_grad, gr + i * V, gs + i * V);
        for (size_t p = 0; p < V; ++p) {
            double n = sqrt(gs[p] * gs[p] + gs[V + p] * gs[V + p] +
                            gs[2 * V + p] * gs[2 * V + p]);
            if (n > gm) gm = n;
        }
        if (!g) free(gs);
    }
    if (L_out) *L_out = L;
    if (gmax_out) *gmax_out = gm;
    if (ccmap) memcpy(ccmap, cc, V * sizeof(double));
    free(J); free(dJ); free(cc); free(a); free(b); free(c); free(Ba);
    free(Bb); free(Bc); free(gr);
}

/* ------------------------------------------------------------------ */
/* Demons as per-voxel LM on MSE, Eq. demons (Section 2.3):             */
/*   r(p) = F(p) - J(p),  n(p) = dJ/du(p) (the gradient of M at p + u),  */
/*   du(p) = r n / (|n|^2 + lambda_p),  lambda_p = alpha^2 r^2           */
/* (0 where r and n both vanish).  du: [3V] (written).                  */
/* ------------------------------------------------------------------ */
void or_demons_force(int nx, int ny, int nz, const double *F,
                     const double *M, const double *u, double alpha,
                     double *du)
{
    size_t V = vox(nx, ny, nz);
    double *J = malloc(V * sizeof(double));
    double *dJ = malloc(3 * V * sizeof(double));
    or_sample(nx, ny, nz, M, u, J, dJ);
    for (size_t p = 0; p < V; ++p) {
        double r = F[p] - J[p];
        double n2 = dJ[p] * dJ[p] + dJ[V + p] * dJ[V + p] +
                    dJ[2 * V + p] * dJ[2 * V + p];
        double den = n2 + alpha * alpha * r * r;
        for (int i = 0; i < 3; ++i)
            du[i * V + p] = den > 0 ? r * dJ[i * V + p] / den : 0.0;
    }
    free(J);
    free(dJ);
}

/* Demons evaluation of a field: L = MSE (as or_eval with OR_MSE) and     */
/* the smoothed update g = G_sigma_grad * du of Eq. demons (reading: the  */
/* Gaussian of the gradient doubles as the fluid-like smoothing of the    */
/* update, Section 2.3 leaves the regulariser open); gmax = max |g|.      */
void or_demons_eval(int nx, int ny, int nz, const double *F, const double *M,
                    const double *u, const or_params *P, double *L_out,
                    double *g, double *gmax_out)
{
    size_t V = vox(nx, ny, nz);
    double *J = malloc(V * sizeof(double));
    double *dJ = malloc(3 * V * sizeof(double));
    double *du = malloc(3 * V * sizeof(double));
    or_sample(nx, ny, nz, M, u, J, dJ);
    double sum = 0;
    for (size_t p = 0; p < V; ++p) sum += (F[p] - J[p]) * (F[p] - J[p]);
    or_demons_force(nx, ny, nz, F, M, u, P->alpha, du);
    for (int i = 0; i < 3; ++i)
        or_smooth(nx, ny, nz, P->sigma_grad, du + i * V, g + i * V);
    double gm = 0;
    for (size_t p = 0; p < V; ++p) {
        double n = sqrt(g[p] * g[p] + g[V + p] * g[V + p] +
                        g[2 * V + p] * g[2 * V + p]);
        if (n > gm) gm = n;
    }
    if (L_out) *L_out = sum / (double)V;
    if (gmax_out) *gmax_out = gm;
    free(J);
    free(dJ);
    free(du);
}

/* ------------------------------------------------------------------ */
/* Compositive update, Eq. compositive (Section 2.1):                  */
/*   out(p) = v(p) + u(p + v(p)), u resampled trilinearly with the      */
/*   cell split taken on v and the corner index clamped to the volume.  */
/* ------------------------------------------------------------------ */
void or_compose(int nx, int ny, int nz, const double *u, const double *v,
                double *out)
{
    size_t V = vox(nx, ny, nz);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t p = at(nx, ny, x, y, z);
                double d[3] = {v[p], v[V + p], v[2 * V + p]};
                double c[3], f[3];
                const double pos[3] = {x, y, z};
                for (int i = 0; i < 3; ++i) {
                    double fl = floor(d[i]);
                    c[i] = pos[i] + fl;
                    f[i] = d[i] - fl;
                }
                for (int comp = 0; comp < 3; ++comp) {
                    const double *U = u + comp * V;
                    double s = 0;
                    for (int sz = 0; sz < 2; ++sz)
                        for (int sy = 0; sy < 2; ++sy)
                            for (int sx = 0; sx < 2; ++sx) {
                                double wx = sx ? f[0] : 1 - f[0];
                                double wy = sy ? f[1] : 1 - f[1];
                                double wz = sz ? f[2] : 1 - f[2];
                                s += wx * wy * wz *
                                     fld_clamp(U, nx, ny, nz, c[0] + sx,
                                               c[1] + sy, c[2] + sz);
                            }
                    out[comp * V + p] = d[comp] + s;
                }
            }
}

/* ------------------------------------------------------------------ */
/* Pooled curvature, Eq. tilen (Section 2.2; tile side k, Section 3):   */
/*   H_T   = |T|^-1 sum_{q in T} ghat(q) ghat(q)^T                       */
/*   du(p) = -(H_T + lambda I)^-1 r ghat(p),   T = the tile holding p    */
/* Readings: the tiles are the non-overlapping k x k x k blocks of the   */
/* grid (p lies in tile floor(p / k) along each axis; the last tile of   */
/* an axis is cut at the volume edge), and the pooling is the mean over  */
/* the tile (a local covariance), so that k = 1 is Eq. tile1 exactly.    */
/* Each 3 x 3 system is solved by Gaussian elimination with partial      */
/* pivoting.  ghat: [3V]; du: [3V] (written).                            */
/* ------------------------------------------------------------------ */
static void solve3(double A[3][3], double b[3], double x[3])
{
    for (int c = 0; c < 3; ++c) {
        int piv = c;
        for (int r = c + 1; r < 3; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (piv != c) {
            for (int j = 0; j < 3; ++j) {
                double t = A[c][j];
                A[c][j] = A[piv][j];
                A[piv][j] = t;
            }
            double t = b[c];
            b[c] = b[piv];
            b[piv] = t;
        }
        for (int r = c + 1; r < 3; ++r) {
            double f = A[r][c] / A[c][c];
            for (int j = c; j < 3; ++j) A[r][j] -= f * A[c][j];
            b[r] -= f * b[c];
        }
    }
    for (int r = 2; r >= 0; --r) {
        double s = b[r];
        for (int j = r + 1; j < 3; ++j) s -= A[r][j] * x[j];
        x[r] = s / A[r][r];
    }
}

void or_tile_du(int nx, int ny, int nz, int k, const double *gh, double r,
                double lambda, double *du)
{
    size_t V = vox(nx, ny, nz);
    int tx = (nx + k - 1) / k, ty = (ny + k - 1) / k, tz = (nz + k - 1) / k;
    size_t nt = (size_t)tx * ty * tz;
    double *H = calloc(nt * 9, sizeof(double));
    double *cnt = calloc(nt, sizeof(double));
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t p = at(nx, ny, x, y, z);
                size_t t = ((size_t)(z / k) * ty + y / k) * tx + x / k;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
                        H[9 * t + 3 * i + j] += gh[i * V + p] * gh[j * V + p];
                cnt[t] += 1.0;
            }
    for (size_t t = 0; t < nt; ++t)
        for (int e = 0; e < 9; ++e) H[9 * t + e] /= cnt[t];
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t p = at(nx, ny, x, y, z);
                size_t t = ((size_t)(z / k) * ty + y / k) * tx + x / k;
                double A[3][3], b[3], sol[3];
                for (int i = 0; i < 3; ++i) {
                    for (int j = 0; j < 3; ++j)
                        A[i][j] = H[9 * t + 3 * i + j] + (i == j ? lambda : 0.0);
                    b[i] = r * gh[i * V + p];
                }
                solve3(A, b, sol);
                for (int i = 0; i < 3; ++i) du[i * V + p] = -sol[i];
            }
    free(H);
    free(cnt);
}

/* ------------------------------------------------------------------ */
/* Steps (c)-(d): the trial field from the current state.              */
/*   ghat = g / gmax (0 if gmax = 0)   (reading of "normalised by the    */
/*   same choice of epsilon": unit max-norm gradient, fixed epsilon)    */
/*   du = -r ghat / (|ghat|^2 + lambda)          Eq. tile1, Appendix A  */
/*   (tile side k > 1: du from the pooled curvature, or_tile_du;        */
/*   Demons: du = g, the smoothed update of Eq. demons, or_demons_eval) */
/*   v = step * du;  u' = v + u o (Id + v)       Eq. compositive        */
/*   u' <- G_sigma_warp * u'  (off when sigma_warp = 0; reading: the    */
/*   field is edge-extended, like the resampling of Eq. compositive)    */
/* Optional: du_out[3V] receives du (before the step scale).            */
/* ------------------------------------------------------------------ */
void or_trial(int nx, int ny, int nz, const double *u, const double *g,
              double gmax, double r, double lambda, const or_params *P,
              double *u_out, double *du_out)
{
    size_t V = vox(nx, ny, nz);
    double *v = malloc(3 * V * sizeof(double));
    if (P->method == OR_DEMONS) {
        /* Demons: g is the smoothed update of Eq. demons; v = step * g */
        for (size_t e = 0; e < 3 * V; ++e) {
            if (du_out) du_out[e] = g[e];
            v[e] = P->step * g[e];
        }
    } else if (P->tile > 1) {
        double *gh = malloc(3 * V * sizeof(double));
        for (size_t e = 0; e < 3 * V; ++e) gh[e] = gmax > 0 ? g[e] / gmax : 0.0;
        or_tile_du(nx, ny, nz, P->tile, gh, r, lambda, v);
        for (size_t e = 0; e < 3 * V; ++e) {
            if (du_out) du_out[e] = v[e];
            v[e] *= P->step;
        }
        free(gh);
    } else {
        for (size_t p = 0; p < V; ++p) {
            double gh[3];
            for (int i = 0; i < 3; ++i)
                gh[i] = gmax > 0 ? g[i * V + p] / gmax : 0.0;
            double n2 = gh[0] * gh[0] + gh[1] * gh[1] + gh[2] * gh[2];
            for (int i = 0; i < 3; ++i) {
                double du = -r * gh[i] / (n2 + lambda);
                if (du_out) du_out[i * V + p] = du;
                v[i * V + p] = P->step * du;
            }
        }
    }
    or_compose(nx, ny, nz, u, v, u_out);
    if (P->sigma_warp > 0) {
        double *tmp = malloc(V * sizeof(double));
        for (int i = 0; i < 3; ++i) {
            or_smooth_field(nx, ny, nz, P->sigma_warp, u_out + i * V, tmp);
            memcpy(u_out + i * V, tmp, V * sizeof(double));
        }
        free(tmp);
    }
    free(v);
}

/* ------------------------------------------------------------------ */
/* Step (e): damping and rejection decision for one evaluated trial.    */
/*   Rejection (Eq. rejection; Eq. delta-loss is tau = 1):              */
/*     prev = |L_t - L_{t-1}| (0 when there is no L_{t-1} yet, reading) */
/*     reject when L_trial - L_t > tau * prev  (strict)                 */
/*     on reject: lambda <- min(mu+ lambda, lambda_max); RETRY while    */
/*     retries < max_retries, else DISCARD (reading: the step is         */
/*     dropped and the state kept after the last retry).                */
/*   Otherwise ACCEPT with Eq. lambda-update: lambda <- mu+ lambda       */
/*     (capped, reading: the cap bounds every increase) when             */
/*     L_trial > L_t, else mu- lambda (ties are good steps).            */
/* ------------------------------------------------------------------ */
int or_decide(double L_trial, double L_t, double L_prev, int has_prev,
              double lambda, int retries, const or_params *P,
              double *lambda_out)
{
    if (P->reject) {
        double prev = has_prev ? fabs(L_t - L_prev) : 0.0;
        if (L_trial - L_t > P->tau * prev) {
            double lam = P->mu_inc * lambda;
            if (lam > P->lambda_max) lam = P->lambda_max;
            *lambda_out = lam;
            return retries < P->max_retries ? OR_RETRY : OR_DISCARD;
        }
    }
    double lam;
    if (L_trial > L_t) {
        lam = P->mu_inc * lambda;
        if (lam > P->lambda_max) lam = P->lambda_max;
    } else {
        lam = P->mu_dec * lambda;
    }
    *lambda_out = lam;
    return OR_ACCEPT;
}

/* ------------------------------------------------------------------ */
/* One LM iteration (steps (a)-(e)) from the state (u, g, gmax, L_t,    */
/* L_{t-1}, lambda), attempting trials until one is accepted or the     */
/* retry budget is spent.  In/out: u, g, gmax, L_t, L_prev, has_prev,   */
/* lambda.  Outputs: first-trial field and loss (optional), accepted    */
/* (1/0), number of retries, number of loss evaluations.                */
/* On DISCARD the field, gradient and loss history stay as they were    */
/* and lambda keeps its raised value.                                   */
/* ------------------------------------------------------------------ */
void or_lm_step(int nx, int ny, int nz, const double *F, const double *M,
                const or_params *P, double *u, double *g, double *gmax,
                double *L_t, double *L_prev, int *has_prev, double *lambda,
                double *u_first, double *L_first, int *accepted,
                int *retries, int *evals)
{
    size_t V = vox(nx, ny, nz);
    double *ut = malloc(3 * V * sizeof(double));
    double *gt = malloc(3 * V * sizeof(double));
    int nret = 0, nev = 0, acc = 0;
    for (;;) {
        double Lt, gmt, lam;
        or_trial(nx, ny, nz, u, g, *gmax, *L_t, *lambda, P, ut, NULL);
        if (P->method == OR_DEMONS)
            or_demons_eval(nx, ny, nz, F, M, ut, P, &Lt, gt, &gmt);
        else
            or_eval(nx, ny, nz, F, M, ut, P, &Lt, NULL, NULL, gt, &gmt, NULL);
        ++nev;
        if (nev == 1) {
            if (u_first) memcpy(u_first, ut, 3 * V * sizeof(double));
            if (L_first) *L_first = Lt;
        }
        /* Demons: no damping rule, every step is kept (Section 2.3) */
        int act = OR_ACCEPT;
        lam = *lambda;
        if (P->method != OR_DEMONS)
            act = or_decide(Lt, *L_t, *L_prev, *has_prev, *lambda, nret, P,
                            &lam);
        *lambda = lam;
        if (act == OR_RETRY) {
            ++nret;
            continue;
        }
        if (act == OR_ACCEPT) {
            memcpy(u, ut, 3 * V * sizeof(double));
            memcpy(g, gt, 3 * V * sizeof(double));
            *gmax = gmt;
            *L_prev = *L_t;
            *has_prev = 1;
            *L_t = Lt;
            acc = 1;
        }
        break;
    }
    *accepted = acc;
    *retries = nret;
    *evals = nev;
    free(ut);
    free(gt);
}

/* ------------------------------------------------------------------ */
/* Coarse-to-fine pyramid (Section 2.1: the warp is inherited from the */
/* coarser level).  Readings: level size n' = max(1, floor(n / f)),      */
/* anti-alias blur with sigma = f/2 (the same zero-padded separable     */
/* Gaussian), level voxel p sits at fine coordinate f p + (f - 1)/2 and */
/* is read trilinearly with zero padding.                               */
/* ------------------------------------------------------------------ */
void or_level_dims(int nx, int ny, int nz, int f, int *ox, int *oy, int *oz)
{
    *ox = nx / f > 0 ? nx / f : 1;
    *oy = ny / f > 0 ? ny / f : 1;
    *oz = nz / f > 0 ? nz / f : 1;
}

static double trilin_zero(const double *X, int nx, int ny, int nz, double x,
                          double y, double z)
{
    double fx = floor(x), fy = floor(y), fz = floor(z);
    double tx = x - fx, ty = y - fy, tz = z - fz;
    double s = 0;
    for (int sz = 0; sz < 2; ++sz)
        for (int sy = 0; sy < 2; ++sy)
            for (int sx = 0; sx < 2; ++sx)
                s += (sx ? tx : 1 - tx) * (sy ? ty : 1 - ty) *
                     (sz ? tz : 1 - tz) *
                     img_zero(X, nx, ny, nz, fx + sx, fy + sy, fz + sz);
    return s;
}

static double trilin_clamp(const double *X, int nx, int ny, int nz, double x,
                           double y, double z)
{
    double fx = floor(x), fy = floor(y), fz = floor(z);
    double tx = x - fx, ty = y - fy, tz = z - fz;
    double s = 0;
    for (int sz = 0; sz < 2; ++sz)
        for (int sy = 0; sy < 2; ++sy)
            for (int sx = 0; sx < 2; ++sx)
                s += (sx ? tx : 1 - tx) * (sy ? ty : 1 - ty) *
                     (sz ? tz : 1 - tz) *
                     fld_clamp(X, nx, ny, nz, fx + sx, fy + sy, fz + sz);
    return s;
}

void or_downsample(int nx, int ny, int nz, int f, const double *X,
                   double *Y)
{
    int ox, oy, oz;
    or_level_dims(nx, ny, nz, f, &ox, &oy, &oz);
    size_t V = vox(nx, ny, nz);
    double *Bl = malloc(V * sizeof(double));
    if (f > 1)
        or_smooth(nx, ny, nz, 0.5 * f, X, Bl);
    else
        memcpy(Bl, X, V * sizeof(double));
    double off = 0.5 * (f - 1);
    for (int z = 0; z < oz; ++z)
        for (int y = 0; y < oy; ++y)
            for (int x = 0; x < ox; ++x)
                Y[at(ox, oy, x, y, z)] = trilin_zero(
                    Bl, nx, ny, nz, f * x + off, f * y + off, f * z + off);
    free(Bl);
}

/* Resample a displacement field from a level of factor fa (dims a*) to a
 * level of factor fb (dims b*): value at level-b voxel p is the level-a
 * field read trilinearly (clamped) at the level-a coordinate of p's centre,
 * times fa / fb (voxel units change with the level). */
void or_resample_field(int ax, int ay, int az, int fa, const double *Ua,
                       int bx, int by, int bz, int fb, double *Ub)
{
    size_t Va = vox(ax, ay, az), Vb = vox(bx, by, bz);
    double scale = (double)fa / (double)fb;
    for (int z = 0; z < bz; ++z)
        for (int y = 0; y < by; ++y)
            for (int x = 0; x < bx; ++x) {
                double p[3] = {x, y, z}, q[3];
                for (int i = 0; i < 3; ++i) {
                    double fine = fb * p[i] + 0.5 * (fb - 1);
                    q[i] = (fine - 0.5 * (fa - 1)) / fa;
                }
                for (int c = 0; c < 3; ++c)
                    Ub[c * Vb + at(bx, by, x, y, z)] =
                        scale * trilin_clamp(Ua + c * Va, ax, ay, az, q[0],
                                             q[1], q[2]);
            }
}

/* ------------------------------------------------------------------ */
/* Whole registration: for each level (factors descending to 1) the      */
/* images are downsampled, the field is carried over from the previous  */
/* level (or from u at level 0), lambda and the loss history restart at */
/* lambda0 (reading), and iters[l] LM iterations run.                    */
/* u: in = initial full-resolution field, out = result.                 */
/* loss_log (optional): the loss after each iteration, levels in order. */
/* ------------------------------------------------------------------ */
void or_register(int nx, int ny, int nz, const double *F, const double *M,
                 const or_params *P, int nlevels, const int *factors,
                 const int *iters, double *u, double *loss_log,
                 int *evals_out)
{
    size_t V = vox(nx, ny, nz);
    double *cur = NULL;
    int cx = nx, cy = ny, cz = nz, cf = 1;
    /* carry the initial field at full resolution */
    cur = malloc(3 * V * sizeof(double));
    memcpy(cur, u, 3 * V * sizeof(double));
    int logi = 0, evals = 0;
    for (int l = 0; l < nlevels; ++l) {
        int f = factors[l], lx, ly, lz;
        or_level_dims(nx, ny, nz, f, &lx, &ly, &lz);
        size_t Vl = vox(lx, ly, lz);
        double *Fl = malloc(Vl * sizeof(double));
        double *Ml = malloc(Vl * sizeof(double));
        double *ul = malloc(3 * Vl * sizeof(double));
        double *gl = malloc(3 * Vl * sizeof(double));
        or_downsample(nx, ny, nz, f, F, Fl);
        or_downsample(nx, ny, nz, f, M, Ml);
        if (cx == lx && cy == ly && cz == lz && cf == f)
            memcpy(ul, cur, 3 * Vl * sizeof(double));
        else
            or_resample_field(cx, cy, cz, cf, cur, lx, ly, lz, f, ul);
        double L, gmax, Lp = 0, lam = P->lambda0;
        int hp = 0;
        if (P->method == OR_DEMONS)
            or_demons_eval(lx, ly, lz, Fl, Ml, ul, P, &L, gl, &gmax);
        else
            or_eval(lx, ly, lz, Fl, Ml, ul, P, &L, NULL, NULL, gl, &gmax, NULL);
        ++evals;
        for (int it = 0; it < iters[l]; ++it) {
            int acc, ret, ev;
            or_lm_step(lx, ly, lz, Fl, Ml, P, ul, gl, &gmax, &L, &Lp, &hp,
                       &lam, NULL, NULL, &acc, &ret, &ev);
            evals += ev;
            if (loss_log) loss_log[logi] = L;
            ++logi;
        }
        free(cur);
        cur = ul;
        cx = lx; cy = ly; cz = lz; cf = f;
        free(Fl); free(Ml); free(gl);
    }
    if (cx == nx && cy == ny && cz == nz && cf == 1)
        memcpy(u, cur, 3 * V * sizeof(double));
    else
        or_resample_field(cx, cy, cz, cf, cur, nx, ny, nz, 1, u);
    free(cur);
    if (evals_out) *evals_out = evals;
}
