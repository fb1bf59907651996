/*
 * scg_oracle.c -- plain, slow FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Everything here is written for a reader checking it against the paper by
 * eye: the system matrix A is evaluated from its definition (exact chord of a
 * line through a unit square), A^T is the literal transpose sum, and every
 * solver follows its algorithm's steps in the paper's order and notation.
 * Loops that write disjoint outputs may run under OpenMP; every sum is taken
 * in a fixed order, so results do not depend on the thread count.
 *
 * Parity status of each function is stated in the comment above it.
 */
#include "scg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Geometry.  Sec. 4 fixes a parallel-beam scan with angles uniformly spaced */
/* over [0, 180) degrees.  cos/sin are snapped to exact values where        */
/* theta is a multiple of pi/2, so that axis-aligned rays are exactly        */
/* axis-aligned.  Pinned by: single-pixel profiles, A.1 = chord of the       */
/* image square, two independent weight derivations agreeing.                */
/* ------------------------------------------------------------------------ */
void orc_angle(int a, int n_angles, double* c, double* s)
{
    if (a == 0) { *c = 1.0; *s = 0.0; return; }
    if (2 * a == n_angles) { *c = 0.0; *s = 1.0; return; }
    /* theta_a = pi a / n_angles; past pi/2 through cos(pi - t) = -cos t,
     * sin(pi - t) = sin t, so that theta and pi - theta are exact mirrors */
    int mirror = 2 * a > n_angles;
    double th = ORC_PI * (double)(mirror ? n_angles - a : a) / (double)n_angles;
    *c = mirror ? -cos(th) : cos(th);
    *s = sin(th);
}

/* A-trap: closed form of the chord of the line x*c + y*s = d' through the
 * unit square centred at the origin, as a function of the signed distance d
 * between the line and the square's centre.  With m = max(|c|,|s|) and
 * n = min(|c|,|s|) the chord is 1/m on the flat top |d| <= (m-n)/2, falls
 * linearly to 0 at |d| = (m+n)/2, and is 0 beyond.  For n = 0 a line on an
 * edge (|d| = 1/2) is shared half-and-half by the two pixels it separates. */
double orc_weight_trap(double d, double c, double s)
{
    double ac = fabs(c), as = fabs(s);
    double m = ac > as ? ac : as;
    double n = ac > as ? as : ac;
    double ad = fabs(d);
    if (n == 0.0) {
        if (ad < 0.5) return 1.0 / m;
        if (ad == 0.5) return 0.5 / m;
        return 0.0;
    }
    if (ad <= 0.5 * (m - n)) return 1.0 / m;
    if (ad < 0.5 * (m + n)) return (0.5 * (m + n) - ad) / (m * n);
    return 0.0;
}

/* A-clip: the same chord by a second, independent route -- clip the ray
 * against the two slabs of the pixel square (parametric slab method).  The
 * ray is P(t) = s_b*(c, s) + t*(-s, c), |direction| = 1, so the chord is the
 * length of the t-interval left after clipping.  A ray lying exactly on an
 * edge of the square counts one half. */
double orc_weight_clip(double xc, double yc, double c, double s, double sb)
{
    double px = sb * c, py = sb * s;      /* point of the ray nearest the origin */
    double dx = -s, dy = c;               /* unit direction                      */
    double tmin = -INFINITY, tmax = INFINITY;
    double share = 1.0;
    /* slab xc-1/2 <= X <= xc+1/2 */
    if (dx != 0.0) {
        double t1 = (xc - 0.5 - px) / dx, t2 = (xc + 0.5 - px) / dx;
        if (t1 > t2) { double t = t1; t1 = t2; t2 = t; }
        if (t1 > tmin) tmin = t1;
        if (t2 < tmax) tmax = t2;
    } else {
        if (px < xc - 0.5 || px > xc + 0.5) return 0.0;
        if (px == xc - 0.5 || px == xc + 0.5) share *= 0.5;
    }
    /* slab yc-1/2 <= Y <= yc+1/2 */
    if (dy != 0.0) {
        double t1 = (yc - 0.5 - py) / dy, t2 = (yc + 0.5 - py) / dy;
        if (t1 > t2) { double t = t1; t1 = t2; t2 = t; }
        if (t1 > tmin) tmin = t1;
        if (t2 < tmax) tmax = t2;
    } else {
        if (py < yc - 0.5 || py > yc + 0.5) return 0.0;
        if (py == yc - 0.5 || py == yc + 0.5) share *= 0.5;
    }
    return tmax > tmin ? share * (tmax - tmin) : 0.0;
}

static double pix_xc(int j, int n) { return (double)j - 0.5 * (double)(n - 1); }
static double pix_yc(int i, int n) { return (double)i - 0.5 * (double)(n - 1); }
static double bin_s(int b, int nb) { return (double)b - 0.5 * (double)(nb - 1); }

/* A x (Eq. LS1: A is the L x J discretisation of the line integrals).
 * y[a,b] = sum_{i,j} T(s_b - xc cos - yc sin) x[i,j], summed over the bins
 * that can be nonzero for each pixel (the chord vanishes for |d| >= 1 > (m+n)/2,
 * so bins outside floor(centre)-1 .. floor(centre)+2 hold exact zeros).
 * Parallel over angles: each angle writes its own sinogram row. */
void orc_project(int n, int na, int nb, const double* x, double* y)
{
    int a;
#pragma omp parallel for schedule(dynamic, 1)
    for (a = 0; a < na; ++a) {
        double c, s;
        orc_angle(a, na, &c, &s);
        double* row = y + (size_t)a * nb;
        for (int b = 0; b < nb; ++b) row[b] = 0.0;
        for (int i = 0; i < n; ++i) {
            double yc = pix_yc(i, n);
            for (int j = 0; j < n; ++j) {
                double v = x[(size_t)i * n + j];
                if (v == 0.0) continue;
                double p = pix_xc(j, n) * c + yc * s;
                double centre = p + 0.5 * (double)(nb - 1);
                int b0 = (int)floor(centre) - 1;
                for (int b = b0; b <= b0 + 3; ++b) {
                    if (b < 0 || b >= nb) continue;
                    double w = orc_weight_trap(bin_s(b, nb) - p, c, s);
                    row[b] += w * v;
                }
            }
        }
    }
}

/* A^T r: the literal transpose sum, x[i,j] = sum_a sum_b T(...) r[a,b],
 * angles in increasing order.  Parallel over pixel rows. */
void orc_backproject(int n, int na, int nb, const double* r, double* x)
{
    int i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i) {
        double yc = pix_yc(i, n);
        for (int j = 0; j < n; ++j) {
            double xc = pix_xc(j, n), acc = 0.0;
            for (int a = 0; a < na; ++a) {
                double c, s;
                orc_angle(a, na, &c, &s);
                double p = xc * c + yc * s;
                double centre = p + 0.5 * (double)(nb - 1);
                int b0 = (int)floor(centre) - 1;
                const double* row = r + (size_t)a * nb;
                for (int b = b0; b <= b0 + 3; ++b) {
                    if (b < 0 || b >= nb) continue;
                    acc += orc_weight_trap(bin_s(b, nb) - p, c, s) * row[b];
                }
            }
            x[(size_t)i * n + j] = acc;
        }
    }
}

static double weight_any(int use_clip, int i, int j, int a, int b, int n, int na, int nb)
{
    double c, s;
    orc_angle(a, na, &c, &s);
    double xc = pix_xc(j, n), yc = pix_yc(i, n), sb = bin_s(b, nb);
    if (use_clip) return orc_weight_clip(xc, yc, c, s, sb);
    return orc_weight_trap(sb - xc * c - yc * s, c, s);
}

/* Dense O(L*J) definitions of A and A^T (every ray against every pixel),
 * with either weight route.  Tiny inputs only; they pin the footprint loops
 * above and the two weight routes against each other. */
void orc_project_dense(int n, int na, int nb, int use_clip, const double* x, double* y)
{
    for (int a = 0; a < na; ++a)
        for (int b = 0; b < nb; ++b) {
            double acc = 0.0;
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j)
                    acc += weight_any(use_clip, i, j, a, b, n, na, nb) * x[(size_t)i * n + j];
            y[(size_t)a * nb + b] = acc;
        }
}

void orc_backproject_dense(int n, int na, int nb, int use_clip, const double* r, double* x)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int a = 0; a < na; ++a)
                for (int b = 0; b < nb; ++b)
                    acc += weight_any(use_clip, i, j, a, b, n, na, nb) * r[(size_t)a * nb + b];
            x[(size_t)i * n + j] = acc;
        }
}

/* Selected rays of A x, each summed over every pixel (for spot checks of
 * full-size outputs). */
void orc_project_rays(int n, int na, int nb, const double* x, int count,
                      const int* a_idx, const int* b_idx, double* out)
{
    int q;
#pragma omp parallel for schedule(dynamic, 4)
    for (q = 0; q < count; ++q) {
        double c, s;
        orc_angle(a_idx[q], na, &c, &s);
        double sb = bin_s(b_idx[q], nb), acc = 0.0;
        for (int i = 0; i < n; ++i) {
            double yc = pix_yc(i, n);
            for (int j = 0; j < n; ++j) {
                double w = orc_weight_trap(sb - pix_xc(j, n) * c - yc * s, c, s);
                if (w != 0.0) acc += w * x[(size_t)i * n + j];
            }
        }
        out[q] = acc;
    }
}

/* Selected pixels of A^T r, each summed over every ray. */
void orc_backproject_pixels(int n, int na, int nb, const double* r, int count,
                            const int* i_idx, const int* j_idx, double* out)
{
    int q;
#pragma omp parallel for schedule(dynamic, 4)
    for (q = 0; q < count; ++q) {
        double xc = pix_xc(j_idx[q], n), yc = pix_yc(i_idx[q], n), acc = 0.0;
        for (int a = 0; a < na; ++a) {
            double c, s;
            orc_angle(a, na, &c, &s);
            for (int b = 0; b < nb; ++b) {
                double w = orc_weight_trap(bin_s(b, nb) - xc * c - yc * s, c, s);
                if (w != 0.0) acc += w * r[(size_t)a * nb + b];
            }
        }
        out[q] = acc;
    }
}

/* ------------------------------------------------------------------------ */
/* Total variation, the secondary criterion (Sec. 1, Sec. 3).  The paper    */
/* names TV without a formula; this is the isotropic forward-difference TV  */
/* over the (N-1)^2 interior terms:                                          */
/*   TV(x) = sum_{i<N-1, j<N-1} sqrt((x[i+1,j]-x[i,j])^2 + (x[i,j+1]-x[i,j])^2) */
/* Pinned by: constant image -> 0; linear ramp -> closed form; gradient vs   */
/* central finite differences.                                               */
/* ------------------------------------------------------------------------ */
double orc_tv(int n, const double* x)
{
    double tv = 0.0;
    for (int i = 0; i + 1 < n; ++i)
        for (int j = 0; j + 1 < n; ++j) {
            double x0 = x[(size_t)i * n + j];
            double du = x[(size_t)(i + 1) * n + j] - x0;
            double dv = x[(size_t)i * n + j + 1] - x0;
            tv += sqrt(du * du + dv * dv);
        }
    return tv;
}

/* A subgradient of TV: each term with nonzero norm contributes its gradient
 * to its three pixels; a term with zero norm contributes 0 (0 is an element
 * of that term's subdifferential).  Returns TV(x). */
double orc_tv_grad(int n, const double* x, double* grad)
{
    size_t J = (size_t)n * n;
    for (size_t q = 0; q < J; ++q) grad[q] = 0.0;
    double tv = 0.0;
    for (int i = 0; i + 1 < n; ++i)
        for (int j = 0; j + 1 < n; ++j) {
            size_t c0 = (size_t)i * n + j, cu = c0 + n, cv = c0 + 1;
            double du = x[cu] - x[c0], dv = x[cv] - x[c0];
            double nrm = sqrt(du * du + dv * dv);
            tv += nrm;
            if (nrm > 0.0) {
                grad[c0] -= (du + dv) / nrm;
                grad[cu] += du / nrm;
                grad[cv] += dv / nrm;
            }
        }
    return tv;
}

/* ------------------------------------------------------------------------ */
/* Preconditioning filter (Sec. 3, "Filters for Preconditioning"):          */
/*   z = A^T F^T C F (A x - y),  c(w) = (|w| + mu)(0.54 + 0.46 cos w).       */
/* F is a unitary DFT of each projection row zero-padded to P, the smallest  */
/* power of two >= 2*n_bins (so the circular product does not wrap); the     */
/* frequency of index k is w_k = 2 pi k / P folded into [-pi, pi].  Done     */
/* here as a naive O(P * n_bins) DFT.  Pinned against numpy's FFT.           */
/* ------------------------------------------------------------------------ */
int orc_filter_length(int nb)
{
    int P = 1;
    while (P < 2 * nb) P *= 2;
    return P;
}

double orc_filter_factor(double omega, double mu)
{
    return (fabs(omega) + mu) * (0.54 + 0.46 * cos(omega));
}

/* The filtering of each row with the factors c(w) of the given mu, exactly
 * as written (mu = 0 allowed). */
static void filter_rows_mu(int na, int nb, double mu, double gain, const double* r, double* out);

void orc_filter_rows(int na, int nb, double mu, double gain, const double* r, double* out)
{
    int P = orc_filter_length(nb);
    if (!(mu > 0.0)) mu = 2.0 * ORC_PI / (double)P;
    filter_rows_mu(na, nb, mu, gain, r, out);
}

static void filter_rows_mu(int na, int nb, double mu, double gain, const double* r, double* out)
{
    int P = orc_filter_length(nb);
    double* cw = (double*)malloc(sizeof(double) * (size_t)P);
    double* sw = (double*)malloc(sizeof(double) * (size_t)P);
    double* cf = (double*)malloc(sizeof(double) * (size_t)P);
    for (int m = 0; m < P; ++m) {
        cw[m] = cos(2.0 * ORC_PI * (double)m / (double)P);
        sw[m] = sin(2.0 * ORC_PI * (double)m / (double)P);
        double w = (m <= P / 2) ? 2.0 * ORC_PI * m / P : 2.0 * ORC_PI * (m - P) / P;
        cf[m] = gain * orc_filter_factor(w, mu);
    }
    double scale = 1.0 / sqrt((double)P);
    int a;
#pragma omp parallel for schedule(dynamic, 1)
    for (a = 0; a < na; ++a) {
        double* re = (double*)malloc(sizeof(double) * (size_t)P);
        double* im = (double*)malloc(sizeof(double) * (size_t)P);
        const double* row = r + (size_t)a * nb;
        for (int k = 0; k < P; ++k) {               /* R = F r (unitary)  */
            double sr = 0.0, si = 0.0;
            for (int t = 0; t < nb; ++t) {
                int idx = (int)(((long long)k * t) % P);
                sr += row[t] * cw[idx];
                si -= row[t] * sw[idx];
            }
            re[k] = cf[k] * sr * scale;              /* Z = C R            */
            im[k] = cf[k] * si * scale;
        }
        for (int t = 0; t < nb; ++t) {               /* z = F^H Z, cropped */
            double acc = 0.0;
            for (int k = 0; k < P; ++k) {
                int idx = (int)(((long long)k * t) % P);
                acc += re[k] * cw[idx] - im[k] * sw[idx];
            }
            out[(size_t)a * nb + t] = acc * scale;
        }
        free(re);
        free(im);
    }
    free(cw);
    free(sw);
    free(cf);
}

/* ------------------------------------------------------------------------ */
/* c = ||A||_2 (Appendix, Eq. lambda) by power iteration on A^T A.           */
/* ------------------------------------------------------------------------ */
double orc_norm_A(int n, int na, int nb, int iters)
{
    size_t J = (size_t)n * n, L = (size_t)na * nb;
    double* v = (double*)malloc(sizeof(double) * J);
    double* w = (double*)malloc(sizeof(double) * J);
    double* q = (double*)malloc(sizeof(double) * L);
    for (size_t k = 0; k < J; ++k) v[k] = 1.0 + 0.001 * (double)(k % 7);
    double lam = 0.0;
    for (int it = 0; it < iters; ++it) {
        double nv = 0.0;
        for (size_t k = 0; k < J; ++k) nv += v[k] * v[k];
        nv = sqrt(nv);
        for (size_t k = 0; k < J; ++k) v[k] /= nv;
        orc_project(n, na, nb, v, q);
        orc_backproject(n, na, nb, q, w);
        lam = 0.0;
        for (size_t k = 0; k < J; ++k) lam += v[k] * w[k];
        memcpy(v, w, sizeof(double) * J);
    }
    free(v);
    free(w);
    free(q);
    return sqrt(lam);
}

/* ------------------------------------------------------------------------ */
/* Filtered backprojection (Sec. 4 shows an FBP reconstruction as the visual  */
/* reference; it names the method of Herman's textbook, Ch. 8, and Sec. 3    */
/* says the preconditioner's Hamming-windowed factors are those commonly     */
/* used there).  Parallel-beam inversion: x(s) = int_0^pi (p_theta * q)(s)   */
/* dtheta with q the ramp |nu| (nu in cycles per bin width).  Discretised:   */
/* each row is filtered by the padded unitary DFT with the factors           */
/*   |nu| (0.54 + 0.46 cos w) = |w|/(2 pi) (0.54 + 0.46 cos w),              */
/* w = 2 pi nu in [-pi, pi]; the angle integral becomes (pi / n_angles)      */
/* times the sum over angles, and that sum at each pixel is A^T (whose       */
/* weights of one pixel and angle add up to the pixel area 1).  In terms of  */
/* the Sec. 3 factors c(w) = (|w| + mu)(0.54 + 0.46 cos w) with mu = 0 this  */
/* is x = A^T F^T (g C) F y with gain g = (pi / n_angles)/(2 pi)             */
/* = 1 / (2 n_angles).                                                       */
/* Pinned by: a numpy FFT route for the filtering, the reconstruction of a   */
/* uniform disk.                                                             */
/* ------------------------------------------------------------------------ */
void orc_fbp(int n, int na, int nb, const double* y, double* x)
{
    double* q = (double*)malloc(sizeof(double) * (size_t)na * nb);
    filter_rows_mu(na, nb, 0.0, 1.0 / (2.0 * (double)na), y, q);
    orc_backproject(n, na, nb, q, x);
    free(q);
}

/* ------------------------------------------------------------------------ */
/* Solvers.                                                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n, na, nb;
    size_t J, L;
    const double* y;
    orc_params prm;
    double* sino;      /* L scratch */
    double* sino2;     /* L scratch */
    double* tvg;       /* J scratch: TV subgradient */
    double* vdir;      /* J scratch: nonascending direction */
    double* ztrial;    /* J scratch: trial point */
    double* gk;        /* J scratch: gradient at x_k (eta rule) */
    long long ell;     /* global gamma index */
    int gamma_fixed;
    double gamma0;
} orc_ctx;

static double dot(const double* u, const double* v, size_t n)
{
    double s = 0.0;
    for (size_t k = 0; k < n; ++k) s += u[k] * v[k];
    return s;
}

static int finite_pos(double v) { return v > 0.0 && isfinite(v); }

static double* vec(size_t n) { return (double*)calloc(n ? n : 1, sizeof(double)); }

/* f(x) = 1/2 ||y - Ax||^2, the primary criterion (Sec. 1). */
static double f_of(orc_ctx* C, const double* x)
{
    orc_project(C->n, C->na, C->nb, x, C->sino);
    double s = 0.0;
    for (size_t k = 0; k < C->L; ++k) {
        double r = C->y[k] - C->sino[k];
        s += r * r;
    }
    return 0.5 * s;
}

/* g = A^T (A x - y) (Eq. g_k+1); returns f(x) as a by-product. */
static double grad_of(orc_ctx* C, const double* x, double* g)
{
    orc_project(C->n, C->na, C->nb, x, C->sino);
    double s = 0.0;
    for (size_t k = 0; k < C->L; ++k) {
        C->sino[k] -= C->y[k];
        s += C->sino[k] * C->sino[k];
    }
    orc_backproject(C->n, C->na, C->nb, C->sino, g);
    return 0.5 * s;
}

/* h = A^T A p */
static void AtA(orc_ctx* C, const double* p, double* h)
{
    orc_project(C->n, C->na, C->nb, p, C->sino);
    orc_backproject(C->n, C->na, C->nb, C->sino, h);
}

/* z = M g at the point x where g = A^T(Ax - y): the filter acts on the
 * residual Ax - y of that same point, z = A^T F^T C F (Ax - y). */
static void M_of(orc_ctx* C, const double* x, double* z)
{
    orc_project(C->n, C->na, C->nb, x, C->sino);
    for (size_t k = 0; k < C->L; ++k) C->sino[k] -= C->y[k];
    if (C->prm.filter_identity) {
        for (size_t k = 0; k < C->L; ++k) C->sino2[k] = C->prm.filter_gain * C->sino[k];
    } else {
        orc_filter_rows(C->na, C->nb, C->prm.mu, C->prm.filter_gain, C->sino, C->sino2);
    }
    orc_backproject(C->n, C->na, C->nb, C->sino2, z);
}

static double* row_of(double* trace, int rows, int it)
{
    if (!trace || it < 0 || it >= rows) return NULL;
    double* r = trace + (size_t)it * ORC_NF;
    for (int q = 0; q < ORC_NF; ++q) r[q] = 0.0;
    return r;
}

/* perturbed(x_k) -> x_{k+1/2} (Eq. superiorized).
 *  gamma rule: v = -dTV/||dTV|| (a nonascending direction of TV); trials
 *    z = x + gamma_0 a^l v, l <- l+1 after every trial, accepted as soon as
 *    TV(z) <= TV(x) (Sec. 1, Eq. superiorization; Eq. gamma_sequence); after
 *    max_trials rejections x is kept.  Zero subgradient: x is kept, l is
 *    unchanged.
 *  eta rule (Appendix, Eq. up bnd u_k): u = eta0 ||g_k|| v with
 *    g_k = A^T(A x_k - y), applied without a TV test.
 *  prox rule (footnote to Eq. superiorized): x_{k+1/2} =
 *    prox_{lambda TV}(x_k), the implicit counterpart of the gamma rule's step
 *    x_k + gamma v = x_k - (gamma / ||dTV||) dTV: lambda = gamma_0 a^l /
 *    ||dTV(x_k)||, gamma_0 fixed as in the gamma rule, FGP with prox_iters
 *    steps.  A prox step cannot raise TV, so there is no trial: l <- l+1 once
 *    per perturbed step.  Zero subgradient: x is kept, l unchanged. */
static void perturb(orc_ctx* C, const double* xk, double* xh, double* trow)
{
    size_t J = C->J;
    double tvx = orc_tv_grad(C->n, xk, C->tvg);
    double gn = sqrt(dot(C->tvg, C->tvg, J));
    if (trow) {
        trow[ORC_T_TV_BEFORE] = tvx;
        trow[ORC_T_ACCEPTED] = -1;
        trow[ORC_T_MARGIN] = INFINITY;
    }
    if (C->prm.perturb == ORC_PERTURB_NONE || gn == 0.0) {
        memcpy(xh, xk, sizeof(double) * J);
        if (trow) { trow[ORC_T_TV_AFTER] = tvx; trow[ORC_T_ELL] = (double)C->ell; }
        return;
    }
    for (size_t k = 0; k < J; ++k) C->vdir[k] = -C->tvg[k] / gn;
    if (C->prm.perturb == ORC_PERTURB_ETA) {
        grad_of(C, xk, C->gk);
        double scale = C->prm.eta0 * sqrt(dot(C->gk, C->gk, J));
        for (size_t k = 0; k < J; ++k) xh[k] = xk[k] + scale * C->vdir[k];
        if (trow) {
            trow[ORC_T_ACCEPTED] = 1;
            trow[ORC_T_GAMMA] = scale;
            trow[ORC_T_TV_AFTER] = orc_tv(C->n, xh);
            trow[ORC_T_ELL] = (double)C->ell;
        }
        return;
    }
    if (!C->gamma_fixed) {
        C->gamma0 = C->prm.gamma0_rel * sqrt(dot(xk, xk, J));
        C->gamma_fixed = 1;
    }
    if (C->prm.perturb == ORC_PERTURB_PROX) {
        double gamma = C->gamma0 * pow(C->prm.a, (double)C->ell);
        double lambda = gamma / gn;
        orc_tv_prox(C->n, xk, lambda, C->prm.prox_iters, 1, xh, NULL, NULL);
        C->ell += 1;
        if (trow) {
            trow[ORC_T_ACCEPTED] = 1;
            trow[ORC_T_GAMMA] = lambda;
            trow[ORC_T_TV_AFTER] = orc_tv(C->n, xh);
            trow[ORC_T_ELL] = (double)C->ell;
        }
        return;
    }
    double margin = INFINITY;
    for (int t = 0; t < C->prm.max_trials; ++t) {
        double gamma = C->gamma0 * pow(C->prm.a, (double)C->ell);
        for (size_t k = 0; k < J; ++k) C->ztrial[k] = xk[k] + gamma * C->vdir[k];
        C->ell += 1;
        double tvz = orc_tv(C->n, C->ztrial);
        double rel = fabs(tvz - tvx) / (tvx > 0.0 ? tvx : 1.0);
        if (rel < margin) margin = rel;
        if (trow) trow[ORC_T_TRIALS] = t + 1;
        if (tvz <= tvx) {
            memcpy(xh, C->ztrial, sizeof(double) * J);
            if (trow) {
                trow[ORC_T_ACCEPTED] = 1;
                trow[ORC_T_GAMMA] = gamma;
                trow[ORC_T_TV_AFTER] = tvz;
                trow[ORC_T_ELL] = (double)C->ell;
                trow[ORC_T_MARGIN] = margin;
            }
            return;
        }
    }
    memcpy(xh, xk, sizeof(double) * J);
    if (trow) {
        trow[ORC_T_ACCEPTED] = 0;
        trow[ORC_T_TV_AFTER] = tvx;
        trow[ORC_T_ELL] = (double)C->ell;
        trow[ORC_T_MARGIN] = margin;
    }
}

/* perturbed(x_k) with several perturbations per step (the superiorization
 * scheme's N nonascending steps per iteration; the printed algorithms take
 * one): the rule is applied perturb_steps times in succession, each time from
 * the current point with its own subgradient; l runs on across the sub-steps
 * and each sub-step has its own trial budget; a sub-step with a zero
 * subgradient ends the sequence.  The trace row keeps TV(x_k) from the first
 * sub-step and the other perturbation fields of the last one.  The eta rule
 * takes one step only. */
static void perturb_all(orc_ctx* C, const double* xk, double* xh, double* trow)
{
    perturb(C, xk, xh, trow);
    int steps = C->prm.perturb_steps;
    if (steps <= 1 || C->prm.perturb == ORC_PERTURB_ETA || C->prm.perturb == ORC_PERTURB_NONE) return;
    if (trow && trow[ORC_T_ACCEPTED] == -1) return;          /* zero subgradient */
    double* cur = vec(C->J);
    double row[ORC_NF];
    for (int s = 1; s < steps; ++s) {
        memcpy(cur, xh, sizeof(double) * C->J);
        for (int q = 0; q < ORC_NF; ++q) row[q] = 0.0;
        perturb(C, cur, xh, row);
        if (trow) {
            double tv0 = trow[ORC_T_TV_BEFORE];
            for (int q = ORC_T_TV_AFTER; q <= ORC_T_GAMMA; ++q) trow[q] = row[q];
            trow[ORC_T_MARGIN] = row[ORC_T_MARGIN];
            trow[ORC_T_TV_BEFORE] = tv0;
        }
        if (row[ORC_T_ACCEPTED] == -1) break;
    }
    free(cur);
}

/* One perturbation step of the gamma rule on its own, for checking the rule
 * against hand-worked cases: x_half = perturbed(x) with the global index l
 * starting at *ell (updated on return), gamma_0 = gamma0 and kernel a.  Runs
 * the same perturb() the solvers call.  *gamma_out = the accepted gamma (0 if
 * none), *trials_out = trials taken, return value = 1 accepted, 0 all
 * rejected (x kept), -1 no perturbation (zero subgradient). */
int orc_perturb_gamma(int n, const double* x, double gamma0, double a, int max_trials,
                      long long* ell, double* x_half, double* gamma_out, int* trials_out)
{
    orc_ctx C;
    memset(&C, 0, sizeof(C));
    C.n = n;
    C.J = (size_t)n * n;
    C.prm.perturb = ORC_PERTURB_GAMMA;
    C.prm.a = a;
    C.prm.max_trials = max_trials;
    C.gamma0 = gamma0;
    C.gamma_fixed = 1;
    C.ell = *ell;
    C.tvg = vec(C.J);
    C.vdir = vec(C.J);
    C.ztrial = vec(C.J);
    double row[ORC_NF];
    for (int q = 0; q < ORC_NF; ++q) row[q] = 0.0;
    perturb(&C, x, x_half, row);
    *ell = C.ell;
    *gamma_out = row[ORC_T_ACCEPTED] == 1 ? row[ORC_T_GAMMA] : 0.0;
    *trials_out = (int)row[ORC_T_TRIALS];
    free(C.tvg);
    free(C.vdir);
    free(C.ztrial);
    return (int)row[ORC_T_ACCEPTED];
}

/* One step of the prox rule on its own (the perturb() the solvers call):
 * x_half = prox_{lambda TV}(x) with lambda = gamma0 a^l / ||dTV(x)||, l
 * starting at *ell (advanced by one when x is perturbed).  *lambda_out =
 * lambda (0 if the subgradient is zero and x is kept).  Returns 1 perturbed,
 * -1 not (zero subgradient). */
int orc_perturb_prox(int n, const double* x, double gamma0, double a, int prox_iters,
                     long long* ell, double* x_half, double* lambda_out)
{
    orc_ctx C;
    memset(&C, 0, sizeof(C));
    C.n = n;
    C.J = (size_t)n * n;
    C.prm.perturb = ORC_PERTURB_PROX;
    C.prm.a = a;
    C.prm.prox_iters = prox_iters;
    C.gamma0 = gamma0;
    C.gamma_fixed = 1;
    C.ell = *ell;
    C.tvg = vec(C.J);
    C.vdir = vec(C.J);
    C.ztrial = vec(C.J);
    double row[ORC_NF];
    for (int q = 0; q < ORC_NF; ++q) row[q] = 0.0;
    perturb(&C, x, x_half, row);
    *ell = C.ell;
    *lambda_out = row[ORC_T_ACCEPTED] == 1 ? row[ORC_T_GAMMA] : 0.0;
    free(C.tvg);
    free(C.vdir);
    free(C.ztrial);
    return (int)row[ORC_T_ACCEPTED];
}

/* Working vectors of one solve; also the exported/imported state. */
typedef struct {
    int k;
    double delta;
    double *x, *xh, *p, *h, *g, *gn, *pn, *hn, *z, *xprev;
} orc_work;

static void work_alloc(orc_work* W, size_t J)
{
    memset(W, 0, sizeof(*W));
    W->x = vec(J); W->xh = vec(J); W->p = vec(J); W->h = vec(J); W->g = vec(J);
    W->gn = vec(J); W->pn = vec(J); W->hn = vec(J); W->z = vec(J); W->xprev = vec(J);
}

static void work_free(orc_work* W)
{
    free(W->x); free(W->xh); free(W->p); free(W->h); free(W->g);
    free(W->gn); free(W->pn); free(W->hn); free(W->z); free(W->xprev);
}

static void cpy(double* dst, const double* src, size_t J)
{
    if (dst && src) memcpy(dst, src, sizeof(double) * J);
}

/* CG (Algorithm 1, steps via CG-STEP, Algorithm 2) and PCG (Algorithm 3,
 * steps via PCG-STEP, Algorithm 4).  Recursive gradient (Eq. recursive). */
static int solve_cg(orc_ctx* C, int precond, const double* x0, int resumed, orc_work* W,
                    orc_result* res, double* trace, int rows, orc_iter_cb cb, void* user)
{
    size_t J = C->J;
    int status = ORC_OK, it = 0;
    if (!resumed) {
        W->k = 0;                                        /* k = 0              */
        cpy(W->x, x0, J);
        grad_of(C, W->x, W->g);                          /* g0 = A^T(Ax0 - y)  */
        if (precond) {
            M_of(C, W->x, W->z);                         /* z0 = M g0          */
            for (size_t q = 0; q < J; ++q) W->p[q] = -W->z[q];   /* p0 = -z0   */
            W->delta = dot(W->g, W->z, J);               /* delta0 = g0^T z0   */
        } else {
            for (size_t q = 0; q < J; ++q) W->p[q] = -W->g[q];   /* p0 = -g0   */
            W->delta = dot(W->g, W->g, J);               /* delta0 = ||g0||^2  */
        }
    }
    double *x = W->x, *g = W->g, *p = W->p, *h = W->h, *z = W->z;
    for (;;) {
        double fx = f_of(C, x);                          /* while f(x_k) > eps */
        if (!(fx > C->prm.eps)) {                    /* f <= eps; NaN f: breakdown */
            if (!(fx <= C->prm.eps)) status = ORC_ERR_BREAKDOWN;
            break;
        }
        if (it >= C->prm.max_iter) { status = ORC_MAX_ITER; break; }
        double* tr = row_of(trace, rows, it);
        if (tr) {
            tr[ORC_T_K] = W->k;
            tr[ORC_T_FTEST] = fx;
            tr[ORC_T_ACCEPTED] = -1;
        }
        /* CG-STEP / PCG-STEP */
        AtA(C, p, h);                                    /* h = A^T A p        */
        double pTh = dot(p, h, J);
        if (!finite_pos(pTh)) {
            if (W->delta == 0.0) break;
            status = ORC_ERR_BREAKDOWN;
            break;
        }
        double alpha = W->delta / pTh;                   /* alpha = delta/p^T h */
        cpy(W->xprev, x, J);
        for (size_t q = 0; q < J; ++q) x[q] += alpha * p[q];   /* x' = x + alpha p */
        for (size_t q = 0; q < J; ++q) g[q] += alpha * h[q];   /* g' = g + alpha h */
        double delta_new;
        if (precond) {
            M_of(C, x, z);                               /* z' = M g'          */
            delta_new = dot(g, z, J);                    /* delta' = g'^T z'   */
        } else {
            delta_new = dot(g, g, J);                    /* delta' = ||g'||^2  */
        }
        double beta = delta_new / W->delta;              /* beta = delta'/delta */
        const double* d = precond ? z : g;
        for (size_t q = 0; q < J; ++q) p[q] = -d[q] + beta * p[q];  /* p' = -g'(z') + beta p */
        W->delta = delta_new;
        if (tr) { tr[ORC_T_ALPHA] = alpha; tr[ORC_T_BETA] = beta; }
        if (cb) cb(it, x, W->xprev, p, h, g, user);
        W->k += 1;                                       /* k = k + 1          */
        ++it;
    }
    cpy(W->xh, x, J);                                    /* x = x_k            */
    res->iters = it;
    res->k_final = W->k;
    res->status = status;
    return status;
}

/* CG-K (Algorithm 6) and PCG-K (Algorithm 12): K CG-STEP / PCG-STEP calls
 * from x0, restarting the recursions.  x, g, p, h, z are work vectors. */
static int cg_k(orc_ctx* C, int precond, const double* x0, double* x,
                double* g, double* p, double* h, double* z)
{
    size_t J = C->J;
    int steps = C->prm.K + (C->prm.k_inclusive ? 1 : 0);
    cpy(x, x0, J);
    grad_of(C, x, g);                                    /* g0 = A^T(Ax0 - y) */
    double delta;
    if (precond) {
        M_of(C, x, z);                                   /* z0 = M g0         */
        for (size_t q = 0; q < J; ++q) p[q] = -z[q];     /* p0 = -z0          */
        delta = dot(g, z, J);                            /* delta0 = g0^T z0  */
    } else {
        for (size_t q = 0; q < J; ++q) p[q] = -g[q];     /* p0 = -g0          */
        delta = dot(g, g, J);                            /* delta0 = ||g0||^2 */
    }
    for (int k = 0; k < steps; ++k) {                    /* while k < K       */
        AtA(C, p, h);
        double pTh = dot(p, h, J);
        if (!finite_pos(pTh)) return delta == 0.0 ? ORC_OK : ORC_ERR_BREAKDOWN;
        double alpha = delta / pTh;
        for (size_t q = 0; q < J; ++q) x[q] += alpha * p[q];
        for (size_t q = 0; q < J; ++q) g[q] += alpha * h[q];
        double delta_new;
        if (precond) {
            M_of(C, x, z);
            delta_new = dot(g, z, J);
        } else {
            delta_new = dot(g, g, J);
        }
        double beta = delta_new / delta;
        const double* d = precond ? z : g;
        for (size_t q = 0; q < J; ++q) p[q] = -d[q] + beta * p[q];
        delta = delta_new;
    }
    return ORC_OK;
}

/* S-CG-K (Algorithm 5) and S-PCG-K (Algorithm 11). */
static int solve_s_k(orc_ctx* C, int precond, const double* x0, int resumed, orc_work* W,
                     orc_result* res, double* trace, int rows, orc_iter_cb cb, void* user)
{
    size_t J = C->J;
    int status = ORC_OK, it = 0;
    if (!resumed) {
        W->k = 0;                                        /* k = 0                 */
        cpy(W->x, x0, J);
        cpy(W->xh, x0, J);                               /* x_{-1/2} = x0         */
    }
    for (;;) {
        double fx = f_of(C, W->xh);                      /* f(x_{k-1/2}) > eps    */
        if (!(fx > C->prm.eps)) {                    /* f <= eps; NaN f: breakdown */
            if (!(fx <= C->prm.eps)) status = ORC_ERR_BREAKDOWN;
            break;
        }
        if (it >= C->prm.max_iter) { status = ORC_MAX_ITER; break; }
        double* tr = row_of(trace, rows, it);
        if (tr) {
            tr[ORC_T_K] = W->k;
            tr[ORC_T_FTEST] = fx;
        }
        perturb_all(C, W->x, W->xh, tr);                     /* x_{k+1/2} = perturbed(x_k) */
        int st = cg_k(C, precond, W->xh, W->x, W->g, W->p, W->h, W->z); /* x_{k+1} = CG-K(x_{k+1/2}) */
        if (st != ORC_OK) { status = st; ++it; W->k += 1; break; }
        if (cb) cb(it, W->x, W->xh, W->p, W->h, W->g, user);
        W->k += 1;
        ++it;
    }
    res->iters = it;                                     /* x = x_{k-1/2}         */
    res->k_final = W->k;
    res->status = status;
    return status;
}

/* S-CG (Algorithm 7 with CG-PR-STEP, Algorithm 8), S-CG-CD (Algorithm 9
 * with CG-CD-STEP, Algorithm 10) and S-PCG (Algorithm 13 with PCG-PR-STEP,
 * Algorithm 14). */
static int solve_s_pr(orc_ctx* C, int variant, const double* x0, int resumed, orc_work* W,
                      orc_result* res, double* trace, int rows, orc_iter_cb cb, void* user)
{
    size_t J = C->J;
    int precond = (variant == ORC_S_PCG);
    int status = ORC_OK, it = 0;
    double *x = W->x, *xh = W->xh, *g = W->g, *gn = W->gn, *p = W->p, *pn = W->pn;
    double *h = W->h, *hn = W->hn, *z = W->z;

    if (!resumed) {
        cpy(xh, x0, J);                                  /* x_{1/2} = x0         */
        grad_of(C, x0, g);                               /* g0 = A^T(Ax0 - y)    */
        if (precond) {
            M_of(C, x0, z);                              /* z0 = M g0            */
            for (size_t q = 0; q < J; ++q) p[q] = -z[q]; /* p0 = -z0             */
        } else {
            for (size_t q = 0; q < J; ++q) p[q] = -g[q]; /* p0 = -g0             */
        }
        AtA(C, p, h);                                    /* h0 = A^T A p0        */
        double pTh = dot(p, h, J);
        double alpha0 = 0.0;
        if (finite_pos(pTh)) alpha0 = -dot(g, p, J) / pTh;   /* alpha = -g0^T p0 / p0^T h0 */
        else if (dot(g, g, J) != 0.0) status = ORC_ERR_BREAKDOWN;
        for (size_t q = 0; q < J; ++q) x[q] = x0[q] + alpha0 * p[q];  /* x1 = x0 + alpha p0 */
        W->k = 1;                                        /* k = 1                */
        if (status != ORC_OK) goto done;
    }

    for (;;) {
        double fx = f_of(C, xh);                         /* while f(x_{k-1/2}) > eps */
        if (!(fx > C->prm.eps)) {                    /* f <= eps; NaN f: breakdown */
            if (!(fx <= C->prm.eps)) status = ORC_ERR_BREAKDOWN;
            break;
        }
        if (it >= C->prm.max_iter) { status = ORC_MAX_ITER; break; }
        double* tr = row_of(trace, rows, it);
        if (tr) {
            tr[ORC_T_K] = W->k;
            tr[ORC_T_FTEST] = fx;
        }
        perturb_all(C, x, xh, tr);                           /* x_{k+1/2} = perturbed(x_k) */

        /* --- the step: CG-PR-STEP / CG-CD-STEP / PCG-PR-STEP --- */
        double f_half = grad_of(C, xh, gn);              /* g' = A^T(A x - y)    */
        double beta;
        const double* d = gn;
        if (variant == ORC_S_CG_CD) {
            double gp = dot(g, p, J);
            double gg = dot(gn, gn, J);
            if (gg == 0.0) beta = 0.0;
            else if (!(gp < 0.0) || !isfinite(gp)) { status = ORC_ERR_BREAKDOWN; ++it; W->k += 1; break; }
            else beta = -gg / gp;                        /* beta = -||g'||^2 / g^T p */
        } else if (precond) {
            M_of(C, xh, z);                              /* z' = M g'            */
            beta = dot(z, h, J) / dot(p, h, J);          /* beta = z'^T h / p^T h */
            d = z;
        } else {
            beta = dot(gn, h, J) / dot(p, h, J);         /* beta = g'^T h / p^T h */
        }
        for (size_t q = 0; q < J; ++q) pn[q] = -d[q] + beta * p[q];   /* p' = -g'(z') + beta p */
        AtA(C, pn, hn);                                  /* h' = A^T A p'        */
        double pnh = dot(pn, hn, J);
        double alpha;
        if (finite_pos(pnh)) alpha = -dot(gn, pn, J) / pnh;   /* alpha = -g'^T p' / p'^T h' */
        else if (dot(gn, gn, J) == 0.0) alpha = 0.0;
        else { status = ORC_ERR_BREAKDOWN; ++it; W->k += 1; break; }
        for (size_t q = 0; q < J; ++q) x[q] = xh[q] + alpha * pn[q];  /* x' = x + alpha p' */
        if (tr) {
            tr[ORC_T_ALPHA] = alpha;
            tr[ORC_T_BETA] = beta;
            tr[ORC_T_F_AFTER] = f_half;
        }
        cpy(p, pn, J);
        cpy(h, hn, J);
        cpy(g, gn, J);
        if (cb) cb(it, x, xh, p, h, g, user);
        W->k += 1;                                       /* k = k + 1            */
        ++it;
    }
done:
    res->iters = it;                                     /* x = x_{k-1/2}        */
    res->k_final = W->k;
    res->status = status;
    return status;
}

int orc_solve(int n, int na, int nb, const double* y, const double* x0,
              const orc_params* prm, double* x_out, orc_result* res,
              double* trace, int trace_rows, orc_iter_cb cb, void* user,
              const orc_state* resume, orc_state* final_state)
{
    if (n <= 0 || na <= 0 || nb <= 0 || !y || !prm || !x_out || !res) return ORC_ERR_INVALID;
    if (!(prm->eps > 0.0) || prm->max_iter < 0) return ORC_ERR_INVALID;
    orc_ctx C;
    memset(&C, 0, sizeof(C));
    C.n = n; C.na = na; C.nb = nb;
    C.J = (size_t)n * n;
    C.L = (size_t)na * nb;
    C.y = y;
    C.prm = *prm;
    C.sino = vec(C.L);
    C.sino2 = vec(C.L);
    C.tvg = vec(C.J);
    C.vdir = vec(C.J);
    C.ztrial = vec(C.J);
    C.gk = vec(C.J);
    C.gamma_fixed = prm->gamma0 > 0.0;
    C.gamma0 = prm->gamma0;
    double* xz = NULL;
    if (!x0) { xz = vec(C.J); x0 = xz; }
    memset(res, 0, sizeof(*res));

    orc_work W;
    work_alloc(&W, C.J);
    int resumed = resume && resume->valid;
    if (resumed) {
        W.k = resume->k;
        W.delta = resume->delta;
        C.ell = resume->ell;
        C.gamma0 = resume->gamma0;
        C.gamma_fixed = resume->gamma_fixed;
        cpy(W.x, resume->x, C.J);
        cpy(W.xh, resume->x_half, C.J);
        cpy(W.p, resume->p, C.J);
        cpy(W.h, resume->h, C.J);
        cpy(W.g, resume->g, C.J);
    }

    int st;
    switch (prm->variant) {
    case ORC_CG:      st = solve_cg(&C, 0, x0, resumed, &W, res, trace, trace_rows, cb, user); break;
    case ORC_PCG:     st = solve_cg(&C, 1, x0, resumed, &W, res, trace, trace_rows, cb, user); break;
    case ORC_S_CG_K:  st = solve_s_k(&C, 0, x0, resumed, &W, res, trace, trace_rows, cb, user); break;
    case ORC_S_PCG_K: st = solve_s_k(&C, 1, x0, resumed, &W, res, trace, trace_rows, cb, user); break;
    case ORC_S_CG:
    case ORC_S_CG_CD:
    case ORC_S_PCG:   st = solve_s_pr(&C, prm->variant, x0, resumed, &W, res, trace, trace_rows, cb, user); break;
    default:          st = ORC_ERR_INVALID; res->status = st; break;
    }
    if (st != ORC_ERR_INVALID) {
        cpy(x_out, W.xh, C.J);                           /* the algorithm's output */
        res->f_final = f_of(&C, x_out);
        res->tv_final = orc_tv(n, x_out);
        res->ell = C.ell;
        res->gamma0_used = C.gamma0;
        if (final_state) {
            final_state->valid = 1;
            final_state->k = W.k;
            final_state->ell = C.ell;
            final_state->gamma0 = C.gamma0;
            final_state->gamma_fixed = C.gamma_fixed;
            final_state->delta = W.delta;
            cpy(final_state->x, W.x, C.J);
            cpy(final_state->x_half, W.xh, C.J);
            cpy(final_state->p, W.p, C.J);
            cpy(final_state->h, W.h, C.J);
            cpy(final_state->g, W.g, C.J);
        }
    }
    work_free(&W);
    free(C.sino); free(C.sino2); free(C.tvg); free(C.vdir); free(C.ztrial); free(C.gk);
    free(xz);
    return st;
}

/* ------------------------------------------------------------------------ */
/* FISTA with a TV proximal operator (Sec. 2: Eq. prox, Eq. FISTA,           */
/* Eq. FISTA-u), the paper's comparison method.                              */
/*                                                                           */
/* TV as a maximum over a dual field: with the interior terms               */
/* (i, j), i, j < N-1, and L x = (x[i+1,j] - x[i,j], x[i,j+1] - x[i,j]) per  */
/* term, TV(x) = max <L x, w> over fields w = (p, q) with p^2 + q^2 <= 1 at  */
/* every term.  The prox of alpha TV at b is then x = b - alpha L^T w*, where */
/* w* minimises ||b - alpha L^T w||^2 over that set: the fast gradient      */
/* projection (FGP) of Beck and Teboulle (2009) solves this dual with a      */
/* gradient step 1/(8 alpha) (||L||^2 <= 8), projection of each term's (p,q) */
/* onto the unit disk, and Nesterov momentum, starting from w = 0.           */
/* Pinned by: a hand-worked 2 x 2 prox in closed form, the duality gap of    */
/* a long FGP run, plain gradient projection converging to the same point.   */
/* ------------------------------------------------------------------------ */
/* L x at every interior term: p = vertical, q = horizontal difference;
 * arrays of (n-1)^2 terms, row-major. */
static void tv_L(int n, const double* x, double* p, double* q)
{
    int m = n - 1;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
            double x0 = x[(size_t)i * n + j];
            p[(size_t)i * m + j] = x[(size_t)(i + 1) * n + j] - x0;
            q[(size_t)i * m + j] = x[(size_t)i * n + j + 1] - x0;
        }
}

/* L^T (p, q): each term sends -(p + q) to its pixel, +p to the pixel below,
 * +q to the pixel on the right. */
static void tv_LT(int n, const double* p, const double* q, double* out)
{
    int m = n - 1;
    for (size_t k = 0; k < (size_t)n * n; ++k) out[k] = 0.0;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
            double pv = p[(size_t)i * m + j], qv = q[(size_t)i * m + j];
            out[(size_t)i * n + j] -= pv + qv;
            out[(size_t)(i + 1) * n + j] += pv;
            out[(size_t)i * n + j + 1] += qv;
        }
}

/* prox_{alpha TV}(b) by `iters` FGP steps (accel = 1) or plain gradient
 * projection steps (accel = 0).  The final dual field is returned in
 * p_out, q_out when they are not NULL. */
void orc_tv_prox(int n, const double* b, double alpha, int iters, int accel, double* x_out,
                 double* p_out, double* q_out)
{
    size_t J = (size_t)n * n, T = (size_t)(n - 1) * (n - 1);
    if (!(alpha > 0.0) || n < 2) {
        memcpy(x_out, b, sizeof(double) * J);
        if (p_out) memset(p_out, 0, sizeof(double) * T);
        if (q_out) memset(q_out, 0, sizeof(double) * T);
        return;
    }
    double* p = vec(T);      /* w_k          */
    double* q = vec(T);
    double* pr = vec(T);     /* r_k: the point the gradient step is taken from */
    double* qr = vec(T);
    double* pn = vec(T);
    double* qn = vec(T);
    double* lp = vec(T);
    double* lq = vec(T);
    double* w = vec(J);
    double t = 1.0;
    for (int k = 0; k < iters; ++k) {
        tv_LT(n, pr, qr, w);                                  /* w = b - alpha L^T r */
        for (size_t e = 0; e < J; ++e) w[e] = b[e] - alpha * w[e];
        tv_L(n, w, lp, lq);
        for (size_t e = 0; e < T; ++e) {                      /* gradient step, projection */
            double a = pr[e] + lp[e] / (8.0 * alpha);
            double c = qr[e] + lq[e] / (8.0 * alpha);
            double nrm = sqrt(a * a + c * c);
            double s = nrm > 1.0 ? nrm : 1.0;
            pn[e] = a / s;
            qn[e] = c / s;
        }
        if (accel) {
            double t1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
            double beta = (t - 1.0) / t1;
            for (size_t e = 0; e < T; ++e) {
                pr[e] = pn[e] + beta * (pn[e] - p[e]);
                qr[e] = qn[e] + beta * (qn[e] - q[e]);
            }
            t = t1;
        } else {
            memcpy(pr, pn, sizeof(double) * T);
            memcpy(qr, qn, sizeof(double) * T);
        }
        memcpy(p, pn, sizeof(double) * T);
        memcpy(q, qn, sizeof(double) * T);
    }
    tv_LT(n, p, q, w);                                        /* x = b - alpha L^T w */
    for (size_t e = 0; e < J; ++e) x_out[e] = b[e] - alpha * w[e];
    if (p_out) memcpy(p_out, p, sizeof(double) * T);
    if (q_out) memcpy(q_out, q, sizeof(double) * T);
    free(p); free(q); free(pr); free(qr); free(pn); free(qn); free(lp); free(lq); free(w);
}

/* FISTA (Eq. FISTA, Eq. FISTA-u):
 *   x_k = prox_{lambda/c^2, TV}(u_k + (1/c^2) A^T (y - A u_k)),
 *   u_{k+1} = x_k + ((t_k - 1)/t_{k+1}) (x_k - x_{k-1}),
 *   t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2,  t_1 = 1,  u_1 = x_0,
 * stopped, like the other methods of Sec. 4, at the first x_k with
 * f(x_k) <= eps (or after max_iter iterations); the output is that x_k.
 * c2 = c^2 = ||A||_2^2.  accel = 0 drops the momentum (ISTA, Eq. ISTA).
 * Trace rows (ORC_NF): k, f(x_k), TV(x_k), t_k, beta = (t_k-1)/t_{k+1}. */
int orc_fista(int n, int na, int nb, const double* y, const double* x0, double eps, double lambda,
              double c2, int prox_iters, int accel, int max_iter, double* x_out, orc_result* res,
              double* trace, int trace_rows)
{
    if (n < 2 || na <= 0 || nb <= 0 || !y || !x_out || !res || !(c2 > 0.0) || lambda < 0.0 ||
        prox_iters < 0 || max_iter < 0 || !(eps > 0.0))
        return ORC_ERR_INVALID;
    size_t J = (size_t)n * n, L = (size_t)na * nb;
    double* x = vec(J);        /* x_k      */
    double* xp = vec(J);       /* x_{k-1}  */
    double* u = vec(J);
    double* g = vec(J);
    double* bvec = vec(J);
    double* sino = vec(L);
    memset(res, 0, sizeof(*res));
    if (x0) memcpy(x, x0, sizeof(double) * J);
    memcpy(u, x, sizeof(double) * J);                        /* u_1 = x_0 */
    double t = 1.0;
    int it = 0, status = ORC_OK;
    for (;;) {
        orc_project(n, na, nb, x, sino);                      /* f(x_k) */
        double f = 0.0;
        for (size_t e = 0; e < L; ++e) {
            double r = y[e] - sino[e];
            f += r * r;
        }
        f *= 0.5;
        if (!(f > eps)) {                            /* f <= eps; NaN f: breakdown */
            if (!(f <= eps)) status = ORC_ERR_BREAKDOWN;
            break;
        }
        if (it >= max_iter) { status = ORC_MAX_ITER; break; }
        orc_project(n, na, nb, u, sino);                      /* A^T (y - A u_k) */
        for (size_t e = 0; e < L; ++e) sino[e] = y[e] - sino[e];
        orc_backproject(n, na, nb, sino, g);
        for (size_t e = 0; e < J; ++e) bvec[e] = u[e] + g[e] / c2;
        memcpy(xp, x, sizeof(double) * J);
        orc_tv_prox(n, bvec, lambda / c2, prox_iters, 1, x, NULL, NULL);   /* x_k */
        double t1 = accel ? 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t)) : 1.0;
        double beta = accel ? (t - 1.0) / t1 : 0.0;
        for (size_t e = 0; e < J; ++e) u[e] = x[e] + beta * (x[e] - xp[e]);   /* u_{k+1} */
        double* tr = row_of(trace, trace_rows, it);
        if (tr) {
            tr[ORC_T_K] = it + 1;
            tr[ORC_T_TV_AFTER] = orc_tv(n, x);
            tr[ORC_T_ALPHA] = t;
            tr[ORC_T_BETA] = beta;
        }
        t = t1;
        ++it;
    }
    memcpy(x_out, x, sizeof(double) * J);
    res->iters = it;
    res->k_final = it;
    res->status = status;
    orc_project(n, na, nb, x, sino);
    double f = 0.0;
    for (size_t e = 0; e < L; ++e) {
        double r = y[e] - sino[e];
        f += r * r;
    }
    res->f_final = 0.5 * f;
    res->tv_final = orc_tv(n, x);
    free(x); free(xp); free(u); free(g); free(bvec); free(sino);
    return status;
}
