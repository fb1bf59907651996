/*
 * scg_oracle.h -- plain, slow FP64 CPU oracle for TV-superiorized conjugate
 * gradient (Zibetti, Lin, Herman, "Total Variation Superiorized Conjugate
 * Gradient Method for Image Reconstruction").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header, table or helper with the CUDA library; the two meet only in
 * the seeded input generators, which hold none of the method's arithmetic.
 *
 * Geometry (the paper's parallel-beam set-up, Sec. 4; exact conventions are
 * this project's reading because the paper states none):
 *   image N x N, unit pixels centred on the origin; pixel (i = row, j = col)
 *     has centre xc = j - (N-1)/2, yc = i - (N-1)/2, stored row-major i*N+j;
 *   angles theta_a = pi * a / n_angles, a = 0..n_angles-1, cos/sin snapped to
 *     exact 0/1 at theta = 0 and theta = pi/2;
 *   bins of unit width, centres s_b = b - (n_bins-1)/2;
 *   ray (a,b) is the line xc*cos + yc*sin = s_b; sinogram stored a*n_bins+b;
 *   A[(a,b),(i,j)] = length of the ray inside pixel (i,j) (exact chord), with
 *     a ray lying exactly on a pixel edge giving half its length to each of
 *     the two pixels it separates.
 */
#ifndef SCG_ORACLE_H
#define SCG_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* variants, Algorithms 1, 3, 7, 9, 5, 13, 11 */
enum { ORC_CG = 0, ORC_PCG = 1, ORC_S_CG = 2, ORC_S_CG_CD = 3, ORC_S_CG_K = 4,
       ORC_S_PCG = 5, ORC_S_PCG_K = 6 };

/* perturbation rules: none, the gamma_l = gamma0 * a^l sequence with a TV
 * acceptance test (Eq. gamma_sequence, Sec. 3), the Appendix's
 * ||u_k|| = eta0 * ||g_k|| rule used by Proposition/Lemma of the Appendix, and
 * the proximal perturbation of the footnote to Eq. superiorized:
 * perturbed(x_k) = prox_{lambda_k TV}(x_k) */
enum { ORC_PERTURB_NONE = 0, ORC_PERTURB_GAMMA = 1, ORC_PERTURB_ETA = 2, ORC_PERTURB_PROX = 3 };

/* status codes */
enum { ORC_OK = 0, ORC_MAX_ITER = 1, ORC_ERR_INVALID = -1, ORC_ERR_BREAKDOWN = -4 };

/* per-iteration trace fields (one row of ORC_NF doubles per loop body) */
enum { ORC_T_K = 0, ORC_T_FTEST, ORC_T_TV_BEFORE, ORC_T_TV_AFTER, ORC_T_TRIALS,
       ORC_T_ACCEPTED, ORC_T_ELL, ORC_T_GAMMA, ORC_T_ALPHA, ORC_T_BETA,
       ORC_T_MARGIN, ORC_T_F_AFTER, ORC_NF };

typedef struct {
    int variant;
    double eps;          /* stopping threshold on f = 0.5 ||y - Ax||^2       */
    int perturb;         /* ORC_PERTURB_*                                      */
    double gamma0;       /* > 0: fixed gamma_0                                 */
    double gamma0_rel;   /* gamma0 <= 0: gamma_0 = gamma0_rel * ||x|| of the
                            first image that is actually perturbed             */
    double a;            /* kernel of gamma_l = gamma_0 a^l, 0 < a < 1         */
    int max_trials;      /* trials of the TV acceptance test per k             */
    double eta0;         /* Appendix rule constant                             */
    int K;               /* CG-K / PCG-K inner steps                           */
    int k_inclusive;     /* 1: literal "while k <= K" (K+1 steps)              */
    double mu;           /* filter offset; <= 0 selects 2*pi/P                 */
    double filter_gain;  /* scale of the filter factors (PCG is invariant)     */
    int filter_identity; /* 1: c(w) = filter_gain for every w (test special
                            case: PCG then reduces to CG)                      */
    int max_iter;        /* cap on loop bodies                                 */
    int prox_iters;      /* FGP steps of the proximal perturbation             */
    int perturb_steps;   /* perturbations per step (<= 1: one, as printed)     */
} orc_params;

typedef struct {
    int iters;           /* loop bodies executed                               */
    int k_final;         /* the algorithm's k when it stopped                  */
    int status;
    double f_final;      /* f(output)                                          */
    double tv_final;     /* TV(output)                                         */
    long long ell;       /* gamma index after the last trial                   */
    double gamma0_used;
} orc_result;

/* Solver state after a loop body (or before the first one).  Which vectors a
 * variant uses:
 *   CG, PCG:             x = x_k, p = p_k, g = g_k, delta = delta_k
 *   S-CG, S-PCG:         x = x_k, x_half = x_{k-1/2}, p = p_{k-1}, h = h_{k-1}
 *   S-CG-CD:             x = x_k, x_half = x_{k-1/2}, p = p_{k-1}, g = g_{k-1}
 *   S-CG-K, S-PCG-K:     x = x_k, x_half = x_{k-1/2}
 * plus the scalars k, ell, gamma0/gamma_fixed.  Vectors are caller-owned
 * arrays of J doubles (unused ones may be NULL).  Passing a state with
 * valid = 1 to orc_solve resumes from it (the initialisation steps are
 * skipped); a non-NULL final state receives the state at exit. */
typedef struct {
    int valid;
    int k;
    long long ell;
    double gamma0;
    int gamma_fixed;
    double delta;
    double* x;
    double* x_half;
    double* p;
    double* h;
    double* g;
} orc_state;

/* After each loop body: iteration index, x_{k+1} (current iterate), x_{k+1/2}
 * (perturbed point the step started from), the search direction p_k, h_k
 * (= A^T A p_k where the variant keeps it, else NULL), g_{k+1/2} (explicit
 * gradient at x_{k+1/2} where computed, else NULL). */
typedef void (*orc_iter_cb)(int it, const double* x_next, const double* x_half,
                            const double* p, const double* h, const double* g,
                            void* user);

int    orc_num_threads(void);
void   orc_angle(int a, int n_angles, double* c, double* s);
double orc_weight_trap(double d, double c, double s);
double orc_weight_clip(double xc, double yc, double c, double s, double sb);

void orc_project(int n, int na, int nb, const double* x, double* y);
void orc_backproject(int n, int na, int nb, const double* r, double* x);
void orc_project_dense(int n, int na, int nb, int use_clip, const double* x, double* y);
void orc_backproject_dense(int n, int na, int nb, int use_clip, const double* r, double* x);
void orc_project_rays(int n, int na, int nb, const double* x, int count,
                      const int* a_idx, const int* b_idx, double* out);
void orc_backproject_pixels(int n, int na, int nb, const double* r, int count,
                            const int* i_idx, const int* j_idx, double* out);

double orc_tv(int n, const double* x);
double orc_tv_grad(int n, const double* x, double* grad);

int    orc_filter_length(int nb);
double orc_filter_factor(double omega, double mu);
void   orc_filter_rows(int na, int nb, double mu, double gain, const double* r, double* out);

double orc_norm_A(int n, int na, int nb, int iters);

void orc_fbp(int n, int na, int nb, const double* y, double* x);

int orc_perturb_gamma(int n, const double* x, double gamma0, double a, int max_trials,
                      long long* ell, double* x_half, double* gamma_out, int* trials_out);
int orc_perturb_prox(int n, const double* x, double gamma0, double a, int prox_iters,
                     long long* ell, double* x_half, double* lambda_out);

void orc_tv_prox(int n, const double* b, double alpha, int iters, int accel, double* x_out,
                 double* p_out, double* q_out);
int orc_fista(int n, int na, int nb, const double* y, const double* x0, double eps, double lambda,
              double c2, int prox_iters, int accel, int max_iter, double* x_out, orc_result* res,
              double* trace, int trace_rows);

int orc_solve(int n, int na, int nb, const double* y, const double* x0,
              const orc_params* prm, double* x_out, orc_result* res,
              double* trace, int trace_rows, orc_iter_cb cb, void* user,
              const orc_state* resume, orc_state* final_state);

#ifdef __cplusplus
}
#endif
#endif
