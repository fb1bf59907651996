/*
 * scg.h -- C ABI of libscg, a GB300 (sm_103a) implementation of the
 * total-variation-superiorized conjugate gradient methods of Zibetti, Lin and
 * Herman ("Total Variation Superiorized Conjugate Gradient Method for Image
 * Reconstruction") for least-squares parallel-beam CT.
 *
 * Problem (Sec. 1, Eq. LS1):  find x minimising f(x) = 1/2 ||y - A x||^2,
 * stopping as soon as f <= eps, with total variation (TV) as the secondary
 * criterion that the superiorized variants lower along the way.
 *
 * Geometry (Sec. 4: parallel beam, angles uniform over [0, 180) degrees; the
 * precise conventions below are this library's, the paper states none):
 *   image   N x N unit pixels centred on the origin, row-major, pixel (i, j)
 *           (row i, column j) centred at xc = j - (N-1)/2, yc = i - (N-1)/2;
 *   angles  theta_a = pi * a / n_angles, a = 0 .. n_angles-1;
 *   bins    unit width, centres s_b = b - (n_bins-1)/2;
 *   rays    ray (a, b) is the line xc cos(theta_a) + yc sin(theta_a) = s_b;
 *   data    sinogram row-major [angle][bin];
 *   A       A[(a,b),(i,j)] = exact length of ray (a,b) inside pixel (i,j); a
 *           ray running along a pixel edge gives half its length to each of
 *           the two pixels it separates.
 *
 * Element types follow scg_precision: double for SCG_F64, float for SCG_F32,
 * IEEE binary16 for SCG_F16, bfloat16 for SCG_BF16.
 *
 * Memory: every array argument is a DEVICE pointer owned by the caller, except
 * where a comment says "host".  Entry points that need scratch take a device
 * workspace (16-byte aligned) whose size the matching *_workspace_bytes query
 * returns; the library itself never allocates device memory.  Workspace
 * contents do not need to be initialised and must not be shared by calls that
 * may run at the same time.
 *
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  Operator
 * calls are asynchronous and stream-ordered.  scg_solve returns when the solve
 * has finished (it reads the device's stop flag); scg_solve_async enqueues the
 * same solve and returns, its result written by the device.
 *
 * Errors: every entry point returns an int status (scg_status).  Nothing
 * prints, aborts or throws; scg_strerror() names a code.  Invalid arguments
 * are rejected before any launch.
 */
#ifndef SCG_H
#define SCG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SCG_OK = 0,               /* finished; for solves: f(output) <= eps         */
    SCG_WARN_MAX_ITER = 1,    /* solve stopped at max_iter with f > eps          */
    SCG_ERR_INVALID = -1,     /* bad geometry/size/pointer/parameter             */
    SCG_ERR_CUDA = -2,        /* a CUDA runtime call failed, or a kernel's       */
                              /* bounded wait for its own copies ran out         */
    SCG_ERR_WORKSPACE = -3,   /* workspace too small or misaligned               */
    SCG_ERR_BREAKDOWN = -4,   /* zero or non-finite CG denominator               */
    SCG_ERR_UNSUPPORTED = -5  /* precision/variant combination not available     */
} scg_status;

/* The seven algorithms of the paper. */
typedef enum {
    SCG_CG = 0,       /* Algorithm 1 (steps: CG-STEP, Algorithm 2)               */
    SCG_PCG = 1,      /* Algorithm 3 (steps: PCG-STEP, Algorithm 4)              */
    SCG_S_CG = 2,     /* Algorithm 7 (steps: CG-PR-STEP, Algorithm 8)            */
    SCG_S_CG_CD = 3,  /* Algorithm 9 (steps: CG-CD-STEP, Algorithm 10)           */
    SCG_S_CG_K = 4,   /* Algorithm 5 (calls CG-K, Algorithm 6)                   */
    SCG_S_PCG = 5,    /* Algorithm 13 (steps: PCG-PR-STEP, Algorithm 14)         */
    SCG_S_PCG_K = 6,  /* Algorithm 11 (calls PCG-K, Algorithm 12)                */
    SCG_FISTA = 7     /* the comparison method of Sec. 4: FISTA (Sec. 2, Eq. FISTA
                         and Eq. FISTA-u) for f(x) + lambda TV(x),
                         x_k = prox_{lambda/c^2, TV}(u_k + A^T(y - A u_k)/c^2),
                         u_{k+1} = x_k + ((t_k - 1)/t_{k+1})(x_k - x_{k-1}),
                         t_{k+1} = (1 + sqrt(1 + 4 t_k^2))/2, t_1 = 1, u_1 = x_0;
                         the prox (Eq. prox) by prox_iters steps of Beck and
                         Teboulle's fast gradient projection on TV's dual, from
                         zero; stopped at the first x_k with f(x_k) <= eps (as
                         the paper's Sec. 4 stops every method) or max_iter.
                         scg_solve only (FP32/FP64; no resume, no final_state);
                         scg_solve_batch and the server return
                         SCG_ERR_UNSUPPORTED.  Trace rows: k, f(x_k) in field
                         11, t_k in field 8, (t_k - 1)/t_{k+1} in field 9.   */
} scg_variant;

typedef enum {
    SCG_F64 = 0,      /* FP64 storage and arithmetic                             */
    SCG_F32 = 1,      /* FP32 storage and arithmetic, FP64 reductions/scalars    */
    SCG_F16 = 2,      /* binary16 storage of every image and sinogram vector,
                         FP32 arithmetic, FP64-quality reductions, FP64 scalars;
                         solves run on the scaled system c A x ~ c y (c a power of
                         two near 1/sqrt(n_angles N), which leaves the iterates
                         unchanged) so that no vector leaves binary16's range;
                         the operator entry points apply A unscaled.  Solves:
                         the superiorized variants only -- CG and PCG update
                         g and r recursively (Algorithms 2, 4), which an 11-
                         or 8-bit mantissa cannot carry (SCG_ERR_UNSUPPORTED) */
    SCG_BF16 = 3      /* as SCG_F16 with bfloat16 storage                        */
} scg_precision;

typedef enum {
    SCG_PERTURB_NONE = 0,   /* no superiorization step (x_{k+1/2} = x_k)          */
    SCG_PERTURB_GAMMA = 1,  /* gamma_l = gamma0 a^l with TV acceptance (Sec. 3)   */
    SCG_PERTURB_ETA = 2,    /* the Appendix's rule (Eq. up bnd u_k):
                               x_{k+1/2} = x_k + u_k, u_k = eta0 ||g_k|| v_k with
                               g_k = A^T (A x_k - y) and v_k = -dTV/||dTV||, no TV
                               test; with 0 < eta0 <= min(1/(4c^2), eta2) (c =
                               ||A||_2, eta2 the positive root of
                               (2 + c^2 eta) eta = 1/(32 c^2)) the Lemma bounds
                               2f(x_k) - 2f(x_{k+1}) >= ||g_k||^2 / (32 c^2).
                               Costs one extra A and A^T pass per loop body.   */
    SCG_PERTURB_PROX = 3    /* proximal perturbation (footnote to Eq.
                               superiorized): x_{k+1/2} = prox_{lambda TV}(x_k)
                               by prox_iters FGP steps, lambda = gamma_0 a^l /
                               ||dTV(x_k)|| (gamma_0 as for the gamma rule); no
                               TV test (a prox step cannot raise TV), l <- l+1
                               per perturbed step.  S-variants only, FP32/FP64
                               storage, scg_solve / scg_solve_async only (the
                               batch and the server return SCG_ERR_UNSUPPORTED);
                               needs scg_solve_workspace_bytes_p's workspace. */
} scg_perturb;

typedef struct {
    int n;            /* image side N (J = N*N pixels), 2 <= N <= 8192          */
    int n_angles;     /* number of projection angles, 1 <= n_angles <= 16384    */
    int n_bins;       /* detector bins per angle, 1 <= n_bins <= 16384          */
} scg_geometry;

/* Solver parameters (Sec. 3 and Sec. 4).  scg_default_params() fills the
 * defaults named below. */
typedef struct {
    int perturb;         /* scg_perturb; default SCG_PERTURB_GAMMA              */
    double gamma0;       /* > 0: gamma_0 of Eq. gamma_sequence.  <= 0: gamma_0 =
                            gamma0_rel * ||x|| of the first image that is
                            perturbed (default 0)                                */
    double gamma0_rel;   /* default 0.05                                         */
    double a;            /* gamma_l = gamma_0 a^l; 0 < a < 1; default 0.975 (Sec. 4) */
    int max_trials;      /* TV-acceptance trials per perturbation; default 32 (a
                            step's first trial pass evaluates 3 candidates, each
                            later pass, run only while none is accepted, up to
                            31)                                                   */
    int K;               /* CG-K/PCG-K inner steps (S-CG-K, S-PCG-K), 1 .. 1000;
                            default 2                                             */
    int k_inclusive;     /* 1: the printed loop "while k <= K" (K+1 steps); default 0 */
    double mu;           /* filter offset of c(w); <= 0 selects 2*pi/P (default)  */
    double filter_gain;  /* scale of c(w); default 1                              */
    int max_iter;        /* cap on loop bodies, 0 .. 10^7; default 100             */
    int host_loop;       /* 0 (default): the while loop runs as one CUDA graph
                            with a conditional node steered by the device.
                            1: one graph per loop body, launched in batches
                            and polled by the host (same kernels; for tools
                            that profile kernels one launch at a time)          */
    double eta0;         /* SCG_PERTURB_ETA only: eta0 > 0 (default 0)          */
    double lambda;       /* SCG_FISTA: weight of TV, >= 0 (default 0: no prox)  */
    int prox_iters;      /* SCG_FISTA and SCG_PERTURB_PROX: FGP steps per prox,
                            0 .. 100000 (default 20; >= 1 for SCG_PERTURB_PROX) */
    double lipschitz;    /* SCG_FISTA: c^2 = ||A||_2^2 (Appendix, Eq. lambda);
                            <= 0 (default): estimated on the device by 100 power
                            iterations on A^T A from 1 + 0.001 (index mod 7) and
                            cached per device, precision and geometry           */
    int proj_shape;      /* 0 (default): the projector's block shape is the one the
                            library's tuner measured fastest for this geometry
                            bucket (the first solve of a bucket in a process
                            times the shapes, so two processes may pick
                            differently); 5..8: blocks of 2^(8-s) angles x 2^s
                            rays, untimed.  Every ray is computed alike in any
                            shape, but f sums the blocks' partial sums, whose
                            rounding depends on the shape: a fixed proj_shape
                            makes solves repeat bit for bit across processes */
    int perturb_steps;   /* perturbations per step, 1 .. 16 (0 or 1: one, as in
                            Algorithms 5-14; default 1).  With more, the rule
                            (SCG_PERTURB_GAMMA or SCG_PERTURB_PROX) is applied
                            in succession, each time from the current point with
                            its own subgradient and trial budget, l running on;
                            the trace row keeps TV(x_k) and the last sub-step's
                            perturbation fields.  SCG_PERTURB_ETA takes one.  */
} scg_params;

typedef struct {
    int iters;           /* loop bodies executed                                   */
    int k_final;         /* the algorithm's counter k when it stopped              */
    int status;          /* scg_status of the solve                                */
    double f_final;      /* f(output), from the device's FP64 reduction            */
    double tv_final;     /* TV(output)                                             */
    long long ell;       /* index l of the gamma sequence after the last trial     */
    double gamma0_used;  /* gamma_0 in force at exit (0 if never fixed)            */
    int kernel_launches; /* kernels this call enqueued (graph nodes counted per
                            launch of the loop-body graph)                       */
    int body_launches;   /* loop bodies started (with the polled loop, bodies
                            launched after the stop flag return at once)         */
    int device_loop;     /* 1: the loop ran as one CUDA graph whose conditional
                            node the device steers; 0: host-polled graph launches */
    double lipschitz_used; /* SCG_FISTA: the c^2 the solve used (else 0)       */
} scg_result;

/* Solver state, for exact checkpoint/resume and for single-step checks.  The
 * vectors are caller-owned device arrays of N*N elements (NULL when a variant
 * does not use them):
 *   CG, PCG:        x = x_k, p = p_k, g = g_k, delta = delta_k
 *   S-CG, S-PCG:    x = x_k, x_half = x_{k-1/2}, p = p_{k-1}, h = h_{k-1}
 *   S-CG-CD:        x = x_k, x_half = x_{k-1/2}, p = p_{k-1}, g = g_{k-1}
 *   S-CG-K, S-PCG-K: x = x_k, x_half = x_{k-1/2}
 * (Appendix, Propositions on h_{k-1} and p_{k-1}: this tuple determines the
 * continuation of Algorithm 7.) */
typedef struct {
    int valid;           /* set to 1 on export; must be 1 to resume               */
    int k;
    long long ell;
    double gamma0;
    int gamma_fixed;
    double delta;
    void* x;
    void* x_half;
    void* p;
    void* h;
    void* g;
} scg_state;

/* Per-iteration trace row written by scg_solve (host array of
 * trace_rows * SCG_TRACE_FIELDS doubles): k, f(x_{k-1/2}) tested at the top of
 * the loop body, TV(x_k), TV(x_{k+1/2}), trials, accepted (1/0, -1 = no
 * perturbation attempted), l after the trials, accepted gamma, alpha, beta,
 * smallest relative TV margin of the trials, f(x_{k+1/2}).  Under
 * SCG_PERTURB_PROX the gamma field holds lambda and TV(x_{k+1/2}) is NaN (not
 * computed). */
#define SCG_TRACE_FIELDS 12

const char* scg_strerror(int status);
void scg_default_params(scg_params* p);

/* Bytes of device workspace for the operator entry points below. */
size_t scg_op_workspace_bytes(const scg_geometry* g, int precision);

/* y = A x (Eq. LS1's system matrix; the ray-driven forward projector).
 * x: N*N image, y: n_angles*n_bins sinogram (both device). */
int scg_project(const scg_geometry* g, int precision, const void* x, void* y,
                void* work, size_t work_bytes, void* stream);

/* x = A^T r (the backprojection in every step of Algorithms 1-14; pixel-driven
 * gather that evaluates the same weights as scg_project, no atomics).  With
 * FP32 arithmetic and n a multiple of 64 it pairs each pixel (x, y) with its
 * mirror (-x, y), which meets angle pi - theta at the same detector position,
 * so the two share one weight evaluation; results agree with the plain gather
 * (other n, angle-block operators) to FP32 rounding, not bit for bit. */
int scg_backproject(const scg_geometry* g, int precision, const void* r, void* x,
                    void* work, size_t work_bytes, void* stream);

/* Release the library's host-side caches: the CUDA graphs captured for earlier
 * solves and batches (keyed by workspace address and geometry) and the
 * per-device side streams and pinned flags; they are rebuilt on the next call.
 * The tuned projector shapes are kept; scg_tv_static's cached scratch
 * addresses are forgotten.  No library call may be running or have work in
 * flight.  The library holds no device memory of its own beyond
 * what these objects use. */
int scg_release(void);

/* Test hook for the error path of the device's bounded waits (fault injection
 * on the host; the paper has no counterpart).  With stall != 0, problems set up
 * afterwards get sinogram copies 16 bytes shorter per angle than the FP32 /
 * 16-bit gather's barriers expect: the copies all complete, but each wait for a
 * chunk runs out after its limit (about 0.13 s), the solve stops at
 * its next loop test and returns SCG_ERR_CUDA (batch and server: that
 * problem's status).  No fault is raised and the context stays usable; the
 * gather's results are not valid meanwhile.  stall = 0 (the default) restores
 * normal operation for problems set up afterwards.  Returns SCG_OK. */
int scg_test_stall_copies(int stall);

/* ---- Prepared operator pair ------------------------------------------------
 * For callers that apply A and A^T many times with one geometry (their own
 * iterative methods): the angle table, descriptors and zero pads are placed in
 * the workspace once, so each application is only device work (a descriptor
 * update and two kernels), asynchronous and capturable in a CUDA graph.  The
 * workspace (scg_op_workspace_bytes) belongs to the operator until
 * scg_operator_destroy; applications through one operator must not overlap in
 * time (they share its workspace).  The paper has no counterpart. */
typedef struct scg_operator scg_operator;    /* opaque */

/* Prepare (blocking: returns after the workspace is set up).  Returns
 * SCG_ERR_INVALID / SCG_ERR_UNSUPPORTED / SCG_ERR_WORKSPACE as scg_project. */
int scg_operator_create(const scg_geometry* g, int precision, void* work, size_t work_bytes,
                        void* stream, scg_operator** out);
/* A prepared operator for one block of consecutive angles of a scan: the rows
 * a_begin .. a_begin + a_count - 1 of A for the scan g (angle a_begin + a of
 * g->n_angles is the operator's angle a).  Projections write a_count x n_bins
 * sinograms; backprojections read them and give that block's share of A^T r
 * (the shares of a partition of the angles add up to A^T r).  This is the
 * local operator of an angle-sharded solve, where each GPU holds one block of
 * the data.  Workspace: scg_op_workspace_bytes of {n, a_count, n_bins}.
 * Returns SCG_ERR_INVALID unless 0 <= a_begin, 1 <= a_count and
 * a_begin + a_count <= g->n_angles.  The paper has no counterpart. */
int scg_operator_create_angles(const scg_geometry* g, int a_begin, int a_count, int precision, void* work,
                               size_t work_bytes, void* stream, scg_operator** out);
/* y = A x, as scg_project (stream-ordered, asynchronous). */
int scg_operator_project(scg_operator* op, const void* x, void* y, void* stream);
/* x = A^T r, as scg_backproject (stream-ordered, asynchronous). */
int scg_operator_backproject(scg_operator* op, const void* r, void* x, void* stream);
/* Turn kernel timing on (enable != 0) or off (0, the default) for the
 * operator's later applications.  While it is on, each application records two
 * CUDA events on its stream immediately before and after the projector (gather)
 * kernel -- about 4 microseconds of device time per application -- except in
 * calls made while the stream is being captured into a graph.  Returns
 * SCG_ERR_INVALID for a NULL operator. */
int scg_operator_timing(scg_operator* op, int enable);
/* Device time, in milliseconds, of the projector (gather) kernel alone in the
 * operator's last timed scg_operator_project (scg_operator_backproject) call,
 * from the events described under scg_operator_timing.  Blocks until that
 * kernel has finished.  Either pointer may be NULL; returns SCG_ERR_INVALID
 * when the requested kernel has no timed call. */
int scg_operator_kernel_ms(scg_operator* op, float* project_ms, float* backproject_ms);
/* Release the host handle (the workspace is the caller's again once the
 * stream work issued through the operator has completed). */
int scg_operator_destroy(scg_operator* op);

/* *tv_out (device double) = TV(x), the secondary criterion: isotropic forward
 * differences over the (N-1)^2 interior terms (the paper names TV without a
 * formula; Sec. 1).  Summed in FP64. */
int scg_tv(int n, int precision, const void* x, double* tv_out,
           void* work, size_t work_bytes, void* stream);

/* *tv_out (device double) = TV(x), exactly as scg_tv computes it, but with no
 * workspace argument: for callers that cannot allocate device memory (a
 * plug-in inside a host program whose memory pool owns the device, a real-time
 * loop that forbids allocator calls, a fixed memory budget set at start-up).
 * The paper has no counterpart; this is an interface convenience.
 * Scratch lives in one array of about 1 MiB that the library defines in device
 * memory; every GPU that loads the library holds it until the process exits.
 * Limits and behaviour:
 *   n must be 2 .. 1024 (larger n returns SCG_ERR_UNSUPPORTED);
 *   precision SCG_F32 or SCG_F64 (the storage formats return SCG_ERR_UNSUPPORTED);
 *   allocates nothing (no cudaMalloc/cudaFree, no allocating library call);
 *   the first call on a device looks up the array's device address with that
 *   device current -- make that first call before any stream capture; the
 *   address belongs to that device's current context: after the context is
 *   destroyed (cudaDeviceReset), call scg_release() before the next call so
 *   that the address is looked up again;
 *   all calls share the array: calls that may overlap on the GPU (e.g. from
 *   two streams at once) race and give undefined results. */
int scg_tv_static(int n, int precision, const void* x, double* tv_out, void* stream);

/* grad = a subgradient of TV at x (terms with zero norm contribute 0) and
 * *tv_out = TV(x); the nonascending direction of the perturbation step is
 * -grad/||grad|| (Sec. 1, Eq. superiorization). */
int scg_tv_grad(int n, int precision, const void* x, void* grad, double* tv_out,
                void* work, size_t work_bytes, void* stream);

/* out = F^T C F r row by row: the filtering part of the preconditioner
 * z = A^T F^T C F (A x - y) of Sec. 3, c(w) = gain (|w| + mu)(0.54 + 0.46 cos w)
 * on a unitary DFT of each row zero-padded to P = 2^ceil(log2(2 n_bins)), w the
 * DFT frequency 2 pi k / P folded into [-pi, pi].  mu <= 0 selects 2*pi/P;
 * gain > 0.  r, out: n_angles*n_bins (device).  The FFT of a padded row pair is
 * held in shared memory: n_bins above 8192 (FP32, FP16, BF16) or 4096 (FP64)
 * returns SCG_ERR_UNSUPPORTED (the same limit applies to the preconditioned
 * solvers, and to scg_fbp). */
int scg_filter(const scg_geometry* g, int precision, double mu, double gain,
               const void* r, void* out, void* work, size_t work_bytes, void* stream);

/* x = filtered backprojection of the sinogram y: the reconstruction Sec. 4
 * shows as its visual reference (the method of Herman's textbook, Ch. 8, with
 * the Hamming-windowed ramp Sec. 3 names).  The parallel-beam inversion
 * x(s) = int_0^pi (p_theta * q)(s) d theta with the ramp q = |nu| (nu in cycles
 * per bin width), discretised: each row is filtered as scg_filter does with
 * mu = 0 and gain 1/(2 n_angles) (= the angle step pi/n_angles over the 2 pi
 * between w and nu), and x = A^T of the filtered rows (A^T spreads each
 * angle's value over a pixel with weights adding up to the pixel area).
 * y: n_angles*n_bins, x: N*N (device); workspace scg_op_workspace_bytes;
 * stream-ordered and asynchronous; n_bins limit as scg_filter. */
int scg_fbp(const scg_geometry* g, int precision, const void* y, void* x,
            void* work, size_t work_bytes, void* stream);

/* Bytes of device workspace for scg_solve with this geometry and variant
 * (default parameters: every perturbation rule but SCG_PERTURB_PROX). */
size_t scg_solve_workspace_bytes(const scg_geometry* g, int variant, int precision);
/* The same for the given parameters (prm may be NULL: the defaults);
 * SCG_PERTURB_PROX adds four dual fields of 2 N^2 stored values.  0 on
 * invalid arguments. */
size_t scg_solve_workspace_bytes_p(const scg_geometry* g, int variant, int precision, const scg_params* prm);

/* Run one solver of the paper from x0 (NULL = zeros) to f <= eps or max_iter.
 *   y      n_angles*n_bins data (device); x_out  N*N output (device): for the
 *          superiorized variants x_{k-1/2}, for CG/PCG x_k (their last steps).
 *   res    host; filled on return.  trace: host, NULL or trace_rows rows.
 *   resume NULL, or a state exported by an earlier call with the same
 *          geometry/variant/precision (its vectors are read, not kept).
 *   final  NULL, or a state whose vector pointers are filled on return.
 * Blocking: returns after the device has finished.  Returns res->status. */
int scg_solve(const scg_geometry* g, int variant, int precision, const scg_params* prm,
              double eps, const void* y, const void* x0, void* x_out,
              void* work, size_t work_bytes, scg_result* res,
              double* trace, int trace_rows,
              const scg_state* resume, scg_state* final_state, void* stream);

/* scg_solve, stream-ordered and asynchronous: the solve is enqueued on
 * `stream` and the call returns; the device writes *res when the stream gets
 * there (its status field then holds the solve's own status, as scg_solve
 * returns it), and x_out is ordered before later work on `stream`.
 *   res   device-accessible memory: device memory, or pinned host memory
 *         (cudaMallocHost / cudaHostAlloc), read after the stream has passed;
 *   no trace and no exported state (use scg_solve for those); host_loop must
 *   be 0 (SCG_ERR_UNSUPPORTED otherwise).
 * Returns SCG_OK once enqueued, or an error found before any launch.  The
 * first call for a geometry bucket and precision times the projector shapes
 * and captures the loop graph, which blocks; later calls do not (a FISTA solve
 * with lipschitz <= 0 estimates c^2 on the device every time: the estimate is
 * not read back here). */
int scg_solve_async(const scg_geometry* g, int variant, int precision, const scg_params* prm,
                    double eps, const void* y, const void* x0, void* x_out,
                    void* work, size_t work_bytes, scg_result* res,
                    const scg_state* resume, void* stream);

/* One problem of a batched solve: its geometry, threshold and buffers (device
 * pointers as for scg_solve; x0 may be NULL). */
typedef struct {
    scg_geometry geometry;
    double eps;
    const void* y;
    const void* x0;
    void* x_out;
} scg_problem;

/* Bytes of device workspace for scg_solve_batch with these problems. */
size_t scg_batch_workspace_bytes(const scg_problem* problems, int count, int variant, int precision);

/* Solve `count` independent problems (each its own geometry, eps, data) with
 * one variant, precision and parameter set, advancing them together: every
 * kernel launch covers the work items of all problems, each problem keeps its
 * own device-resident state and stops on its own test, and the loop runs until
 * every problem has stopped (Sec. 3's algorithms, batched; the paper solves
 * one problem at a time).  Each problem's output equals what scg_solve gives
 * for it alone, bit for bit.  results: host array of `count`.  Blocking.
 * Returns SCG_OK when every problem ended with f <= eps, else the first
 * problem's non-OK status (each result carries its own). */
int scg_solve_batch(const scg_problem* problems, int count, int variant, int precision,
                    const scg_params* prm, void* work, size_t work_bytes, scg_result* results,
                    void* stream);

/* ---- Serving: continuous batching over a request stream ------------------
 *
 * A server holds a set of resident requests in a caller-owned device pool and
 * advances all of them together, one launch per kernel of the loop body over
 * the work items of every resident request (as scg_solve_batch does).  A
 * request joins at the next step after it is submitted, once a slot and pool
 * memory are free (admission in submission order, by the bytes its state
 * needs), keeps its whole solver state in the pool while it runs, and leaves
 * the step after it stops, freeing its memory.  Each result equals what
 * scg_solve gives for the same request alone, bit for bit.  The paper solves
 * one problem at a time; serving is this library's. */
typedef struct scg_server scg_server;       /* opaque */

typedef struct {
    int variant;            /* one SCG_* variant for every request */
    int precision;          /* an scg_precision */
    scg_params params;      /* shared by every request (eps is per request); host_loop must be 0 */
    void* pool;             /* caller-owned device memory for resident states and work lists,
                               16-byte aligned; must outlive the server */
    size_t pool_bytes;
    int max_active;         /* most requests resident at once, 1..65535 */
    int bodies_per_step;    /* loop bodies each resident request advances per step, >= 1 */
} scg_server_config;

typedef struct {
    unsigned long long tag; /* the tag given to scg_server_submit */
    scg_result result;      /* as scg_solve's; x_out has been written */
} scg_completion;

/* Pool bytes one resident request of this geometry holds (its state, vectors
 * and work items); 0 on invalid arguments. */
size_t scg_server_footprint(const scg_geometry* g, int variant, int precision);

/* Create a server (host memory only; the pool is not touched until the first
 * step).  *out receives the handle.  Returns SCG_ERR_INVALID on bad
 * arguments. */
int scg_server_create(const scg_server_config* cfg, scg_server** out);

/* Queue one request.  The problem's buffers (y, x0, x_out) are device
 * pointers that must stay valid until its completion is returned.  Returns
 * SCG_ERR_INVALID on bad arguments, SCG_ERR_WORKSPACE if its footprint can
 * never fit the pool.  Host-only; does not block. */
int scg_server_submit(scg_server* srv, const scg_problem* req, unsigned long long tag);

/* One step: admit queued requests that fit (in submission order; a request
 * that does not fit yet waits, and so do the ones behind it; one that cannot
 * fit even with nothing resident completes at once with status
 * SCG_ERR_WORKSPACE), advance every
 * resident request by bodies_per_step loop bodies, finish the ones that
 * stopped and write up to max_done completions to done[] (*n_done gets the
 * count; completions beyond max_done are kept for the next step).  Blocking:
 * returns after the device has finished the step; the completed outputs are
 * ordered before later work on `stream`. */
int scg_server_step(scg_server* srv, void* stream, scg_completion* done, int max_done, int* n_done);

/* Requests queued (not yet admitted) and resident. */
int scg_server_pending(const scg_server* srv, int* queued, int* active);

/* Destroy the server (pending requests are dropped).  The pool is the
 * caller's to free afterwards.
 *
 * A server is driven by one host thread at a time.  After a step returns an
 * error (SCG_ERR_CUDA, SCG_ERR_WORKSPACE) its requests' states are undefined:
 * destroy it. */
int scg_server_destroy(scg_server* srv);

#ifdef __cplusplus
}
#endif
#endif
