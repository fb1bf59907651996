// solver.cu -- host side of libscg: workspace layout, the per-variant kernel
// programs of Algorithms 1-14, CUDA-graph capture of the loop body, the
// operator entry points and scg_solve.
//
// A solve runs as: an initialisation program (the algorithm's set-up steps),
// then repeated launches of one captured CUDA graph holding a whole loop body.
// Every scalar decision (beta, alpha, the TV acceptance index l, the eps test,
// the iteration cap, breakdown) is taken on the device by the block that
// finishes the relevant reduction; once the device sets its stop flag, every
// kernel of later bodies returns at once.  The host only reads the flag
// between batches of bodies, one batch ahead of the device.
#include <math.h>
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "scg_kernels.h"

using namespace scg;

namespace {

constexpr int kMaxTraceRows = 4096;
constexpr size_t kAlign = 256;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
int round_up4(int v) { return (v + 3) / 4 * 4; }

bool valid_geometry(const scg_geometry* g) {
    return g && g->n >= 2 && g->n <= 8192 && g->n_angles >= 1 && g->n_angles <= 16384 &&
           g->n_bins >= 1 && g->n_bins <= 16384;
}

int filter_length(int nb) {
    int P = 1;
    while (P < 2 * nb) P *= 2;
    return P;
}

int family_of(int v) {
    if (v == SCG_CG || v == SCG_PCG) return FAM_CG;
    if (v == SCG_S_CG_K || v == SCG_S_PCG_K) return FAM_S_K;
    return FAM_S_PR;
}

bool uses_filter(int v) { return v == SCG_PCG || v == SCG_S_PCG || v == SCG_S_PCG_K; }

// Workspace plan: byte offsets of every segment.
struct Plan {
    size_t state, prob, ang, taps, partials, counter, trace;
    size_t img[IB_COUNT];
    size_t view_rm, view_cm;
    size_t sino[SB_COUNT];
    size_t total;
    int S, SB, cnt_ray, cnt_img, cnt_row, tiles_x, ray_blocks, filt_blocks, P;
    int cnt_proj, proj_blocks;
};

enum PlanKind { PLAN_OP = 0, PLAN_SOLVE = 1 };

Plan make_plan(const scg_geometry& g, int variant, size_t tsize, int kind) {
    Plan p;
    memset(&p, 0, sizeof(p));
    const int N = g.n, na = g.n_angles, nb = g.n_bins;
    p.S = round_up4(N + 2 * kPad);          // pairs per view line
    p.SB = round_up4(nb + 2 * kSPad);       // pairs per sinogram-view row
    p.ray_blocks = (nb + kRayBlock - 1) / kRayBlock;
    p.tiles_x = (N + kTileW - 1) / kTileW;
    p.cnt_ray = na * p.ray_blocks;
    p.cnt_img = ((N + kTileH - 1) / kTileH) * p.tiles_x;
    p.filt_blocks = (nb + kFilterBlock - 1) / kFilterBlock;
    p.cnt_row = na * p.filt_blocks;
    p.proj_blocks = (nb + kProjRays - 1) / kProjRays;
    p.cnt_proj = ((na + kProjAngles - 1) / kProjAngles) * p.proj_blocks;
    p.P = filter_length(nb);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, kAlign); return o; };
    const size_t J = (size_t)N * N;
    p.state = take(sizeof(DevState));
    p.prob = take(sizeof(Prob<double>));
    p.ang = take(sizeof(Angle<double>) * na);
    p.taps = take(tsize * (2 * (size_t)nb - 1));
    int maxcnt = p.cnt_ray > p.cnt_img ? p.cnt_ray : p.cnt_img;
    if (p.cnt_row > maxcnt) maxcnt = p.cnt_row;
    if (p.cnt_proj > maxcnt) maxcnt = p.cnt_proj;
    p.partials = take(sizeof(double) * kSlots * (size_t)maxcnt);
    p.counter = take(sizeof(unsigned) * 4);
    p.view_rm = take(2 * tsize * (size_t)N * p.S);
    p.view_cm = take(2 * tsize * (size_t)N * p.S);
    const size_t sino_bytes = 2 * tsize * (size_t)na * p.SB;
    for (int q = 0; q < IB_COUNT; ++q) p.img[q] = (size_t)-1;
    for (int q = 0; q < SB_COUNT; ++q) p.sino[q] = (size_t)-1;
    if (kind == PLAN_OP) {
        p.trace = (size_t)-1;
        p.sino[SB_R] = take(sino_bytes);
    } else {
        p.trace = take(sizeof(double) * TR_NF * kMaxTraceRows);
        const int fam = family_of(variant);
        p.img[IB_X] = take(tsize * J);
        p.img[IB_P] = take(tsize * J);
        p.img[IB_H] = take(tsize * J);
        p.img[IB_G] = take(tsize * J);
        if (fam != FAM_CG) {
            p.img[IB_XH] = take(tsize * J);
            p.img[IB_TVG] = take(tsize * J);
        }
        if (uses_filter(variant)) p.img[IB_Z] = take(tsize * J);
        p.sino[SB_R] = take(sino_bytes);
        p.sino[SB_Q] = take(sino_bytes);
        if (uses_filter(variant)) p.sino[SB_W] = take(sino_bytes);
    }
    p.total = off;
    return p;
}

template <typename T>
void fill_angles(std::vector<Angle<T>>& out, int na, int n) {
    out.resize(na);
    const double off_n = 0.5 * (n - 1);
    for (int a = 0; a < na; ++a) {
        double c, s;
        if (a == 0) { c = 1.0; s = 0.0; }
        else if (2 * a == na) { c = 0.0; s = 1.0; }
        else { const double th = M_PI * (double)a / (double)na; c = cos(th); s = sin(th); }
        const double ac = fabs(c), as = fabs(s);
        const double m = ac > as ? ac : as, mn = ac > as ? as : ac;
        const double hs = 0.5 * (m + mn);
        Angle<T> g;
        memset(&g, 0, sizeof(g));
        g.c = (T)c;
        g.s = (T)s;
        g.inv_m = (T)(1.0 / m);
        if (mn == 0.0) {
            g.k2 = (T)1.0; g.h2 = (T)1.0; g.h2p = (T)2.0;
            g.kb = (T)1.0; g.hb0 = (T)1.0; g.hb1 = (T)0.0;
            g.hb0p = (T)2.0; g.hb1p = (T)-1.0;
        } else {
            g.k2 = (T)(m / mn); g.h2 = (T)(hs / mn); g.h2p = (T)(hs / mn + m / mn);
            g.kb = (T)(1.0 / mn); g.hb0 = (T)(hs / mn); g.hb1 = (T)((hs - 1.0) / mn);
            g.hb0p = (T)(hs / mn + 1.0 / mn); g.hb1p = (T)((hs - 1.0) / mn - 1.0 / mn);
        }
        g.c24 = (int)llrint(c * 16777216.0);
        g.s24 = (int)llrint(s * 16777216.0);
        g.col_driven = as >= ac ? 1 : 0;
        const double inv = g.col_driven ? 1.0 / s : 1.0 / c;
        const double e = g.col_driven ? c : s;
        const double slope = -e * inv, c0_off = off_n * (e * inv + 1.0);
        g.slope = (T)slope;
        g.inv_drive = (T)inv;
        g.c0_off = (T)c0_off;
        g.inv_slope = slope == 0.0 ? (T)0 : (T)(1.0 / slope);
        g.c_d = c;
        g.s_d = s;
        g.inv_d = inv;
        g.c0_off_d = c0_off;
        g.slope_d = slope;
        const double two32 = 4294967296.0;
        g.c_fx = llrint(c * two32);
        g.s_fx = llrint(s * two32);
        g.inv_fx = llrint(inv * two32);
        g.c0_off_fx = llrint(c0_off * two32);
        g.slope_fx = llrint(slope * two32);
        out[a] = g;
    }
}

template <typename T>
Prob<T> make_prob(const scg_geometry& g, const Plan& pl, unsigned char* base) {
    Prob<T> P;
    memset(&P, 0, sizeof(P));
    P.n = g.n;
    P.na = g.n_angles;
    P.nb = g.n_bins;
    P.S = pl.S;
    P.SB = pl.SB;
    P.cnt_ray = pl.cnt_ray;
    P.cnt_img = pl.cnt_img;
    P.cnt_row = pl.cnt_row;
    P.tiles_x = pl.tiles_x;
    P.ray_blocks = pl.ray_blocks;
    P.filt_blocks = pl.filt_blocks;
    P.cnt_proj = pl.cnt_proj;
    P.proj_blocks = pl.proj_blocks;
    P.P = pl.P;
    P.off_n = (T)(0.5 * (g.n - 1));
    P.off_b = (T)(0.5 * (g.n_bins - 1));
    P.ang = reinterpret_cast<const Angle<T>*>(base + pl.ang);
    P.taps = reinterpret_cast<const T*>(base + pl.taps);
    for (int q = 0; q < IB_COUNT; ++q)
        P.img[q] = pl.img[q] == (size_t)-1 ? nullptr : reinterpret_cast<T*>(base + pl.img[q]);
    using T2 = typename Vec2<T>::type;
    for (int q = 0; q < SB_COUNT; ++q)
        P.sino[q] = pl.sino[q] == (size_t)-1 ? nullptr : reinterpret_cast<T2*>(base + pl.sino[q]);
    P.view_rm = reinterpret_cast<T2*>(base + pl.view_rm);
    P.view_cm = reinterpret_cast<T2*>(base + pl.view_cm);
    P.partials = reinterpret_cast<double*>(base + pl.partials);
    P.counter = reinterpret_cast<unsigned*>(base + pl.counter);
    P.st = reinterpret_cast<DevState*>(base + pl.state);
    P.trace = pl.trace == (size_t)-1 ? nullptr : reinterpret_cast<double*>(base + pl.trace);
    P.trace_rows = pl.trace == (size_t)-1 ? 0 : kMaxTraceRows;
    return P;
}

#define CK(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return SCG_ERR_CUDA; \
    } while (0)

// Kernel launch sequence helper for one problem.
// Kernel launch sequence helper: one problem (item lists null, blocks decode
// their item from blockIdx) or a batch (explicit item lists over problems).
template <typename T>
struct Runner {
    const Prob<T>* d;
    int g_ray, g_img, g_row, g_proj, nb;
    cudaStream_t s;
    int launches;
    const Item* i_ray = nullptr;
    const Item* i_img = nullptr;
    const Item* i_row = nullptr;
    const Item* i_proj = nullptr;
    void project(int dst, int mode, int step) { ++launches; launch_project<T>(d, i_proj, g_proj, dst, mode, step, s); }
    void back1(int src, int dst, int step) { ++launches; launch_backproject<T>(d, i_img, g_img, 1, src, src, dst, dst, step, s); }
    void back2(int s0, int s1, int d0, int d1, int step) { ++launches; launch_backproject<T>(d, i_img, g_img, 2, s0, s1, d0, d1, step, s); }
    void vec(int op, int sel, int step) { ++launches; launch_vec<T>(d, i_img, g_img, op, sel, step, s); }
    void tvgrad(int src, int fuse, int wg, int step) { ++launches; launch_tvgrad<T>(d, i_img, g_img, src, fuse, wg, step, s); }
    void trial() { ++launches; launch_trial<T>(d, i_img, g_img, s); }
    void axpy(int step) { ++launches; launch_sino_axpy<T>(d, i_ray, g_ray, step, s); }
    void filter(int src, int dst) { ++launches; launch_filter<T>(d, i_row, g_row, nb, src, dst, 0, s); }
};

struct Program {
    int variant, trial_passes, ksteps;
};

// The algorithms' set-up steps (before the first loop test).
template <typename T>
void run_init(Runner<T>& R, const Program& pg) {
    const int v = pg.variant, fam = family_of(v);
    const bool pre = uses_filter(v);
    const int dsel = pre ? IB_Z : IB_G;
    R.vec(VEC_INIT, 0, FIN_NONE);                      // x_{1/2} = x0 (S-CG family), x_{-1/2} = x0 (S-K)
    R.project(SB_R, PROJ_RESIDUAL, FIN_F);             // r = A x0 - y, f(x0)
    if (fam == FAM_S_K) {
        R.tvgrad(IB_X, 0, 1, FIN_END);                 // TV and dTV of x_0; first loop test
        return;
    }
    if (pre) R.filter(SB_R, SB_W);
    if (fam == FAM_CG) {
        if (pre) R.back2(SB_R, SB_W, IB_G, IB_Z, FIN_CG_DELTA);   // g0 = A^T r, z0 = M g0
        else R.back1(SB_R, IB_G, FIN_CG_DELTA);                    // g0 = A^T r
        R.vec(VEC_FORM_P0, dsel, FIN_CG_END);          // p0 = -g0 (-z0); first loop test
        return;
    }
    if (pre) R.back2(SB_R, SB_W, IB_G, IB_Z, FIN_BETA);
    else R.back1(SB_R, IB_G, FIN_BETA);                // g0 = A^T (A x0 - y)
    R.vec(VEC_FORM_P0, dsel, FIN_NUM);                 // p0 = -g0 (-z0), g0^T p0
    R.project(SB_Q, PROJ_PLAIN, FIN_NONE);             // A p0
    R.back1(SB_Q, IB_H, FIN_ALPHA);                    // h0 = A^T A p0, alpha
    R.tvgrad(IB_X, 1, 1, FIN_END);                     // x1 = x0 + alpha p0 (+ dTV(x1)); k = 1; loop test
}

// One loop body of the variant's while loop.
template <typename T>
void run_body(Runner<T>& R, const Program& pg) {
    const int v = pg.variant, fam = family_of(v);
    const bool pre = uses_filter(v);
    const int dsel = pre ? IB_Z : IB_G;
    if (fam == FAM_CG) {                               // CG-STEP / PCG-STEP
        R.project(SB_Q, PROJ_PLAIN, FIN_NONE);         // A p
        R.back1(SB_Q, IB_H, FIN_CG_ALPHA);             // h = A^T A p, alpha = delta / p^T h
        R.axpy(FIN_CG_F);                              // r' = r + alpha A p, f(x')
        if (pre) {
            R.filter(SB_R, SB_W);
            R.back1(SB_W, IB_Z, FIN_NONE);             // z' = M g'
        }
        R.vec(VEC_CG_UPDATE, IB_X, FIN_CG_BETA);       // x' = x + alpha p, g' = g + alpha h, beta
        R.vec(VEC_FORM_P, dsel, FIN_CG_END);           // p' = -g' (-z') + beta p; k = k+1; loop test
        return;
    }
    for (int t = 0; t < pg.trial_passes; ++t) R.trial();  // TV trials of x_k + gamma_l v
    R.vec(VEC_PERTURB, 0, FIN_NONE);                   // x_{k+1/2} = perturbed(x_k)
    R.project(SB_R, PROJ_RESIDUAL, FIN_F);             // A x_{k+1/2} - y, f(x_{k+1/2})
    if (pre) R.filter(SB_R, SB_W);
    if (fam == FAM_S_K) {                              // CG-K / PCG-K from x_{k+1/2}
        if (pre) R.back2(SB_R, SB_W, IB_G, IB_Z, FIN_CG_DELTA);
        else R.back1(SB_R, IB_G, FIN_CG_DELTA);
        R.vec(VEC_FORM_P0, dsel, FIN_NONE);
        for (int q = 0; q < pg.ksteps; ++q) {
            R.project(SB_Q, PROJ_PLAIN, FIN_NONE);
            R.back1(SB_Q, IB_H, FIN_CG_ALPHA);
            if (pre) {
                R.axpy(FIN_NONE);
                R.filter(SB_R, SB_W);
                R.back1(SB_W, IB_Z, FIN_NONE);
            }
            R.vec(VEC_CG_UPDATE, q == 0 ? IB_XH : IB_X, FIN_CG_BETA);
            if (q + 1 < pg.ksteps) R.vec(VEC_FORM_P, dsel, FIN_NONE);
        }
        R.tvgrad(IB_X, 0, 1, FIN_END);                 // dTV(x_{k+1}); k = k+1; loop test
        return;
    }
    // CG-PR-STEP / CG-CD-STEP / PCG-PR-STEP
    if (pre) R.back2(SB_R, SB_W, IB_G, IB_Z, FIN_BETA);   // g', z' = M g'
    else R.back1(SB_R, IB_G, FIN_BETA);                // g' = A^T (A x - y), beta
    R.vec(VEC_FORM_P, dsel, FIN_NUM);                  // p' = -g' (-z') + beta p, g'^T p'
    R.project(SB_Q, PROJ_PLAIN, FIN_NONE);             // A p'
    R.back1(SB_Q, IB_H, FIN_ALPHA);                    // h' = A^T A p', alpha
    R.tvgrad(IB_X, 1, 1, FIN_END);                     // x' = x + alpha p' (+ dTV); k = k+1; loop test
}

// Resume from an imported state: recompute f at the tested point, the dots
// the next step needs, and dTV(x_k); then take the loop test.
template <typename T>
void run_resume(Runner<T>& R, const Program& pg) {
    const int fam = family_of(pg.variant);
    if (fam == FAM_CG) {
        R.vec(VEC_VIEWS, IB_X, FIN_NONE);
        R.project(SB_R, PROJ_RESIDUAL, FIN_F);         // r_k = A x_k - y, f(x_k)
        R.vec(VEC_VIEWS, IB_P, FIN_CG_END);            // loop test
        return;
    }
    R.vec(VEC_VIEWS, IB_XH, FIN_NONE);
    R.project(SB_R, PROJ_RESIDUAL, FIN_F);             // f(x_{k-1/2})
    if (fam == FAM_S_PR) R.vec(VEC_DOTS_RESUME, 0, FIN_RESUME);   // p^T h, g^T p
    R.tvgrad(IB_X, 0, 1, FIN_END);                     // dTV(x_k); loop test
}

struct GraphKey {
    int dev;
    const void* work;
    int prec, variant, trial_passes, ksteps, n, na, nb, host_loop;
    bool operator<(const GraphKey& o) const {
        return std::tie(dev, work, prec, variant, trial_passes, ksteps, n, na, nb, host_loop) <
               std::tie(o.dev, o.work, o.prec, o.variant, o.trial_passes, o.ksteps, o.n, o.na, o.nb,
                        o.host_loop);
    }
};

struct BodyGraph {
    cudaGraphExec_t exec;
    int kernels;
    bool device_loop;    // whole while loop in one graph (conditional node)
};

std::mutex g_mu;
std::map<GraphKey, BodyGraph> g_graphs;
std::map<int, cudaStream_t> g_streams;
std::map<int, int*> g_pinned;

cudaError_t side_stream(int dev, cudaStream_t* out, int** pinned) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_streams.find(dev);
    if (it == g_streams.end()) {
        cudaStream_t s;
        cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        int* h = nullptr;
        e = cudaHostAlloc((void**)&h, 2 * sizeof(int), cudaHostAllocDefault);
        if (e != cudaSuccess) return e;
        g_streams[dev] = s;
        g_pinned[dev] = h;
        it = g_streams.find(dev);
    }
    *out = it->second;
    *pinned = g_pinned[dev];
    return cudaSuccess;
}

template <typename T>
int solve_impl(const scg_geometry* g, int variant, int precision, const scg_params* prm, double eps,
               const void* y, const void* x0, void* x_out, void* work, size_t work_bytes,
               scg_result* res, double* trace, int trace_rows, const scg_state* resume,
               scg_state* final_state, cudaStream_t user_stream) {
    const Plan pl = make_plan(*g, variant, sizeof(T), PLAN_SOLVE);
    if (work_bytes < pl.total || ((uintptr_t)work & 15u)) return SCG_ERR_WORKSPACE;
    unsigned char* base = (unsigned char*)work;
    const int N = g->n, fam = family_of(variant);
    const size_t J = (size_t)N * N;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    cudaStream_t s;
    int* pinned = nullptr;
    CK(side_stream(dev, &s, &pinned));
    // order the side stream after the caller's work
    cudaEvent_t ev;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CK(cudaEventRecord(ev, user_stream));
    CK(cudaStreamWaitEvent(s, ev, 0));

    Prob<T> P = make_prob<T>(*g, pl, base);
    P.y = (const T*)y;
    P.img[IB_AUX] = (T*)x0;
    std::vector<Angle<T>> ang;
    fill_angles<T>(ang, g->n_angles, g->n);

    DevState st;
    memset(&st, 0, sizeof(st));
    st.eps = eps;
    st.max_iter = prm->max_iter;
    st.perturb = prm->perturb;
    st.gamma0 = prm->gamma0 > 0.0 ? prm->gamma0 : 0.0;
    st.gamma_fixed = prm->gamma0 > 0.0 ? 1 : 0;
    st.gamma0_rel = prm->gamma0_rel;
    st.a = prm->a;
    st.max_trials = prm->max_trials;
    st.variant = variant;
    st.family = fam;
    st.in_init = 1;
    st.k = (fam == FAM_S_PR) ? 1 : 0;
    const bool resumed = resume && resume->valid == 1;
    if (resumed) {
        st.k = resume->k;
        st.ell = resume->ell;
        st.gamma0 = resume->gamma0;
        st.gamma_fixed = resume->gamma_fixed;
        st.delta = resume->delta;
    }

    CK(cudaMemsetAsync(base, 0, pl.total, s));
    CK(cudaMemcpyAsync(base + pl.state, &st, sizeof(st), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(base + pl.prob, &P, sizeof(P), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(base + pl.ang, ang.data(), sizeof(Angle<T>) * ang.size(), cudaMemcpyHostToDevice, s));
    if (uses_filter(variant)) {
        const double mu = prm->mu > 0.0 ? prm->mu : 2.0 * M_PI / pl.P;
        launch_taps<T>(reinterpret_cast<T*>(base + pl.taps), g->n_bins, pl.P, mu, prm->filter_gain, s);
        size_t smem = (size_t)(3 * g->n_bins) * sizeof(T);
        if (smem > 227 * 1024) return SCG_ERR_UNSUPPORTED;
    }
    Runner<T> R{reinterpret_cast<const Prob<T>*>(base + pl.prob), pl.cnt_ray, pl.cnt_img, pl.cnt_row,
                pl.cnt_proj, g->n_bins, s, 0};
    Program pg;
    pg.variant = variant;
    pg.trial_passes = prm->perturb == SCG_PERTURB_GAMMA ? (prm->max_trials + kTrials - 1) / kTrials : 0;
    pg.ksteps = prm->K + (prm->k_inclusive ? 1 : 0);

    if (resumed) {
        const size_t vb = sizeof(T) * J;
        if (resume->x) CK(cudaMemcpyAsync(P.img[IB_X], resume->x, vb, cudaMemcpyDeviceToDevice, s));
        if (resume->x_half && P.img[IB_XH]) CK(cudaMemcpyAsync(P.img[IB_XH], resume->x_half, vb, cudaMemcpyDeviceToDevice, s));
        if (resume->p) CK(cudaMemcpyAsync(P.img[IB_P], resume->p, vb, cudaMemcpyDeviceToDevice, s));
        if (resume->h) CK(cudaMemcpyAsync(P.img[IB_H], resume->h, vb, cudaMemcpyDeviceToDevice, s));
        if (resume->g) CK(cudaMemcpyAsync(P.img[IB_G], resume->g, vb, cudaMemcpyDeviceToDevice, s));
        run_resume<T>(R, pg);
    } else {
        run_init<T>(R, pg);
    }
    CK(cudaGetLastError());

    // The while loop.  Preferred: one CUDA graph holding the whole loop as a
    // conditional WHILE node whose condition a one-thread kernel sets on the
    // device after every body (no host round trip per iteration).  Fallback:
    // one graph per body, launched in batches and polled one batch ahead.
    GraphKey key{dev, work, precision, variant, pg.trial_passes, pg.ksteps, g->n, g->n_angles, g->n_bins,
                 prm->host_loop ? 1 : 0};
    BodyGraph bg{nullptr, 0, false};
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_graphs.find(key);
        if (it != g_graphs.end()) bg = it->second;
    }
    DevState* dst_mut = reinterpret_cast<DevState*>(base + pl.state);
    if (!bg.exec) {
        cudaStream_t cap;
        CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        Runner<T> RC = R;
        RC.s = cap;
        RC.launches = 0;
        // device loop
        cudaGraph_t g0 = nullptr;
        bool ok = !prm->host_loop && cudaGraphCreate(&g0, 0) == cudaSuccess;
        cudaGraphConditionalHandle h = 0;
        if (ok) ok = cudaGraphConditionalHandleCreate(&h, g0, 1, cudaGraphCondAssignDefault) == cudaSuccess;
        cudaGraph_t tmp = nullptr;
        if (ok) ok = cudaStreamBeginCaptureToGraph(cap, g0, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            launch_loop_cond(dst_mut, h, cap);
            ok = cudaStreamEndCapture(cap, &tmp) == cudaSuccess;
        }
        cudaGraphNode_t pre = nullptr;
        size_t nn = 1;
        if (ok) ok = cudaGraphGetNodes(g0, &pre, &nn) == cudaSuccess && nn == 1;
        alignas(cudaGraphNodeParams) unsigned char npbuf[sizeof(cudaGraphNodeParams)];
        memset(npbuf, 0, sizeof(npbuf));
        cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(npbuf);
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t wnode = nullptr;
        if (ok) ok = cudaGraphAddNode(&wnode, g0, &pre, nullptr, 1, &np) == cudaSuccess;
        if (ok) {
            cudaGraph_t body = np.conditional.phGraph_out[0];
            ok = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                run_body<T>(RC, pg);
                launch_loop_cond(dst_mut, h, cap);
                ok = cudaStreamEndCapture(cap, &tmp) == cudaSuccess;
            }
        }
        if (ok) ok = cudaGraphInstantiate(&bg.exec, g0, 0) == cudaSuccess;
        if (g0) cudaGraphDestroy(g0);
        if (ok) {
            bg.kernels = RC.launches;
            bg.device_loop = true;
        } else {
            cudaGetLastError();                     // clear, and fall back
            bg.exec = nullptr;
            RC.launches = 0;
            CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
            run_body<T>(RC, pg);
            cudaGraph_t graph;
            cudaError_t e = cudaStreamEndCapture(cap, &graph);
            if (e != cudaSuccess) { cudaStreamDestroy(cap); return SCG_ERR_CUDA; }
            e = cudaGraphInstantiate(&bg.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) { cudaStreamDestroy(cap); return SCG_ERR_CUDA; }
            bg.kernels = RC.launches;
            bg.device_loop = false;
        }
        cudaStreamDestroy(cap);
        std::lock_guard<std::mutex> lk(g_mu);
        g_graphs[key] = bg;
    }

    const DevState* dst = reinterpret_cast<const DevState*>(base + pl.state);
    const int max_bodies = prm->max_iter + 2;
    int launched = 0;
    if (bg.device_loop) {
        int mb[2] = {0, max_bodies};                // bodies, max_bodies
        CK(cudaMemcpyAsync(&dst_mut->bodies, mb, sizeof(mb), cudaMemcpyHostToDevice, s));
        CK(cudaGraphLaunch(bg.exec, s));
    } else {
        // loop bodies, polled one batch ahead
        int polled = 0;
        cudaEvent_t evs[2];
        CK(cudaEventCreateWithFlags(&evs[0], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&evs[1], cudaEventDisableTiming));
        int chunk = 2;
        bool finished = false;
        int pending = -1;
        while (!finished) {
            if (launched < max_bodies) {
                int cnt = chunk;
                if (launched + cnt > max_bodies) cnt = max_bodies - launched;
                for (int q = 0; q < cnt; ++q) CK(cudaGraphLaunch(bg.exec, s));
                launched += cnt;
                const int slot = polled & 1;
                CK(cudaMemcpyAsync(pinned + slot, &dst->done, sizeof(int), cudaMemcpyDeviceToHost, s));
                CK(cudaEventRecord(evs[slot], s));
                if (chunk < 8) chunk *= 2;
            }
            if (pending >= 0) {
                CK(cudaEventSynchronize(evs[pending & 1]));
                if (pinned[pending & 1]) finished = true;
            }
            pending = polled;
            ++polled;
            if (launched >= max_bodies && !finished) {
                CK(cudaEventSynchronize(evs[pending & 1]));
                finished = true;
            }
        }
        cudaEventDestroy(evs[0]);
        cudaEventDestroy(evs[1]);
    }
    const int body_kernels = bg.kernels;

    // output, f and TV of the output
    const int out_sel = fam == FAM_CG ? IB_X : IB_XH;
    CK(cudaMemcpyAsync(x_out, P.img[out_sel], sizeof(T) * J, cudaMemcpyDeviceToDevice, s));
    DevState* dstm = reinterpret_cast<DevState*>(base + pl.state);
    int zero = 0;
    CK(cudaMemcpyAsync(&dstm->done, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
    R.tvgrad(out_sel, 0, 0, FIN_FINAL_TV);
    if (fam == FAM_CG) {
        R.vec(VEC_VIEWS, IB_X, FIN_NONE);
        R.project(SB_Q, PROJ_RESIDUAL, FIN_FINAL_F);
    }
    CK(cudaGetLastError());
    DevState hs;
    CK(cudaMemcpyAsync(&hs, dstm, sizeof(hs), cudaMemcpyDeviceToHost, s));
    if (trace && trace_rows > 0) {
        int rows = trace_rows < kMaxTraceRows ? trace_rows : kMaxTraceRows;
        CK(cudaMemcpyAsync(trace, P.trace, sizeof(double) * TR_NF * rows, cudaMemcpyDeviceToHost, s));
    }
    if (final_state) {
        const size_t vb = sizeof(T) * J;
        if (final_state->x) CK(cudaMemcpyAsync(final_state->x, P.img[IB_X], vb, cudaMemcpyDeviceToDevice, s));
        if (final_state->x_half && P.img[IB_XH]) CK(cudaMemcpyAsync(final_state->x_half, P.img[IB_XH], vb, cudaMemcpyDeviceToDevice, s));
        if (final_state->p) CK(cudaMemcpyAsync(final_state->p, P.img[IB_P], vb, cudaMemcpyDeviceToDevice, s));
        if (final_state->h) CK(cudaMemcpyAsync(final_state->h, P.img[IB_H], vb, cudaMemcpyDeviceToDevice, s));
        if (final_state->g) CK(cudaMemcpyAsync(final_state->g, P.img[IB_G], vb, cudaMemcpyDeviceToDevice, s));
    }
    CK(cudaStreamSynchronize(s));
    // the caller's stream sees the outputs
    CK(cudaEventRecord(ev, s));
    CK(cudaStreamWaitEvent(user_stream, ev, 0));
    cudaEventDestroy(ev);

    res->iters = hs.iters;
    res->k_final = hs.k;
    res->status = hs.status;
    res->f_final = fam == FAM_CG ? hs.f_final : hs.f_half;
    res->tv_final = hs.tv_final;
    res->ell = hs.ell;
    res->gamma0_used = hs.gamma0;
    if (bg.device_loop) {
        res->body_launches = hs.bodies;
        res->kernel_launches = R.launches + 1 + hs.bodies * (body_kernels + 1);
    } else {
        res->body_launches = launched;
        res->kernel_launches = R.launches + launched * body_kernels;
    }
    res->device_loop = bg.device_loop ? 1 : 0;
    if (final_state) {
        final_state->valid = 1;
        final_state->k = hs.k;
        final_state->ell = hs.ell;
        final_state->gamma0 = hs.gamma0;
        final_state->gamma_fixed = hs.gamma_fixed;
        final_state->delta = hs.delta;
    }
    return hs.status;
}

// ---------------------------------------------------------------------------
// Operator entry points share this set-up.
template <typename T>
int op_setup(const scg_geometry& g, void* work, size_t work_bytes, cudaStream_t s, Plan* pl_out,
             Prob<T>* P_out) {
    const Plan pl = make_plan(g, SCG_S_CG, sizeof(T), PLAN_OP);
    if (work_bytes < pl.total || ((uintptr_t)work & 15u)) return SCG_ERR_WORKSPACE;
    unsigned char* base = (unsigned char*)work;
    Prob<T> P = make_prob<T>(g, pl, base);
    std::vector<Angle<T>> ang;
    fill_angles<T>(ang, g.n_angles, g.n);
    CK(cudaMemsetAsync(base + pl.state, 0, sizeof(DevState), s));
    CK(cudaMemsetAsync(base + pl.counter, 0, 16, s));
    CK(cudaMemcpyAsync(base + pl.ang, ang.data(), sizeof(Angle<T>) * ang.size(), cudaMemcpyHostToDevice, s));
    *pl_out = pl;
    *P_out = P;
    return SCG_OK;
}

template <typename T>
int upload_prob(const Prob<T>& P, const Plan& pl, void* work, cudaStream_t s) {
    CK(cudaMemcpyAsync((unsigned char*)work + pl.prob, &P, sizeof(P), cudaMemcpyHostToDevice, s));
    return SCG_OK;
}

template <typename T>
int project_impl(const scg_geometry& g, const void* x, void* y, void* work, size_t wb, cudaStream_t s) {
    Plan pl;
    Prob<T> P;
    int rc = op_setup<T>(g, work, wb, s, &pl, &P);
    if (rc) return rc;
    unsigned char* base = (unsigned char*)work;
    CK(cudaMemsetAsync(base + pl.view_rm, 0, 2 * sizeof(T) * (size_t)g.n * pl.S, s));
    CK(cudaMemsetAsync(base + pl.view_cm, 0, 2 * sizeof(T) * (size_t)g.n * pl.S, s));
    P.img[IB_AUX] = (T*)x;
    P.user_out = (T*)y;
    rc = upload_prob<T>(P, pl, work, s);
    if (rc) return rc;
    const Prob<T>* d = reinterpret_cast<const Prob<T>*>(base + pl.prob);
    launch_vec<T>(d, nullptr, pl.cnt_img, VEC_VIEWS, IB_AUX, FIN_NONE, s);
    launch_project<T>(d, nullptr, pl.cnt_proj, SB_Q, PROJ_PLAIN_OUT, FIN_NONE, s);
    CK(cudaGetLastError());
    return SCG_OK;
}

template <typename T>
int backproject_impl(const scg_geometry& g, const void* r, void* x, void* work, size_t wb, cudaStream_t s) {
    Plan pl;
    Prob<T> P;
    int rc = op_setup<T>(g, work, wb, s, &pl, &P);
    if (rc) return rc;
    unsigned char* base = (unsigned char*)work;
    CK(cudaMemsetAsync(base + pl.sino[SB_R], 0, 2 * sizeof(T) * (size_t)g.n_angles * pl.SB, s));
    P.img[IB_AUX] = (T*)x;
    P.user_in = (const T*)r;
    rc = upload_prob<T>(P, pl, work, s);
    if (rc) return rc;
    const Prob<T>* d = reinterpret_cast<const Prob<T>*>(base + pl.prob);
    launch_sino_pairs<T>(d, pl.cnt_ray, SB_R, s);
    launch_backproject<T>(d, nullptr, pl.cnt_img, 1, SB_R, SB_R, IB_AUX, IB_AUX, FIN_NONE, s);
    CK(cudaGetLastError());
    return SCG_OK;
}

template <typename T>
int tv_impl(int n, const void* x, void* grad, double* tv_out, void* work, size_t wb, cudaStream_t s) {
    scg_geometry g{n, 1, 1};
    Plan pl;
    Prob<T> P;
    int rc = op_setup<T>(g, work, wb, s, &pl, &P);
    if (rc) return rc;
    unsigned char* base = (unsigned char*)work;
    P.img[IB_AUX] = (T*)x;
    P.img[IB_TVG] = (T*)grad;
    P.trace = tv_out;
    P.trace_rows = 1;
    rc = upload_prob<T>(P, pl, work, s);
    if (rc) return rc;
    const Prob<T>* d = reinterpret_cast<const Prob<T>*>(base + pl.prob);
    launch_tvgrad<T>(d, nullptr, pl.cnt_img, IB_AUX, 0, grad ? 1 : 0, FIN_TV, s);
    CK(cudaGetLastError());
    return SCG_OK;
}

template <typename T>
int filter_impl(const scg_geometry& g, double mu, double gain, const void* r, void* out, void* work,
                size_t wb, cudaStream_t s) {
    Plan pl;
    Prob<T> P;
    int rc = op_setup<T>(g, work, wb, s, &pl, &P);
    if (rc) return rc;
    if ((size_t)(3 * g.n_bins) * sizeof(T) > 227 * 1024) return SCG_ERR_UNSUPPORTED;
    unsigned char* base = (unsigned char*)work;
    P.user_in = (const T*)r;
    P.user_out = (T*)out;
    rc = upload_prob<T>(P, pl, work, s);
    if (rc) return rc;
    const double mu_eff = mu > 0.0 ? mu : 2.0 * M_PI / pl.P;
    launch_taps<T>(reinterpret_cast<T*>(base + pl.taps), g.n_bins, pl.P, mu_eff, gain, s);
    const Prob<T>* d = reinterpret_cast<const Prob<T>*>(base + pl.prob);
    CK(launch_filter<T>(d, nullptr, pl.cnt_row, g.n_bins, SB_R, SB_W, 1, s));
    CK(cudaGetLastError());
    return SCG_OK;
}

// ---------------------------------------------------------------------------
// Batched solves.  Workspace: [BatchState][an always-stopped DevState][Prob x
// capacity][item lists for the projector, image-tile, sinogram-row and
// filter-row kinds][one single-solve region per problem].  Items carry
// (problem, u, v, local) with local the index the problem's own single-solve
// launch would give, so each problem's reductions add in exactly the order of
// a solve of that problem alone.
//
// The problem capacity and the item-list lengths are rounded up to a few
// steps per octave, and the padding items name a placeholder problem whose
// state is permanently stopped (its blocks return at once).  The captured loop
// graph then depends only on those rounded sizes, so batches of different
// geometry mixes reuse it.
enum { K_PROJ = 0, K_IMG = 1, K_RAY = 2, K_ROW = 3, K_COUNT = 4 };

int round_up_bucket(int n) {
    if (n <= 16) return n;
    int lg = 31 - __builtin_clz((unsigned)n);
    const int step = 1 << (lg - 3);                 // 8 steps per octave: <= 12.5 % padding
    return (n + step - 1) / step * step;
}

struct BatchPlan {
    size_t state, dummy, probs, items[K_COUNT];
    int n_items[K_COUNT], cap_items[K_COUNT];
    int cap_probs;
    std::vector<size_t> region;
    std::vector<Plan> plans;
    size_t total;
    int nb_cap;
};

BatchPlan make_batch_plan(const scg_problem* pr, int count, int variant, size_t tsize) {
    BatchPlan b;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, kAlign); return o; };
    b.state = take(sizeof(BatchState));
    b.dummy = take(sizeof(DevState));
    b.cap_probs = round_up_bucket(count + 1);
    b.probs = take(sizeof(Prob<double>) * (size_t)b.cap_probs);
    for (int k = 0; k < K_COUNT; ++k) b.n_items[k] = 0;
    int max_nb = 1;
    b.plans.resize(count);
    for (int i = 0; i < count; ++i) {
        b.plans[i] = make_plan(pr[i].geometry, variant, tsize, PLAN_SOLVE);
        b.n_items[K_PROJ] += b.plans[i].cnt_proj;
        b.n_items[K_IMG] += b.plans[i].cnt_img;
        b.n_items[K_RAY] += b.plans[i].cnt_ray;
        b.n_items[K_ROW] += b.plans[i].cnt_row;
        if (pr[i].geometry.n_bins > max_nb) max_nb = pr[i].geometry.n_bins;
    }
    b.nb_cap = (max_nb + 127) / 128 * 128;
    for (int k = 0; k < K_COUNT; ++k) {
        b.cap_items[k] = round_up_bucket(b.n_items[k]);
        b.items[k] = take(sizeof(Item) * (size_t)b.cap_items[k]);
    }
    b.region.resize(count);
    for (int i = 0; i < count; ++i) b.region[i] = take(b.plans[i].total);
    b.total = off;
    return b;
}

struct BatchKey {
    int dev;
    const void* work;
    int prec, variant, trial_passes, ksteps, cap_probs, nb_cap;
    int cap_items[K_COUNT];
    bool operator<(const BatchKey& o) const {
        return std::tie(dev, work, prec, variant, trial_passes, ksteps, cap_probs, nb_cap, cap_items[0],
                        cap_items[1], cap_items[2], cap_items[3]) <
               std::tie(o.dev, o.work, o.prec, o.variant, o.trial_passes, o.ksteps, o.cap_probs, o.nb_cap,
                        o.cap_items[0], o.cap_items[1], o.cap_items[2], o.cap_items[3]);
    }
};
std::map<BatchKey, BodyGraph> g_batch_graphs;

template <typename T>
int batch_impl(const scg_problem* pr, int count, int variant, int precision, const scg_params* prm,
               void* work, size_t work_bytes, scg_result* results, cudaStream_t user_stream) {
    const BatchPlan bp = make_batch_plan(pr, count, variant, sizeof(T));
    if (work_bytes < bp.total || ((uintptr_t)work & 15u)) return SCG_ERR_WORKSPACE;
    if (uses_filter(variant) && (size_t)(3 * bp.nb_cap) * sizeof(T) > 227 * 1024) return SCG_ERR_UNSUPPORTED;
    unsigned char* base = (unsigned char*)work;
    const int fam = family_of(variant);
    int dev = 0;
    CK(cudaGetDevice(&dev));
    cudaStream_t s;
    int* pinned = nullptr;
    CK(side_stream(dev, &s, &pinned));
    cudaEvent_t ev;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CK(cudaEventRecord(ev, user_stream));
    CK(cudaStreamWaitEvent(s, ev, 0));

    std::vector<Prob<T>> probs(bp.cap_probs);
    memset(probs.data(), 0, sizeof(Prob<T>) * probs.size());
    std::vector<std::vector<Item>> items(K_COUNT);
    for (int k = 0; k < K_COUNT; ++k) items[k].reserve(bp.cap_items[k]);
    CK(cudaMemsetAsync(base, 0, bp.total, s));
    for (int i = 0; i < count; ++i) {
        const Plan& pl = bp.plans[i];
        unsigned char* rb = base + bp.region[i];
        Prob<T> P = make_prob<T>(pr[i].geometry, pl, rb);
        P.y = (const T*)pr[i].y;
        P.img[IB_AUX] = (T*)pr[i].x0;
        probs[i] = P;
        for (int q = 0; q < pl.cnt_proj; ++q) items[K_PROJ].push_back(Item{i, q / pl.proj_blocks, q % pl.proj_blocks, q});
        for (int q = 0; q < pl.cnt_img; ++q) items[K_IMG].push_back(Item{i, q / pl.tiles_x, q % pl.tiles_x, q});
        for (int q = 0; q < pl.cnt_ray; ++q) items[K_RAY].push_back(Item{i, q / pl.ray_blocks, q % pl.ray_blocks, q});
        for (int q = 0; q < pl.cnt_row; ++q) items[K_ROW].push_back(Item{i, q / pl.filt_blocks, q % pl.filt_blocks, q});
        DevState st;
        memset(&st, 0, sizeof(st));
        st.eps = pr[i].eps;
        st.max_iter = prm->max_iter;
        st.perturb = prm->perturb;
        st.gamma0 = prm->gamma0 > 0.0 ? prm->gamma0 : 0.0;
        st.gamma_fixed = prm->gamma0 > 0.0 ? 1 : 0;
        st.gamma0_rel = prm->gamma0_rel;
        st.a = prm->a;
        st.max_trials = prm->max_trials;
        st.variant = variant;
        st.family = fam;
        st.in_init = 1;
        st.k = (fam == FAM_S_PR) ? 1 : 0;
        CK(cudaMemcpyAsync(rb + pl.state, &st, sizeof(st), cudaMemcpyHostToDevice, s));
        std::vector<Angle<T>> ang;
        fill_angles<T>(ang, pr[i].geometry.n_angles, pr[i].geometry.n);
        CK(cudaMemcpyAsync(rb + pl.ang, ang.data(), sizeof(Angle<T>) * ang.size(), cudaMemcpyHostToDevice, s));
        if (uses_filter(variant)) {
            const double mu = prm->mu > 0.0 ? prm->mu : 2.0 * M_PI / pl.P;
            launch_taps<T>(reinterpret_cast<T*>(rb + pl.taps), pr[i].geometry.n_bins, pl.P, mu, prm->filter_gain, s);
        }
        // (pageable host sources are staged before cudaMemcpyAsync returns,
        // so st and ang may be reused for the next problem)
    }
    // placeholder problem for the padding items: stopped for good
    DevState stopped;
    memset(&stopped, 0, sizeof(stopped));
    stopped.done = 1;
    CK(cudaMemcpyAsync(base + bp.dummy, &stopped, sizeof(stopped), cudaMemcpyHostToDevice, s));
    for (int i = count; i < bp.cap_probs; ++i) probs[i].st = reinterpret_cast<DevState*>(base + bp.dummy);
    for (int k = 0; k < K_COUNT; ++k)
        while ((int)items[k].size() < bp.cap_items[k]) items[k].push_back(Item{count, 0, 0, 0});
    BatchState bs{0, prm->max_iter + 2, count, 0};
    CK(cudaMemcpyAsync(base + bp.state, &bs, sizeof(bs), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(base + bp.probs, probs.data(), sizeof(Prob<T>) * bp.cap_probs, cudaMemcpyHostToDevice, s));
    for (int k = 0; k < K_COUNT; ++k)
        if (bp.cap_items[k])
            CK(cudaMemcpyAsync(base + bp.items[k], items[k].data(), sizeof(Item) * bp.cap_items[k],
                               cudaMemcpyHostToDevice, s));
    const Prob<T>* d = reinterpret_cast<const Prob<T>*>(base + bp.probs);
    Runner<T> R{d, bp.cap_items[K_RAY], bp.cap_items[K_IMG], bp.cap_items[K_ROW], bp.cap_items[K_PROJ],
                bp.nb_cap, s, 0};
    R.i_ray = reinterpret_cast<const Item*>(base + bp.items[K_RAY]);
    R.i_img = reinterpret_cast<const Item*>(base + bp.items[K_IMG]);
    R.i_row = reinterpret_cast<const Item*>(base + bp.items[K_ROW]);
    R.i_proj = reinterpret_cast<const Item*>(base + bp.items[K_PROJ]);
    Program pg;
    pg.variant = variant;
    pg.trial_passes = prm->perturb == SCG_PERTURB_GAMMA ? (prm->max_trials + kTrials - 1) / kTrials : 0;
    pg.ksteps = prm->K + (prm->k_inclusive ? 1 : 0);
    run_init<T>(R, pg);
    CK(cudaGetLastError());

    BatchState* bsd = reinterpret_cast<BatchState*>(base + bp.state);
    BatchKey key{dev, work, precision, variant, pg.trial_passes, pg.ksteps, bp.cap_probs, bp.nb_cap,
                 {bp.cap_items[0], bp.cap_items[1], bp.cap_items[2], bp.cap_items[3]}};
    BodyGraph bg{nullptr, 0, false};
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_batch_graphs.find(key);
        if (it != g_batch_graphs.end()) bg = it->second;
    }
    if (!bg.exec) {
        cudaStream_t cap;
        CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        Runner<T> RC = R;
        RC.s = cap;
        RC.launches = 0;
        cudaGraph_t g0 = nullptr;
        bool ok = cudaGraphCreate(&g0, 0) == cudaSuccess;
        cudaGraphConditionalHandle h = 0;
        if (ok) ok = cudaGraphConditionalHandleCreate(&h, g0, 1, cudaGraphCondAssignDefault) == cudaSuccess;
        cudaGraph_t tmp = nullptr;
        if (ok) ok = cudaStreamBeginCaptureToGraph(cap, g0, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            launch_loop_cond_batch<T>(d, bsd, h, cap);
            ok = cudaStreamEndCapture(cap, &tmp) == cudaSuccess;
        }
        cudaGraphNode_t pre = nullptr;
        size_t nn = 1;
        if (ok) ok = cudaGraphGetNodes(g0, &pre, &nn) == cudaSuccess && nn == 1;
        alignas(cudaGraphNodeParams) unsigned char npbuf[sizeof(cudaGraphNodeParams)];
        memset(npbuf, 0, sizeof(npbuf));
        cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(npbuf);
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t wnode = nullptr;
        if (ok) ok = cudaGraphAddNode(&wnode, g0, &pre, nullptr, 1, &np) == cudaSuccess;
        if (ok) {
            cudaGraph_t body = np.conditional.phGraph_out[0];
            ok = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                run_body<T>(RC, pg);
                launch_loop_cond_batch<T>(d, bsd, h, cap);
                ok = cudaStreamEndCapture(cap, &tmp) == cudaSuccess;
            }
        }
        if (ok) ok = cudaGraphInstantiate(&bg.exec, g0, 0) == cudaSuccess;
        if (g0) cudaGraphDestroy(g0);
        cudaStreamDestroy(cap);
        if (!ok) { cudaGetLastError(); return SCG_ERR_CUDA; }
        bg.kernels = RC.launches;
        bg.device_loop = true;
        std::lock_guard<std::mutex> lk(g_mu);
        g_batch_graphs[key] = bg;
    }
    CK(cudaGraphLaunch(bg.exec, s));

    // outputs, f and TV of every output
    const int out_sel = fam == FAM_CG ? IB_X : IB_XH;
    for (int i = 0; i < count; ++i) {
        const size_t J = (size_t)pr[i].geometry.n * pr[i].geometry.n;
        CK(cudaMemcpyAsync(pr[i].x_out, probs[i].img[out_sel], sizeof(T) * J, cudaMemcpyDeviceToDevice, s));
    }
    launch_set_done<T>(d, count, 0, s);
    R.tvgrad(out_sel, 0, 0, FIN_FINAL_TV);
    if (fam == FAM_CG) {
        R.vec(VEC_VIEWS, IB_X, FIN_NONE);
        R.project(SB_Q, PROJ_RESIDUAL, FIN_FINAL_F);
    }
    CK(cudaGetLastError());
    std::vector<DevState> hs(count);
    for (int i = 0; i < count; ++i)
        CK(cudaMemcpyAsync(&hs[i], base + bp.region[i] + bp.plans[i].state, sizeof(DevState),
                           cudaMemcpyDeviceToHost, s));
    BatchState hb;
    CK(cudaMemcpyAsync(&hb, bsd, sizeof(hb), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaEventRecord(ev, s));
    CK(cudaStreamWaitEvent(user_stream, ev, 0));
    cudaEventDestroy(ev);

    int rc = SCG_OK;
    const int launches = R.launches + 1 + hb.bodies * (bg.kernels + 1);
    for (int i = 0; i < count; ++i) {
        scg_result& r = results[i];
        memset(&r, 0, sizeof(r));
        r.iters = hs[i].iters;
        r.k_final = hs[i].k;
        r.status = hs[i].status;
        r.f_final = fam == FAM_CG ? hs[i].f_final : hs[i].f_half;
        r.tv_final = hs[i].tv_final;
        r.ell = hs[i].ell;
        r.gamma0_used = hs[i].gamma0;
        r.body_launches = hb.bodies;
        r.kernel_launches = launches;
        r.device_loop = 1;
        if (rc == SCG_OK && r.status != SCG_OK) rc = r.status;
    }
    return rc;
}

bool valid_prec(int p) { return p == SCG_F32 || p == SCG_F64; }
size_t tsize_of(int p) { return p == SCG_F64 ? sizeof(double) : sizeof(float); }

}  // namespace

extern "C" {

const char* scg_strerror(int status) {
    switch (status) {
    case SCG_OK: return "ok";
    case SCG_WARN_MAX_ITER: return "stopped at max_iter with f > eps";
    case SCG_ERR_INVALID: return "invalid argument";
    case SCG_ERR_CUDA: return "CUDA runtime error";
    case SCG_ERR_WORKSPACE: return "workspace too small or not 16-byte aligned";
    case SCG_ERR_BREAKDOWN: return "zero or non-finite CG denominator";
    case SCG_ERR_UNSUPPORTED: return "unsupported precision/variant/size";
    default: return "unknown status";
    }
}

void scg_default_params(scg_params* p) {
    if (!p) return;
    p->perturb = SCG_PERTURB_GAMMA;
    p->gamma0 = 0.0;
    p->gamma0_rel = 0.05;
    p->a = 0.975;
    p->max_trials = 31;
    p->K = 2;
    p->k_inclusive = 0;
    p->mu = 0.0;
    p->filter_gain = 1.0;
    p->max_iter = 100;
    p->host_loop = 0;
}

size_t scg_op_workspace_bytes(const scg_geometry* g, int precision) {
    if (!valid_geometry(g) || !valid_prec(precision)) return 0;
    return make_plan(*g, SCG_S_CG, tsize_of(precision), PLAN_OP).total;
}

size_t scg_solve_workspace_bytes(const scg_geometry* g, int variant, int precision) {
    if (!valid_geometry(g) || !valid_prec(precision) || variant < SCG_CG || variant > SCG_S_PCG_K)
        return 0;
    return make_plan(*g, variant, tsize_of(precision), PLAN_SOLVE).total;
}

int scg_project(const scg_geometry* g, int precision, const void* x, void* y, void* work,
                size_t work_bytes, void* stream) {
    if (!valid_geometry(g) || !x || !y || !work) return SCG_ERR_INVALID;
    if (!valid_prec(precision)) return SCG_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    return precision == SCG_F64 ? project_impl<double>(*g, x, y, work, work_bytes, s)
                                : project_impl<float>(*g, x, y, work, work_bytes, s);
}

int scg_backproject(const scg_geometry* g, int precision, const void* r, void* x, void* work,
                    size_t work_bytes, void* stream) {
    if (!valid_geometry(g) || !x || !r || !work) return SCG_ERR_INVALID;
    if (!valid_prec(precision)) return SCG_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    return precision == SCG_F64 ? backproject_impl<double>(*g, r, x, work, work_bytes, s)
                                : backproject_impl<float>(*g, r, x, work, work_bytes, s);
}

int scg_tv(int n, int precision, const void* x, double* tv_out, void* work, size_t work_bytes,
           void* stream) {
    if (n < 2 || n > 8192 || !x || !tv_out || !work) return SCG_ERR_INVALID;
    if (!valid_prec(precision)) return SCG_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    return precision == SCG_F64 ? tv_impl<double>(n, x, nullptr, tv_out, work, work_bytes, s)
                                : tv_impl<float>(n, x, nullptr, tv_out, work, work_bytes, s);
}

int scg_tv_grad(int n, int precision, const void* x, void* grad, double* tv_out, void* work,
                size_t work_bytes, void* stream) {
    if (n < 2 || n > 8192 || !x || !grad || !tv_out || !work) return SCG_ERR_INVALID;
    if (!valid_prec(precision)) return SCG_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    return precision == SCG_F64 ? tv_impl<double>(n, x, grad, tv_out, work, work_bytes, s)
                                : tv_impl<float>(n, x, grad, tv_out, work, work_bytes, s);
}

int scg_filter(const scg_geometry* g, int precision, double mu, double gain, const void* r, void* out,
               void* work, size_t work_bytes, void* stream) {
    if (!valid_geometry(g) || !r || !out || !work) return SCG_ERR_INVALID;
    if (!valid_prec(precision)) return SCG_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    return precision == SCG_F64 ? filter_impl<double>(*g, mu, gain, r, out, work, work_bytes, s)
                                : filter_impl<float>(*g, mu, gain, r, out, work, work_bytes, s);
}

int scg_solve(const scg_geometry* g, int variant, int precision, const scg_params* prm, double eps,
              const void* y, const void* x0, void* x_out, void* work, size_t work_bytes,
              scg_result* res, double* trace, int trace_rows, const scg_state* resume,
              scg_state* final_state, void* stream) {
    if (!valid_geometry(g) || !prm || !y || !x_out || !work || !res) return SCG_ERR_INVALID;
    if (variant < SCG_CG || variant > SCG_S_PCG_K) return SCG_ERR_INVALID;
    if (!(eps > 0.0) || !isfinite(eps) || prm->max_iter < 0 || prm->max_iter > 10000000 ||
        prm->max_trials < 1 || prm->max_trials > 100000 || prm->K < 1 || prm->K > 1000 ||
        !(prm->a > 0.0 && prm->a < 1.0) || !(prm->filter_gain > 0.0))
        return SCG_ERR_INVALID;
    if (prm->perturb != SCG_PERTURB_NONE && prm->perturb != SCG_PERTURB_GAMMA) return SCG_ERR_INVALID;
    if (prm->host_loop != 0 && prm->host_loop != 1) return SCG_ERR_INVALID;
    if (resume && resume->valid != 1) return SCG_ERR_INVALID;
    if (!valid_prec(precision)) return SCG_ERR_UNSUPPORTED;
    memset(res, 0, sizeof(*res));
    cudaStream_t s = (cudaStream_t)stream;
    int rc = precision == SCG_F64
                 ? solve_impl<double>(g, variant, precision, prm, eps, y, x0, x_out, work, work_bytes,
                                      res, trace, trace_rows, resume, final_state, s)
                 : solve_impl<float>(g, variant, precision, prm, eps, y, x0, x_out, work, work_bytes,
                                     res, trace, trace_rows, resume, final_state, s);
    if (rc < 0 && rc != SCG_ERR_BREAKDOWN) res->status = rc;
    return rc;
}

size_t scg_batch_workspace_bytes(const scg_problem* problems, int count, int variant, int precision) {
    if (!problems || count < 1 || count > 65536 || !valid_prec(precision) || variant < SCG_CG ||
        variant > SCG_S_PCG_K)
        return 0;
    for (int i = 0; i < count; ++i)
        if (!valid_geometry(&problems[i].geometry)) return 0;
    return make_batch_plan(problems, count, variant, tsize_of(precision)).total;
}

int scg_solve_batch(const scg_problem* problems, int count, int variant, int precision,
                    const scg_params* prm, void* work, size_t work_bytes, scg_result* results,
                    void* stream) {
    if (!problems || count < 1 || count > 65536 || !prm || !work || !results) return SCG_ERR_INVALID;
    if (variant < SCG_CG || variant > SCG_S_PCG_K) return SCG_ERR_INVALID;
    if (prm->max_iter < 0 || prm->max_iter > 10000000 || prm->max_trials < 1 || prm->max_trials > 100000 ||
        prm->K < 1 || prm->K > 1000 || !(prm->a > 0.0 && prm->a < 1.0) || !(prm->filter_gain > 0.0))
        return SCG_ERR_INVALID;
    if (prm->perturb != SCG_PERTURB_NONE && prm->perturb != SCG_PERTURB_GAMMA) return SCG_ERR_INVALID;
    if (prm->host_loop != 0) return SCG_ERR_UNSUPPORTED;
    for (int i = 0; i < count; ++i) {
        const scg_problem& p = problems[i];
        if (!valid_geometry(&p.geometry) || !p.y || !p.x_out || !(p.eps > 0.0) || !isfinite(p.eps))
            return SCG_ERR_INVALID;
    }
    if (!valid_prec(precision)) return SCG_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = precision == SCG_F64
                 ? batch_impl<double>(problems, count, variant, precision, prm, work, work_bytes, results, s)
                 : batch_impl<float>(problems, count, variant, precision, prm, work, work_bytes, results, s);
    if (rc < 0 && rc != SCG_ERR_BREAKDOWN)
        for (int i = 0; i < count; ++i) results[i].status = rc;
    return rc;
}

}  // extern "C"
