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
#include <atomic>
#include <mutex>
#include <tuple>
#include <vector>

#include "host_programs.h"

using namespace scg;
using namespace scg::host;

namespace {

struct GraphKey {
    int dev;
    const void* work;
    int prec, variant, trial_passes, ksteps, n, na, nb, host_loop, proj_shift, eta, prox_iters, pert_steps, prox;
    bool operator<(const GraphKey& o) const {
        return std::tie(dev, work, prec, variant, trial_passes, ksteps, n, na, nb, host_loop, proj_shift, eta,
                        prox_iters, pert_steps, prox) <
               std::tie(o.dev, o.work, o.prec, o.variant, o.trial_passes, o.ksteps, o.n, o.na, o.nb,
                        o.host_loop, o.proj_shift, o.eta, o.prox_iters, o.pert_steps, o.prox);
    }
};

struct BodyGraph {
    cudaGraphExec_t exec;
    int kernels;
    bool device_loop;    // whole while loop in one graph (conditional node)
};

std::mutex g_mu;
std::map<GraphKey, BodyGraph> g_graphs;

struct ShapeKey {
    int dev, prec, bn, ba, bb;
    bool operator<(const ShapeKey& o) const {
        return std::tie(dev, prec, bn, ba, bb) < std::tie(o.dev, o.prec, o.bn, o.ba, o.bb);
    }
};
std::mutex g_shape_mu;
std::map<ShapeKey, int> g_shapes;
ShapeKey shape_key(int dev, int precision, const scg_geometry& g) {
    auto bucket = [](int v) { return (int)lround(2.0 * log2((double)v)); };
    return ShapeKey{dev, precision, bucket(g.n), bucket(g.n_angles), bucket(g.n_bins)};
}
// Projector work lists (longest blocks first), per exact geometry, shape and
// angle block
struct OrderKey {
    int n, na, nb, shift, a_begin, na_total;
    bool operator<(const OrderKey& o) const {
        return std::tie(n, na, nb, shift, a_begin, na_total) < std::tie(o.n, o.na, o.nb, o.shift, o.a_begin, o.na_total);
    }
};
std::mutex g_order_mu;
std::map<OrderKey, std::shared_ptr<const ProjOrder>> g_orders;
// FISTA's c^2 estimates, per device, precision and exact geometry
std::map<std::tuple<int, int, int, int, int>, double> g_lipschitz;
constexpr int kPowerIters = 100;
double lipschitz_lookup(int dev, int precision, const scg_geometry& g) {
    std::lock_guard<std::mutex> lk(g_shape_mu);
    auto it = g_lipschitz.find(std::make_tuple(dev, precision, g.n, g.n_angles, g.n_bins));
    return it == g_lipschitz.end() ? 0.0 : it->second;
}
void lipschitz_store(int dev, int precision, const scg_geometry& g, double c2) {
    std::lock_guard<std::mutex> lk(g_shape_mu);
    g_lipschitz[std::make_tuple(dev, precision, g.n, g.n_angles, g.n_bins)] = c2;
}
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
               scg_state* final_state, cudaStream_t user_stream, scg_result* res_async = nullptr) {
    using E = typename Tr<T>::S;
    using C = typename Tr<T>::C;
    Plan pl = make_plan(*g, variant, prec_of<T>(), PLAN_SOLVE, prm->perturb == SCG_PERTURB_PROX);
    if (work_bytes < pl.total || ((uintptr_t)work & 15u)) return SCG_ERR_WORKSPACE;
    if (uses_filter(variant) && !filter_fits(g->n_bins, prec_of<T>())) return SCG_ERR_UNSUPPORTED;
    unsigned char* base = (unsigned char*)work;
    const int N = g->n, fam = family_of(variant);
    const double scale = system_scale(*g, prec_of<T>()), s2 = scale * scale;
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

    Prob<T> P = make_prob<T>(*g, pl, base, scale);
    P.y = (const E*)y;
    P.img[IB_AUX] = (E*)x0;
    if (fam == FAM_FISTA) P.user_out = (E*)x_out;        // written by the output pass
    std::vector<Angle<C>> ang;
    fill_angles<C>(ang, g->n_angles, g->n, scale);

    DevState st = initial_state(prm, eps * s2, variant);
    // FISTA's c^2: given, cached for this geometry, or estimated below
    bool need_power = false;
    if (fam == FAM_FISTA && !(prm->lipschitz > 0.0)) {
        const double c2 = lipschitz_lookup(dev, prec_of<T>(), *g);
        if (c2 > 0.0) st.ex.c2 = c2;
        else need_power = true;
    }
    const bool resumed = resume && resume->valid == 1;
    if (resumed) {
        st.k = resume->k;
        st.ell = resume->ell;
        st.a_ell = pow(prm->a, (double)resume->ell);
        st.gamma0 = resume->gamma0;
        st.gamma_fixed = resume->gamma_fixed;
        st.delta = resume->delta;
    }

    CK(cudaMemsetAsync(base, 0, pl.total, s));
    {
        const int rc = upload_sino_maps<T>(P, pl, base, s);
        if (rc != SCG_OK) return rc;
    }
    CK(cudaMemcpyAsync(base + pl.state, &st, sizeof(st), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(base + pl.prob, &P, sizeof(P), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(base + pl.ang, ang.data(), sizeof(Angle<C>) * ang.size(), cudaMemcpyHostToDevice, s));
    std::vector<C> ftab;
    if (uses_filter(variant)) {
        const double mu = prm->mu > 0.0 ? prm->mu : 2.0 * M_PI / pl.P;
        fill_filter_tables<C>(ftab, pl.P, mu, prm->filter_gain);
        CK(cudaMemcpyAsync(base + pl.taps, ftab.data(), sizeof(C) * ftab.size(), cudaMemcpyHostToDevice, s));
    }
    {
        const int rc = tune_proj_shape<T>(P, pl, reinterpret_cast<Prob<T>*>(base + pl.prob), *g, s,
                                          reinterpret_cast<Item*>(base + pl.proj_items), prm->proj_shape);
        if (rc != SCG_OK) return rc;
    }
    Runner<T> R{reinterpret_cast<const Prob<T>*>(base + pl.prob), pl.cnt_ray, pl.cnt_img, pl.cnt_row,
                pl.cnt_proj, g->n_bins, s, 0};
    R.g_bp = pl.cnt_bp;
    R.i_proj = reinterpret_cast<const Item*>(base + pl.proj_items);   // longest first
    const Program pg = make_program(prm, variant);

    if (resumed) {
        const size_t vb = sizeof(E) * J;
        if (resume->x) CK(cudaMemcpyAsync(P.img[IB_X], resume->x, vb, cudaMemcpyDeviceToDevice, s));
        if (resume->x_half && P.img[IB_XH]) CK(cudaMemcpyAsync(P.img[IB_XH], resume->x_half, vb, cudaMemcpyDeviceToDevice, s));
        if (resume->p) CK(cudaMemcpyAsync(P.img[IB_P], resume->p, vb, cudaMemcpyDeviceToDevice, s));
        if (resume->h) CK(cudaMemcpyAsync(P.img[IB_H], resume->h, vb, cudaMemcpyDeviceToDevice, s));
        if (resume->g) CK(cudaMemcpyAsync(P.img[IB_G], resume->g, vb, cudaMemcpyDeviceToDevice, s));
        run_resume<T>(R, pg);
    } else {
        if (need_power) run_power<T>(R, kPowerIters);
        run_init<T>(R, pg);
    }
    CK(cudaGetLastError());

    // The while loop.  Preferred: one CUDA graph holding the whole loop as a
    // conditional WHILE node whose condition a one-thread kernel sets on the
    // device after every body (no host round trip per iteration).  Fallback:
    // one graph per body, launched in batches and polled one batch ahead.
    GraphKey key{dev, work, precision, variant, pg.trial_passes, pg.ksteps, g->n, g->n_angles, g->n_bins,
                 prm->host_loop ? 1 : 0, pl.proj_shift, pg.eta ? 1 : 0, pg.prox_iters, pg.pert_steps,
                 pg.prox ? 1 : 0};
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
    // (a FISTA body holds three iterations)
    const int max_bodies = (fam == FAM_FISTA ? prm->max_iter / 3 : prm->max_iter) + 2;
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
    const int out_sel = fam == FAM_CG ? IB_X : fam == FAM_FISTA ? IB_Z : IB_XH;
    if (fam != FAM_FISTA) CK(cudaMemcpyAsync(x_out, P.img[out_sel], sizeof(E) * J, cudaMemcpyDeviceToDevice, s));
    DevState* dstm = reinterpret_cast<DevState*>(base + pl.state);
    int zero = 0;
    CK(cudaMemcpyAsync(&dstm->done, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
    if (fam == FAM_FISTA) R.vec(VEC_FISTA_OUT, 0, FIN_NONE);   // x_k of the device's k, to Z and x_out
    R.tvgrad(out_sel, 0, 0, FIN_FINAL_TV);
    if (fam == FAM_CG) {
        R.vec(VEC_VIEWS, IB_X, FIN_NONE);
        R.project(SB_Q, PROJ_RESIDUAL, FIN_FINAL_F);
    }
    CK(cudaGetLastError());
    if (res_async) {
        // stream-ordered: the device writes the result when it gets there
        launch_write_result(dstm, res_async, s2, fam == FAM_CG ? 1 : 0, R.launches + 1, body_kernels, s);
        CK(cudaGetLastError());
        CK(cudaEventRecord(ev, s));
        CK(cudaStreamWaitEvent(user_stream, ev, 0));
        cudaEventDestroy(ev);
        return SCG_OK;
    }
    DevState hs;
    CK(cudaMemcpyAsync(&hs, dstm, sizeof(hs), cudaMemcpyDeviceToHost, s));
    if (trace && trace_rows > 0) {
        int rows = trace_rows < kMaxTraceRows ? trace_rows : kMaxTraceRows;
        CK(cudaMemcpyAsync(trace, P.trace, sizeof(double) * TR_NF * rows, cudaMemcpyDeviceToHost, s));
    }
    if (final_state) {
        const size_t vb = sizeof(E) * J;
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

    if (trace && trace_rows > 0 && scale != 1.0) {   // f and alpha back to the unscaled system
        const int rows = trace_rows < kMaxTraceRows ? trace_rows : kMaxTraceRows;
        for (int r = 0; r < rows; ++r) {
            trace[r * TR_NF + TR_FTEST] /= s2;
            trace[r * TR_NF + TR_F_AFTER] /= s2;
            trace[r * TR_NF + TR_ALPHA] *= s2;
        }
    }
    res->iters = hs.iters;
    res->k_final = hs.k;
    const int status = hs.dev_error ? SCG_ERR_CUDA : hs.status;   // dev_error: a device-side wait ran out
    res->status = status;
    res->f_final = (fam == FAM_CG ? hs.f_final : hs.f_half) / s2;
    res->tv_final = hs.tv_final;
    res->ell = hs.ell;
    res->gamma0_used = hs.gamma0;
    res->lipschitz_used = fam == FAM_FISTA ? hs.ex.c2 : 0.0;
    if (need_power && hs.ex.c2 > 0.0) lipschitz_store(dev, prec_of<T>(), *g, hs.ex.c2);
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
    return status;
}

// ---------------------------------------------------------------------------
// Operator entry points share this set-up.
// `g` is the geometry the operator applies (for an angle block: n_angles =
// the block's angles), angle a of it is angle a_begin + a of a scan of
// na_total angles.
template <typename T>
int op_setup(const scg_geometry& g, void* work, size_t work_bytes, cudaStream_t s, Plan* pl_out,
             Prob<T>* P_out, int a_begin = 0, int na_total = -1) {
    using C = typename Tr<T>::C;
    Plan pl = make_plan(g, SCG_S_CG, prec_of<T>(), PLAN_OP);
    if (work_bytes < pl.total || ((uintptr_t)work & 15u)) return SCG_ERR_WORKSPACE;
    if (a_begin != 0 || (na_total >= 0 && na_total != g.n_angles)) pl.bp_mirror = 0;   // an angle block
    unsigned char* base = (unsigned char*)work;
    Prob<T> P = make_prob<T>(g, pl, base);
    std::vector<Angle<C>> ang;
    fill_angles<C>(ang, g.n_angles, g.n, 1.0, a_begin, na_total);
    {
        const int rc = upload_sino_maps<T>(P, pl, base, s);
        if (rc != SCG_OK) return rc;
    }
    CK(cudaMemsetAsync(base + pl.state, 0, sizeof(DevState), s));
    CK(cudaMemsetAsync(base + pl.counter, 0, 16, s));
    CK(cudaMemcpyAsync(base + pl.ang, ang.data(), sizeof(Angle<C>) * ang.size(), cudaMemcpyHostToDevice, s));
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
    using E = typename Tr<T>::S;
    CK(cudaMemsetAsync(base + pl.view_rm, 0, 2 * sizeof(E) * (size_t)g.n * pl.S, s));
    CK(cudaMemsetAsync(base + pl.view_cm, 0, 2 * sizeof(E) * (size_t)g.n * pl.S, s));
    P.img[IB_AUX] = (E*)x;
    P.user_out = (E*)y;
    rc = upload_prob<T>(P, pl, work, s);
    if (rc) return rc;
    const Prob<T>* d = reinterpret_cast<const Prob<T>*>(base + pl.prob);
    rc = upload_proj_order(pl, base + pl.proj_items, g, s);
    if (rc) return rc;
    launch_vec<T>(d, nullptr, pl.cnt_img, VEC_VIEWS, IB_AUX, FIN_NONE, s);
    launch_project<T>(d, reinterpret_cast<const Item*>(base + pl.proj_items), pl.cnt_proj, SB_Q, PROJ_PLAIN_OUT,
                      FIN_NONE, s);
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
    using E = typename Tr<T>::S;
    CK(cudaMemsetAsync(base + pl.sino[SB_R], 0, 2 * sizeof(E) * (size_t)g.n_angles * pl.SB, s));
    P.img[IB_AUX] = (E*)x;
    P.user_in = (const E*)r;
    rc = upload_prob<T>(P, pl, work, s);
    if (rc) return rc;
    const Prob<T>* d = reinterpret_cast<const Prob<T>*>(base + pl.prob);
    launch_sino_pairs<T>(d, pl.cnt_ray, SB_R, s);
    launch_backproject<T>(d, nullptr, pl.cnt_bp, 1, SB_R, SB_R, IB_AUX, IB_AUX, FIN_NONE, s);
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
    using E = typename Tr<T>::S;
    P.img[IB_AUX] = (E*)x;
    P.img[IB_TVG] = (E*)grad;
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
    using E = typename Tr<T>::S;
    using C = typename Tr<T>::C;
    unsigned char* base = (unsigned char*)work;
    P.user_in = (const E*)r;
    P.user_out = (E*)out;
    rc = upload_prob<T>(P, pl, work, s);
    if (rc) return rc;
    const double mu_eff = mu > 0.0 ? mu : 2.0 * M_PI / pl.P;
    std::vector<C> ftab;
    fill_filter_tables<C>(ftab, pl.P, mu_eff, gain);
    CK(cudaMemcpyAsync(base + pl.taps, ftab.data(), sizeof(C) * ftab.size(), cudaMemcpyHostToDevice, s));
    const Prob<T>* d = reinterpret_cast<const Prob<T>*>(base + pl.prob);
    CK(launch_filter<T>(d, nullptr, pl.cnt_row, g.n_bins, SB_R, SB_W, FILT_PLAIN, s));
    CK(cudaGetLastError());
    return SCG_OK;
}

// Filtered backprojection: the rows filtered with the Hamming-windowed ramp
// (mu = 0, gain 1/(2 n_angles): the angle step pi/n_angles over the 2 pi that
// turns the radian factors into the ramp |nu|), written into the pair view the
// gather reads, then A^T.
template <typename T>
int fbp_impl(const scg_geometry& g, const void* y, void* x, void* work, size_t wb, cudaStream_t s) {
    if (!filter_fits(g.n_bins, prec_of<T>())) return SCG_ERR_UNSUPPORTED;
    Plan pl;
    Prob<T> P;
    int rc = op_setup<T>(g, work, wb, s, &pl, &P);
    if (rc) return rc;
    unsigned char* base = (unsigned char*)work;
    using E = typename Tr<T>::S;
    using C = typename Tr<T>::C;
    CK(cudaMemsetAsync(base + pl.sino[SB_R], 0, 2 * sizeof(E) * (size_t)g.n_angles * pl.SB, s));
    P.img[IB_AUX] = (E*)x;
    P.user_in = (const E*)y;
    rc = upload_prob<T>(P, pl, work, s);
    if (rc) return rc;
    std::vector<C> ftab;
    fill_filter_tables<C>(ftab, pl.P, 0.0, 1.0 / (2.0 * (double)g.n_angles));
    CK(cudaMemcpyAsync(base + pl.taps, ftab.data(), sizeof(C) * ftab.size(), cudaMemcpyHostToDevice, s));
    const Prob<T>* d = reinterpret_cast<const Prob<T>*>(base + pl.prob);
    CK(launch_filter<T>(d, nullptr, pl.cnt_row, g.n_bins, SB_R, SB_R, FILT_FBP, s));
    launch_backproject<T>(d, nullptr, pl.cnt_bp, 1, SB_R, SB_R, IB_AUX, IB_AUX, FIN_NONE, s);
    CK(cudaGetLastError());
    return SCG_OK;
}

// ---------------------------------------------------------------------------
// Prepared operator pair: set up once, then each application is device work
// only (descriptor update by a one-thread kernel, view or pair-row pass, and
// the projector or backprojector).
// With timing on, each application records CUDA events on its stream around
// the projector (or gather) kernel alone -- not while the stream is being
// captured into a graph -- so that scg_operator_kernel_ms can report that
// kernel's device time.  Off by default: the two records cost about 4 us of
// device time per application.
struct OperatorBase {
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};   // project start/end, backproject start/end
    bool timed[2] = {false, false};
    bool timing = false;
    virtual ~OperatorBase() {
        for (auto e : ev)
            if (e) cudaEventDestroy(e);
    }
    int make_events() {
        for (auto& e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) return SCG_ERR_CUDA;
        return SCG_OK;
    }
    // record event i on s unless s is capturing; returns whether it was recorded
    bool mark(int i, cudaStream_t s) {
        if (!timing) return false;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return false;
        return cudaEventRecord(ev[i], s) == cudaSuccess;
    }
    virtual int project(const void* x, void* y, cudaStream_t s) = 0;
    virtual int backproject(const void* r, void* x, cudaStream_t s) = 0;
};

template <typename T>
struct Operator final : OperatorBase {
    using E = typename Tr<T>::S;
    scg_geometry g;
    Plan pl;
    Prob<T>* d = nullptr;
    const Item* order = nullptr;       // projector blocks, longest first

    int init(const scg_geometry& geo, void* work, size_t wb, cudaStream_t s, int a_begin = 0, int na_total = -1) {
        g = geo;
        Prob<T> P;
        int rc = op_setup<T>(g, work, wb, s, &pl, &P, a_begin, na_total);
        if (rc) return rc;
        // projector shape: the one tuned for this geometry bucket, if any (an
        // operator workspace has no scratch sinogram to tune on)
        int dev = 0;
        CK(cudaGetDevice(&dev));
        const int sh = prec_of<T>() == SCG_F64 ? -1 : proj_shape_lookup(dev, prec_of<T>(), g);
        if (sh >= 0) {
            set_proj_shape(pl, g.n_angles, g.n_bins, sh);
            P.cnt_proj = pl.cnt_proj; P.proj_blocks = pl.proj_blocks; P.proj_shift = sh;
        }
        unsigned char* base = (unsigned char*)work;
        order = reinterpret_cast<const Item*>(base + pl.proj_items);
        rc = upload_proj_order(pl, base + pl.proj_items, g, s, a_begin, na_total);
        if (rc) return rc;
        // zero pads of the views and of the pair rows, once
        CK(cudaMemsetAsync(base + pl.view_rm, 0, 2 * sizeof(E) * (size_t)g.n * pl.S, s));
        CK(cudaMemsetAsync(base + pl.view_cm, 0, 2 * sizeof(E) * (size_t)g.n * pl.S, s));
        CK(cudaMemsetAsync(base + pl.sino[SB_R], 0, 2 * sizeof(E) * (size_t)g.n_angles * pl.SB, s));
        rc = upload_prob<T>(P, pl, work, s);
        if (rc) return rc;
        d = reinterpret_cast<Prob<T>*>(base + pl.prob);
        CK(cudaStreamSynchronize(s));
        return SCG_OK;
    }
    int project(const void* x, void* y, cudaStream_t s) override {
        launch_set_io<T>(d, nullptr, (E*)y, (E*)const_cast<void*>(x), s);
        launch_vec<T>(d, nullptr, pl.cnt_img, VEC_VIEWS, IB_AUX, FIN_NONE, s);
        const bool t0 = mark(0, s);
        launch_project<T>(d, order, pl.cnt_proj, SB_Q, PROJ_PLAIN_OUT, FIN_NONE, s);
        if (t0) timed[0] = mark(1, s);
        CK(cudaGetLastError());
        return SCG_OK;
    }
    int backproject(const void* r, void* x, cudaStream_t s) override {
        launch_set_io<T>(d, (const E*)r, nullptr, (E*)x, s);
        launch_sino_pairs<T>(d, pl.cnt_ray, SB_R, s);
        const bool t0 = mark(2, s);
        launch_backproject<T>(d, nullptr, pl.cnt_bp, 1, SB_R, SB_R, IB_AUX, IB_AUX, FIN_NONE, s);
        if (t0) timed[1] = mark(3, s);
        CK(cudaGetLastError());
        return SCG_OK;
    }
};

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
struct BatchPlan {
    size_t state, dummy, probs, items[K_COUNT];
    int n_items[K_COUNT], cap_items[K_COUNT];
    int cap_probs;
    std::vector<size_t> region;
    std::vector<Plan> plans;
    size_t total;
    int nb_cap;
};

BatchPlan make_batch_plan(const scg_problem* pr, int count, int variant, int precision) {
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
        b.plans[i] = make_plan(pr[i].geometry, variant, precision, PLAN_SOLVE);
        b.n_items[K_PROJ] += max_proj_items(pr[i].geometry.n_angles, pr[i].geometry.n_bins);
        b.n_items[K_IMG] += b.plans[i].cnt_img;
        b.n_items[K_RAY] += b.plans[i].cnt_ray;
        b.n_items[K_ROW] += b.plans[i].cnt_row;
        b.n_items[K_BP] += b.plans[i].cnt_bp;
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
    int prec, variant, trial_passes, ksteps, cap_probs, nb_cap, eta, pert_steps;
    int cap_items[K_COUNT];
    bool operator<(const BatchKey& o) const {
        return std::tie(dev, work, prec, variant, trial_passes, ksteps, cap_probs, nb_cap, eta, pert_steps,
                        cap_items[0], cap_items[1], cap_items[2], cap_items[3], cap_items[4]) <
               std::tie(o.dev, o.work, o.prec, o.variant, o.trial_passes, o.ksteps, o.cap_probs, o.nb_cap, o.eta,
                        o.pert_steps, o.cap_items[0], o.cap_items[1], o.cap_items[2], o.cap_items[3],
                        o.cap_items[4]);
    }
};
std::map<BatchKey, BodyGraph> g_batch_graphs;

template <typename T>
int batch_impl(const scg_problem* pr, int count, int variant, int precision, const scg_params* prm,
               void* work, size_t work_bytes, scg_result* results, cudaStream_t user_stream) {
    using E = typename Tr<T>::S;
    using C = typename Tr<T>::C;
    BatchPlan bp = make_batch_plan(pr, count, variant, prec_of<T>());
    if (work_bytes < bp.total || ((uintptr_t)work & 15u)) return SCG_ERR_WORKSPACE;
    if (uses_filter(variant) && !filter_fits(bp.nb_cap, prec_of<T>())) return SCG_ERR_UNSUPPORTED;
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
    std::vector<double> scales(count, 1.0);
    memset(probs.data(), 0, sizeof(Prob<T>) * probs.size());
    std::vector<std::vector<Item>> items(K_COUNT);
    for (int k = 0; k < K_COUNT; ++k) items[k].reserve(bp.cap_items[k]);
    CK(cudaMemsetAsync(base, 0, bp.total, s));
    Prob<T>* slots = reinterpret_cast<Prob<T>*>(base + bp.probs);
    for (int i = 0; i < count; ++i) {
        Plan& pl = bp.plans[i];
        unsigned char* rb = base + bp.region[i];
        const double scale = system_scale(pr[i].geometry, prec_of<T>());
        scales[i] = scale;
        Prob<T> P = make_prob<T>(pr[i].geometry, pl, rb, scale);
        {
            const int rc = upload_sino_maps<T>(P, pl, rb, s);
            if (rc != SCG_OK) return rc;
        }
        P.y = (const E*)pr[i].y;
        P.img[IB_AUX] = (E*)pr[i].x0;
        DevState st = initial_state(prm, pr[i].eps * scale * scale, variant);
        CK(cudaMemcpyAsync(rb + pl.state, &st, sizeof(st), cudaMemcpyHostToDevice, s));
        std::vector<Angle<C>> ang;
        fill_angles<C>(ang, pr[i].geometry.n_angles, pr[i].geometry.n, scale);
        CK(cudaMemcpyAsync(rb + pl.ang, ang.data(), sizeof(Angle<C>) * ang.size(), cudaMemcpyHostToDevice, s));
        if (uses_filter(variant)) {
            const double mu = prm->mu > 0.0 ? prm->mu : 2.0 * M_PI / pl.P;
            std::vector<C> ftab;
            fill_filter_tables<C>(ftab, pl.P, mu, prm->filter_gain);
            CK(cudaMemcpyAsync(rb + pl.taps, ftab.data(), sizeof(C) * ftab.size(), cudaMemcpyHostToDevice, s));
        }
        // the problem's own slot serves the shape tuner (a single-problem launch)
        // (blocks in index order: a batch's launch holds many problems' blocks,
        // so no longest-first list is built for it)
        const int rc = tune_proj_shape<T>(P, pl, slots + i, pr[i].geometry, s, nullptr, prm->proj_shape);
        if (rc != SCG_OK) return rc;
        probs[i] = P;
        append_items(pl, i, items.data());
        // (pageable host sources are staged before cudaMemcpyAsync returns,
        // so st and ang may be reused for the next problem)
    }
    // placeholder problem for the padding items: stopped for good
    DevState stopped;
    memset(&stopped, 0, sizeof(stopped));
    stopped.done = 1;
    CK(cudaMemcpyAsync(base + bp.dummy, &stopped, sizeof(stopped), cudaMemcpyHostToDevice, s));
    for (int i = count; i < bp.cap_probs; ++i) probs[i].st = reinterpret_cast<DevState*>(base + bp.dummy);
    // projector items depend on the tuned shapes: launch their rounded count
    int grid[K_COUNT];
    for (int k = 0; k < K_COUNT; ++k) grid[k] = k == K_PROJ ? round_up_bucket((int)items[k].size()) : bp.cap_items[k];
    for (int k = 0; k < K_COUNT; ++k)
        while ((int)items[k].size() < grid[k]) items[k].push_back(Item{count, 0, 0, 0});
    BatchState bs{0, prm->max_iter + 2, count, 0};
    CK(cudaMemcpyAsync(base + bp.state, &bs, sizeof(bs), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(base + bp.probs, probs.data(), sizeof(Prob<T>) * bp.cap_probs, cudaMemcpyHostToDevice, s));
    for (int k = 0; k < K_COUNT; ++k)
        if (grid[k])
            CK(cudaMemcpyAsync(base + bp.items[k], items[k].data(), sizeof(Item) * grid[k],
                               cudaMemcpyHostToDevice, s));
    const Prob<T>* d = reinterpret_cast<const Prob<T>*>(base + bp.probs);
    Runner<T> R{d, grid[K_RAY], grid[K_IMG], grid[K_ROW], grid[K_PROJ], bp.nb_cap, s, 0};
    R.i_ray = reinterpret_cast<const Item*>(base + bp.items[K_RAY]);
    R.i_img = reinterpret_cast<const Item*>(base + bp.items[K_IMG]);
    R.i_row = reinterpret_cast<const Item*>(base + bp.items[K_ROW]);
    R.i_proj = reinterpret_cast<const Item*>(base + bp.items[K_PROJ]);
    R.g_bp = grid[K_BP];
    R.i_bp = reinterpret_cast<const Item*>(base + bp.items[K_BP]);
    const Program pg = make_program(prm, variant);
    run_init<T>(R, pg);
    CK(cudaGetLastError());

    BatchState* bsd = reinterpret_cast<BatchState*>(base + bp.state);
    BatchKey key{dev, work, precision, variant, pg.trial_passes, pg.ksteps, bp.cap_probs, bp.nb_cap,
                 pg.eta ? 1 : 0, pg.pert_steps, {grid[0], grid[1], grid[2], grid[3], grid[4]}};
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
        CK(cudaMemcpyAsync(pr[i].x_out, probs[i].img[out_sel], sizeof(E) * J, cudaMemcpyDeviceToDevice, s));
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
        r.status = hs[i].dev_error ? SCG_ERR_CUDA : hs[i].status;
        r.f_final = (fam == FAM_CG ? hs[i].f_final : hs[i].f_half) / (scales[i] * scales[i]);
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

// Run F<T>(...) for the precision code p.
#define SCG_DISPATCH(p, F, ...)                                              \
    ((p) == SCG_F64 ? F<double>(__VA_ARGS__)                                 \
     : (p) == SCG_F32 ? F<float>(__VA_ARGS__)                                \
     : (p) == SCG_F16 ? F<__half>(__VA_ARGS__) : F<__nv_bfloat16>(__VA_ARGS__))

}  // namespace

namespace scg {
namespace host {
int proj_shape_lookup(int dev, int precision, const scg_geometry& g) {
    std::lock_guard<std::mutex> lk(g_shape_mu);
    auto it = g_shapes.find(shape_key(dev, precision, g));
    return it == g_shapes.end() ? -1 : it->second;
}
void proj_shape_store(int dev, int precision, const scg_geometry& g, int shift) {
    std::lock_guard<std::mutex> lk(g_shape_mu);
    g_shapes[shape_key(dev, precision, g)] = shift;
}
std::atomic<int> g_test_stall{0};
bool test_stall_copies() { return g_test_stall.load() != 0; }

EncodeTiledFn tensor_map_encoder() {
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

std::shared_ptr<const ProjOrder> proj_order(int n, int na, int nb, int shift, int a_begin, int na_total) {
    if (na_total < 0) na_total = na;
    const OrderKey key{n, na, nb, shift, a_begin, na_total};
    std::lock_guard<std::mutex> lk(g_order_mu);
    auto it = g_orders.find(key);
    if (it != g_orders.end()) return it->second;
    std::vector<Angle<double>> ang;
    fill_angles<double>(ang, na, n, 1.0, a_begin, na_total);
    auto o = std::make_shared<const ProjOrder>(make_proj_order(n, nb, shift, ang));
    if (g_orders.size() >= 1024) g_orders.clear();
    g_orders[key] = o;
    return o;
}
}  // namespace host
}  // namespace scg

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
    p->max_trials = 32;
    p->K = 2;
    p->k_inclusive = 0;
    p->mu = 0.0;
    p->filter_gain = 1.0;
    p->max_iter = 100;
    p->host_loop = 0;
    p->eta0 = 0.0;
    p->lambda = 0.0;
    p->prox_iters = 20;
    p->lipschitz = 0.0;
    p->proj_shape = 0;
    p->perturb_steps = 1;
}

size_t scg_op_workspace_bytes(const scg_geometry* g, int precision) {
    if (!valid_geometry(g) || !valid_prec(precision)) return 0;
    return make_plan(*g, SCG_S_CG, precision, PLAN_OP).total;
}

size_t scg_solve_workspace_bytes(const scg_geometry* g, int variant, int precision) {
    if (!valid_geometry(g) || !valid_prec(precision) || !valid_variant(variant) ||
        !solve_supported(variant, precision))
        return 0;
    return make_plan(*g, variant, precision, PLAN_SOLVE).total;
}

size_t scg_solve_workspace_bytes_p(const scg_geometry* g, int variant, int precision, const scg_params* prm) {
    if (!prm) return scg_solve_workspace_bytes(g, variant, precision);
    if (!valid_geometry(g) || !valid_prec(precision) || !valid_variant(variant) ||
        !solve_supported(variant, precision) || !valid_params(prm) || !perturb_supported(prm, precision))
        return 0;
    return make_plan(*g, variant, precision, PLAN_SOLVE, prm->perturb == SCG_PERTURB_PROX).total;
}

int scg_project(const scg_geometry* g, int precision, const void* x, void* y, void* work,
                size_t work_bytes, void* stream) {
    if (!valid_geometry(g) || !x || !y || !work) return SCG_ERR_INVALID;
    if (!valid_prec(precision)) return SCG_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    return SCG_DISPATCH(precision, project_impl, *g, x, y, work, work_bytes, s);
}

int scg_backproject(const scg_geometry* g, int precision, const void* r, void* x, void* work,
                    size_t work_bytes, void* stream) {
    if (!valid_geometry(g) || !x || !r || !work) return SCG_ERR_INVALID;
    if (!valid_prec(precision)) return SCG_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    return SCG_DISPATCH(precision, backproject_impl, *g, r, x, work, work_bytes, s);
}

int scg_tv(int n, int precision, const void* x, double* tv_out, void* work, size_t work_bytes,
           void* stream) {
    if (n < 2 || n > 8192 || !x || !tv_out || !work) return SCG_ERR_INVALID;
    if (!valid_prec(precision)) return SCG_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    return SCG_DISPATCH(precision, tv_impl, n, x, nullptr, tv_out, work, work_bytes, s);
}

int scg_tv_grad(int n, int precision, const void* x, void* grad, double* tv_out, void* work,
                size_t work_bytes, void* stream) {
    if (n < 2 || n > 8192 || !x || !grad || !tv_out || !work) return SCG_ERR_INVALID;
    if (!valid_prec(precision)) return SCG_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    return SCG_DISPATCH(precision, tv_impl, n, x, grad, tv_out, work, work_bytes, s);
}

int scg_filter(const scg_geometry* g, int precision, double mu, double gain, const void* r, void* out,
               void* work, size_t work_bytes, void* stream) {
    if (!valid_geometry(g) || !r || !out || !work || !(gain > 0.0) || !isfinite(mu)) return SCG_ERR_INVALID;
    if (!valid_prec(precision) || !filter_fits(g->n_bins, precision)) return SCG_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    return SCG_DISPATCH(precision, filter_impl, *g, mu, gain, r, out, work, work_bytes, s);
}

int scg_solve_async(const scg_geometry* g, int variant, int precision, const scg_params* prm, double eps,
                    const void* y, const void* x0, void* x_out, void* work, size_t work_bytes, scg_result* res,
                    const scg_state* resume, void* stream) {
    if (!valid_geometry(g) || !prm || !y || !x_out || !work || !res) return SCG_ERR_INVALID;
    if (!valid_variant(variant)) return SCG_ERR_INVALID;
    if (!(eps > 0.0) || !isfinite(eps) || !valid_params(prm)) return SCG_ERR_INVALID;
    if (resume && resume->valid != 1) return SCG_ERR_INVALID;
    if (prm->host_loop != 0 || (variant == SCG_FISTA && resume)) return SCG_ERR_UNSUPPORTED;
    if (!valid_prec(precision) || !solve_supported(variant, precision) || !perturb_supported(prm, precision))
        return SCG_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    scg_result dummy;
    return SCG_DISPATCH(precision, solve_impl, g, variant, precision, prm, eps, y, x0, x_out, work, work_bytes,
                        &dummy, nullptr, 0, resume, nullptr, s, res);
}

int scg_fbp(const scg_geometry* g, int precision, const void* y, void* x, void* work, size_t work_bytes,
            void* stream) {
    if (!valid_geometry(g) || !y || !x || !work) return SCG_ERR_INVALID;
    if (!valid_prec(precision)) return SCG_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    return SCG_DISPATCH(precision, fbp_impl, *g, y, x, work, work_bytes, s);
}

int scg_solve(const scg_geometry* g, int variant, int precision, const scg_params* prm, double eps,
              const void* y, const void* x0, void* x_out, void* work, size_t work_bytes,
              scg_result* res, double* trace, int trace_rows, const scg_state* resume,
              scg_state* final_state, void* stream) {
    if (!valid_geometry(g) || !prm || !y || !x_out || !work || !res) return SCG_ERR_INVALID;
    if (!valid_variant(variant)) return SCG_ERR_INVALID;
    if (variant == SCG_FISTA && resume) return SCG_ERR_UNSUPPORTED;
    if (!(eps > 0.0) || !isfinite(eps) || !valid_params(prm)) return SCG_ERR_INVALID;
    if (prm->host_loop != 0 && prm->host_loop != 1) return SCG_ERR_INVALID;
    if (resume && resume->valid != 1) return SCG_ERR_INVALID;
    if (!valid_prec(precision) || !solve_supported(variant, precision) || !perturb_supported(prm, precision))
        return SCG_ERR_UNSUPPORTED;
    memset(res, 0, sizeof(*res));
    cudaStream_t s = (cudaStream_t)stream;
    int rc = SCG_DISPATCH(precision, solve_impl, g, variant, precision, prm, eps, y, x0, x_out, work,
                          work_bytes, res, trace, trace_rows, resume, final_state, s);
    if (rc < 0 && rc != SCG_ERR_BREAKDOWN) res->status = rc;
    return rc;
}

}  // extern "C"

struct scg_operator {
    OperatorBase* impl;
};

extern "C" {

int scg_test_stall_copies(int stall) {
    scg::host::g_test_stall.store(stall ? 1 : 0);
    return SCG_OK;
}

int scg_release(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    int rc = SCG_OK;
    for (auto& kv : g_streams)
        if (cudaStreamSynchronize(kv.second) != cudaSuccess) rc = SCG_ERR_CUDA;
    for (auto& kv : g_graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    g_graphs.clear();
    for (auto& kv : g_batch_graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    g_batch_graphs.clear();
    for (auto& kv : g_streams) cudaStreamDestroy(kv.second);
    g_streams.clear();
    for (auto& kv : g_pinned) cudaFreeHost(kv.second);
    g_pinned.clear();
    scg::noalloc_forget();
    {
        std::lock_guard<std::mutex> lo(g_order_mu);
        g_orders.clear();
    }
    return rc;
}

int scg_operator_create_angles(const scg_geometry* g, int a_begin, int a_count, int precision, void* work,
                               size_t work_bytes, void* stream, scg_operator** out) {
    if (!valid_geometry(g) || !work || !out || a_begin < 0 || a_count < 1 || a_begin + a_count > g->n_angles)
        return SCG_ERR_INVALID;
    if (!valid_prec(precision)) return SCG_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    const scg_geometry gl{g->n, a_count, g->n_bins};       // the block as the operator's own scan
    OperatorBase* impl = nullptr;
    int rc;
    switch (precision) {
    case SCG_F64: { auto* o = new Operator<double>(); rc = o->init(gl, work, work_bytes, s, a_begin, g->n_angles); impl = o; break; }
    case SCG_F32: { auto* o = new Operator<float>(); rc = o->init(gl, work, work_bytes, s, a_begin, g->n_angles); impl = o; break; }
    case SCG_F16: { auto* o = new Operator<__half>(); rc = o->init(gl, work, work_bytes, s, a_begin, g->n_angles); impl = o; break; }
    default: { auto* o = new Operator<__nv_bfloat16>(); rc = o->init(gl, work, work_bytes, s, a_begin, g->n_angles); impl = o; break; }
    }
    if (rc == SCG_OK) rc = impl->make_events();
    if (rc != SCG_OK) { delete impl; return rc; }
    *out = new scg_operator{impl};
    return SCG_OK;
}

int scg_operator_timing(scg_operator* op, int enable) {
    if (!op) return SCG_ERR_INVALID;
    op->impl->timing = enable != 0;
    return SCG_OK;
}

int scg_operator_kernel_ms(scg_operator* op, float* project_ms, float* backproject_ms) {
    if (!op || (!project_ms && !backproject_ms)) return SCG_ERR_INVALID;
    OperatorBase* o = op->impl;
    if ((project_ms && !o->timed[0]) || (backproject_ms && !o->timed[1])) return SCG_ERR_INVALID;
    if (project_ms) {
        if (cudaEventSynchronize(o->ev[1]) != cudaSuccess) return SCG_ERR_CUDA;
        if (cudaEventElapsedTime(project_ms, o->ev[0], o->ev[1]) != cudaSuccess) return SCG_ERR_CUDA;
    }
    if (backproject_ms) {
        if (cudaEventSynchronize(o->ev[3]) != cudaSuccess) return SCG_ERR_CUDA;
        if (cudaEventElapsedTime(backproject_ms, o->ev[2], o->ev[3]) != cudaSuccess) return SCG_ERR_CUDA;
    }
    return SCG_OK;
}

int scg_operator_create(const scg_geometry* g, int precision, void* work, size_t work_bytes, void* stream,
                        scg_operator** out) {
    if (!valid_geometry(g)) return SCG_ERR_INVALID;
    return scg_operator_create_angles(g, 0, g->n_angles, precision, work, work_bytes, stream, out);
}

int scg_operator_project(scg_operator* op, const void* x, void* y, void* stream) {
    if (!op || !x || !y) return SCG_ERR_INVALID;
    return op->impl->project(x, y, (cudaStream_t)stream);
}

int scg_operator_backproject(scg_operator* op, const void* r, void* x, void* stream) {
    if (!op || !r || !x) return SCG_ERR_INVALID;
    return op->impl->backproject(r, x, (cudaStream_t)stream);
}

int scg_operator_destroy(scg_operator* op) {
    if (!op) return SCG_ERR_INVALID;
    delete op->impl;
    delete op;
    return SCG_OK;
}

size_t scg_batch_workspace_bytes(const scg_problem* problems, int count, int variant, int precision) {
    if (!problems || count < 1 || count > 65536 || !valid_prec(precision) || variant < SCG_CG ||
        variant > SCG_S_PCG_K || !solve_supported(variant, precision))
        return 0;
    for (int i = 0; i < count; ++i)
        if (!valid_geometry(&problems[i].geometry)) return 0;
    return make_batch_plan(problems, count, variant, precision).total;
}

int scg_solve_batch(const scg_problem* problems, int count, int variant, int precision,
                    const scg_params* prm, void* work, size_t work_bytes, scg_result* results,
                    void* stream) {
    if (!problems || count < 1 || count > 65536 || !prm || !work || !results) return SCG_ERR_INVALID;
    if (variant == SCG_FISTA) return SCG_ERR_UNSUPPORTED;          // FISTA: scg_solve only
    if (variant < SCG_CG || variant > SCG_S_PCG_K) return SCG_ERR_INVALID;
    if (!valid_params(prm)) return SCG_ERR_INVALID;
    if (prm->perturb == SCG_PERTURB_PROX) return SCG_ERR_UNSUPPORTED;   // proximal perturbation: scg_solve only
    if (prm->host_loop != 0) return SCG_ERR_UNSUPPORTED;
    for (int i = 0; i < count; ++i) {
        const scg_problem& p = problems[i];
        if (!valid_geometry(&p.geometry) || !p.y || !p.x_out || !(p.eps > 0.0) || !isfinite(p.eps))
            return SCG_ERR_INVALID;
    }
    if (!valid_prec(precision) || !solve_supported(variant, precision)) return SCG_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = SCG_DISPATCH(precision, batch_impl, problems, count, variant, precision, prm, work, work_bytes,
                          results, s);
    if (rc < 0 && rc != SCG_ERR_BREAKDOWN)
        for (int i = 0; i < count; ++i) results[i].status = rc;
    return rc;
}

}  // extern "C"
