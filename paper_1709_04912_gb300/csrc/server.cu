// server.cu -- continuous-batching request server (scg_server_*).
//
// Resident requests live in a caller-owned device pool: one solve region per
// request (the same layout a solo scg_solve uses), a descriptor array with one
// slot per resident request plus a permanently stopped placeholder slot, and
// per-kind work lists.  A step admits queued requests in submission order
// while a slot and pool memory are free, runs their set-up program over a work
// list of the newcomers alone, advances every resident request by a fixed
// number of loop bodies through one captured graph over the work lists of all
// of them, gathers the stop flags, and finishes the requests that stopped
// (their final TV / f, the output copy and the state read-back) before their
// memory returns to the pool.  Work items keep each request's single-solve
// block indices, so every result is bit-identical to its solo solve.
#include <deque>
#include <map>
#include <tuple>
#include <vector>

#include "host_programs.h"

using namespace scg;
using namespace scg::host;

namespace {

#define SCK(call)                                  \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return SCG_ERR_CUDA; \
    } while (0)

// First-fit allocator over the pool, with coalescing of freed neighbours.
class PoolAllocator {
public:
    void reset(size_t bytes) {
        free_.clear();
        if (bytes) free_[0] = bytes;
    }
    bool alloc(size_t bytes, size_t* off) {
        bytes = align_up(bytes ? bytes : 1, kAlign);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes, at = it->first + bytes;
            free_.erase(it);
            if (rest) free_[at] = rest;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = align_up(bytes ? bytes : 1, kAlign);
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t largest() const {
        size_t m = 0;
        for (auto& f : free_) m = f.second > m ? f.second : m;
        return m;
    }

private:
    std::map<size_t, size_t> free_;
};

// Pinned host staging for uploads and read-backs (bump allocation; when full,
// the stream is drained and the buffer reused or grown).
class Staging {
public:
    ~Staging() { if (buf_) cudaFreeHost(buf_); }
    cudaError_t get(size_t bytes, cudaStream_t s, unsigned char** out) {
        bytes = align_up(bytes ? bytes : 1, 64);
        if (off_ + bytes > cap_) {
            cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return e;
            off_ = 0;
            if (bytes > cap_) {
                if (buf_) cudaFreeHost(buf_);
                buf_ = nullptr;
                cap_ = 0;
                size_t c = bytes > (size_t)(1 << 20) ? bytes : (size_t)(1 << 20);
                e = cudaHostAlloc((void**)&buf_, c, cudaHostAllocDefault);
                if (e != cudaSuccess) return e;
                cap_ = c;
            }
        }
        *out = buf_ + off_;
        off_ += bytes;
        return cudaSuccess;
    }
    void reset() { off_ = 0; }

private:
    unsigned char* buf_ = nullptr;
    size_t cap_ = 0, off_ = 0;
};

struct Request {
    scg_problem p;
    unsigned long long tag;
    Plan plan;
    double scale;      // system scale c (f is reported / c^2)
    size_t off;
    int slot, bodies;
};

// A device work list of one kind, held in the pool.
struct DevList {
    size_t off = 0;
    int cap = 0;
};

struct ServerBase {
    virtual ~ServerBase() {}
    virtual int submit(const scg_problem* req, unsigned long long tag) = 0;
    virtual int step(cudaStream_t user, scg_completion* done, int max_done, int* n_done) = 0;
    virtual void pending(int* queued, int* active) const = 0;
};

// Pool bytes of one resident request: its solve region, and its share of the
// active (rounded up) and set-up/final work lists.
size_t footprint_bytes(const Plan& pl, const scg_geometry& g) {
    int n[K_COUNT];
    n[K_PROJ] = max_proj_items(g.n_angles, g.n_bins);
    n[K_IMG] = pl.cnt_img;
    n[K_RAY] = pl.cnt_ray;
    n[K_ROW] = pl.cnt_row;
    n[K_BP] = pl.cnt_bp;
    size_t b = align_up(pl.total, kAlign);
    for (int k = 0; k < K_COUNT; ++k)
        b += align_up(sizeof(Item) * (size_t)round_up_bucket(n[k]), kAlign) + align_up(sizeof(Item) * (size_t)n[k], kAlign);
    return b;
}

template <typename T>
class Server final : public ServerBase {
public:
    explicit Server(const scg_server_config& c) : cfg_(c) {
        fam_ = family_of(c.variant);
        prog_ = make_program(&c.params, c.variant);
        base_ = static_cast<unsigned char*>(c.pool);
        alloc_.reset(c.pool_bytes);
        slots_.assign(c.max_active, nullptr);
    }
    ~Server() override {
        if (stream_) cudaStreamSynchronize(stream_);
        for (auto& g : graphs_) cudaGraphExecDestroy(g.second.exec);
        for (Request* r : queue_) delete r;
        for (Request* r : slots_) delete r;
        if (stream_) cudaStreamDestroy(stream_);
        if (ev_) cudaEventDestroy(ev_);
    }

    int init() {
        const int cap = cfg_.max_active + 1;
        if (!alloc_.alloc(sizeof(Prob<T>) * (size_t)cap, &probs_off_) ||
            !alloc_.alloc(sizeof(DevState), &dummy_off_) ||
            !alloc_.alloc(sizeof(int) * (size_t)cfg_.max_active, &slot_ids_off_) ||
            !alloc_.alloc(sizeof(int) * (size_t)cfg_.max_active, &flags_off_))
            return SCG_ERR_WORKSPACE;
        reserved_ = alloc_.largest();
        return SCG_OK;
    }

    int submit(const scg_problem* req, unsigned long long tag) override {
        Request* r = new Request();
        r->p = *req;
        r->tag = tag;
        if (uses_filter(cfg_.variant) && !filter_fits(req->geometry.n_bins, prec_of<T>())) {
            delete r;
            return SCG_ERR_UNSUPPORTED;
        }
        r->plan = make_plan(req->geometry, cfg_.variant, prec_of<T>(), PLAN_SOLVE);
        r->scale = system_scale(req->geometry, prec_of<T>());
        r->off = 0;
        r->slot = -1;
        r->bodies = 0;
        // region plus its share of the work lists (active and set-up/final)
        if (footprint_bytes(r->plan, req->geometry) > reserved_) {
            delete r;
            return SCG_ERR_WORKSPACE;
        }
        queue_.push_back(r);
        return SCG_OK;
    }

    void pending(int* queued, int* active) const override {
        if (queued) *queued = (int)queue_.size();
        if (active) *active = n_active_;
    }

    int step(cudaStream_t user, scg_completion* done, int max_done, int* n_done) override {
        if (!stream_) {
            SCK(cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking));
            SCK(cudaEventCreateWithFlags(&ev_, cudaEventDisableTiming));
            DevState stopped;
            memset(&stopped, 0, sizeof(stopped));
            stopped.done = 1;
            SCK(upload(base_ + dummy_off_, &stopped, sizeof(stopped)));
            std::vector<Prob<T>> ph(cfg_.max_active + 1);
            memset(ph.data(), 0, sizeof(Prob<T>) * ph.size());
            for (auto& P : ph) P.st = reinterpret_cast<DevState*>(base_ + dummy_off_);
            SCK(upload(probs(), ph.data(), sizeof(Prob<T>) * ph.size()));
        }
        SCK(cudaEventRecord(ev_, user));
        SCK(cudaStreamWaitEvent(stream_, ev_, 0));
        int rc = SCG_OK;
        if (queue_.size() || n_active_) rc = advance();
        SCK(cudaStreamSynchronize(stream_));           // staged copies and freed regions are idle
        staging_.reset();
        for (auto& f : deferred_free_) alloc_.release(f.first, f.second);
        deferred_free_.clear();
        SCK(cudaEventRecord(ev_, stream_));
        SCK(cudaStreamWaitEvent(user, ev_, 0));
        int k = 0;
        while (k < max_done && !completions_.empty()) {
            done[k++] = completions_.front();
            completions_.pop_front();
        }
        if (n_done) *n_done = k;
        return rc;
    }

private:
    Prob<T>* probs() { return reinterpret_cast<Prob<T>*>(base_ + probs_off_); }
    const Item* list_ptr(const DevList& l) const { return reinterpret_cast<const Item*>(base_ + l.off); }

    cudaError_t upload(void* dst, const void* src, size_t bytes) {
        unsigned char* h = nullptr;
        cudaError_t e = staging_.get(bytes, stream_, &h);
        if (e != cudaSuccess) return e;
        memcpy(h, src, bytes);
        return cudaMemcpyAsync(dst, h, bytes, cudaMemcpyHostToDevice, stream_);
    }

    // Make `l` hold at least `need` items (old storage is freed after the step).
    int reserve_list(DevList& l, int need) {
        if (need <= l.cap) return SCG_OK;
        int cap = need + need / 2;
        size_t off = 0;
        if (!alloc_.alloc(sizeof(Item) * (size_t)cap, &off)) {
            cap = need;
            if (!alloc_.alloc(sizeof(Item) * (size_t)cap, &off)) return SCG_ERR_WORKSPACE;
        }
        if (l.cap) deferred_free_.push_back({l.off, sizeof(Item) * (size_t)l.cap});
        l.off = off;
        l.cap = cap;
        graphs_dirty_ = true;
        return SCG_OK;
    }

    // Free every work list now (only when no request is resident and nothing
    // is in flight); cached graphs name list addresses, so they go too.
    void drop_lists() {
        for (auto& f : deferred_free_) alloc_.release(f.first, f.second);
        deferred_free_.clear();
        for (int k = 0; k < K_COUNT; ++k) {
            if (active_lists_[k].cap) alloc_.release(active_lists_[k].off, sizeof(Item) * (size_t)active_lists_[k].cap);
            if (aux_lists_[k].cap) alloc_.release(aux_lists_[k].off, sizeof(Item) * (size_t)aux_lists_[k].cap);
            active_lists_[k] = DevList();
            aux_lists_[k] = DevList();
        }
        for (auto& g : graphs_) cudaGraphExecDestroy(g.second.exec);
        graphs_.clear();
        graphs_dirty_ = true;
    }

    // Upload work lists over the given slots; `bucket` pads each list with
    // placeholder items to its rounded length.  Returns the launch grids.
    int build_lists(const std::vector<int>& slots, DevList* lists, bool bucket, int* grid, int* nb_max) {
        std::vector<Item> v[K_COUNT];
        *nb_max = 1;
        for (int sl : slots) {
            append_items(slots_[sl]->plan, sl, v);
            if (slots_[sl]->p.geometry.n_bins > *nb_max) *nb_max = slots_[sl]->p.geometry.n_bins;
        }
        for (int k = 0; k < K_COUNT; ++k) {
            const int n = (int)v[k].size();
            const int g = bucket ? round_up_bucket(n) : n;
            while ((int)v[k].size() < g) v[k].push_back(Item{cfg_.max_active, 0, 0, 0});
            grid[k] = g;
            if (!g) continue;
            int rc = reserve_list(lists[k], g);
            if (rc != SCG_OK) return rc;
            SCK(upload(base_ + lists[k].off, v[k].data(), sizeof(Item) * (size_t)g));
        }
        return SCG_OK;
    }

    Runner<T> runner(const DevList* lists, const int* grid, int nb, cudaStream_t s) {
        Runner<T> R{probs(), grid[K_RAY], grid[K_IMG], grid[K_ROW], grid[K_PROJ], nb, s, 0};
        R.i_ray = list_ptr(lists[K_RAY]);
        R.i_img = list_ptr(lists[K_IMG]);
        R.i_row = list_ptr(lists[K_ROW]);
        R.i_proj = list_ptr(lists[K_PROJ]);
        R.g_bp = grid[K_BP];
        R.i_bp = list_ptr(lists[K_BP]);
        return R;
    }

    // Work items of each kind one request can add (projector: its largest shape).
    static void request_items(const Request* r, int* n) {
        n[K_PROJ] = max_proj_items(r->p.geometry.n_angles, r->p.geometry.n_bins);
        n[K_IMG] = r->plan.cnt_img;
        n[K_RAY] = r->plan.cnt_ray;
        n[K_ROW] = r->plan.cnt_row;
        n[K_BP] = r->plan.cnt_bp;
    }

    int admit(std::vector<int>* newcomers) {
        // items of the resident requests, and of this step's newcomers
        int act[K_COUNT] = {0, 0, 0, 0, 0}, fresh[K_COUNT] = {0, 0, 0, 0, 0}, n[K_COUNT];
        for (Request* q : slots_) {
            if (!q) continue;
            request_items(q, n);
            for (int k = 0; k < K_COUNT; ++k) act[k] += n[k];
        }
        bool lists_dropped = false;
        while (!queue_.empty() && n_active_ < cfg_.max_active) {
            Request* r = queue_.front();
            // the work lists must hold the newcomer before its state is placed
            request_items(r, n);
            bool ok = true;
            for (int k = 0; k < K_COUNT && ok; ++k)
                ok = reserve_list(active_lists_[k], round_up_bucket(act[k] + n[k])) == SCG_OK &&
                     reserve_list(aux_lists_[k], fresh[k] + n[k]) == SCG_OK;
            size_t off = 0;
            if (ok) ok = alloc_.alloc(r->plan.total, &off);
            if (!ok) {
                if (n_active_ > 0 || !newcomers->empty()) break;   // wait for memory to free up
                // nothing resident and nothing in flight: drop the work lists (they
                // only grow) and retry once; a request that still does not fit can
                // never run, and completes with SCG_ERR_WORKSPACE
                if (!lists_dropped) {
                    drop_lists();
                    lists_dropped = true;
                    continue;
                }
                scg_completion c;
                memset(&c, 0, sizeof(c));
                c.tag = r->tag;
                c.result.status = SCG_ERR_WORKSPACE;
                completions_.push_back(c);
                queue_.pop_front();
                delete r;
                lists_dropped = false;
                continue;
            }
            lists_dropped = false;
            for (int k = 0; k < K_COUNT; ++k) { act[k] += n[k]; fresh[k] += n[k]; }
            int slot = 0;
            while (slots_[slot]) ++slot;
            r->off = off;
            r->slot = slot;
            unsigned char* rb = base_ + off;
            const Plan& pl = r->plan;
            using E = typename Tr<T>::S;
            using C = typename Tr<T>::C;
            Prob<T> P = make_prob<T>(r->p.geometry, pl, rb, r->scale);
            P.y = static_cast<const E*>(r->p.y);
            P.img[IB_AUX] = static_cast<E*>(const_cast<void*>(r->p.x0));
            SCK(cudaMemsetAsync(rb, 0, pl.total, stream_));
            {
                const int rc = upload_sino_maps<T>(P, pl, rb, stream_);
                if (rc != SCG_OK) return rc;
            }
            DevState st = initial_state(&cfg_.params, r->p.eps * r->scale * r->scale, cfg_.variant);
            SCK(upload(rb + pl.state, &st, sizeof(st)));
            std::vector<Angle<C>> ang;
            fill_angles<C>(ang, r->p.geometry.n_angles, r->p.geometry.n, r->scale);
            SCK(upload(rb + pl.ang, ang.data(), sizeof(Angle<C>) * ang.size()));
            if (uses_filter(cfg_.variant)) {
                const double mu = cfg_.params.mu > 0.0 ? cfg_.params.mu : 2.0 * M_PI / pl.P;
                std::vector<C> ftab;
                fill_filter_tables<C>(ftab, pl.P, mu, cfg_.params.filter_gain);
                SCK(upload(rb + pl.taps, ftab.data(), sizeof(C) * ftab.size()));
            }
            SCK(upload(probs() + slot, &P, sizeof(P)));
            {
                const int rc = tune_proj_shape<T>(P, r->plan, probs() + slot, r->p.geometry, stream_, nullptr,
                                                  cfg_.params.proj_shape);
                if (rc != SCG_OK) return rc;
            }
            slots_[slot] = r;
            ++n_active_;
            queue_.pop_front();
            newcomers->push_back(slot);
            membership_changed_ = true;
        }
        return SCG_OK;
    }

    struct Key {
        size_t off[K_COUNT];
        int grid[K_COUNT];
        int nb;
        bool operator<(const Key& o) const {
            return std::tie(off[0], off[1], off[2], off[3], off[4], grid[0], grid[1], grid[2], grid[3], grid[4],
                            nb) <
                   std::tie(o.off[0], o.off[1], o.off[2], o.off[3], o.off[4], o.grid[0], o.grid[1], o.grid[2],
                            o.grid[3], o.grid[4], o.nb);
        }
    };
    struct Graph {
        cudaGraphExec_t exec;
        int kernels;
    };

    int body_graph(const Key& key, Graph* out) {
        auto it = graphs_.find(key);
        if (it != graphs_.end()) { *out = it->second; return SCG_OK; }
        if (graphs_.size() >= 32) {                      // nothing in flight: the stream is drained
            SCK(cudaStreamSynchronize(stream_));
            for (auto& g : graphs_) cudaGraphExecDestroy(g.second.exec);
            graphs_.clear();
        }
        cudaStream_t cap;
        SCK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        Runner<T> R = runner(active_lists_, key.grid, key.nb, cap);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            run_body<T>(R, prog_);
            e = cudaStreamEndCapture(cap, &g);
        }
        Graph G{nullptr, R.launches};
        if (e == cudaSuccess) e = cudaGraphInstantiate(&G.exec, g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) { cudaGetLastError(); return SCG_ERR_CUDA; }
        graphs_[key] = G;
        *out = G;
        return SCG_OK;
    }

    int advance() {
        std::vector<int> newcomers;
        int rc = admit(&newcomers);
        if (rc != SCG_OK) return rc;
        int grid[K_COUNT], nb = 1;
        if (!newcomers.empty()) {                        // set-up programs of the newcomers
            rc = build_lists(newcomers, aux_lists_, false, grid, &nb);
            if (rc != SCG_OK) return rc;
            Runner<T> R = runner(aux_lists_, grid, nb, stream_);
            run_init<T>(R, prog_);
            SCK(cudaGetLastError());
        }
        std::vector<int> act;
        for (int i = 0; i < cfg_.max_active; ++i)
            if (slots_[i]) act.push_back(i);
        if (act.empty()) return SCG_OK;
        if (membership_changed_ || graphs_dirty_) {
            rc = build_lists(act, active_lists_, true, active_grid_, &nb);
            if (rc != SCG_OK) return rc;
            active_nb_ = (nb + 127) / 128 * 128;
            SCK(upload(base_ + slot_ids_off_, act.data(), sizeof(int) * act.size()));
            membership_changed_ = false;
            graphs_dirty_ = false;
        }
        Key key;
        for (int k = 0; k < K_COUNT; ++k) {
            key.off[k] = active_lists_[k].off;
            key.grid[k] = active_grid_[k];
        }
        key.nb = active_nb_;
        Graph G;
        rc = body_graph(key, &G);
        if (rc != SCG_OK) return rc;
        for (int b = 0; b < cfg_.bodies_per_step; ++b) SCK(cudaGraphLaunch(G.exec, stream_));
        for (int sl : act) slots_[sl]->bodies += cfg_.bodies_per_step;
        // stop flags
        int* flags_dev = reinterpret_cast<int*>(base_ + flags_off_);
        launch_slots_done<T>(probs(), reinterpret_cast<const int*>(base_ + slot_ids_off_), (int)act.size(),
                             flags_dev, 0, 0, stream_);
        unsigned char* hf = nullptr;
        SCK(staging_.get(sizeof(int) * act.size(), stream_, &hf));
        SCK(cudaMemcpyAsync(hf, flags_dev, sizeof(int) * act.size(), cudaMemcpyDeviceToHost, stream_));
        SCK(cudaStreamSynchronize(stream_));
        std::vector<int> fin;
        const int* flags = reinterpret_cast<const int*>(hf);
        for (size_t i = 0; i < act.size(); ++i)
            if (flags[i] || slots_[act[i]]->bodies > cfg_.params.max_iter + 2) fin.push_back(act[i]);
        if (fin.empty()) return SCG_OK;
        return finish(fin);
    }

    int finish(const std::vector<int>& fin) {
        const int n = (int)fin.size();
        int* ids = reinterpret_cast<int*>(base_ + flags_off_);   // reuse: flags already read
        SCK(upload(ids, fin.data(), sizeof(int) * n));
        launch_slots_done<T>(probs(), ids, n, nullptr, 1, 0, stream_);
        int grid[K_COUNT], nb = 1;
        int rc = build_lists(fin, aux_lists_, false, grid, &nb);
        if (rc != SCG_OK) return rc;
        Runner<T> R = runner(aux_lists_, grid, nb, stream_);
        const int out_sel = fam_ == FAM_CG ? IB_X : IB_XH;
        R.tvgrad(out_sel, 0, 0, FIN_FINAL_TV);
        if (fam_ == FAM_CG) {
            R.vec(VEC_VIEWS, IB_X, FIN_NONE);
            R.project(SB_Q, PROJ_RESIDUAL, FIN_FINAL_F);
        }
        SCK(cudaGetLastError());
        unsigned char* hs = nullptr;
        SCK(staging_.get(sizeof(DevState) * n, stream_, &hs));
        for (int i = 0; i < n; ++i) {
            Request* r = slots_[fin[i]];
            const size_t J = (size_t)r->p.geometry.n * r->p.geometry.n;
            unsigned char* rb = base_ + r->off;
            const Prob<T> P = make_prob<T>(r->p.geometry, r->plan, rb);
            SCK(cudaMemcpyAsync(r->p.x_out, P.img[out_sel], sizeof(typename Tr<T>::S) * J,
                                cudaMemcpyDeviceToDevice, stream_));
            SCK(cudaMemcpyAsync(hs + i * sizeof(DevState), rb + r->plan.state, sizeof(DevState),
                                cudaMemcpyDeviceToHost, stream_));
        }
        SCK(cudaStreamSynchronize(stream_));
        for (int i = 0; i < n; ++i) {
            Request* r = slots_[fin[i]];
            DevState st;
            memcpy(&st, hs + i * sizeof(DevState), sizeof(DevState));
            scg_completion c;
            memset(&c, 0, sizeof(c));
            c.tag = r->tag;
            c.result.iters = st.iters;
            c.result.k_final = st.k;
            c.result.status = st.dev_error ? SCG_ERR_CUDA : st.status;
            c.result.f_final = (fam_ == FAM_CG ? st.f_final : st.f_half) / (r->scale * r->scale);
            c.result.tv_final = st.tv_final;
            c.result.ell = st.ell;
            c.result.gamma0_used = st.gamma0;
            c.result.body_launches = r->bodies;
            c.result.device_loop = 0;
            completions_.push_back(c);
            deferred_free_.push_back({r->off, r->plan.total});
            slots_[fin[i]] = nullptr;
            delete r;
            --n_active_;
        }
        membership_changed_ = true;
        return SCG_OK;
    }

    scg_server_config cfg_;
    int fam_ = 0;
    Program prog_;
    unsigned char* base_ = nullptr;
    PoolAllocator alloc_;
    Staging staging_;
    size_t probs_off_ = 0, dummy_off_ = 0, slot_ids_off_ = 0, flags_off_ = 0, reserved_ = 0;
    std::deque<Request*> queue_;
    std::vector<Request*> slots_;
    int n_active_ = 0;
    DevList active_lists_[K_COUNT], aux_lists_[K_COUNT];
    int active_grid_[K_COUNT] = {0, 0, 0, 0, 0};
    int active_nb_ = 128;
    bool membership_changed_ = true, graphs_dirty_ = true;
    std::vector<std::pair<size_t, size_t>> deferred_free_;
    std::deque<scg_completion> completions_;
    std::map<Key, Graph> graphs_;
    cudaStream_t stream_ = nullptr;
    cudaEvent_t ev_ = nullptr;
};

}  // namespace

struct scg_server {
    ServerBase* impl;
};

extern "C" {

size_t scg_server_footprint(const scg_geometry* g, int variant, int precision) {
    if (!valid_geometry(g) || variant < SCG_CG || variant > SCG_S_PCG_K || !valid_prec(precision) ||
        !solve_supported(variant, precision))
        return 0;
    const Plan pl = make_plan(*g, variant, precision, PLAN_SOLVE);
    return footprint_bytes(pl, *g);
}

int scg_server_create(const scg_server_config* cfg, scg_server** out) {
    if (!cfg || !out || !cfg->pool || ((uintptr_t)cfg->pool & 15u)) return SCG_ERR_INVALID;
    if (cfg->variant == SCG_FISTA) return SCG_ERR_UNSUPPORTED;     // FISTA: scg_solve only
    if (cfg->params.perturb == SCG_PERTURB_PROX) return SCG_ERR_UNSUPPORTED;   // scg_solve only
    if (cfg->variant < SCG_CG || cfg->variant > SCG_S_PCG_K) return SCG_ERR_INVALID;
    if (!valid_prec(cfg->precision) || !solve_supported(cfg->variant, cfg->precision)) return SCG_ERR_UNSUPPORTED;
    if (cfg->max_active < 1 || cfg->max_active > 65535 || cfg->bodies_per_step < 1 ||
        cfg->bodies_per_step > 1000)
        return SCG_ERR_INVALID;
    if (!valid_params(&cfg->params) || cfg->params.host_loop != 0) return SCG_ERR_INVALID;
    ServerBase* impl = nullptr;
    int rc;
    switch (cfg->precision) {
    case SCG_F64: { auto* s = new Server<double>(*cfg); rc = s->init(); impl = s; break; }
    case SCG_F32: { auto* s = new Server<float>(*cfg); rc = s->init(); impl = s; break; }
    case SCG_F16: { auto* s = new Server<__half>(*cfg); rc = s->init(); impl = s; break; }
    default: { auto* s = new Server<__nv_bfloat16>(*cfg); rc = s->init(); impl = s; break; }
    }
    if (rc != SCG_OK) { delete impl; return rc; }
    *out = new scg_server{impl};
    return SCG_OK;
}

int scg_server_submit(scg_server* srv, const scg_problem* req, unsigned long long tag) {
    if (!srv || !req) return SCG_ERR_INVALID;
    if (!valid_geometry(&req->geometry) || !req->y || !req->x_out || !(req->eps > 0.0) || !isfinite(req->eps))
        return SCG_ERR_INVALID;
    return srv->impl->submit(req, tag);
}

int scg_server_step(scg_server* srv, void* stream, scg_completion* done, int max_done, int* n_done) {
    if (!srv || max_done < 0 || (max_done > 0 && !done)) return SCG_ERR_INVALID;
    return srv->impl->step(static_cast<cudaStream_t>(stream), done, max_done, n_done);
}

int scg_server_pending(const scg_server* srv, int* queued, int* active) {
    if (!srv) return SCG_ERR_INVALID;
    srv->impl->pending(queued, active);
    return SCG_OK;
}

int scg_server_destroy(scg_server* srv) {
    if (!srv) return SCG_ERR_INVALID;
    delete srv->impl;
    delete srv;
    return SCG_OK;
}

}  // extern "C"
