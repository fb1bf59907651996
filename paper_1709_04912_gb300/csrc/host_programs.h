// host_programs.h -- host-side pieces shared by the solve, batch and serving
// entry points: the per-problem workspace plan, the angle table, the device
// problem descriptor, the per-variant kernel programs (Algorithms 1-14) and
// the work-item lists of batched launches.
#pragma once
#include <math.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <vector>

#include <cuda.h>   // CUtensorMap and its encoder's signature (the encoder is resolved at run time)

#include "scg_kernels.h"

namespace scg {
namespace host {

constexpr int kMaxTraceRows = 4096;
constexpr size_t kAlign = 256;
constexpr size_t kMapBytes = kSinoMapBytes;       // one CUtensorMap

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
inline int round_up4(int v) { return (v + 3) / 4 * 4; }

inline bool valid_geometry(const scg_geometry* g) {
    return g && g->n >= 2 && g->n <= 8192 && g->n_angles >= 1 && g->n_angles <= 16384 &&
           g->n_bins >= 1 && g->n_bins <= 16384;
}

inline int filter_length(int nb) { return filter_length_of(nb); }

inline int family_of(int v) {
    if (v == SCG_CG || v == SCG_PCG) return FAM_CG;
    if (v == SCG_S_CG_K || v == SCG_S_PCG_K) return FAM_S_K;
    if (v == SCG_FISTA) return FAM_FISTA;
    return FAM_S_PR;
}
inline bool valid_variant(int v) { return v >= SCG_CG && v <= SCG_FISTA; }

inline bool uses_filter(int v) { return v == SCG_PCG || v == SCG_S_PCG || v == SCG_S_PCG_K; }

// The row filter holds a whole padded row pair's FFT in shared memory.
inline bool filter_fits(int nb, int precision) {
    return (precision == SCG_F64 ? filter_smem_bytes<double>(nb) : filter_smem_bytes<float>(nb)) <= kFilterSmemMax;
}

// Filter tables of one geometry (Sec. 3, Eq. filter_factors_pre): P factors
// gain c(w_k) / P with c(w) = (|w| + mu)(0.54 + 0.46 cos w), w_k = 2 pi k / P
// folded into [-pi, pi] (the 1/P completes the unitary transform pair), stored
// at the bit reversal of k (the order in which the filter kernel's forward FFT
// leaves the spectrum), then the twiddles exp(-2 pi i j / P), j < P/2, as
// (cos, -sin) pairs; all in FP64, rounded once to the arithmetic type.
template <typename C>
void fill_filter_tables(std::vector<C>& out, int P, double mu, double gain) {
    out.assign(2 * (size_t)P, C(0));
    int lg = 0;
    while ((1 << lg) < P) ++lg;
    for (int k = 0; k < P; ++k) {
        const double w = (k <= P / 2) ? 2.0 * M_PI * k / P : 2.0 * M_PI * (k - P) / P;
        int r = 0;                                    // k with its lg bits reversed
        for (int b = 0; b < lg; ++b) r |= ((k >> b) & 1) << (lg - 1 - b);
        out[r] = (C)(gain * (fabs(w) + mu) * (0.54 + 0.46 * cos(w)) / (double)P);
    }
    for (int j = 0; j < P / 2; ++j) {
        const double a = 2.0 * M_PI * (double)j / (double)P;
        out[P + 2 * j] = (C)cos(a);
        out[P + 2 * j + 1] = (C)(-sin(a));
    }
}

constexpr int kProjShiftMin = 5, kProjShiftMax = 8;   // projector blocks 8 x 32 ... 1 x 256

// Parameter ranges shared by every solving entry point.
inline bool valid_params(const scg_params* p) {
    if (p->max_iter < 0 || p->max_iter > 10000000 || p->max_trials < 1 || p->max_trials > 100000 || p->K < 1 ||
        p->K > 1000 || !(p->a > 0.0 && p->a < 1.0) || !(p->filter_gain > 0.0))
        return false;
    if (!(p->lambda >= 0.0) || !isfinite(p->lambda) || p->prox_iters < 0 || p->prox_iters > 100000 ||
        !isfinite(p->lipschitz))
        return false;
    if (p->proj_shape != 0 && (p->proj_shape < kProjShiftMin || p->proj_shape > kProjShiftMax)) return false;
    if (p->perturb_steps < 0 || p->perturb_steps > 16) return false;
    if (p->perturb == SCG_PERTURB_ETA) return p->eta0 > 0.0 && isfinite(p->eta0) && p->perturb_steps <= 1;
    if (p->perturb == SCG_PERTURB_PROX) return p->prox_iters >= 1;
    return p->perturb == SCG_PERTURB_NONE || p->perturb == SCG_PERTURB_GAMMA;
}

inline bool valid_prec(int p) { return p == SCG_F32 || p == SCG_F64 || p == SCG_F16 || p == SCG_BF16; }
// bytes of one stored element, and of one arithmetic value
inline size_t elem_size(int p) { return p == SCG_F64 ? 8 : p == SCG_F32 ? 4 : 2; }
inline size_t calc_size(int p) { return p == SCG_F64 ? 8 : 4; }
template <typename T> constexpr int prec_of();
template <> constexpr int prec_of<float>() { return SCG_F32; }
template <> constexpr int prec_of<double>() { return SCG_F64; }
template <> constexpr int prec_of<__half>() { return SCG_F16; }
template <> constexpr int prec_of<__nv_bfloat16>() { return SCG_BF16; }

// Half and bfloat16 storage serve the superiorized variants, whose gradient
// is recomputed from x in every loop body.  CG and PCG update g and r
// recursively (g' = g + alpha h, Algorithms 2 and 4): with an 8- or 11-bit
// mantissa the cancellation in that update loses the gradient.
inline bool solve_supported(int variant, int precision) {
    if (precision == SCG_F32 || precision == SCG_F64) return true;
    return variant != SCG_CG && variant != SCG_PCG && variant != SCG_FISTA;
}
// The proximal perturbation runs the FGP kernels, which exist for FP32 and
// FP64 storage only (as FISTA).
inline bool perturb_supported(const scg_params* p, int precision) {
    return p->perturb != SCG_PERTURB_PROX || precision == SCG_F32 || precision == SCG_F64;
}

// Scale c of the system a solve works on: c A x ~ c y, f scaled by c^2.  CG's
// iterates do not change when A and y are scaled together, and a power of two
// scales every value exactly, so this only moves magnitudes: for half storage
// A^T (A x - y) grows with n_angles * N and would overflow at 1024^2 / 1440
// angles.  c = 2^-round(log2(sqrt(n_angles N))) keeps the residual, gradient
// and direction vectors near 1.  FP32 and FP64 solve the unscaled system.
inline double system_scale(const scg_geometry& g, int precision) {
    if (precision == SCG_F32 || precision == SCG_F64) return 1.0;
    const double e = 0.5 * log2((double)g.n_angles * (double)g.n);
    return ldexp(1.0, -(int)llround(e));
}

// Workspace plan: byte offsets of every segment.
struct Plan {
    size_t state, prob, ang, taps, partials, counter, trace, proj_items, maps;
    size_t img[IB_COUNT];
    size_t dual[4];
    size_t view_rm, view_cm;
    size_t sino[SB_COUNT];
    size_t total;
    int S, SB, cnt_ray, cnt_img, cnt_row, tiles_x, ray_blocks, filt_blocks, P;
    int cnt_proj, proj_blocks, proj_shift;
    int cnt_bp;
    int bp_mirror;          // the gather may take the mirror-paired kernel (64 | N, FP32 arithmetic,
                            // the scan's full angle set)
    int part_cap;           // work items the partial-sum buffer holds per slot
};

// Projector items for the block shape 2^(8-shift) angles x 2^shift rays.
inline void set_proj_shape(Plan& p, int na, int nb, int shift) {
    const int R = 1 << shift, A = kProjThreads >> shift;
    p.proj_shift = shift;
    p.proj_blocks = (nb + R - 1) / R;
    p.cnt_proj = ((na + A - 1) / A) * p.proj_blocks;
}
inline int max_proj_items(int na, int nb) {
    Plan p;
    int m = 0;
    for (int sh = kProjShiftMin; sh <= kProjShiftMax; ++sh) {
        set_proj_shape(p, na, nb, sh);
        if (p.cnt_proj > m) m = p.cnt_proj;
    }
    return m;
}

enum PlanKind { PLAN_OP = 0, PLAN_SOLVE = 1 };

// prox_duals: the proximal perturbation's four dual fields (S-variants).
inline Plan make_plan(const scg_geometry& g, int variant, int precision, int kind, bool prox_duals = false) {
    const size_t tsize = elem_size(precision), csize = calc_size(precision);
    Plan p;
    memset(&p, 0, sizeof(p));
    const int N = g.n, na = g.n_angles, nb = g.n_bins;
    p.S = round_up4(N + 2 * kPad);          // pairs per view line
    p.SB = round_up4(nb + 2 * kSPad);       // pairs per sinogram-view row
    p.ray_blocks = (nb + kRayBlock - 1) / kRayBlock;
    p.tiles_x = (N + kTileW - 1) / kTileW;
    p.cnt_ray = na * p.ray_blocks;
    p.cnt_img = ((N + kTileH - 1) / kTileH) * p.tiles_x;
    p.filt_blocks = 1;                      // one item per pair of rows
    p.cnt_row = (na + 1) / 2;
    // partials are sized for the largest item count of any projector shape
    const int max_proj = max_proj_items(na, nb);
    set_proj_shape(p, na, nb, kProjShiftDefault);
    const int bp_th = precision == SCG_F64 ? kBpTileH64 : kBpTileH32;
    p.cnt_bp = ((N + bp_th - 1) / bp_th) * p.tiles_x;
    p.bp_mirror = (precision != SCG_F64 && N % 64 == 0) ? 1 : 0;
    p.P = filter_length(nb);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, kAlign); return o; };
    const size_t J = (size_t)N * N;
    p.state = take(sizeof(DevState));
    p.prob = take(sizeof(Prob<double>));
    p.ang = take(sizeof(Angle<double>) * na);
    p.taps = take(csize * 2 * (size_t)p.P);
    int maxcnt = p.cnt_ray > p.cnt_img ? p.cnt_ray : p.cnt_img;
    if (p.cnt_row > maxcnt) maxcnt = p.cnt_row;
    if (max_proj > maxcnt) maxcnt = max_proj;
    if (p.cnt_bp > maxcnt) maxcnt = p.cnt_bp;
    p.partials = take(sizeof(double) * kSlots * (size_t)maxcnt);
    p.part_cap = maxcnt;
    p.proj_items = take(sizeof(Item) * (size_t)max_proj);
    p.maps = take(kMapBytes * SB_COUNT);          // TMA maps of the sinogram views (kAlign >= 128)
    p.counter = take(sizeof(unsigned) * 4);
    p.view_rm = take(2 * tsize * (size_t)N * p.S);
    p.view_cm = take(2 * tsize * (size_t)N * p.S);
    const size_t sino_bytes = 2 * tsize * (size_t)na * p.SB;
    for (int q = 0; q < IB_COUNT; ++q) p.img[q] = (size_t)-1;
    for (int q = 0; q < SB_COUNT; ++q) p.sino[q] = (size_t)-1;
    for (int q = 0; q < 4; ++q) p.dual[q] = (size_t)-1;
    if (kind == PLAN_OP) {
        p.trace = (size_t)-1;
        p.sino[SB_R] = take(sino_bytes);
    } else {
        p.trace = take(sizeof(double) * TR_NF * kMaxTraceRows);
        const int fam = family_of(variant);
        if (fam == FAM_FISTA) {                 // x in three slots, b, A^T r, the dual fields, A x in three slots
            p.img[IB_X] = take(tsize * J);
            p.img[IB_XH] = take(tsize * J);
            p.img[IB_P] = take(tsize * J);
            p.img[IB_H] = take(tsize * J);
            p.img[IB_G] = take(tsize * J);
            p.img[IB_Z] = take(tsize * J);
            for (int q = 0; q < 4; ++q) p.dual[q] = take(2 * tsize * J);
            p.sino[SB_R] = take(sino_bytes);
            p.sino[SB_Q] = take(sino_bytes);
            p.sino[SB_W] = take(sino_bytes);
            p.sino[SB_V] = take(sino_bytes);
            p.total = off;
            return p;
        }
        p.img[IB_X] = take(tsize * J);
        p.img[IB_P] = take(tsize * J);
        p.img[IB_H] = take(tsize * J);
        p.img[IB_G] = take(tsize * J);
        if (fam != FAM_CG) {
            p.img[IB_XH] = take(tsize * J);
            p.img[IB_TVG] = take(tsize * J);
        }
        if (uses_filter(variant)) p.img[IB_Z] = take(tsize * J);
        if (prox_duals && fam != FAM_CG)
            for (int q = 0; q < 4; ++q) p.dual[q] = take(2 * tsize * J);
        p.sino[SB_R] = take(sino_bytes);
        p.sino[SB_Q] = take(sino_bytes);
        if (uses_filter(variant)) p.sino[SB_W] = take(sino_bytes);
    }
    p.total = off;
    return p;
}

// Per-angle constants; `scale` multiplies every chord (1/m), i.e. A -> scale A.
// Entry a describes angle a_begin + a of a scan of na_total angles (a block of
// consecutive angles for an angle-sharded operator; by default the whole scan).
template <typename T>
void fill_angles(std::vector<Angle<T>>& out, int na, int n, double scale = 1.0, int a_begin = 0,
                 int na_total = -1) {
    out.resize(na);
    if (na_total < 0) na_total = na;
    const double off_n = 0.5 * (n - 1);
    for (int a = 0; a < na; ++a) {
        const int ga = a_begin + a;
        double c, s;
        if (ga == 0) { c = 1.0; s = 0.0; }
        else if (2 * ga == na_total) { c = 0.0; s = 1.0; }
        else {
            // past pi/2 through cos(pi - t) = -cos t, sin(pi - t) = sin t, so that
            // theta and pi - theta are exact mirrors (as the oracle computes them)
            const bool mirror = 2 * ga > na_total;
            const double th = M_PI * (double)(mirror ? na_total - ga : ga) / (double)na_total;
            c = mirror ? -cos(th) : cos(th);
            s = sin(th);
        }
        const double ac = fabs(c), as = fabs(s);
        const double m = ac > as ? ac : as, mn = ac > as ? as : ac;
        const double hs = 0.5 * (m + mn);
        Angle<T> g;
        memset(&g, 0, sizeof(g));
        g.c = (T)c;
        g.s = (T)s;
        g.inv_m = (T)(scale / m);
        g.m_w = (T)(m / scale);
        if (mn == 0.0) {
            g.k2 = (T)1.0; g.h2 = (T)1.0; g.h2p = (T)2.0;
            g.kb = (T)1.0; g.hb0 = (T)1.0; g.hb1 = (T)0.0;
            g.hb0p = (T)2.0; g.hb1p = (T)-1.0;
        } else {
            g.k2 = (T)(m / mn); g.h2 = (T)(hs / mn); g.h2p = (T)(hs / mn + m / mn);
            g.kb = (T)(1.0 / mn); g.hb0 = (T)(hs / mn); g.hb1 = (T)((hs - 1.0) / mn);
            g.hb0p = (T)(hs / mn + 1.0 / mn); g.hb1p = (T)((hs - 1.0) / mn - 1.0 / mn);
        }
        g.c23 = (int)llrint(c * 8388608.0);
        g.s23 = (int)llrint(s * 8388608.0);
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

// Projector work list, longest blocks first.  The blocks of one launch differ
// widely in work -- rays near the ends of the detector are short or miss the
// image -- and in block-index order long blocks are still starting when most
// SMs have run out of work (about a fifth of the launch at 512^2 / 720 x 725,
// 3.4 waves).  Handing the blocks out longest first (list scheduling) ends the
// launch close to the mean load of an SM.  A block's cost is the number of
// strips its warps walk: each warp walks the union of its rays' strip ranges in
// lockstep, in whole pairs, plus a fixed set-up cost.  Only the order changes:
// every item keeps its block index (local), so the partial sums are added in
// the same order and the results are bit-identical to the block-index order.
struct ProjOrder {
    std::vector<Item> items;    // longest first
};
constexpr int kWarpSetupStrips = 12;

inline ProjOrder make_proj_order(int n, int nb, int shift, const std::vector<Angle<double>>& ang) {
    const int na = (int)ang.size();
    const int lab = kProjLog2 - shift, law = lab < 2 ? lab : 2, lrw = 5 - law, lwpr = shift - lrw;
    const int ablocks = (na + (1 << lab) - 1) >> lab, bblocks = (nb + (1 << shift) - 1) >> shift;
    // strip range [lo, hi] of every ray: -1 <= c0 + t slope < n, 0 <= t < n
    std::vector<int> lo((size_t)na * nb), hi((size_t)na * nb);
    for (int a = 0; a < na; ++a) {
        const Angle<double>& g = ang[a];
        for (int b = 0; b < nb; ++b) {
            const double c0 = ((double)b - 0.5 * (nb - 1)) * g.inv_d + g.c0_off_d;
            double t0 = 0.0, t1 = n - 1.0;
            if (g.slope_d == 0.0) {
                if (!(c0 >= -1.0 && c0 < (double)n)) { t0 = 1.0; t1 = 0.0; }
            } else {
                const double ta = (-1.0 - c0) / g.slope_d, tb = ((double)n - c0) / g.slope_d;
                t0 = std::max(t0, ceil(std::min(ta, tb)));
                t1 = std::min(t1, floor(std::max(ta, tb)));
            }
            const size_t q = (size_t)a * nb + b;
            if (t0 > t1) { lo[q] = 1; hi[q] = 0; }
            else { lo[q] = (int)t0; hi[q] = (int)t1; }
        }
    }
    ProjOrder o;
    const int cnt = ablocks * bblocks;
    std::vector<std::pair<float, int>> by_cost(cnt);
    for (int u = 0; u < ablocks; ++u)
        for (int v = 0; v < bblocks; ++v) {
            float c = 0.f;
            for (int w = 0; w < kProjThreads / 32; ++w) {
                int mlo = 1 << 30, mhi = -1;
                for (int lane = 0; lane < 32; ++lane) {
                    const int a = (u << lab) + ((w >> lwpr) << law) + (lane >> lrw);
                    const int b = (v << shift) + ((w & ((1 << lwpr) - 1)) << lrw) + (lane & ((1 << lrw) - 1));
                    if (a >= na || b >= nb) continue;
                    const size_t q = (size_t)a * nb + b;
                    if (lo[q] > hi[q]) continue;
                    mlo = std::min(mlo, lo[q]);
                    mhi = std::max(mhi, hi[q]);
                }
                c += mhi < mlo ? 1.f : (float)((mhi | 1) - (mlo & ~1) + 1 + kWarpSetupStrips);
            }
            by_cost[u * bblocks + v] = {c, u * bblocks + v};
        }
    std::stable_sort(by_cost.begin(), by_cost.end(),
                     [](const std::pair<float, int>& x, const std::pair<float, int>& y) { return x.first > y.first; });
    o.items.resize(cnt);
    for (int k = 0; k < cnt; ++k) {
        const int q = by_cost[k].second;
        o.items[k] = Item{0, q / bblocks, q % bblocks, q};
    }
    return o;
}

template <typename T>
Prob<T> make_prob(const scg_geometry& g, const Plan& pl, unsigned char* base, double scale = 1.0) {
    using E = typename Tr<T>::S;
    using E2 = typename Tr<T>::S2;
    using C = typename Tr<T>::C;
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
    P.proj_shift = pl.proj_shift;
    P.cnt_bp = pl.cnt_bp;
    P.bp_mirror = pl.bp_mirror;
    P.P = pl.P;
    P.off_n = (C)(0.5 * (g.n - 1));
    P.off_b = (C)(0.5 * (g.n_bins - 1));
    P.y_scale = (C)scale;
    P.ang = reinterpret_cast<const Angle<C>*>(base + pl.ang);
    P.taps = reinterpret_cast<const C*>(base + pl.taps);
    for (int q = 0; q < IB_COUNT; ++q)
        P.img[q] = pl.img[q] == (size_t)-1 ? nullptr : reinterpret_cast<E*>(base + pl.img[q]);
    for (int q = 0; q < SB_COUNT; ++q)
        P.sino[q] = pl.sino[q] == (size_t)-1 ? nullptr : reinterpret_cast<E2*>(base + pl.sino[q]);
    for (int q = 0; q < 4; ++q)
        P.dual[q] = pl.dual[q] == (size_t)-1 ? nullptr : reinterpret_cast<E2*>(base + pl.dual[q]);
    P.view_rm = reinterpret_cast<E2*>(base + pl.view_rm);
    P.view_cm = reinterpret_cast<E2*>(base + pl.view_cm);
    P.partials = reinterpret_cast<double*>(base + pl.partials);
    P.part_cap = pl.part_cap;
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

// cuTensorMapEncodeTiled, resolved once through the runtime's driver entry
// point (no link against the driver library); null if unavailable.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn tensor_map_encoder();
bool test_stall_copies();             // scg_test_stall_copies's setting

// TMA maps of a problem's sinogram views, written to base + pl.maps and
// pointed to by P.sino_map (FP32 and 16-bit storage; the FP64 gather copies
// with cp.async and gets none).  Map q describes sino[q] as na rows of SB
// pairs, each pair one 8-byte (FP32) or 4-byte (16-bit) element; a box is one
// row of band_slots pairs, the gather's band of one angle.  Elements outside
// the view read as zero, as the band's zero-fill requires.  Call after every
// change of the sinogram views' addresses (a map holds the address).
template <typename T>
int upload_sino_maps(Prob<T>& P, const Plan& pl, unsigned char* base, cudaStream_t s) {
    P.sino_map = nullptr;
    if constexpr (!std::is_same<T, double>::value) {
        using S2 = typename Tr<T>::S2;
        static_assert(sizeof(CUtensorMap) == kMapBytes, "one map per 128 bytes");
        const EncodeTiledFn enc = tensor_map_encoder();
        if (!enc) return SCG_ERR_CUDA;
        CUtensorMap maps[SB_COUNT];
        memset(maps, 0, sizeof(maps));
        for (int q = 0; q < SB_COUNT; ++q) {
            if (!P.sino[q]) continue;
            const cuuint64_t dims[2] = {(cuuint64_t)P.SB, (cuuint64_t)P.na};
            const cuuint64_t strides[1] = {(cuuint64_t)P.SB * sizeof(S2)};
            // (under scg_test_stall_copies the box is 16 bytes narrower than the
            // band the gather's barrier expects, so no chunk's bytes ever add up)
            const cuuint32_t box[2] = {(cuuint32_t)(band_slots<S2>() - (test_stall_copies() ? 16 / (int)sizeof(S2) : 0)),
                                       1u};
            const cuuint32_t estr[2] = {1u, 1u};
            const CUresult r = enc(&maps[q], sizeof(S2) == 8 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32,
                                   2, (void*)P.sino[q], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return SCG_ERR_CUDA;
        }
        CK(cudaMemcpyAsync(base + pl.maps, maps, sizeof(maps), cudaMemcpyHostToDevice, s));
        P.sino_map = base + pl.maps;
    }
    return SCG_OK;
}

// The projector work list of one geometry and shape (make_proj_order), cached
// for the life of the process; a_begin / na_total as for fill_angles.
std::shared_ptr<const ProjOrder> proj_order(int n, int na, int nb, int shift, int a_begin = 0, int na_total = -1);

// Writes the work list of shape pl.proj_shift to dst (a device array of
// pl.cnt_proj items, normally base + pl.proj_items).
inline int upload_proj_order(const Plan& pl, void* dst, const scg_geometry& g, cudaStream_t s, int a_begin = 0,
                             int na_total = -1) {
    const auto o = proj_order(g.n, g.n_angles, g.n_bins, pl.proj_shift, a_begin, na_total);
    if ((int)o->items.size() != pl.cnt_proj) return SCG_ERR_INVALID;
    CK(cudaMemcpyAsync(dst, o->items.data(), sizeof(Item) * o->items.size(), cudaMemcpyHostToDevice, s));
    return SCG_OK;
}

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
    int g_bp = 0;                      // backprojector tiles
    const Item* i_bp = nullptr;
    void project(int dst, int mode, int step) { ++launches; launch_project<T>(d, i_proj, g_proj, dst, mode, step, s); }
    void back1(int src, int dst, int step) { ++launches; launch_backproject<T>(d, i_bp, g_bp, 1, src, src, dst, dst, step, s); }
    void back2(int s0, int s1, int d0, int d1, int step) { ++launches; launch_backproject<T>(d, i_bp, g_bp, 2, s0, s1, d0, d1, step, s); }
    void vec(int op, int sel, int step) { ++launches; launch_vec<T>(d, i_img, g_img, op, sel, step, s); }
    void tvgrad(int src, int fuse, int wg, int step) { ++launches; launch_tvgrad<T>(d, i_img, g_img, src, fuse, wg, step, s); }
    void trial(int ncand) { ++launches; launch_trial<T>(d, i_bp, g_bp, ncand, s); }
    void axpy(int step) { ++launches; launch_sino_axpy<T>(d, i_ray, g_ray, step, s); }
    void filter(int src, int dst) { ++launches; launch_filter<T>(d, i_row, g_row, nb, src, dst, FILT_VIEW, s); }
    void sino_comb(int cur, int prev) { ++launches; launch_sino_comb<T>(d, i_ray, g_ray, cur, prev, s); }
    void fgp(int j, double beta, int mode = 0) { ++launches; launch_fgp<T>(d, i_img, g_img, j, beta, mode, s); }
    void fgp2(int p, double b0, double b1, int mode) { ++launches; launch_fgp2<T>(d, i_img, g_img, p, b0, b1, mode, s); }
    void sino_norm(int src, int step) { ++launches; launch_sino_norm<T>(d, i_ray, g_ray, src, step, s); }
};

struct Program {
    int variant, trial_passes, ksteps;
    bool eta;          // Appendix rule: the gradient at x_k sizes the perturbation
    bool prox;         // proximal perturbation (S-variants): x_{k+1/2} = prox_{lambda_k TV}(x_k)
    int prox_iters;    // FISTA and the proximal perturbation: FGP steps per prox (0: no prox)
    int pert_steps;    // perturbations per step (S-variants, gamma and prox rules; 1 otherwise)
};

// g'^T p' for the step length: FIN_BETA derives it from the gradient pass's
// sums (-g'^T d + beta g'^T p, exact for the unrounded p'); with 16-bit
// storage p' is rounded to 11 or 8 bits, and the dot is taken again on the
// stored p' when it is formed, so that alpha is the exact line search along
// the direction actually used.
template <typename T>
constexpr int num_step() { return sizeof(typename Tr<T>::S) < 4 ? FIN_NUM : FIN_NONE; }

// Power iteration for c^2 = ||A^T A||_2 (Appendix, Eq. lambda and Eq. gamma):
// p <- A^T A p / ||A^T A p|| from the start vector 1 + 0.001 (index mod 7);
// the device keeps the Rayleigh quotient p^T A^T A p / ||p||^2 as c^2.
template <typename T>
void run_power(Runner<T>& R, int iters) {
    R.vec(VEC_POWER_START, 0, FIN_POWER_NORM);
    for (int q = 0; q < iters; ++q) {
        R.project(SB_Q, PROJ_PLAIN, FIN_NONE);         // A p (views written by the vector pass)
        R.back1(SB_Q, IB_H, FIN_NONE);                 // h = A^T A p
        R.vec(VEC_POWER_DOTS, 0, FIN_POWER);           // c^2 = p^T h / ||p||^2, 1/||h||
        R.vec(VEC_NORMALIZE, 0, FIN_POWER_NORM);       // p = h / ||h||
    }
}

// The FGP steps of one TV prox (momentum (t_j - 1)/t_{j+1}, t_1 = 1), two per
// launch (k_fgp2) and a last single step when the count is odd; mode 0 is
// FISTA's prox, 1 the proximal perturbation.  Returns the dual buffer (0 or 1)
// that holds the final w, or 2 if no step was taken.
template <typename T>
int run_fgp(Runner<T>& R, int iters, int mode) {
    double t = 1.0;
    int p = 0;                                        // launch index: selects the buffers
    for (int j = 0; j < iters; ++p) {
        const double t1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        const double b0 = (t - 1.0) / t1;
        t = t1;
        if (j + 1 < iters) {
            const double t2 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
            const double b1 = (t - 1.0) / t2;
            t = t2;
            R.fgp2(p, b0, b1, mode);
            j += 2;
        } else {
            R.fgp(p, b0, mode);
            j += 1;
        }
    }
    return p > 0 ? (p - 1) & 1 : 2;
}

// FISTA (Eq. FISTA, Eq. FISTA-u): x_0 is projected once; each iteration forms
// A u_k - y from the two latest residuals, backprojects it, takes the gradient
// step, the prox by FGP, and projects x_k (its residual r_k = A x_k - y, the
// stop test, t_{k+1}, beta_k).  x_k lives in kFistaX[k % 3] and r_k in
// kFistaQ[k % 3]; a loop body holds three iterations so that every buffer
// choice is static.
template <typename T>
void run_fista_iteration(Runner<T>& R, const Program& pg, int k3) {
    const int cur = (k3 + 2) % 3, prev = (k3 + 1) % 3;    // x_{k-1}, x_{k-2}
    R.sino_comb(kFistaQ[cur], kFistaQ[prev]);          // A u_k - y = (1 + beta) r_{k-1} - beta r_{k-2}
    R.back1(SB_R, IB_G, FIN_NONE);                     // A^T (A u_k - y)
    R.vec(VEC_FISTA_B, kFistaX[cur] | (kFistaX[prev] << 4), FIN_NONE);   // b = u_k - A^T(A u_k - y)/c^2
    const int w = run_fgp<T>(R, pg.prox_iters, 0);    // FGP on the prox's dual
    R.vec(VEC_FGP_FINAL, kFistaX[k3] | (w << 4), FIN_NONE);              // x_k = prox(b), views
    R.project(kFistaQ[k3], PROJ_RESIDUAL, FIN_NONE);  // r_k = A x_k - y
    R.sino_norm(kFistaQ[k3], FIN_FISTA_F);             // f(x_k): stop test, t_{k+1}, beta_k
}

// The algorithms' set-up steps (before the first loop test).
template <typename T>
void run_init(Runner<T>& R, const Program& pg) {
    const int v = pg.variant, fam = family_of(v);
    const bool pre = uses_filter(v);
    const int dsel = pre ? IB_Z : IB_G;
    if (fam == FAM_FISTA) {
        R.vec(VEC_INIT, 0, FIN_NONE);                  // x_0 (u_1 = x_0), views
        R.project(kFistaQ[0], PROJ_RESIDUAL, FIN_NONE);  // r_0 = A x_0 - y
        R.sino_norm(kFistaQ[0], FIN_FISTA_F);          // f(x_0): first loop test
        return;
    }
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
    R.vec(VEC_FORM_P0, dsel, num_step<T>());           // p0 = -g0 (-z0) (g0^T p0: see num_step)
    R.project(SB_Q, PROJ_PLAIN, FIN_NONE);             // A p0
    R.back1(SB_Q, IB_H, FIN_ALPHA);                    // h0 = A^T A p0, alpha
    R.tvgrad(IB_X, 1, 1, FIN_END);                     // x1 = x0 + alpha p0 (+ dTV(x1)); k = 1; loop test
}

// One loop body of the variant's while loop (FISTA: three iterations).
template <typename T>
void run_body(Runner<T>& R, const Program& pg) {
    const int v = pg.variant, fam = family_of(v);
    const bool pre = uses_filter(v);
    const int dsel = pre ? IB_Z : IB_G;
    if (fam == FAM_FISTA) {
        for (int k3 = 1; k3 <= 3; ++k3) run_fista_iteration<T>(R, pg, k3 % 3);
        return;
    }
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
    for (int sub = 0; sub < pg.pert_steps; ++sub) {
        if (sub > 0) {                                 // the next perturbation starts from x_{k+1/2}
            R.vec(VEC_COPY_HALF, 0, FIN_NONE);         // (x_k is not used again in the step)
            R.tvgrad(IB_X, 0, 1, FIN_PERTURB_NEXT);    // its TV and subgradient; trial set-up
        }
        if (pg.prox) {                                 // x_{k+1/2} = prox_{lambda_k TV}(x_k): FGP from a zero dual
            const int w = run_fgp<T>(R, pg.prox_iters, 1);
            R.vec(VEC_FGP_FINAL, IB_XH | (w << 4) | (1 << 8), FIN_PROX_END);   // x_{k+1/2}, views; l <- l+1
        } else {
            for (int t = 0; t < pg.trial_passes; ++t)     // TV trials of x_k + gamma_l v
                R.trial(t == 0 ? kTrialsFirst : kTrials);
            if (pg.eta) {                              // ||g_k||, g_k = A^T (A x_k - y)
                R.vec(VEC_VIEWS, IB_X, FIN_NONE);
                R.project(SB_R, PROJ_RESIDUAL, FIN_NONE);
                R.back1(SB_R, IB_G, FIN_NONE);
                R.vec(VEC_NORM_G, 0, FIN_ETA_SIZE);
            }
            R.vec(VEC_PERTURB, 0, FIN_NONE);           // x_{k+1/2} = perturbed(x_k)
        }
    }
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
    R.vec(VEC_FORM_P, dsel, num_step<T>());            // p' = -g' (-z') + beta p (g'^T p': see num_step)
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

// ---------------------------------------------------------------------------
// Projector block-shape tuner.  The best shape depends on the geometry (how
// long the rays are, how many angles share image spans); it is measured once
// per geometry bucket (two buckets per octave of N, n_angles and n_bins) and
// precision on each device, and cached for the life of the process.  The
// choice changes only the block decomposition: every ray's value is computed
// identically, and only the order in which the blocks' partial sums of r^2 are
// added differs.  FP64 solves keep the default shape.
int proj_shape_lookup(int dev, int precision, const scg_geometry& g);   // -1 if not tuned
void proj_shape_store(int dev, int precision, const scg_geometry& g, int shift);

// Time the candidate shapes on problem slot d (a solve plan, DevState not
// stopped, angles uploaded; the SB_Q view is overwritten), each launched over
// its longest-first work list in order_dst (pl.cnt_proj items of the problem's
// workspace), and leave the best shape in P, pl and the slot and its list in
// order_dst.  order_dst = nullptr: blocks in index order, no list (batched
// launches, whose many problems' blocks already fill the last wave).
template <typename T>
int tune_proj_shape(Prob<T>& P, Plan& pl, Prob<T>* d, const scg_geometry& g, cudaStream_t s, Item* order_dst,
                    int forced = 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SCG_ERR_CUDA;
    int best = prec_of<T>() == SCG_F64 ? kProjShiftDefault : proj_shape_lookup(dev, prec_of<T>(), g);
    if (forced >= kProjShiftMin && forced <= kProjShiftMax) best = forced;     // the caller's shape
    if (best < 0) {
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) != cudaSuccess) return SCG_ERR_CUDA;
        if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return SCG_ERR_CUDA; }
        float best_ms = 1e30f;
        for (int sh = kProjShiftMin; sh <= kProjShiftMax; ++sh) {
            set_proj_shape(pl, g.n_angles, g.n_bins, sh);
            P.cnt_proj = pl.cnt_proj; P.proj_blocks = pl.proj_blocks; P.proj_shift = sh;
            if (cudaMemcpyAsync(d, &P, sizeof(P), cudaMemcpyHostToDevice, s) != cudaSuccess) break;
            if (order_dst && upload_proj_order(pl, order_dst, g, s) != SCG_OK) break;
            launch_project<T>(d, order_dst, pl.cnt_proj, SB_Q, PROJ_PLAIN, FIN_NONE, s);
            cudaEventRecord(e0, s);
            for (int r = 0; r < 3; ++r) launch_project<T>(d, order_dst, pl.cnt_proj, SB_Q, PROJ_PLAIN, FIN_NONE, s);
            cudaEventRecord(e1, s);
            float ms = 1e30f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) break;
            if (ms < best_ms) { best_ms = ms; best = sh; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (cudaGetLastError() != cudaSuccess || best < 0) return SCG_ERR_CUDA;
        proj_shape_store(dev, prec_of<T>(), g, best);
    }
    set_proj_shape(pl, g.n_angles, g.n_bins, best);
    P.cnt_proj = pl.cnt_proj; P.proj_blocks = pl.proj_blocks; P.proj_shift = best;
    if (cudaMemcpyAsync(d, &P, sizeof(P), cudaMemcpyHostToDevice, s) != cudaSuccess) return SCG_ERR_CUDA;
    return order_dst ? upload_proj_order(pl, order_dst, g, s) : SCG_OK;
}

// Initial device state of one solve.
inline DevState initial_state(const scg_params* prm, double eps, int variant) {
    DevState st;
    memset(&st, 0, sizeof(st));
    const int fam = family_of(variant);
    st.eps = eps;
    st.max_iter = prm->max_iter;
    st.perturb = prm->perturb;
    st.gamma0 = prm->gamma0 > 0.0 ? prm->gamma0 : 0.0;
    st.gamma_fixed = prm->gamma0 > 0.0 ? 1 : 0;
    st.gamma0_rel = prm->gamma0_rel;
    st.a = prm->a;
    st.a_ell = 1.0;                                  // ell = 0
    if (prm->perturb == SCG_PERTURB_ETA || fam == FAM_FISTA) {   // no gamma trials: the table holds these
        st.ex.eta0 = prm->eta0;
        st.ex.lam = prm->lambda;
        st.ex.c2 = prm->lipschitz > 0.0 ? prm->lipschitz : 0.0;
        st.ex.tk = 1.0;
    } else {
        st.apow[0] = 1.0;
        for (int t = 1; t < kTrials; ++t) st.apow[t] = st.apow[t - 1] * prm->a;
    }
    st.max_trials = prm->max_trials;
    st.variant = variant;
    st.family = fam;
    st.in_init = 1;
    st.k = (fam == FAM_S_PR) ? 1 : 0;
    return st;
}

inline Program make_program(const scg_params* prm, int variant) {
    Program pg;
    pg.variant = variant;
    pg.trial_passes = prm->perturb == SCG_PERTURB_GAMMA ? trial_passes_for(prm->max_trials) : 0;
    pg.ksteps = prm->K + (prm->k_inclusive ? 1 : 0);
    pg.eta = prm->perturb == SCG_PERTURB_ETA && family_of(variant) != FAM_CG && family_of(variant) != FAM_FISTA;
    pg.prox = prm->perturb == SCG_PERTURB_PROX && family_of(variant) != FAM_CG && family_of(variant) != FAM_FISTA;
    if (family_of(variant) == FAM_FISTA) pg.prox_iters = prm->lambda > 0.0 ? prm->prox_iters : 0;
    else pg.prox_iters = pg.prox ? prm->prox_iters : 0;
    const bool multi = family_of(variant) != FAM_CG && family_of(variant) != FAM_FISTA &&
                       (prm->perturb == SCG_PERTURB_GAMMA || prm->perturb == SCG_PERTURB_PROX);
    pg.pert_steps = multi && prm->perturb_steps > 1 ? prm->perturb_steps : 1;
    if (family_of(variant) == FAM_FISTA) pg.trial_passes = 0;
    return pg;
}

// Work items of batched launches, one list per launch kind.  A problem's
// items keep the (u, v) and block index (local) of its own single-problem
// launch, so its reductions add in the single-problem order.
enum { K_PROJ = 0, K_IMG = 1, K_RAY = 2, K_ROW = 3, K_BP = 4, K_COUNT = 5 };

inline void append_items(const Plan& pl, int prob, std::vector<Item>* lists) {
    for (int q = 0; q < pl.cnt_proj; ++q) lists[K_PROJ].push_back(Item{prob, q / pl.proj_blocks, q % pl.proj_blocks, q});
    for (int q = 0; q < pl.cnt_img; ++q) lists[K_IMG].push_back(Item{prob, q / pl.tiles_x, q % pl.tiles_x, q});
    for (int q = 0; q < pl.cnt_ray; ++q) lists[K_RAY].push_back(Item{prob, q / pl.ray_blocks, q % pl.ray_blocks, q});
    for (int q = 0; q < pl.cnt_row; ++q) lists[K_ROW].push_back(Item{prob, q / pl.filt_blocks, q % pl.filt_blocks, q});
    for (int q = 0; q < pl.cnt_bp; ++q) lists[K_BP].push_back(Item{prob, q / pl.tiles_x, q % pl.tiles_x, q});
}

// List lengths rounded up to eight steps per octave (<= 12.5 % padding), so
// launches captured for one mix of problems serve other mixes.
inline int round_up_bucket(int n) {
    if (n <= 16) return n;
    int lg = 31 - __builtin_clz((unsigned)n);
    const int step = 1 << (lg - 3);
    return (n + step - 1) / step * step;
}

}  // namespace host
}  // namespace scg
