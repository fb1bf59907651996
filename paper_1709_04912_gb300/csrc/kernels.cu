// kernels.cu -- the CUDA kernels of the TV-superiorized CG hot path.
//
//   k_project      ray-driven forward projector A (Eq. LS1), fused residual
//                  epilogue r = Ax - y and FP64 sum of squares (f of Sec. 1)
//   k_sino_norm    ||r||^2 of a residual view (FISTA's f)
//   k_backproject  pixel-driven gather A^T (1 or 2 right-hand sides), fused
//                  FP64 inner products of Algorithms 2/4/8/10/14; with one
//                  right-hand side, 64 | N and a full angle set, a
//                  mirror-paired path (pixel (x, y) at theta and (-x, y) at
//                  pi - theta share one band index and weight pair)
//   k_vec          CG vector updates (p' = -g' + beta p, x' = x + alpha p,
//                  g' = g + alpha h), perturbation apply, projector views
//   k_tvgrad       TV, TV subgradient, ||dTV||^2, ||x||^2 (optionally fused
//                  with x_{k+1} = x_{k+1/2} + alpha p')
//   k_trial        TV of several trial points x + gamma_l v in one pass
//                  (Eq. gamma_sequence, acceptance TV(z) <= TV(x))
//   k_sino_axpy    recursive residual r' = r + alpha A p (CG/PCG)
//   k_filter       row filter of the preconditioner (Sec. 3): radix-2 FFT of
//                  two rows at once in shared memory, factors, inverse FFT
//   k_sino_pairs   a caller's plain sinogram into the pair layout
// No kernel uses atomics on data; reductions are deterministic.
#include <cstring>
#include <type_traits>

#include "scg_kernels.h"

namespace scg {

// Work item `bid` (normally the block index) of a launch: from the caller's
// item list, or computed from the single problem's shape.
template <typename T>
__device__ __forceinline__ Item decode_item(const Prob<T>* probs, const Item* items, int kind,
                                            int bid = -1) {
    if (bid < 0) bid = blockIdx.x;
    if (items) return items[bid];
    const Prob<T>& P = probs[0];
    Item it;
    it.prob = 0;
    it.local = bid;
    if (kind == 0) { it.u = bid / P.ray_blocks; it.v = bid % P.ray_blocks; }
    else if (kind == 1) { it.u = bid / P.tiles_x; it.v = bid % P.tiles_x; }
    else if (kind == 2) { it.u = bid / P.filt_blocks; it.v = bid % P.filt_blocks; }
    else if (kind == 3) { it.u = bid / P.proj_blocks; it.v = bid % P.proj_blocks; }
    else { it.u = bid / P.tiles_x; it.v = bid % P.tiles_x; }   // backprojector tiles
    return it;
}

// ---------------------------------------------------------------------------
// Forward projector.  One thread per ray (a, b); a block holds
// 2^(8-proj_shift) adjacent angles x 2^proj_shift consecutive bins, so
// sinogram writes are coalesced and the block's warps read nearly the same
// image spans.  The ray
// is walked along its driving axis (columns when |sin| >= |cos|, else rows);
// in each strip its chord is 1/m and falls on the two pixels nearest the
// crossing, split u : (1-u) by one saturating FMA of the crossing's
// fractional part (see Angle).  The two pixels are one pair-layout load from
// the view whose lines run across the driving axis.  Crossing at driving
// index t: c*(t) = c0 + t*slope, c0 = (b - (nb-1)/2) * inv_drive + c0_off.
//
// Address of the view element whose index is D's high word, formed by one wide
// integer multiply-add.  Written as plain pointer arithmetic it cost about one
// more instruction per strip on the integer ALU pipe, the pipe that bounds this
// walk (ncu on GB300 at 512^2 / 720 x 725: 5.93 -> 5.01 ALU-pipe instructions
// per strip, k_project 92.2 -> 87.0 us; the index and the data read are the same).
template <typename V2>
__device__ __forceinline__ const V2* view_at(const V2* view, long long D) {
    const V2* p;
    asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(p) : "r"((int)(D >> 32)), "n"((int)sizeof(V2)), "l"(view));
    return p;
}

// FP32 walk: c* is carried in 32.32 fixed point C, so every increment is
// exact; the high word is floor(c*) and the fraction's top 23 bits become a
// float in [1, 2) as the mantissa under the exponent of 1 (an add of the
// shifted word, which cannot carry into the exponent).
// D carries the view element index of the pair at the crossing in its high
// word (line t*S, pad kPad, floor(c*)) and the crossing's fraction in its low
// word; adding DL = slope + S (both in 32.32) steps to the next strip.
// The walk is software-pipelined in three register groups of four strips that
// take turns: a strip's weight is formed when its load is issued (so its 32.32
// position dies at once), and while two groups' loads are in flight the third
// group is summed.  Every index read lies inside
// the view because [tlo, thi] holds exactly the strips whose crossing
// satisfies -1 <= floor(c*) <= N-1 (kPad >= 1), and no load runs ahead of
// strip n-1.
#define SCG_W(D_) __saturatef(fmaf(-__int_as_float(0x3F800000u + ((unsigned)(D_) >> 9)), k2, h2p))
#define SCG_LD(D_) to_c2(__ldg(view_at(view, (D_))))
#define SCG_ISSUE4(V_, W_)                                                     \
    V_[0] = SCG_LD(D); W_[0] = SCG_W(D); D += DL;                              \
    V_[1] = SCG_LD(D); W_[1] = SCG_W(D); D += DL;                              \
    V_[2] = SCG_LD(D); W_[2] = SCG_W(D); D += DL;                              \
    V_[3] = SCG_LD(D); W_[3] = SCG_W(D); D += DL;
#define SCG_SUM4(V_, W_)                                                       \
    u0 = fmaf(W_[0], V_[0].x - V_[0].y, u0); y0 += V_[0].y;                    \
    u1 = fmaf(W_[1], V_[1].x - V_[1].y, u1); y1 += V_[1].y;                    \
    u0 = fmaf(W_[2], V_[2].x - V_[2].y, u0); y0 += V_[2].y;                    \
    u1 = fmaf(W_[3], V_[3].x - V_[3].y, u1); y1 += V_[3].y;
// Sums go to two accumulator pairs by the parity of the ABSOLUTE strip index
// (u0, y0: even strips; u1, y1: odd), each receiving its strips in increasing
// order, so a ray's value does not depend on how its strips are split between
// the unmasked walk and the masked edges (that split follows the warp's lanes).
// The walk starts on an even strip, and groups start at multiples of four.
template <typename V2>
__device__ __forceinline__ void walk_ray_f32(const V2* view, int n, long long D, long long DL,
                                             float k2, float h2p, float& u0, float& u1, float& y0, float& y1) {
    int t = 0;
    float2 va[4], vb[4], vc[4];
    float wa[4], wb[4], wc[4];
    if (n >= 8) {
        // at the top of each iteration group a holds strips t-8 .. t-5 and
        // group b t-4 .. t-1 (issued), and D is strip t
        SCG_ISSUE4(va, wa)
        SCG_ISSUE4(vb, wb)
        for (t = 8; t + 12 <= n; t += 12) {
            SCG_ISSUE4(vc, wc)
            SCG_SUM4(va, wa)
            SCG_ISSUE4(va, wa)
            SCG_SUM4(vb, wb)
            SCG_ISSUE4(vb, wb)
            SCG_SUM4(vc, wc)
        }
        SCG_SUM4(va, wa)
        SCG_SUM4(vb, wb)
    }
    // fewer than 12 strips left (t a multiple of four): whole groups, then the rest
    for (; t + 4 <= n; t += 4) {
        SCG_ISSUE4(vc, wc)
        SCG_SUM4(vc, wc)
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        vc[k] = t + k < n ? SCG_LD(D) : make_float2(0.f, 0.f);
        wc[k] = SCG_W(D);
        D += DL;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
        if (t + k < n) {
            if (k & 1) { u1 = fmaf(wc[k], vc[k].x - vc[k].y, u1); y1 += vc[k].y; }
            else { u0 = fmaf(wc[k], vc[k].x - vc[k].y, u0); y0 += vc[k].y; }
        }
}
#undef SCG_ISSUE4
#undef SCG_SUM4
#undef SCG_W
#undef SCG_LD

// Strips t in [0, N) whose crossing C(t) = C0 + t*SL (32.32) has floor in
// [-1, N-1]: a FP32 estimate, then corrected exactly in integer arithmetic.
__device__ __forceinline__ void walk_range(long long C0, long long SL, int N, float c0f, float inv_slope,
                                           int& tlo, int& thi) {
    const long long lo = -(1LL << 32), hi = (long long)N << 32;   // valid: lo <= C < hi
    auto ok = [&](int t) { const long long C = C0 + (long long)t * SL; return C >= lo && C < hi; };
    if (SL == 0) {
        tlo = 0;
        thi = (C0 >= lo && C0 < hi) ? N - 1 : -1;
        return;
    }
    const float ta = (-1.f - c0f) * inv_slope, tb = ((float)N - c0f) * inv_slope;
    tlo = max(0, min(N, (int)floorf(fminf(ta, tb))));
    thi = min(N - 1, max(-1, (int)floorf(fmaxf(ta, tb)) + 1));
    for (int q = 0; q < 3 && tlo <= thi && !ok(tlo); ++q) ++tlo;
    for (int q = 0; q < 3 && tlo > 0 && ok(tlo - 1); ++q) --tlo;
    for (int q = 0; q < 3 && thi >= tlo && !ok(thi); ++q) --thi;
    for (int q = 0; q < 3 && thi < N - 1 && ok(thi + 1); ++q) ++thi;
    // after the corrections every t in [tlo, thi] is valid (the valid set is
    // an interval and both ends were checked); anything left unconfirmed is
    // dropped rather than read out of range
    if (tlo > thi || !ok(tlo) || !ok(thi)) { tlo = 0; thi = -1; }
}

// FP32 arithmetic (float, half and bfloat16 storage).  The 32 rays of a warp
// walk the same absolute strip t together: the lanes' loads then fall in one
// line of the view, a short contiguous span (walking each ray from its own
// first strip puts the lanes in different lines wherever rays enter through
// the image's far sides).  Strips are taken in pairs (even t, t+1).  The pairs
// inside every non-empty lane's range [tlo, thi] run unmasked through the
// pipelined walk; the pairs before and after run masked, each lane loading
// only inside its own range (a masked strip adds an exact zero).  A lane with
// no strip (ray misses the image, or past the last bin) walks element kPad of
// each line of the warp's union -- always in bounds -- and discards the sum.
// Every lane of the warp must call this (warp shuffles).
template <typename T>
__device__ __forceinline__ float project_ray_f32(const Prob<T>& P, const Angle<float>& g, int b, bool valid) {
    const int N = P.n, B2 = 2 * b - (P.nb - 1);           // 2 (b - (nb-1)/2)
    const long long C0 = (((long long)B2 * g.inv_fx) >> 1) + g.c0_off_fx;
    const float c0f = fmaf(0.5f * (float)B2, g.inv_drive, g.c0_off);
    int tlo = 0, thi = -1;
    if (valid) walk_range(C0, g.slope_fx, N, c0f, g.inv_slope, tlo, thi);
    const bool empty = thi < tlo;
    int mlo = empty ? 0x7fffffff : tlo, mhi = empty ? -1 : thi;          // union of the lanes' ranges
    int ilo = empty ? -1 : tlo, ihi = empty ? 0x7fffffff : thi;          // intersection (non-empty lanes)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mlo = min(mlo, __shfl_xor_sync(0xffffffffu, mlo, o));
        mhi = max(mhi, __shfl_xor_sync(0xffffffffu, mhi, o));
        ilo = max(ilo, __shfl_xor_sync(0xffffffffu, ilo, o));
        ihi = min(ihi, __shfl_xor_sync(0xffffffffu, ihi, o));
    }
    if (mhi < mlo) return 0.f;                            // the whole warp misses the image
    mlo &= ~1;                                            // first pair
    ilo += ilo & 1;                                       // whole pairs inside the intersection
    ihi -= (ihi & 1) ^ 1;
    const int mend = mhi | 1;                             // last strip of the last pair
    const bool shared = ilo < ihi;
    const int m0 = shared ? ilo : mend + 1, m1 = shared ? ihi : mend;   // unmasked pairs [m0, m1]
    const long long S32 = (long long)P.S << 32;
    const long long DL = empty ? S32 : g.slope_fx + S32;
    long long D = (empty ? 0 : C0 + (long long)mlo * g.slope_fx) + (long long)mlo * S32 + ((long long)kPad << 32);
    const auto* view = g.col_driven ? P.view_cm : P.view_rm;
    const float k2 = g.k2, h2p = g.h2p;
    const int lo = empty ? mlo : tlo;                     // the strips this lane loads: [lo, lo + span]
    const unsigned span = empty ? (unsigned)(mhi - mlo) : (unsigned)(thi - tlo);
    float uE = 0.f, uO = 0.f, yE = 0.f, yO = 0.f;        // even / odd strips (see walk_ray_f32)
    auto edge = [&](int t, int tend) {                    // pairs [t, tend), masked
        for (; t < tend; t += 2, D += 2 * DL) {
            const long long D1 = D + DL;
            const float2 v0 = (unsigned)(t - lo) <= span ? to_c2(__ldg(view_at(view, D))) : make_float2(0.f, 0.f);
            const float2 v1 = (unsigned)(t + 1 - lo) <= span ? to_c2(__ldg(view_at(view, D1))) : make_float2(0.f, 0.f);
            uE = fmaf(__saturatef(fmaf(-__int_as_float(0x3F800000u + ((unsigned)D >> 9)), k2, h2p)), v0.x - v0.y, uE);
            yE += v0.y;
            uO = fmaf(__saturatef(fmaf(-__int_as_float(0x3F800000u + ((unsigned)D1 >> 9)), k2, h2p)), v1.x - v1.y, uO);
            yO += v1.y;
        }
    };
    edge(mlo, m0);
    if (shared) {
        const int n = m1 - m0 + 1;
        walk_ray_f32(view, n, D, DL, k2, h2p, uE, uO, yE, yO);
        D += (long long)n * DL;
    }
    edge(m1 + 1, mend + 1);
    return empty ? 0.f : ((uE + uO) + (yE + yO)) * g.inv_m;
}

__device__ __forceinline__ double project_ray_f64(const Prob<double>& P, const Angle<double>& g, int b) {
    const int N = P.n;
    const double c0d = fma((double)b - 0.5 * (double)(P.nb - 1), g.inv_d, g.c0_off_d);
    int tlo = 0, thi = N - 1;
    if (g.slope_d == 0.0) {
        if (!(c0d >= -1.5 && c0d <= (double)N + 0.5)) thi = -1;
    } else {
        const double t1 = (-1.5 - c0d) / g.slope_d, t2 = ((double)N + 0.5 - c0d) / g.slope_d;
        const double lo = fmax(fmin(t1, t2), -1.0), hi = fmin(fmax(t1, t2), (double)N);
        tlo = max(0, (int)floor(lo));
        thi = min(N - 1, (int)floor(hi) + 1);
    }
    const double c0i = floor(c0d);
    const double c0f = c0d - c0i;
    const int cbase = (int)c0i + kPad;
    const unsigned top = (unsigned)(N + 2 * kPad - 2);
    const double2* line = (g.col_driven ? P.view_cm : P.view_rm) + (size_t)tlo * P.S;
    double acc = 0.0;
    for (int t = tlo; t <= thi; ++t, line += P.S) {
        const double cs = fma((double)t, g.slope_d, c0f);
        const double fl = floor(cs);
        const unsigned sl = min((unsigned)((int)fl + cbase), top);
        const double2 v = __ldg(line + sl);
        acc += fma(sat(fma(fl - cs, g.k2, g.h2)), v.x - v.y, v.y);
    }
    return acc * g.inv_m;
}

template <typename T>
__device__ __forceinline__ typename Tr<T>::C project_ray(const Prob<T>& P, const Angle<typename Tr<T>::C>& g, int b,
                                                         bool valid) {
    if constexpr (std::is_same<T, double>::value) return valid ? project_ray_f64(P, g, b) : 0.0;
    else return project_ray_f32(P, g, b, valid);
}

// Resident projector blocks per SM the register allocation is sized for: at
// 4 (64 registers) the walk keeps more loads in flight than at 5 (48), which
// measured 15-20 % slower on GB300 at 512^2 and 1024^2.
constexpr int kProjMinBlocks = 4;

// One block: 2^(8-proj_shift) adjacent angles x 2^proj_shift consecutive bins
// (the shape is tuned per geometry on the host).  Rays of neighbouring angles
// cross the image almost together, so the warps of a block read nearly the
// same view spans and most of those reads hit L1.
template <typename T>
__global__ void __launch_bounds__(kProjThreads, kProjMinBlocks)
k_project(const Prob<T>* __restrict__ probs, const Item* __restrict__ items, int dst_sel,
          int mode, int step) {
    const Item it = decode_item(probs, items, 3);
    const Prob<T>& P = probs[it.prob];
    if (P.st->done) return;
    const int nb = P.nb;
    // block: AB = 2^(8-sh) angles x R = 2^sh rays; warp: AW adjacent angles x
    // 32/AW consecutive rays (AW = min(4, AB)), so the lanes' rays cross the
    // image close together and their loads share cache lines
    const int sh = P.proj_shift;
    const int lab = kProjLog2 - sh;                      // log2 angles per block
    const int law = lab < 2 ? lab : 2;                   // log2 angles per warp
    const int lrw = 5 - law;                             // log2 rays per warp
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lwpr = sh - lrw;                           // log2 warps along the rays
    const int a = (it.u << lab) + ((warp >> lwpr) << law) + (lane >> lrw);
    const int b = (it.v << sh) + ((warp & ((1 << lwpr) - 1)) << lrw) + (lane & ((1 << lrw) - 1));
    using C = typename Tr<T>::C;
    Acc<T> v[1];
    acc_zero(v[0]);
    const bool valid = a < P.na && b < nb;
    const Angle<C> g = P.ang[valid ? a : 0];
    // the residual's data value, loaded before the walk so that its latency is
    // hidden (y_scale is 1 except for half/bfloat16 storage; the product is exact)
    C yv = C(0);
    if (valid && mode == PROJ_RESIDUAL) yv = to_c(P.y[(size_t)a * nb + b]) * P.y_scale;
    C out = project_ray<T>(P, g, b, valid);                // every lane: the FP32 walk is warp-wide
    if (valid) {
        if (mode == PROJ_RESIDUAL) out = out - yv;
        if (mode == PROJ_PLAIN_OUT) P.user_out[(size_t)a * nb + b] = to_s<typename Tr<T>::S>(out);
        else store_pair<T>(P.sino[dst_sel] + (size_t)a * P.SB + kSPad, b, out * g.inv_m);   // weighted view
        v[0] = acc_prod(out, out);
    }
    if (step != FIN_NONE) reduce_and_finalize<T, 1, true>(v, P, it.local, P.cnt_proj, step);
}

// ---------------------------------------------------------------------------
// Backprojector: a 32 x TH tile per cluster of CL blocks of 128 threads, PIX
// pixels per thread (rows ty, ty + TH/PIX, ...), each block 1/CL of the
// angles.  A pixel whose centre projects to bin coordinate cb can only meet
// bins floor(cb) and floor(cb)+1
// ((m+n)/2 <= 1/sqrt(2)); their weights are two saturating FMAs of cb's
// fractional part (see Angle), and the two bins are one pair-layout load.  The
// sinogram views hold r[a,b] / m_a (the chord factor 1/m of the angle is
// applied when a view is written), so the gather is two FMAs per pixel.
//
// Angles are processed in chunks.  For each angle the band of sinogram pairs
// the tile can touch is copied into shared memory with cp.async,
// double-buffered so the next chunk's copies overlap this chunk's arithmetic;
// parts of a band beyond the detector are zero-filled by the copy itself, so
// the inner loop needs no bounds test.  A band starts at the slot of
// floor(projection of the tile origin) + floor(31 min(c, 0)) - 1, rounded
// down to a 16-byte boundary (g slots of g = 16 / sizeof(pair)), and the
// tile's pixels then reach at most 31 (|c| + |s|) + g + 2 < 44 + g + 2 slots
// further (|c| + |s| <= sqrt 2, 32 x 32 tile): kBand = 48 slots for FP32
// pairs (g = 2), 52 for 16-bit pairs (g = 4).  The projection of the tile's
// first pixel comes from 32.32 fixed point (FP64 in the FP64 kernel), split
// into integer + fraction; each pixel adds only its small in-tile offset
// (9.23 fixed point in the FP32 kernel: the fraction bits are directly a
// float mantissa).
// Tile height, pixels per thread, angles per chunk, and blocks per tile (CL
// blocks -- a thread-block cluster -- take consecutive parts of the angles of
// one tile; blocks 1..CL-1 hand their sums to block 0 through distributed
// shared memory).  32 x 32 tiles with 8 pixels per thread spread each angle's
// set-up (row of constants, tile-origin position, chunk copies) over twice
// the pixels of 32 x 16 tiles; four blocks per tile keep 1024 blocks in
// flight at 512^2.  Measured on GB300 (one right-hand side): 32 x 16 tiles in
// clusters of 2 -> 32 x 32 in clusters of 4: 97.8 -> 86.1 us at 512^2 / 720
// angles, 664 -> 610 us at 1024^2 / 1440 ...
template <typename T, int NRHS> struct BpCfg {
    static constexpr int TH = kBpTileH32, PIX = 8, CL = 4;
    // the hand-over of three blocks' sums reuses the band storage
    static constexpr int CH = (NRHS == 1 || sizeof(typename Tr<T>::S2) == 4) ? 32 : 16;
};
// ... and FP64 (48 KB static shared memory)
template <int NRHS> struct BpCfg<double, NRHS> {
    static constexpr int TH = kBpTileH64, PIX = 2, CH = 8, CL = 1;
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// TMA and mbarrier (FP32 / 16-bit gather).  One mbarrier per band buffer, one
// arrival (the expect_tx of the chunk's bytes) per phase.
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned mb) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned mb, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes) : "memory");
}
// Waits for the phase of the given parity to complete, for at most about
// 2^28 SM cycles (~0.13 s); returns false if the wait ran out.
__device__ __forceinline__ bool mbar_wait(unsigned mb, unsigned parity) {
    const long long t0 = clock64();
    for (;;) {
        unsigned done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(mb), "r"(parity) : "memory");
        if (done) return true;
        if (clock64() - t0 > (1LL << 28)) return false;
    }
}
// One box of a 2-D tensor map (x innermost, in elements) into shared memory,
// completing its bytes on mbarrier mb.
__device__ __forceinline__ void tma_load_2d(unsigned dst, const void* map, int x, int y, unsigned mb) {
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                 ::"r"(dst), "l"(map), "r"(x), "r"(y), "r"(mb) : "memory");
}

// Per-slot row of the mirror-paired gather (below): an angle a and its mirror.
struct __align__(16) BpRowM {
    int baseA, baseB;    // band index of the tile's origin in windows A and B, in 9.23 fixed point
    int c23, s23;        // cos, sin of angle a in 9.23
    float kb, hb0p, hb1p;
    int pad_;
};
constexpr int kBpMirrorCH = 8;    // slots per chunk of the mirror-paired gather
constexpr int kBpMirrorNB = 4;    // bands per slot

// Per-angle row of the FP32 gather (two 16-byte shared loads).
struct __align__(16) BpRowF {
    int base;        // band index of the tile origin's projection, in 9.23 fixed point
    int c23, s23;    // cos, sin in 9.23
    float kb, hb0p, hb1p;
    int pad_[2];
};
// Per-angle row of the FP64 gather.
struct __align__(16) BpRowD {
    double c, s, kb, hb0, hb1, frac;
    int rel;
};

// Tile origin projection (integer part I and fraction) for one angle:
// off_b + xc0 c + yc0 s with xc0 = X2/2, yc0 = Y2/2, in 32.32 fixed point.
__device__ __forceinline__ long long tile_origin_fx(const Angle<float>& g, int X2, int Y2, int nb) {
    return ((long long)(nb - 1) << 31) + (((long long)X2 * g.c_fx + (long long)Y2 * g.s_fx) >> 1);
}

// ---------------------------------------------------------------------------
// Mirror-paired gather (FP32 arithmetic, one right-hand side; N a multiple of
// 64 and a scan's full angle set).  Pixel (x, y) at angle theta and pixel
// (-x, y) at pi - theta project to the same detector position (cos(pi - t) =
// -cos t, sin(pi - t) = sin t; the angle table holds these mirrors exactly),
// so one band index and one pair of weights serve both.  A work item is a
// 32 x 16 tile T of the image's left half together with its mirror image T'
// in the right half, four pixels of each per thread.  Angles come in slots:
// angle 0, the pairs (a, na - a) for 0 < a < na/2, and angle na/2 when na is
// even.  For a slot (a, a') and a thread's pixel p of T (mirror p' of T'):
//   window A = the positions of T at angle a:        p at a,  p' at a'
//   window B = the positions of T at the mirror of a: p at a', p' at a
// so a slot stages four bands (rows a and a' over each window) and takes two
// weight evaluations and four pair loads per pixel pair, where the plain
// gather takes four evaluations.  A slot with a single angle (0, na/2) has no
// second row: the two bands of the missing row are zero-filled in shared
// memory, so every slot takes the same path.  Item q is the plain gather's item q (64 | N makes
// the counts equal: (N/64) x (N/16) = (N/32)^2), so work lists and partial
// sums are shared with it, and a batch or a server step mixes problems of
// either path in one launch (each problem always takes the same one, so its
// result does not depend on its company); bands arrive by TMA as in the plain
// gather, four boxes per slot, eight slots per chunk, in the plain gather's
// shared storage (the same number of band bytes).  Called by the plain
// gather's blocks for a problem with bp_mirror set.
template <typename T>
__device__ __forceinline__ void backproject_mirror(const Prob<T>& P, const Item& it, int part, int src, int dst,
                                                   int step, void* rows_smem, void* band_smem,
                                                   unsigned long long* mbar) {
    using S2 = typename Tr<T>::S2;
    using C = typename Tr<T>::C;
    static_assert(std::is_same<C, float>::value, "FP32 arithmetic");
    constexpr int TH = 16, PIX = 4, kStep = TH / PIX, CH = kBpMirrorCH, CL = 4, NB = kBpMirrorNB;
    static_assert(kTileW * kStep == kBackThreads && kBackThreads == 128, "one thread per column and row group");
    static_assert(CH * NB == 32, "one box per staging lane: lanes 0..7 of the four warps");
    constexpr int kBand = band_slots<S2>();
    constexpr int kSlotsPerSeg = 16 / (int)sizeof(S2);
    constexpr int kBandS = (kBand * (int)sizeof(S2) + 127) / 128 * 128 / (int)sizeof(S2);
    constexpr unsigned kBoxBytes = (unsigned)(kBand * (int)sizeof(S2));
    using Row = BpRowM;
    Row (&rows)[2][CH] = *reinterpret_cast<Row(*)[2][CH]>(rows_smem);
    // bands: a over A, a' over A, a' over B, a over B
    S2 (&band)[2][CH][NB][kBandS] = *reinterpret_cast<S2(*)[2][CH][NB][kBandS]>(band_smem);
    const int N = P.n, na = P.na, nb = P.nb;
    const int tl = threadIdx.x, tx = tl % kTileW, ty = tl / kTileW;
    const int mcols = N / 64;                    // left-half tile columns
    const int i0 = (it.local / mcols) * TH, j0 = (it.local % mcols) * kTileW;
    const int X2 = 2 * j0 - (N - 1), Y2 = 2 * i0 - (N - 1);
    const int npairs = (na - 1) / 2;             // slots 1..npairs: (a, na - a)
    const int nslots = npairs + 1 + ((na & 1) ? 0 : 1);
    const int nsp = (nslots + CL - 1) / CL;      // slots of each block
    const int s_begin = min(nslots, part * nsp), s_end = min(nslots, s_begin + nsp);
    const int nchunks = (nsp + CH - 1) / CH;     // the same for every block of the cluster
    const unsigned char* map = P.sino_map + (size_t)src * kSinoMapBytes;

    bool ok = true;                              // every wait of this thread on its block's copies completed
    // Rows and bands of chunk ch: lane l < 8 of warp w takes box b = 8 w + l,
    // slot b / 4 of the chunk, band b % 4.  A lane of window B places T at the
    // mirror of a (cos -> -cos, in 32.32 fixed point: exact); box origin = the
    // window's first slot, rounded down to a 16-byte boundary as TMA requires.
    // Thread 0 adds the chunk's TMA bytes to the barrier's expected count (a
    // copy may complete first; the phase still ends only after that arrival).
    auto stage = [&](int ch) {
        const int buf = ch & 1;
        const int s0 = s_begin + ch * CH;
        const int cnt = min(CH, s_end - s0);             // may be <= 0 (a part with no slots)
        if (tl == 0 && ok) {
            int single = 0;                              // slots of one angle in this chunk (two boxes fewer each)
            if (cnt > 0 && s0 == 0) ++single;
            if (cnt > 0 && (na & 1) == 0 && s0 <= npairs + 1 && npairs + 1 < s0 + cnt) ++single;
            mbar_expect_tx(smem_addr(&mbar[buf]), cnt > 0 ? (unsigned)(cnt * NB - 2 * single) * kBoxBytes : 0u);
        }
        const int lane = tl & 31;
        const int b = (tl >> 5) * 8 + lane;
        const int q = b >> 2, which = b & 3;
        if (lane < 8 && q < cnt) {
            const int sl = s0 + q;
            const bool pair = sl >= 1 && sl <= npairs;
            const int a = sl <= npairs ? sl : na / 2;
            const Angle<C> g = P.ang[a];
            const bool wB = which >= 2;
            const long long cfx = wB ? -g.c_fx : g.c_fx;
            const long long cb = ((long long)(nb - 1) << 31) + (((long long)X2 * cfx + (long long)Y2 * g.s_fx) >> 1);
            const int lo = (int)floorf((float)(kTileW - 1) * fminf(wB ? -g.c : g.c, 0.f)) - 1;
            const int I = (int)(cb >> 32);
            const int s_lo = (I + kSPad + lo) & ~(kSlotsPerSeg - 1);
            const int base = ((I + kSPad - s_lo) << 23) | (int)((unsigned)cb >> 9);
            Row& r = rows[buf][q];
            if (which == 0) {
                r.baseA = base;
                r.c23 = g.c23; r.s23 = g.s23;
                r.kb = g.kb; r.hb0p = g.hb0p; r.hb1p = g.hb1p;
                r.pad_ = 0;
            } else if (which == 2) {
                r.baseB = base;
            }
            S2* dstb = &band[buf][q][which][0];
            if (pair || which == 0 || which == 3) {
                // this buffer was last read through the generic proxy (before the
                // block barrier that ended that chunk); order those reads first
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                tma_load_2d(smem_addr(dstb), map, s_lo, (which == 0 || which == 3) ? a : na - a, smem_addr(&mbar[buf]));
            } else {
                // no second angle: zeros (visible to the block after the barrier
                // that ends the current chunk)
                uint4* z = reinterpret_cast<uint4*>(dstb);
                for (int k = 0; k < kBand * (int)sizeof(S2) / 16; ++k) z[k] = make_uint4(0u, 0u, 0u, 0u);
            }
        }
    };

    float acc[2 * PIX];                          // p (rows ty + 4k of T), then p' (the same rows of T')
#pragma unroll
    for (int k = 0; k < 2 * PIX; ++k) acc[k] = 0.f;
    if (tl == 0) {
        mbar_init(smem_addr(&mbar[0]));
        mbar_init(smem_addr(&mbar[1]));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    stage(0);
    __syncthreads();
    for (int ch = 0; ch < nchunks; ++ch) {
        // stage the next chunk (into the other buffer, free since the barrier
        // that ended the previous chunk), then wait for this chunk's bands --
        // always, even after a wait ran out, so that no copy is in flight when
        // the block ends
        if (ch + 1 < nchunks) stage(ch + 1);
        const bool w = mbar_wait(smem_addr(&mbar[ch & 1]), (unsigned)((ch >> 1) & 1));
        ok = ok && w;
        const int cnt = min(CH, s_end - (s_begin + ch * CH));
        const int buf = ch & 1;
        if (ok) {
#pragma unroll 2
            for (int q = 0; q < cnt; ++q) {
                const Row r = rows[buf][q];
                // 9.23 positions of the thread's first pixel in windows A and B (> 0)
                const int pA0 = r.baseA + tx * r.c23 + ty * r.s23;
                const int pB0 = r.baseB - tx * r.c23 + ty * r.s23;
                const int dp = kStep * r.s23;
                const S2* bq = &band[buf][q][0][0];
#pragma unroll
                for (int k = 0; k < PIX; ++k) {
                    const int pA = pA0 + k * dp, pB = pB0 + k * dp;
                    // 1 + fraction as a float in [1, 2): the fraction bits are the mantissa
                    const float fA = __int_as_float(0x3F800000 | ((unsigned)pA & 0x7FFFFFu));
                    const float fB = __int_as_float(0x3F800000 | ((unsigned)pB & 0x7FFFFFu));
                    const float wA0 = __saturatef(fmaf(-fA, r.kb, r.hb0p)), wA1 = __saturatef(fmaf(fA, r.kb, r.hb1p));
                    const float wB0 = __saturatef(fmaf(-fB, r.kb, r.hb0p)), wB1 = __saturatef(fmaf(fB, r.kb, r.hb1p));
                    const int iA = pA >> 23, iB = pB >> 23;
                    const float2 e0 = to_c2(bq[iA]);                 // row a,  window A: p  at a
                    const float2 e1 = to_c2(bq[kBandS + iA]);        // row a', window A: p' at a'
                    const float2 e2 = to_c2(bq[2 * kBandS + iB]);    // row a', window B: p  at a'
                    const float2 e3 = to_c2(bq[3 * kBandS + iB]);    // row a,  window B: p' at a
                    acc[k] = fmaf(wA0, e0.x, fmaf(wA1, e0.y, acc[k]));
                    acc[PIX + k] = fmaf(wA0, e1.x, fmaf(wA1, e1.y, acc[PIX + k]));
                    acc[k] = fmaf(wB0, e2.x, fmaf(wB1, e2.y, acc[k]));
                    acc[PIX + k] = fmaf(wB0, e3.x, fmaf(wB1, e3.y, acc[PIX + k]));
                }
            }
        }
        __syncthreads();
    }
    if (!ok) atomicExch(&P.st->dev_error, 1);     // a band never arrived: the sums are not valid
    // pixel k of this thread: row i0 + ty + 4 (k % PIX), column j0 + tx (k < PIX)
    // or its mirror N - 1 - j0 - tx
    auto pix = [&](int k) {
        const int i = i0 + ty + (k % PIX) * kStep;
        const int j = k < PIX ? j0 + tx : N - 1 - j0 - tx;
        return (size_t)i * N + j;
    };
    // block 0's epilogue operands (h and p for the fused dots), loaded before
    // the cluster barriers so that their latency overlaps the hand-over
    const bool want_h = step == FIN_BETA;
    const bool want_p = step == FIN_BETA || step == FIN_ALPHA || step == FIN_CG_ALPHA;
    C hv[2 * PIX], pv[2 * PIX];
#pragma unroll
    for (int k = 0; k < 2 * PIX; ++k) {
        const size_t idx = pix(k);
        hv[k] = part == 0 && want_h ? to_c(P.img[IB_H][idx]) : C(0);
        pv[k] = part == 0 && want_p ? to_c(P.img[IB_P][idx]) : C(0);
    }
    // blocks 1..3 write their sums into block 0's band storage (free once every
    // block of the cluster has passed the first cluster barrier; release /
    // acquire), and block 0 adds them in rank order after the second
    float* xs = reinterpret_cast<float*>(&band[0][0][0][0]);
    static_assert(sizeof(float) * (CL - 1) * 2 * PIX * kBackThreads <= sizeof(band), "hand-over fits");
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    if (part != 0) {
        const unsigned local = (unsigned)__cvta_generic_to_shared(&xs[tl]);
        unsigned remote;
        asm volatile("mapa.shared::cluster.u32 %0, %1, 0;" : "=r"(remote) : "r"(local));
#pragma unroll
        for (int k = 0; k < 2 * PIX; ++k)
            asm volatile("st.shared::cluster.f32 [%0], %1;"
                         ::"r"(remote + (unsigned)(sizeof(float) * ((part - 1) * 2 * PIX + k) * kBackThreads)),
                         "f"(acc[k]) : "memory");
    }
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    if (part != 0) return;
#pragma unroll
    for (int r = 1; r < CL; ++r)
#pragma unroll
        for (int k = 0; k < 2 * PIX; ++k) acc[k] = acc[k] + xs[((r - 1) * 2 * PIX + k) * kBackThreads + tl];
    using S = typename Tr<T>::S;
    Acc<T> v[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) acc_zero(v[q]);
#pragma unroll
    for (int k = 0; k < 2 * PIX; ++k) {
        const size_t idx = pix(k);
        // stored values are rounded to the storage format; the dots use them
        const C g0 = rnd<T>(acc[k]);
        P.img[dst][idx] = to_s<S>(g0);
        if (step == FIN_BETA) {
            v[0] = acc_add(v[0], acc_prod(g0, hv[k]));               // g'^T h
            v[1] = acc_add(v[1], acc_prod(g0, g0));                  // ||g'||^2
            v[2] = acc_add(v[2], acc_prod(g0, pv[k]));               // g'^T p
        } else if (step == FIN_ALPHA || step == FIN_CG_ALPHA) {
            v[0] = acc_add(v[0], acc_prod(pv[k], g0));               // p^T h
        } else if (step == FIN_CG_DELTA) {
            v[0] = acc_add(v[0], acc_prod(g0, g0));                  // ||g||^2
            v[1] = acc_add(v[1], acc_prod(g0, g0));                  // g^T z (z = g)
        }
    }
    if (step == FIN_NONE) return;
    reduce_and_finalize<T, 3>(v, P, it.local, P.cnt_bp, step);
}

// Gather blocks per SM the register allocation is sized for: seven with one
// right-hand side (72 registers; at 512^2 the 1024 blocks then run in one wave
// on 152 SMs), six with two, whose sums need more registers.
template <int NRHS> constexpr int back_min_blocks() { return NRHS == 1 ? 7 : 6; }

template <typename T, int NRHS>
__global__ void __launch_bounds__(kBackThreads, back_min_blocks<NRHS>())
k_backproject(const Prob<T>* __restrict__ probs, const Item* __restrict__ items, int src0,
              int src1, int dst0, int dst1, int step) {
    using S2 = typename Tr<T>::S2;
    using C = typename Tr<T>::C;
    using Row = typename std::conditional<std::is_same<C, float>::value, BpRowF, BpRowD>::type;
    constexpr bool kF32 = std::is_same<C, float>::value;
    constexpr int TH = BpCfg<T, NRHS>::TH, PIX = BpCfg<T, NRHS>::PIX, CH = BpCfg<T, NRHS>::CH;
    constexpr int CL = BpCfg<T, NRHS>::CL;
    constexpr int kStep = TH / PIX;                   // rows between a thread's pixels
    static_assert(kTileW * kStep == kBackThreads, "one thread per column and row group");
    constexpr int kBand = band_slots<S2>();
    constexpr int kSlotsPerSeg = 16 / (int)sizeof(S2);
    static_assert(kBand % kSlotsPerSeg == 0, "whole 16-byte copies");
    constexpr int kSegs = kBand / kSlotsPerSeg;       // 16-byte copies per band
    // launched in clusters of CL blocks along x: block rank blockIdx.x % CL
    const int part = (int)(blockIdx.x % CL);
    const Item it = decode_item(probs, items, 4, (int)(blockIdx.x / CL));
    const Prob<T>& P = probs[it.prob];
    if (P.st->done) return;                      // the same flag for every block of a cluster
    // FP32 / 16-bit: bands arrive by TMA, one box (one angle row of kBand pairs)
    // per angle into a row padded to 128 bytes; FP64: cp.async, 16 bytes a copy
    constexpr int kBandS = kF32 ? (kBand * (int)sizeof(S2) + 127) / 128 * 128 / (int)sizeof(S2) : kBand;
    __shared__ Row rows[2][CH];
    __shared__ int slo[2][CH];                   // first slot of each band in its sinogram row (FP64)
    __shared__ __align__(128) S2 band[2][NRHS][CH][kBandS];
    __shared__ __align__(8) unsigned long long mbar[2];   // TMA completion per band buffer
    if constexpr (kF32 && NRHS == 1) {
        if (P.bp_mirror) {
            static_assert(sizeof(rows) >= 2 * kBpMirrorCH * sizeof(BpRowM) &&
                          sizeof(band) >= 2 * kBpMirrorCH * kBpMirrorNB * kBandS * sizeof(S2),
                          "the mirror-paired path fits the plain gather's storage");
            backproject_mirror<T>(P, it, part, src0, dst0, step, &rows[0][0], &band[0][0][0][0], mbar);
            return;
        }
    }
    const int N = P.n, na = P.na, nb = P.nb, SB = P.SB;
    const int tl = threadIdx.x;
    const int nap = (na + CL - 1) / CL;          // angles of each block
    const int a_begin = min(na, part * nap), a_end = min(na, a_begin + nap);
    const int ti0 = it.u * TH, tj0 = it.v * kTileW;
    const int tx = tl % kTileW, ty = tl / kTileW;
    const int j = tj0 + tx;
    const int X2 = 2 * tj0 - (N - 1), Y2 = 2 * ti0 - (N - 1);
    const S2* R[2] = {P.sino[src0], NRHS == 2 ? P.sino[src1] : P.sino[src0]};
    const int nchunks = (nap + CH - 1) / CH;     // the same for every block of the cluster

    // FP64: the row constants of chunk ch (threads q < CH) for the cp.async copies
    auto stage_rows = [&](int ch) {
        if constexpr (!kF32) {
            const int q = tl;
            const int a = a_begin + ch * CH + q;
            if (q < CH && a < a_end) {
                const Angle<C> g = P.ang[a];
                // band: slots the tile can touch, from floor(projection of the origin)
                // + floor((kTileW-1) min(c, 0)) - 1, rounded down to a 16-byte boundary
                const int lo = (int)tfloor(C(kTileW - 1) * tmin(g.c, C(0))) - 1;
                const double cbt = 0.5 * (double)(nb - 1) + 0.5 * (double)X2 * g.c_d + 0.5 * (double)Y2 * g.s_d;
                const double fl = floor(cbt);
                const int I = (int)fl;
                const int s_lo = (I + kSPad + lo) & ~(kSlotsPerSeg - 1);
                BpRowD r;
                r.c = g.c; r.s = g.s; r.kb = g.kb; r.hb0 = g.hb0; r.hb1 = g.hb1;
                r.frac = cbt - fl;
                r.rel = I + kSPad - s_lo;
                rows[ch & 1][q] = r;
                slo[ch & 1][q] = s_lo;
            }
        }
    };
    bool ok = true;                              // every wait of this thread on its block's copies completed
    // FP32 / 16-bit: the row constants of chunk ch and the TMA copies of its
    // bands, spread over the block: lanes 0..CH/4-1 of warp w take the chunk's
    // angles w*CH/4 .. (w+1)*CH/4-1 (box origin: the band's first slot, rounded
    // down to a 16-byte boundary as TMA requires; slots beyond the row read as
    // zero).  Thread 0 adds the chunk's bytes to the barrier's expected count;
    // a copy may complete before that (the count may go below zero), and the
    // phase still ends only after thread 0's arrival.
    auto stage_tma = [&](int ch) {
        if constexpr (kF32) {
            constexpr int kPerWarp = CH / 4;
            static_assert(kBackThreads == 128 && CH % 4 == 0, "four warps share a chunk's rows");
            const int buf = ch & 1;
            const int a0 = a_begin + ch * CH;
            const int cnt = min(CH, a_end - a0);          // may be <= 0 (a part with no angles)
            const unsigned mb = smem_addr(&mbar[buf]);
            // (only while thread 0's own waits all completed: a barrier phase is the
            // same for every thread, so it never arrives twice in one phase)
            if (tl == 0 && ok) mbar_expect_tx(mb, cnt > 0 ? (unsigned)(cnt * NRHS * kBand * (int)sizeof(S2)) : 0u);
            const int lane = tl & 31;
            const int q = (tl >> 5) * kPerWarp + lane;
            if (lane < kPerWarp && q < cnt) {
                const Angle<C> g = P.ang[a0 + q];
                const int lo = (int)tfloor(C(kTileW - 1) * tmin(g.c, C(0))) - 1;
                const long long cb = tile_origin_fx(g, X2, Y2, nb);
                const int I = (int)(cb >> 32);
                const int s_lo = (I + kSPad + lo) & ~(kSlotsPerSeg - 1);
                BpRowF r;
                r.base = ((I + kSPad - s_lo) << 23) | (int)((unsigned)cb >> 9);
                r.c23 = g.c23; r.s23 = g.s23;
                r.kb = g.kb; r.hb0p = g.hb0p; r.hb1p = g.hb1p;
                r.pad_[0] = r.pad_[1] = 0;
                rows[buf][q] = r;
                // this buffer was last read through the generic proxy (before the
                // block barrier that ended that chunk); order those reads first
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
#pragma unroll
                for (int h = 0; h < NRHS; ++h)
                    tma_load_2d(smem_addr(&band[buf][h][q][0]),
                                P.sino_map + (size_t)(h == 0 ? src0 : src1) * kSinoMapBytes, s_lo, a0 + q, mb);
            }
        }
    };
    auto stage_copy = [&](int ch) {
        const int a0 = a_begin + ch * CH;
        const int cnt = min(CH, a_end - a0);
#pragma unroll
        for (int h = 0; h < NRHS; ++h) {
            for (int sg = tl; sg < cnt * kSegs; sg += kBackThreads) {
                const int q = sg / kSegs, k = sg - q * kSegs;
                const int slot = slo[ch & 1][q] + k * kSlotsPerSeg;
                const S2* row = R[h] + (size_t)(a0 + q) * SB;
                const bool ok = slot >= 0 && slot + kSlotsPerSeg <= SB;
                cp_async16(&band[ch & 1][h][q][k * kSlotsPerSeg], ok ? row + slot : row, ok ? 16 : 0);
            }
        }
        cp_async_commit();
    };

    C acc[NRHS][PIX];
#pragma unroll
    for (int h = 0; h < NRHS; ++h)
#pragma unroll
        for (int k = 0; k < PIX; ++k) acc[h][k] = C(0);
    if constexpr (kF32) {
        if (tl == 0) {
            mbar_init(smem_addr(&mbar[0]));
            mbar_init(smem_addr(&mbar[1]));
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        stage_tma(0);
        __syncthreads();
    } else {
        stage_rows(0);
        __syncthreads();
        stage_copy(0);
    }
    for (int ch = 0; ch < nchunks; ++ch) {
        const bool more = ch + 1 < nchunks;
        if constexpr (kF32) {
            // stage the next chunk (rows and copies into the other buffer, free
            // since the barrier that ended the previous chunk), then wait for this
            // chunk's bands -- always, even after a wait ran out, so that no copy
            // is in flight when the block ends
            if (more) stage_tma(ch + 1);
            const bool w = mbar_wait(smem_addr(&mbar[ch & 1]), (unsigned)((ch >> 1) & 1));
            ok = ok && w;
        } else {
            if (more) stage_rows(ch + 1);
            __syncthreads();
            if (more) { stage_copy(ch + 1); cp_async_wait<1>(); }
            else cp_async_wait<0>();
            __syncthreads();
        }
        const int cnt = min(CH, a_end - (a_begin + ch * CH));
        const int buf = ch & 1;
        if (ok && j < N && ti0 + ty < N) {
            if constexpr (kF32) {
#pragma unroll 4
                for (int q = 0; q < cnt; ++q) {              // 4 angles in flight: measured 5 % faster than 2
                    const BpRowF g = rows[buf][q];
                    // 9.23 position of the thread's first pixel in band coordinates (> 0)
                    const int p0 = g.base + tx * g.c23 + ty * g.s23;
                    const int dp = kStep * g.s23;
#pragma unroll
                    for (int k = 0; k < PIX; ++k) {
                        const int p = p0 + k * dp;
                        // 1 + fraction as a float in [1, 2): the fraction bits are the mantissa
                        const float f = __int_as_float(0x3F800000 | ((unsigned)p & 0x7FFFFFu));
                        const float w0 = __saturatef(fmaf(-f, g.kb, g.hb0p));
                        const float w1 = __saturatef(fmaf(f, g.kb, g.hb1p));
#pragma unroll
                        for (int h = 0; h < NRHS; ++h) {
                            const float2 e = to_c2(band[buf][h][q][p >> 23]);
                            acc[h][k] = fmaf(w0, e.x, fmaf(w1, e.y, acc[h][k]));
                        }
                    }
                }
            } else {
                const double dj = double(tx);
                for (int q = 0; q < cnt; ++q) {
                    const BpRowD& g = *reinterpret_cast<const BpRowD*>(&rows[buf][q]);
                    const double djc = dj * g.c;
#pragma unroll
                    for (int k = 0; k < PIX; ++k) {
                        const double v = g.frac + fma(double(ty + k * kStep), g.s, djc);
                        int qi;
                        const double f = v - floor_split(v, qi);
                        const unsigned kk = min((unsigned)(qi + g.rel), (unsigned)(kBand - 2));
                        const double w0 = sat(fma(-f, g.kb, g.hb0)), w1 = sat(fma(f, g.kb, g.hb1));
#pragma unroll
                        for (int h = 0; h < NRHS; ++h) {
                            const double2 e = to_c2(band[buf][h][q][kk]);
                            acc[h][k] = fma(w0, e.x, fma(w1, e.y, acc[h][k]));
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
    if constexpr (kF32) {
        if (!ok) atomicExch(&P.st->dev_error, 1);   // a band never arrived: the sums are not valid
    }
    // block 0's epilogue operands (h and p for the fused dots), loaded before
    // the cluster barriers so that their latency overlaps the hand-over
    const bool want_h = step == FIN_BETA;
    const bool want_p = step == FIN_BETA || step == FIN_ALPHA || step == FIN_CG_ALPHA;
    C hv[PIX], pv[PIX];
#pragma unroll
    for (int k = 0; k < PIX; ++k) {
        const int i = ti0 + ty + k * kStep;
        const bool in = part == 0 && i < N && j < N;
        const size_t idx = (size_t)i * N + j;
        hv[k] = in && want_h ? to_c(P.img[IB_H][idx]) : C(0);
        pv[k] = in && want_p ? to_c(P.img[IB_P][idx]) : C(0);
    }
    if constexpr (CL > 1) {
        // blocks 1..CL-1 write their sums into block 0's band storage (free once
        // every block of the cluster has passed the first cluster barrier;
        // release / acquire), and block 0 adds them in rank order after the
        // second: first part of the angles + second + ...
        C* xs = reinterpret_cast<C*>(&band[0][0][0][0]);
        static_assert(sizeof(C) * (CL - 1) * NRHS * PIX * kBackThreads <= sizeof(band), "hand-over fits");
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
        if (part != 0) {
            const unsigned local = (unsigned)__cvta_generic_to_shared(&xs[tl]);
            unsigned remote;
            asm volatile("mapa.shared::cluster.u32 %0, %1, 0;" : "=r"(remote) : "r"(local));
#pragma unroll
            for (int h = 0; h < NRHS; ++h)
#pragma unroll
                for (int k = 0; k < PIX; ++k)
                    asm volatile("st.shared::cluster.f32 [%0], %1;"
                                 ::"r"(remote + (unsigned)(sizeof(C) * (((part - 1) * NRHS + h) * PIX + k) * kBackThreads)),
                                 "f"((float)acc[h][k]) : "memory");
        }
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
        if (part != 0) return;
#pragma unroll
        for (int r = 1; r < CL; ++r)
#pragma unroll
            for (int h = 0; h < NRHS; ++h)
#pragma unroll
                for (int k = 0; k < PIX; ++k)
                    acc[h][k] = acc[h][k] + xs[(((r - 1) * NRHS + h) * PIX + k) * kBackThreads + tl];
    }
    using S = typename Tr<T>::S;
    const int dst[2] = {dst0, dst1};
    constexpr int NSUM = NRHS == 2 ? 4 : 3;
    Acc<T> v[NSUM];
#pragma unroll
    for (int q = 0; q < NSUM; ++q) acc_zero(v[q]);
#pragma unroll
    for (int k = 0; k < PIX; ++k) {
        const int i = ti0 + ty + k * kStep;
        if (i >= N || j >= N) continue;
        const size_t idx = (size_t)i * N + j;
        // stored values are rounded to the storage format; the dots use them
#pragma unroll
        for (int h = 0; h < NRHS; ++h) {
            acc[h][k] = rnd<T>(acc[h][k]);
            P.img[dst[h]][idx] = to_s<S>(acc[h][k]);
        }
        if (step == FIN_NONE) continue;
        const C g0 = acc[0][k], g1 = acc[NRHS - 1][k];
        if (step == FIN_BETA) {
            v[0] = acc_add(v[0], acc_prod(NRHS == 2 ? g1 : g0, hv[k]));                   // g'^T h (z'^T h)
            v[1] = acc_add(v[1], acc_prod(g0, g0));                                       // ||g'||^2
            v[2] = acc_add(v[2], acc_prod(g0, pv[k]));                                    // g'^T p
            if constexpr (NRHS == 2) v[NSUM - 1] = acc_add(v[NSUM - 1], acc_prod(g0, g1)); // g'^T z'
        } else if (step == FIN_ALPHA || step == FIN_CG_ALPHA) {
            v[0] = acc_add(v[0], acc_prod(pv[k], g0));                                    // p^T h
        } else if (step == FIN_CG_DELTA) {
            v[0] = acc_add(v[0], acc_prod(g0, g0));                                       // ||g||^2
            v[1] = acc_add(v[1], acc_prod(g0, g1));                                       // g^T z
        }
    }
    if (step == FIN_NONE) return;
    reduce_and_finalize<T, NSUM>(v, P, it.local, P.cnt_bp, step);
}

// ---------------------------------------------------------------------------
// Write one tile of an image into both projector views (pair layout: each
// element is written into its own slot and the previous slot's second half).
// `val` is this thread's pixel value (ignored outside the image).
template <typename T>
__device__ __forceinline__ void write_views(const Prob<T>& P, int ti, int tj, typename Tr<T>::C val, bool in) {
    __shared__ typename Tr<T>::C tile[kTileH][kTileW + 1];
    const int ty = threadIdx.x / kTileW, tx = threadIdx.x % kTileW;
    const int i = ti * kTileH + ty, j = tj * kTileW + tx;
    if (in) store_pair<T>(P.view_rm + (size_t)i * P.S + kPad, j, val);
    tile[ty][tx] = val;
    __syncthreads();
    const int jj = threadIdx.x / kTileH, ii = threadIdx.x % kTileH;
    const int i2 = ti * kTileH + ii, j2 = tj * kTileW + jj;
    if (i2 < P.n && j2 < P.n) store_pair<T>(P.view_cm + (size_t)j2 * P.S + kPad, i2, tile[ii][jj]);
}

// Elementwise operations on one image tile (see VecOp).
template <typename T>
__global__ void __launch_bounds__(kTileThreads)
k_vec(const Prob<T>* __restrict__ probs, const Item* __restrict__ items, int op, int sel, int step) {
    const Item it = decode_item(probs, items, 1);
    const Prob<T>& P = probs[it.prob];
    const DevState& st = *P.st;
    if (st.done) return;
    const int N = P.n;
    const int i = it.u * kTileH + threadIdx.x / kTileW;
    const int j = it.v * kTileW + threadIdx.x % kTileW;
    const bool in = (i < N) && (j < N);
    const size_t idx = (size_t)i * N + j;
    using C = typename Tr<T>::C;
    using S = typename Tr<T>::S;
    // every value written is rounded to storage first (rnd: identity for
    // float/double), and the dots use the stored value
    Acc<T> v[2];
    acc_zero(v[0]);
    acc_zero(v[1]);
    C val = C(0);
    switch (op) {
    case VEC_INIT: {            // X = XH = x0 (AUX, or zeros), views of X
        const S* src = P.img[IB_AUX];
        if (in) {
            val = src ? to_c(src[idx]) : C(0);
            P.img[IB_X][idx] = to_s<S>(val);
            if (P.img[IB_XH]) P.img[IB_XH][idx] = to_s<S>(val);
        }
        write_views(P, it.u, it.v, val, in);
        break;
    }
    case VEC_VIEWS: {           // views of img[sel]
        if (in) val = to_c(P.img[sel][idx]);
        write_views(P, it.u, it.v, val, in);
        break;
    }
    case VEC_PERTURB: {         // x_{k+1/2} = x_k + coef * dTV(x_k), views
        const C coef = (C)st.coef;
        if (in) {
            const C x = to_c(P.img[IB_X][idx]);
            val = (st.accepted == 1) ? rnd<T>(fma_rn(coef, to_c(P.img[IB_TVG][idx]), x)) : x;
            P.img[IB_XH][idx] = to_s<S>(val);
        }
        write_views(P, it.u, it.v, val, in);
        break;
    }
    case VEC_FORM_P: {          // p' = -d + beta p (d = g' or z'), views; S0 = g'^T p' (if summed)
        const C beta = (C)st.beta;
        if (in) {
            const C d = to_c(P.img[sel][idx]);
            val = rnd<T>(fma(beta, to_c(P.img[IB_P][idx]), -d));
            P.img[IB_P][idx] = to_s<S>(val);
            if (step != FIN_NONE) v[0] = acc_prod(to_c(P.img[IB_G][idx]), val);
        }
        write_views(P, it.u, it.v, val, in);
        break;
    }
    case VEC_FORM_P0: {         // p_0 = -d (first direction), views; S0 = g^T p_0 (if summed)
        if (in) {
            val = -to_c(P.img[sel][idx]);
            P.img[IB_P][idx] = to_s<S>(val);
            if (step != FIN_NONE) v[0] = acc_prod(to_c(P.img[IB_G][idx]), val);
        }
        write_views(P, it.u, it.v, val, in);
        break;
    }
    case VEC_FORM_P_NOVIEW: {   // p' = -d + beta p without views (last CG-K step unused)
        const C beta = (C)st.beta;
        if (in) {
            const C d = to_c(P.img[sel][idx]);
            val = rnd<T>(fma(beta, to_c(P.img[IB_P][idx]), -d));
            P.img[IB_P][idx] = to_s<S>(val);
            v[0] = acc_prod(to_c(P.img[IB_G][idx]), val);
        }
        break;
    }
    case VEC_CG_UPDATE: {       // x' = base + alpha p, g' = g + alpha h; S0 = ||g'||^2, S1 = g'^T z
        const C alpha = (C)st.alpha;
        if (in) {
            const C base = to_c(P.img[sel][idx]);
            P.img[IB_X][idx] = to_s<S>(fma(alpha, to_c(P.img[IB_P][idx]), base));
            const C gn = rnd<T>(fma(alpha, to_c(P.img[IB_H][idx]), to_c(P.img[IB_G][idx])));
            P.img[IB_G][idx] = to_s<S>(gn);
            v[0] = acc_prod(gn, gn);
            if (P.img[IB_Z]) v[1] = acc_prod(gn, to_c(P.img[IB_Z][idx]));
        }
        break;
    }
    case VEC_DOTS_RESUME: {     // S0 = p^T h, S1 = g^T p
        if (in) {
            const C p = to_c(P.img[IB_P][idx]);
            if (P.img[IB_H]) v[0] = acc_prod(p, to_c(P.img[IB_H][idx]));
            if (P.img[IB_G]) v[1] = acc_prod(p, to_c(P.img[IB_G][idx]));
        }
        break;
    }
    case VEC_POWER_START: {     // the power iteration's start vector 1 + 0.001 (index mod 7)
        if (in) {
            val = C(1) + C(0.001) * C((int)(idx % 7));
            P.img[IB_P][idx] = to_s<S>(val);
            v[0] = acc_prod(val, val);
        }
        write_views(P, it.u, it.v, val, in);
        break;
    }
    case VEC_NORM_G: {          // S0 = ||g||^2
        if (in) {
            const C g = to_c(P.img[IB_G][idx]);
            v[0] = acc_prod(g, g);
        }
        break;
    }
    case VEC_POWER_DOTS: {      // S0 = ||h||^2, S1 = p^T h (h = A^T A p)
        if (in) {
            const C h = to_c(P.img[IB_H][idx]);
            v[0] = acc_prod(h, h);
            v[1] = acc_prod(to_c(P.img[IB_P][idx]), h);
        }
        break;
    }
    case VEC_NORMALIZE: {       // p = h / ||h||
        const C c = (C)st.coef;
        if (in) {
            val = rnd<T>(to_c(P.img[IB_H][idx]) * c);
            P.img[IB_P][idx] = to_s<S>(val);
            v[0] = acc_prod(val, val);
        }
        write_views(P, it.u, it.v, val, in);
        break;
    }
    case VEC_FISTA_B: {         // b = u_k + A^T (y - A u_k) / c^2, u_k = x_{k-1} + beta (x_{k-1} - x_{k-2})
        if (in) {
            const C xc = to_c(P.img[sel & 15][idx]), xp = to_c(P.img[sel >> 4][idx]);
            const C u = fma((C)st.beta, xc - xp, xc);
            P.img[IB_Z][idx] = to_s<S>(u - to_c(P.img[IB_G][idx]) * (C)(1.0 / st.ex.c2));
        }
        break;
    }
    case VEC_FGP_FINAL: {       // x = b - alpha L^T w: the prox of Eq. FISTA (mode 0, b = img[IB_Z],
                                // alpha = lambda / c^2) or the proximal perturbation (mode 1, b = x_k,
                                // alpha = prox_lambda); sel = output | w << 4 | mode << 8
        const int w = (sel >> 4) & 15, mode = sel >> 8;
        const double a64 = mode ? prox_lambda(st) : st.ex.lam / st.ex.c2;
        if (in) {
            val = to_c(P.img[mode ? IB_X : IB_Z][idx]);
            if (w < 2 && a64 > 0.0) {
                const auto* D = P.dual[w];
                const int m = N - 1;
                C lt = C(0);                                        // (L^T w) at pixel (i, j)
                if (i < m && j < m) { const auto e = D[idx]; lt -= to_c(e.x) + to_c(e.y); }
                if (i > 0 && j < m) lt += to_c(D[idx - N].x);
                if (j > 0 && i < m) lt += to_c(D[idx - 1].y);
                val = fma(-(C)a64, lt, val);
            }
            P.img[sel & 15][idx] = to_s<S>(val);
        }
        write_views(P, it.u, it.v, val, in);
        break;
    }
    case VEC_COPY_HALF:         // x <- x_{k+1/2} (several perturbations per step)
        if (in) P.img[IB_X][idx] = P.img[IB_XH][idx];
        break;
    case VEC_FISTA_OUT: {       // the output x_k, from the buffer of k mod 3
        if (in) {
            const int ks = st.k % 3;
            const S xv = P.img[ks == 0 ? IB_X : ks == 1 ? IB_XH : IB_P][idx];   // kFistaX[k % 3]
            P.img[IB_Z][idx] = xv;
            if (P.user_out) P.user_out[idx] = xv;
        }
        break;
    }
    default:
        break;
    }
    if (step >= kFirstRareStep) reduce_and_finalize<T, 2, false, true>(v, P, it.local, P.cnt_img, step);
    else if (step != FIN_NONE) reduce_and_finalize<T, 2>(v, P, it.local, P.cnt_img, step);
}

// ---------------------------------------------------------------------------
// TV stencil.  TV(x) = sum over interior (i,j) of ||(x[i+1,j]-x[i,j], x[i,j+1]-x[i,j])||;
// the subgradient at (i,j) collects the unit vectors of the terms (i,j),
// (i-1,j) and (i,j-1) (terms of zero norm contribute 0).  With fuse_update the
// tile first forms x_{k+1} = x_{k+1/2} + alpha p' (written to X) and takes the
// stencil of that.  src selects the image when not fused; write_grad = 0 only
// sums TV.
// Norms of the TV terms.  FP32: the hardware square-root approximations
// (relative error below 2^-22, against twice the instructions for the
// correctly rounded forms); FP64: sqrt and division, as the definition reads.
__device__ __forceinline__ float tv_norm(float v) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float tv_rsqrt(float v) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ double tv_norm(double v) { return sqrt(v); }

template <typename T>
__global__ void __launch_bounds__(kTileThreads)
k_tvgrad(const Prob<T>* __restrict__ probs, const Item* __restrict__ items, int src,
         int fuse_update, int write_grad, int step) {
    const Item it = decode_item(probs, items, 1);
    const Prob<T>& P = probs[it.prob];
    const DevState& st = *P.st;
    if (st.done) return;
    using C = typename Tr<T>::C;
    using S = typename Tr<T>::S;
    __shared__ C xs[kTileH + 2][kTileW + 3];
    __shared__ C tu[kTileH + 1][kTileW + 2];
    __shared__ C tv[kTileH + 1][kTileW + 2];
    const int N = P.n;
    const int i0 = it.u * kTileH - 1, j0 = it.v * kTileW - 1;     // smem origin
    const C alpha = (C)st.alpha;
    const S* XH = P.img[IB_XH];
    const S* PP = P.img[IB_P];
    const S* SRC = P.img[src];
    for (int q = threadIdx.x; q < (kTileH + 2) * (kTileW + 2); q += kTileThreads) {
        const int ii = q / (kTileW + 2), jj = q % (kTileW + 2);
        const int gi = i0 + ii, gj = j0 + jj;
        C val = C(0);
        if (gi >= 0 && gi < N && gj >= 0 && gj < N) {
            const size_t g = (size_t)gi * N + gj;
            // the fused x_{k+1} is rounded to storage: the stencil sees the stored x
            val = fuse_update ? rnd<T>(fma(alpha, to_c(PP[g]), to_c(XH[g]))) : to_c(SRC[g]);
        }
        xs[ii][jj] = val;
    }
    __syncthreads();
    const int ty = threadIdx.x / kTileW, tx = threadIdx.x % kTileW;
    // terms for smem rows 0..kTileH (global i0..i0+kTileH), cols 0..kTileW
    for (int q = threadIdx.x; q < (kTileH + 1) * (kTileW + 1); q += kTileThreads) {
        const int ii = q / (kTileW + 1), jj = q % (kTileW + 1);
        const int gi = i0 + ii, gj = j0 + jj;
        C a = C(0), c = C(0);
        if (gi >= 0 && gi < N - 1 && gj >= 0 && gj < N - 1) {
            const C x0 = xs[ii][jj];
            const C du = xs[ii + 1][jj] - x0, dv = xs[ii][jj + 1] - x0;
            const C n2 = du * du + dv * dv;
            if (n2 > C(0)) {
                if constexpr (std::is_same<C, double>::value) {
                    const C nrm = sqrt(n2);
                    a = du / nrm; c = dv / nrm;
                } else {
                    const C r = tv_rsqrt(n2);
                    a = du * r; c = dv * r;
                }
            }
        }
        tu[ii][jj] = a;
        tv[ii][jj] = c;
    }
    __syncthreads();
    const int i = i0 + 1 + ty, j = j0 + 1 + tx;
    const bool in = (i < N) && (j < N);
    Acc<T> v[3];
    acc_zero(v[0]); acc_zero(v[1]); acc_zero(v[2]);
    if (in) {
        const size_t g = (size_t)i * N + j;
        const C x = xs[ty + 1][tx + 1];
        if (fuse_update) P.img[IB_X][g] = to_s<S>(x);
        if (i < N - 1 && j < N - 1) {         // this tile's own term (i, j)
            const C du = xs[ty + 2][tx + 1] - x, dv = xs[ty + 1][tx + 2] - x;
            v[0] = acc_val(tv_norm(du * du + dv * dv));
        }
        const C gr = rnd<T>(-(tu[ty + 1][tx + 1] + tv[ty + 1][tx + 1]) + tu[ty][tx + 1] + tv[ty + 1][tx]);
        if (write_grad) P.img[IB_TVG][g] = to_s<S>(gr);
        v[1] = acc_prod(gr, gr);
        v[2] = acc_prod(x, x);
    }
    if (step >= kFirstRareStep) reduce_and_finalize<T, 3, true, true>(v, P, it.local, P.cnt_img, step);
    else if (step != FIN_NONE) reduce_and_finalize<T, 3, true>(v, P, it.local, P.cnt_img, step);
}

// ---------------------------------------------------------------------------
// NC trial points z_t = x + coef_t * dTV(x) (coef_t = -gamma_{l+t}/||dTV||)
// and x itself, their TVs summed in one pass over x and dTV.  A step's first
// pass tries kTrialsFirst candidates (after the first steps the first one is
// normally accepted); the passes after it, which run only while nothing has
// been accepted, try kTrials each.  The accepted point is later formed by
// k_vec(VEC_PERTURB) with the same coefficient and the same fma, so the stored
// x_{k+1/2} is exactly the point that was tested.
// Blocks take the backprojector's tiles (32 x kBpTileH, 128 threads), each
// thread TH/4 pixels of one column, so a thread adds its pixels' terms before
// the warp-level sums.  The FP32 kernel takes each term's square root with the
// hardware approximation (relative error below 2^-22, where the correctly
// rounded sqrtf costs half the pass): every TV this pass compares -- the
// candidates' and x's own -- is summed the same way, so the acceptance test
// TV(z) <= TV(x) compares like with like.
template <typename A>
__device__ __forceinline__ A ld_acc(const A* p) {
    if constexpr (std::is_same<A, double>::value) return __ldcg(p);
    else {
        const float2 w = __ldcg(reinterpret_cast<const float2*>(p));
        A r;
        r.hi = w.x; r.lo = w.y;
        return r;
    }
}

template <typename T, int NC>
__global__ void __launch_bounds__(kBackThreads)
k_trial(const Prob<T>* __restrict__ probs, const Item* __restrict__ items) {
    using A = Acc<T>;
    using C = typename Tr<T>::C;
    using S = typename Tr<T>::S;
    static_assert(NC >= 1 && NC <= kTrials, "candidates per pass");
    constexpr int NS = NC + 1;                      // candidates + x itself
    constexpr int G = NS < 8 ? NS : 8;              // sums reduced together
    static_assert(NS % G == 0, "whole groups");
    constexpr int NW = kBackThreads / 32;
    constexpr int SPW = NS / NW;                    // slots per warp in the final sum
    static_assert(SPW * NW == NS, "the final sum splits the slots evenly over the warps");
    constexpr int TH = std::is_same<T, double>::value ? kBpTileH64 : kBpTileH32;
    constexpr int PIX = TH / NW, kStep = NW;        // pixels per thread, row step
    const Item it = decode_item(probs, items, 4);
    const Prob<T>& P = probs[it.prob];
    const DevState& st = *P.st;
    if (st.done || st.accepted != 0) return;
    __shared__ A wsum[NW][NS];
    __shared__ C coef_s[NC];
    __shared__ unsigned s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < NC) coef_s[threadIdx.x] = (C)(st.trial_c0 * st.apow[threadIdx.x]);
    __syncthreads();
    const int N = P.n;
    const int j = it.v * kTileW + lane;
    C x0[PIX], xu[PIX], xv[PIX], q0[PIX], qu[PIX], qv[PIX];
    bool in[PIX];
#pragma unroll
    for (int k = 0; k < PIX; ++k) {
        const int i = it.u * TH + warp + k * kStep;
        in[k] = (i < N - 1) && (j < N - 1);
        x0[k] = xu[k] = xv[k] = q0[k] = qu[k] = qv[k] = C(0);
        if (in[k]) {
            const S* X = P.img[IB_X];
            const S* Gr = P.img[IB_TVG];
            const size_t g0 = (size_t)i * N + j;
            x0[k] = to_c(X[g0]); xu[k] = to_c(X[g0 + N]); xv[k] = to_c(X[g0 + 1]);
            q0[k] = to_c(Gr[g0]); qu[k] = to_c(Gr[g0 + N]); qv[k] = to_c(Gr[g0 + 1]);
        }
    }
#pragma unroll
    for (int grp = 0; grp < NS / G; ++grp) {
        A v[G];
#pragma unroll
        for (int kk = 0; kk < G; ++kk) {
            const int t = grp * G + kk;
            C sum = C(0);                          // this thread's pixels: non-negative terms
#pragma unroll
            for (int k = 0; k < PIX; ++k) {
                C du, dv;
                if (t < NC) {
                    // trial points as they would be stored (VEC_PERTURB rounds the same way)
                    const C c = coef_s[t];
                    const C z0 = rnd<T>(fma_rn(c, q0[k], x0[k])), zu = rnd<T>(fma_rn(c, qu[k], xu[k])),
                            zv = rnd<T>(fma_rn(c, qv[k], xv[k]));
                    du = zu - z0; dv = zv - z0;
                } else {
                    du = xu[k] - x0[k]; dv = xv[k] - x0[k];
                }
                sum += in[k] ? tv_norm(du * du + dv * dv) : C(0);
            }
            v[kk] = acc_val(sum);
        }
#pragma unroll
        for (int kk = 0; kk < G; ++kk) v[kk] = warp_sum<true>(v[kk]);
        if (lane == 0) {
#pragma unroll
            for (int kk = 0; kk < G; ++kk) wsum[warp][grp * G + kk] = v[kk];
        }
    }
    __syncthreads();
    A* parts = reinterpret_cast<A*>(P.partials);
    if (threadIdx.x < NS) {
        A b = wsum[0][threadIdx.x];
        for (int w = 1; w < NW; ++w) b = acc_add(b, wsum[w][threadIdx.x]);
        parts[(size_t)threadIdx.x * P.part_cap + it.local] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) s_last = arrive_last(P.counter, (unsigned)P.cnt_bp);
    __syncthreads();
    if (!s_last) return;
    StateCopy sc;
    sc.load(P.st);                                    // in flight during the sums below
    // last block: warp w adds slots SPW*w .. SPW*w+SPW-1 over all items (lane l
    // takes items l, l+32, ...), then across its lanes in a fixed order;
    // thread 0 collects the warps' results
    __shared__ double red[NS];
    {
        A acc[SPW];
#pragma unroll
        for (int k = 0; k < SPW; ++k) acc_zero(acc[k]);
#pragma unroll 4
        for (int q = lane; q < P.cnt_bp; q += 32) {      // loads of 4 items in flight
#pragma unroll
            for (int k = 0; k < SPW; ++k)
                acc[k] = acc_add(acc[k], ld_acc(parts + (size_t)(warp * SPW + k) * P.part_cap + q));
        }
#pragma unroll
        for (int k = 0; k < SPW; ++k) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[k] = acc_add(acc[k], acc_shfl_down(acc[k], o));
        }
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < SPW; ++k) red[warp * SPW + k] = acc_to_double(acc[k]);
        }
    }
    __shared__ DevState sst;
    sc.to_smem(sst);
    __syncthreads();
    if (threadIdx.x == 0) {
        *P.counter = 0u;
        sst.pass_cands = NC;
        finalize<T>(FIN_TRIAL, P, sst, red);          // the sums, from shared memory
    }
    __syncthreads();
    StateCopy::store(sst, P.st);
}

// ---------------------------------------------------------------------------
// r' = r + alpha q on the sinogram views; S0 = ||r'||^2.
template <typename T>
__global__ void __launch_bounds__(kRayBlock)
k_sino_axpy(const Prob<T>* __restrict__ probs, const Item* __restrict__ items, int step) {
    const Item it = decode_item(probs, items, 0);
    const Prob<T>& P = probs[it.prob];
    const DevState& st = *P.st;
    if (st.done) return;
    const int a = it.u, b = it.v * kRayBlock + threadIdx.x;
    Acc<T> v[1];
    acc_zero(v[0]);
    if (b < P.nb) {
        const size_t o = (size_t)a * P.SB + kSPad;
        // reads the first half of slot b, writes it and the second half of
        // slot b-1: no other thread touches those words
        using C = typename Tr<T>::C;
        // weighted views (r / m_a): the update is linear; ||r'||^2 unweights
        const C r = rnd<T>(fma((C)st.alpha, to_c(P.sino[SB_Q][o + b].x), to_c(P.sino[SB_R][o + b].x)));
        store_pair<T>(P.sino[SB_R] + o, b, r);
        const C ru = r * P.ang[a].m_w;
        v[0] = acc_prod(ru, ru);
    }
    reduce_and_finalize<T, 1, true>(v, P, it.local, P.cnt_ray, step);
}

// FISTA's gradient residual A u_k - y on the sinogram views, without
// projecting u_k: u_k = x_{k-1} + beta (x_{k-1} - x_{k-2}) is linear in the
// iterates, so A u_k - y = (1 + beta) r_{k-1} - beta r_{k-2} from the residuals
// r_j = A x_j - y of the two projections already taken.
template <typename T>
__global__ void __launch_bounds__(kRayBlock)
k_sino_comb(const Prob<T>* __restrict__ probs, const Item* __restrict__ items, int cur, int prev) {
    const Item it = decode_item(probs, items, 0);
    const Prob<T>& P = probs[it.prob];
    const DevState& st = *P.st;
    if (st.done) return;
    using C = typename Tr<T>::C;
    const int a = it.u, b = it.v * kRayBlock + threadIdx.x;
    if (b >= P.nb) return;
    const size_t o = (size_t)a * P.SB + kSPad;
    const C beta = (C)st.beta;
    const C qc = to_c(P.sino[cur][o + b].x), qp = to_c(P.sino[prev][o + b].x);
    store_pair<T>(P.sino[SB_R] + o, b, fma(beta, qc - qp, qc));
}

// ||r||^2 of a residual view (r / m_a stored; the chord factor is undone), for
// FISTA's f(x_k) = ||A x_k - y||^2 / 2.
template <typename T>
__global__ void __launch_bounds__(kRayBlock)
k_sino_norm(const Prob<T>* __restrict__ probs, const Item* __restrict__ items, int src, int step) {
    const Item it = decode_item(probs, items, 0);
    const Prob<T>& P = probs[it.prob];
    if (P.st->done) return;
    using C = typename Tr<T>::C;
    const int a = it.u, b = it.v * kRayBlock + threadIdx.x;
    Acc<T> v[1];
    acc_zero(v[0]);
    if (b < P.nb) {
        const C r = to_c(P.sino[src][(size_t)a * P.SB + kSPad + b].x) * P.ang[a].m_w;
        v[0] = acc_prod(r, r);
    }
    if (step >= kFirstRareStep) reduce_and_finalize<T, 1, true, true>(v, P, it.local, P.cnt_ray, step);
    else reduce_and_finalize<T, 1, true>(v, P, it.local, P.cnt_ray, step);
}

// One step of the fast gradient projection (Beck and Teboulle) for the dual
// of a TV prox at b with step alpha -- mode 0: FISTA's prox, b = img[IB_Z],
// alpha = lambda / c^2; mode 1: the proximal perturbation, b = x_k = img[IB_X],
// alpha = prox_lambda (a block with alpha = 0, zero subgradient, does nothing:
// the final pass then keeps x_k).  With r the
// momentum point, w = b - alpha L^T r at every pixel, then per interior term
// w_j = proj_{|.| <= 1}(r + L w / (8 alpha)) and the next momentum point
// r' = w_j + beta_j (w_j - w_{j-1}).  dual[j % 2] receives w_j (w_{j-1} is
// read from the other), dual[2 + (j+1) % 2] receives r' (r is read from
// dual[2 + j % 2]); step j = 0 starts from r = w_{-1} = 0.  A block takes the
// 8 x 32 terms of an image tile; r is staged with a one-term halo and w on the
// tile's pixels plus one row and column.
template <typename T>
__global__ void __launch_bounds__(kTileThreads)
k_fgp(const Prob<T>* __restrict__ probs, const Item* __restrict__ items, int j, typename Tr<T>::C beta,
      int mode) {
    using C = typename Tr<T>::C;
    using C2 = typename Vec2<C>::type;
    if constexpr (!std::is_same<typename Tr<T>::S, C>::value) {
        return;                                              // FISTA runs in FP32 / FP64 storage only
    } else {
    const Item it = decode_item(probs, items, 1);
    const Prob<T>& P = probs[it.prob];
    const DevState& st = *P.st;
    if (st.done) return;
    __shared__ C2 rs[kTileH + 2][kTileW + 2];
    __shared__ C ws[kTileH + 1][kTileW + 1];
    const int N = P.n, m = N - 1;
    const int i0 = it.u * kTileH, j0 = it.v * kTileW;
    const double a64 = mode ? prox_lambda(st) : st.ex.lam / st.ex.c2;
    if (!(a64 > 0.0)) return;
    const C alpha = (C)a64;
    const C inv8a = C(1) / (C(8) * alpha);
    const bool start = j == 0;
    const C2* R = reinterpret_cast<const C2*>(P.dual[2 + (j & 1)]);
    const C2* Wold = reinterpret_cast<const C2*>(P.dual[(j + 1) & 1]);
    C2* Wnew = reinterpret_cast<C2*>(P.dual[j & 1]);
    C2* Rnext = reinterpret_cast<C2*>(P.dual[2 + ((j + 1) & 1)]);
    // the loads that need nothing staged -- b on the w points, the previous dual
    // field at this thread's term -- are issued first, so that their latency
    // overlaps the halo's
    constexpr int kWPts = (kTileH + 1) * (kTileW + 1);
    constexpr int kWIters = (kWPts + kTileThreads - 1) / kTileThreads;
    const C* B = P.img[mode ? IB_X : IB_Z];
    C bv[kWIters];
#pragma unroll
    for (int k = 0; k < kWIters; ++k) {
        const int q = threadIdx.x + k * kTileThreads;
        const int a = i0 + q / (kTileW + 1), b = j0 + q % (kTileW + 1);
        bv[k] = q < kWPts && a < N && b < N ? B[(size_t)a * N + b] : C(0);
    }
    const int ty = threadIdx.x / kTileW, tx = threadIdx.x % kTileW;
    const int i = i0 + ty, jc = j0 + tx;
    const bool term = i < m && jc < m;
    const size_t idx = (size_t)i * N + jc;
    C2 wo;
    wo.x = C(0);
    wo.y = C(0);
    if (!start && term) wo = Wold[idx];
    for (int q = threadIdx.x; q < (kTileH + 2) * (kTileW + 2); q += kTileThreads) {
        const int ii = q / (kTileW + 2), jj = q % (kTileW + 2);
        const int ti = i0 - 1 + ii, tj = j0 - 1 + jj;
        C2 v;
        v.x = C(0);
        v.y = C(0);
        if (!start && ti >= 0 && ti < m && tj >= 0 && tj < m) v = R[(size_t)ti * N + tj];
        rs[ii][jj] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kWIters; ++k) {
        const int q = threadIdx.x + k * kTileThreads;
        if (q >= kWPts) break;
        const int ii = q / (kTileW + 1), jj = q % (kTileW + 1);
        const int a = i0 + ii, b = j0 + jj;
        C w = C(0);
        if (a < N && b < N) {
            // (L^T r) at pixel (a, b): -(p + q) of term (a, b), +p of (a-1, b), +q of (a, b-1)
            const C lt = -(rs[ii + 1][jj + 1].x + rs[ii + 1][jj + 1].y) + rs[ii][jj + 1].x + rs[ii + 1][jj].y;
            w = fma(-alpha, lt, bv[k]);
        }
        ws[ii][jj] = w;
    }
    __syncthreads();
    if (!term) return;
    const C w0 = ws[ty][tx];
    const C2 r = rs[ty + 1][tx + 1];
    const C ax = fma(ws[ty + 1][tx] - w0, inv8a, r.x);      // r + (L w) / (8 alpha)
    const C ay = fma(ws[ty][tx + 1] - w0, inv8a, r.y);
    const C nrm = sqrt(ax * ax + ay * ay);
    const C sc = nrm > C(1) ? C(1) / nrm : C(1);
    C2 wn;
    wn.x = ax * sc;
    wn.y = ay * sc;
    C2 rn;
    rn.x = fma(beta, wn.x - wo.x, wn.x);
    rn.y = fma(beta, wn.y - wo.y, wn.y);
    Wnew[idx] = wn;
    Rnext[idx] = rn;
    }
}

// Two FGP steps (j, j+1) in one launch, with the buffers of launch index p as
// k_fgp with j = p (reads dual[2 + (p & 1)] and dual[(p + 1) & 1], writes
// dual[p & 1] and dual[2 + ((p + 1) & 1)]): step j is computed on the tile
// grown by one term on every side (from the momentum point with a two-term
// halo), kept in shared memory, and step j+1 on the tile, so one launch and one
// round of dual fields through L2 serve two steps.  Every value is formed by the
// same expressions as in k_fgp, so the iterates are bit-identical.
template <typename T>
__global__ void __launch_bounds__(kTileThreads)
k_fgp2(const Prob<T>* __restrict__ probs, const Item* __restrict__ items, int p, typename Tr<T>::C beta0,
       typename Tr<T>::C beta1, int mode) {
    using C = typename Tr<T>::C;
    using C2 = typename Vec2<C>::type;
    if constexpr (!std::is_same<typename Tr<T>::S, C>::value) {
        return;                                              // FP32 / FP64 storage only
    } else {
    constexpr int H = kTileH, W = kTileW;
    const Item it = decode_item(probs, items, 1);
    const Prob<T>& P = probs[it.prob];
    const DevState& st = *P.st;
    if (st.done) return;
    __shared__ C2 rs0[H + 4][W + 4];     // r_j on terms (i0-2+ii, j0-2+jj)
    __shared__ C bs[H + 3][W + 3];       // b on pixels (i0-1+ii, j0-1+jj)
    __shared__ C ws0[H + 3][W + 3];      // b - alpha L^T r_j on the same pixels
    __shared__ C2 w1s[H + 2][W + 2];     // w_j on terms (i0-1+ii, j0-1+jj)
    __shared__ C2 r1s[H + 2][W + 2];     // r_{j+1} on the same terms
    __shared__ C ws1[H + 1][W + 1];      // b - alpha L^T r_{j+1} on pixels (i0+ii, j0+jj)
    const int N = P.n, m = N - 1;
    const int i0 = it.u * H, j0 = it.v * W;
    const double a64 = mode ? prox_lambda(st) : st.ex.lam / st.ex.c2;
    if (!(a64 > 0.0)) return;
    const C alpha = (C)a64;
    const C inv8a = C(1) / (C(8) * alpha);
    const bool start = p == 0;
    const C2* R = reinterpret_cast<const C2*>(P.dual[2 + (p & 1)]);
    const C2* Wold = reinterpret_cast<const C2*>(P.dual[(p + 1) & 1]);
    C2* Wnew = reinterpret_cast<C2*>(P.dual[p & 1]);
    C2* Rnext = reinterpret_cast<C2*>(P.dual[2 + ((p + 1) & 1)]);
    const C* B = P.img[mode ? IB_X : IB_Z];
    const int tl = threadIdx.x;
    auto valid_term = [&](int ti, int tj) { return ti >= 0 && ti < m && tj >= 0 && tj < m; };
    constexpr int kR1 = (H + 2) * (W + 2);
    constexpr int kR1Iters = (kR1 + kTileThreads - 1) / kTileThreads;
    // every load first: r_j with its two-term halo, b, w_{j-1} on the grown tile
    for (int q = tl; q < (H + 4) * (W + 4); q += kTileThreads) {
        const int ii = q / (W + 4), jj = q % (W + 4);
        const int ti = i0 - 2 + ii, tj = j0 - 2 + jj;
        C2 v;
        v.x = C(0);
        v.y = C(0);
        if (!start && valid_term(ti, tj)) v = R[(size_t)ti * N + tj];
        rs0[ii][jj] = v;
    }
    for (int q = tl; q < (H + 3) * (W + 3); q += kTileThreads) {
        const int ii = q / (W + 3), jj = q % (W + 3);
        const int a = i0 - 1 + ii, b = j0 - 1 + jj;
        bs[ii][jj] = a >= 0 && a < N && b >= 0 && b < N ? B[(size_t)a * N + b] : C(0);
    }
    C2 wo[kR1Iters];
#pragma unroll
    for (int k = 0; k < kR1Iters; ++k) {
        const int q = tl + k * kTileThreads;
        const int ti = i0 - 1 + q / (W + 2), tj = j0 - 1 + q % (W + 2);
        wo[k].x = C(0);
        wo[k].y = C(0);
        if (q < kR1 && !start && valid_term(ti, tj)) wo[k] = Wold[(size_t)ti * N + tj];
    }
    __syncthreads();
    // w = b - alpha L^T r_j on the pixels of the grown tile plus a row and column
    for (int q = tl; q < (H + 3) * (W + 3); q += kTileThreads) {
        const int ii = q / (W + 3), jj = q % (W + 3);
        const int a = i0 - 1 + ii, b = j0 - 1 + jj;
        C w = C(0);
        if (a >= 0 && a < N && b >= 0 && b < N) {
            // (L^T r) at pixel (a, b): -(p + q) of term (a, b), +p of (a-1, b), +q of (a, b-1)
            const C lt = -(rs0[ii + 1][jj + 1].x + rs0[ii + 1][jj + 1].y) + rs0[ii][jj + 1].x + rs0[ii + 1][jj].y;
            w = fma(-alpha, lt, bs[ii][jj]);
        }
        ws0[ii][jj] = w;
    }
    __syncthreads();
    // step j on the grown tile: w_j and r_{j+1} (zero on terms outside the image)
#pragma unroll
    for (int k = 0; k < kR1Iters; ++k) {
        const int q = tl + k * kTileThreads;
        if (q >= kR1) break;
        const int ii = q / (W + 2), jj = q % (W + 2);
        const int ti = i0 - 1 + ii, tj = j0 - 1 + jj;
        C2 wn, rn;
        wn.x = wn.y = rn.x = rn.y = C(0);
        if (valid_term(ti, tj)) {
            const C w0 = ws0[ii][jj];
            const C2 r = rs0[ii + 1][jj + 1];
            const C ax = fma(ws0[ii + 1][jj] - w0, inv8a, r.x);      // r + (L w) / (8 alpha)
            const C ay = fma(ws0[ii][jj + 1] - w0, inv8a, r.y);
            const C nrm = sqrt(ax * ax + ay * ay);
            const C sc = nrm > C(1) ? C(1) / nrm : C(1);
            wn.x = ax * sc;
            wn.y = ay * sc;
            rn.x = fma(beta0, wn.x - wo[k].x, wn.x);
            rn.y = fma(beta0, wn.y - wo[k].y, wn.y);
        }
        w1s[ii][jj] = wn;
        r1s[ii][jj] = rn;
    }
    __syncthreads();
    // w = b - alpha L^T r_{j+1} on the tile's pixels plus a row and column
    for (int q = tl; q < (H + 1) * (W + 1); q += kTileThreads) {
        const int ii = q / (W + 1), jj = q % (W + 1);
        const int a = i0 + ii, b = j0 + jj;
        C w = C(0);
        if (a < N && b < N) {
            const C lt = -(r1s[ii + 1][jj + 1].x + r1s[ii + 1][jj + 1].y) + r1s[ii][jj + 1].x + r1s[ii + 1][jj].y;
            w = fma(-alpha, lt, bs[ii + 1][jj + 1]);
        }
        ws1[ii][jj] = w;
    }
    __syncthreads();
    // step j+1 on the tile
    const int ty = tl / W, tx = tl % W;
    const int i = i0 + ty, jc = j0 + tx;
    if (i >= m || jc >= m) return;
    const C w0 = ws1[ty][tx];
    const C2 r = r1s[ty + 1][tx + 1];
    const C ax = fma(ws1[ty + 1][tx] - w0, inv8a, r.x);
    const C ay = fma(ws1[ty][tx + 1] - w0, inv8a, r.y);
    const C nrm = sqrt(ax * ax + ay * ay);
    const C sc = nrm > C(1) ? C(1) / nrm : C(1);
    C2 wn;
    wn.x = ax * sc;
    wn.y = ay * sc;
    const C2 wp = w1s[ty + 1][tx + 1];
    C2 rn;
    rn.x = fma(beta1, wn.x - wp.x, wn.x);
    rn.y = fma(beta1, wn.y - wp.y, wn.y);
    const size_t idx = (size_t)i * N + jc;
    Wnew[idx] = wn;
    Rnext[idx] = rn;
    }
}

// Caller's plain sinogram [na][nb] into the pair view sino[dst].
template <typename T>
__global__ void __launch_bounds__(kRayBlock)
k_sino_pairs(const Prob<T>* __restrict__ probs, int dst) {
    const Prob<T>& P = probs[0];
    const int a = blockIdx.x / P.ray_blocks, b = (blockIdx.x % P.ray_blocks) * kRayBlock + threadIdx.x;
    if (b < P.nb)
        store_pair<T>(P.sino[dst] + (size_t)a * P.SB + kSPad, b,
                      to_c(P.user_in[(size_t)a * P.nb + b]) * P.ang[a].inv_m);   // weighted view
}

// ---------------------------------------------------------------------------
// Row filter of Sec. 3 (Filters for Preconditioning): each sinogram row r is
// zero-padded to P (a power of two >= 2 n_bins, so the circular product does
// not wrap), transformed by a DFT, multiplied by the real factors
// fac[k] = gain c(w_k) / P (c(w) = (|w| + mu)(0.54 + 0.46 cos w), w_k = 2 pi
// k / P folded into [-pi, pi]; the 1/P is the unitary pair F^T ... F), and
// transformed back; the first n_bins outputs are kept.
//
// One block per pair of rows: rows 2u and 2u+1 are the real and imaginary
// parts of one complex sequence z = a + i b.  The factors are real and even
// (fac[k] = fac[P-k]), so filtering z filters a and b separately: the result
// is filter(a) + i filter(b), one complex FFT pair for two rows.  The FFT is
// radix-2 in shared memory: the forward transform decimates in frequency
// (natural order in, spectrum out in bit-reversed order), the factors -- which
// the host stores in that bit-reversed order -- are applied in place, and the
// inverse transform decimates in time with conjugate twiddles (bit-reversed
// order in, natural order out).  So rows are read and written in natural
// order and no pass touches shared memory through a bit reversal (whose
// power-of-two strides put a warp's accesses in one bank).  The twiddles
// w_j = exp(-2 pi i j / P) come from a quarter table staged in shared memory
// once per block (w_{j + P/4} = -i w_j), not from global memory in every
// stage.  Twiddles and factors come from a table the host fills in FP64 once
// per problem.
//
// mode: FILT_VIEW  pair view src -> pair view dst (the solvers' sinograms)
//       FILT_PLAIN the caller's plain rows user_in -> user_out
//       FILT_FBP   the caller's plain rows user_in -> pair view dst, scaled by
//                  the angle's chord factor like every sinogram view
template <typename T>
__global__ void __launch_bounds__(kFilterThreads)
k_filter(const Prob<T>* __restrict__ probs, const Item* __restrict__ items, int src, int dst, int mode) {
    using C = typename Tr<T>::C;
    using C2 = typename Vec2<C>::type;
    const Item it = decode_item(probs, items, 2);
    const Prob<T>& P = probs[it.prob];
    if (P.st->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nb = P.nb, na = P.na, L = P.P;
    const int lg = 31 - __clz(L);
    const int quarter = max(L >> 2, 1);
    C2* z = reinterpret_cast<C2*>(smem_raw);              // [L] the row pair, natural order
    C2* twq = z + L;                                       // [quarter] w_k = exp(-2 pi i k / L), k < L/4
    const int ra = 2 * it.u, rb = ra + 1;                 // the block's two rows (rb may be past the end)
    const bool has_b = rb < na;
    const C* fac = P.taps;                                // [L] factors in bit-reversed order
    const C2* tw = reinterpret_cast<const C2*>(P.taps + L);   // [L/2] twiddles
    for (int q = threadIdx.x; q < quarter; q += blockDim.x) twq[q] = tw[q];
    for (int q = threadIdx.x; q < L; q += blockDim.x) {
        C va = C(0), vb = C(0);
        if (q < nb) {
            if (mode == FILT_VIEW) {
                const typename Tr<T>::S2* R = P.sino[src] + kSPad;
                va = to_c(R[(size_t)ra * P.SB + q].x);
                if (has_b) vb = to_c(R[(size_t)rb * P.SB + q].x);
            } else {
                va = to_c(P.user_in[(size_t)ra * nb + q]);
                if (has_b) vb = to_c(P.user_in[(size_t)rb * nb + q]);
            }
        }
        C2 v;
        v.x = va;
        v.y = vb;
        z[q] = v;
    }
    __syncthreads();
    // w_k for k < L/2 from the quarter table: w_{k + L/4} = -i w_k
    auto W = [&](int k) -> C2 {
        if (k < quarter) return twq[k];
        const C2 a = twq[k - quarter];
        return C2{a.y, -a.x};
    };
    // forward: decimation in frequency (natural order in, bit-reversed out),
    // spans L, L/2, ..., 2
    for (int st = lg; st >= 1; --st) {
        const int half = 1 << (st - 1);
#pragma unroll 4
        for (int t = threadIdx.x; t < (L >> 1); t += blockDim.x) {
            const int pos = t & (half - 1);
            const int i0 = ((t >> (st - 1)) << st) + pos, i1 = i0 + half;
            const C2 w = W(pos << (lg - st));
            const C2 u = z[i0], v = z[i1];
            const C dr = u.x - v.x, di = u.y - v.y;
            z[i0] = C2{u.x + v.x, u.y + v.y};
            z[i1] = C2{dr * w.x - di * w.y, dr * w.y + di * w.x};   // (u - v) w
        }
        __syncthreads();
    }
    // the factors, stored in the spectrum's bit-reversed order
#pragma unroll 4
    for (int q = threadIdx.x; q < L; q += blockDim.x) {
        const C f = fac[q];
        const C2 v = z[q];
        z[q] = C2{v.x * f, v.y * f};
    }
    __syncthreads();
    // inverse: decimation in time with conjugate twiddles (bit-reversed order
    // in, natural out), spans 2, 4, ..., L
    for (int st = 1; st <= lg; ++st) {
        const int half = 1 << (st - 1);
#pragma unroll 4
        for (int t = threadIdx.x; t < (L >> 1); t += blockDim.x) {
            const int pos = t & (half - 1);
            const int i0 = ((t >> (st - 1)) << st) + pos, i1 = i0 + half;
            const C2 w = W(pos << (lg - st));
            const C2 u = z[i0], v = z[i1];
            const C vr = v.x * w.x + v.y * w.y, vi = v.y * w.x - v.x * w.y;   // v conj(w)
            z[i0] = C2{u.x + vr, u.y + vi};
            z[i1] = C2{u.x - vr, u.y - vi};
        }
        __syncthreads();
    }
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const C2 v = z[b];
        if (mode == FILT_PLAIN) {
            P.user_out[(size_t)ra * nb + b] = to_s<typename Tr<T>::S>(v.x);
            if (has_b) P.user_out[(size_t)rb * nb + b] = to_s<typename Tr<T>::S>(v.y);
        } else {
            const C sa = mode == FILT_FBP ? P.ang[ra].inv_m : C(1);
            store_pair<T>(P.sino[dst] + (size_t)ra * P.SB + kSPad, b, v.x * sa);
            if (has_b) {
                const C sb = mode == FILT_FBP ? P.ang[rb].inv_m : C(1);
                store_pair<T>(P.sino[dst] + (size_t)rb * P.SB + kSPad, b, v.y * sb);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Loop condition of the device-driven while loop (one thread): continue while
// the solver has not stopped, and never past max_bodies bodies, so the loop
// ends even if the stop flag were never set.
__global__ void k_loop_cond(DevState* st, cudaGraphConditionalHandle h) {
    if (threadIdx.x != 0) return;
    if (st->dev_error) st->done = 1;          // a bounded wait ran out: stop (reported as SCG_ERR_CUDA)
    unsigned more = st->done ? 0u : 1u;
    if (st->bodies >= st->max_bodies) more = 0u;
    st->bodies += (int)more;
    cudaGraphSetConditional(h, more);
}

void launch_loop_cond(DevState* st, cudaGraphConditionalHandle h, cudaStream_t s) {
    k_loop_cond<<<1, 32, 0, s>>>(st, h);
}

// The result of an asynchronous solve, written by the device from its state
// when the stream reaches it (f is reported on the unscaled system).
__global__ void k_write_result(const DevState* st, scg_result* res, double s2, int cg_family, int base_launches,
                               int body_kernels) {
    const bool fista = st->family == FAM_FISTA;
    if (threadIdx.x != 0) return;
    res->iters = st->iters;
    res->k_final = st->k;
    res->status = st->dev_error ? SCG_ERR_CUDA : st->status;
    res->f_final = (cg_family ? st->f_final : st->f_half) / s2;
    res->tv_final = st->tv_final;
    res->ell = st->ell;
    res->gamma0_used = st->gamma0;
    res->kernel_launches = base_launches + st->bodies * (body_kernels + 1);
    res->body_launches = st->bodies;
    res->device_loop = 1;
    res->lipschitz_used = fista ? st->ex.c2 : 0.0;
}
void launch_write_result(const DevState* st, scg_result* res, double s2, int cg_family, int base_launches,
                         int body_kernels, cudaStream_t s) {
    k_write_result<<<1, 32, 0, s>>>(st, res, s2, cg_family, base_launches, body_kernels);
}

// Point a prepared operator's descriptor at the caller's buffers (one thread;
// keeps every application stream-ordered and free of host copies).
template <typename T>
__global__ void k_set_io(Prob<T>* d, const typename Tr<T>::S* in_sino, typename Tr<T>::S* out_sino,
                         typename Tr<T>::S* image) {
    if (threadIdx.x != 0) return;
    d->user_in = in_sino;
    d->user_out = out_sino;
    d->img[IB_AUX] = image;
}
template <typename T>
void launch_set_io(Prob<T>* d, const typename Tr<T>::S* in_sino, typename Tr<T>::S* out_sino,
                   typename Tr<T>::S* image, cudaStream_t s) {
    k_set_io<T><<<1, 32, 0, s>>>(d, in_sino, out_sino, image);
}

// Set every problem's stop flag (used around the final kernels of a batch).
template <typename T>
__global__ void k_set_done(const Prob<T>* probs, int count, int value) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) probs[i].st->done = value;
}
template <typename T>
void launch_set_done(const Prob<T>* d, int count, int value, cudaStream_t s) {
    k_set_done<T><<<(count + 127) / 128, 128, 0, s>>>(d, count, value);
}

// Serving: stop flags of the listed problem slots, gathered (out[i] = done of
// slots[i]) or set (done = value).
template <typename T>
__global__ void k_slots_done(const Prob<T>* probs, const int* slots, int count, int* out, int set, int value) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    DevState* st = probs[slots[i]].st;
    if (set) st->done = value;
    else out[i] = st->done;
}
template <typename T>
void launch_slots_done(const Prob<T>* d, const int* slots, int count, int* out, int set, int value,
                       cudaStream_t s) {
    if (count > 0) k_slots_done<T><<<(count + 127) / 128, 128, 0, s>>>(d, slots, count, out, set, value);
}

// Batched loop condition: continue while any problem is still running, and
// never past max_bodies bodies.
template <typename T>
__global__ void k_loop_cond_batch(const Prob<T>* probs, BatchState* bs, cudaGraphConditionalHandle h) {
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < bs->count; i += blockDim.x) {
        DevState* st = probs[i].st;
        if (st->dev_error) st->done = 1;      // a bounded wait ran out: stop that problem
        if (!st->done) atomicOr(&any, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned more = any ? 1u : 0u;
        if (bs->bodies >= bs->max_bodies) more = 0u;
        bs->bodies += (int)more;
        cudaGraphSetConditional(h, more);
    }
}

template <typename T>
void launch_loop_cond_batch(const Prob<T>* d, BatchState* bs, cudaGraphConditionalHandle h, cudaStream_t s) {
    k_loop_cond_batch<T><<<1, 256, 0, s>>>(d, bs, h);
}

// ---------------------------------------------------------------------------
// Host launchers.
template <typename T>
void launch_project(const Prob<T>* d, const Item* items, int grid, int dst, int mode, int step,
                    cudaStream_t s) {
    k_project<T><<<grid, kProjThreads, 0, s>>>(d, items, dst, mode, step);
}
// `grid` tiles (work items), each taken by a cluster of BpCfg::CL blocks.
template <typename T, int NRHS>
void launch_bp(const Prob<T>* d, const Item* items, int grid, int src0, int src1, int dst0, int dst1,
               int step, cudaStream_t s) {
    constexpr int CL = BpCfg<T, NRHS>::CL;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)(grid * CL));
    cfg.blockDim = dim3(kBackThreads);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_backproject<T, NRHS>, d, items, src0, src1, dst0, dst1, step);
}
template <typename T>
void launch_backproject(const Prob<T>* d, const Item* items, int grid, int nrhs, int src0,
                        int src1, int dst0, int dst1, int step, cudaStream_t s) {
    if (nrhs == 2) launch_bp<T, 2>(d, items, grid, src0, src1, dst0, dst1, step, s);
    else launch_bp<T, 1>(d, items, grid, src0, src1, dst0, dst1, step, s);
}
template <typename T>
void launch_sino_comb(const Prob<T>* d, const Item* items, int grid, int cur, int prev, cudaStream_t s) {
    k_sino_comb<T><<<grid, kRayBlock, 0, s>>>(d, items, cur, prev);
}
template <typename T>
void launch_sino_norm(const Prob<T>* d, const Item* items, int grid, int src, int step, cudaStream_t s) {
    k_sino_norm<T><<<grid, kRayBlock, 0, s>>>(d, items, src, step);
}
template <typename T>
void launch_fgp(const Prob<T>* d, const Item* items, int grid, int j, double beta, int mode, cudaStream_t s) {
    k_fgp<T><<<grid, kTileThreads, 0, s>>>(d, items, j, (typename Tr<T>::C)beta, mode);
}
template <typename T>
void launch_fgp2(const Prob<T>* d, const Item* items, int grid, int p, double beta0, double beta1, int mode,
                 cudaStream_t s) {
    using C = typename Tr<T>::C;
    k_fgp2<T><<<grid, kTileThreads, 0, s>>>(d, items, p, (C)beta0, (C)beta1, mode);
}
template <typename T>
void launch_sino_pairs(const Prob<T>* d, int grid, int dst, cudaStream_t s) {
    k_sino_pairs<T><<<grid, kRayBlock, 0, s>>>(d, dst);
}
template <typename T>
void launch_vec(const Prob<T>* d, const Item* items, int grid, int op, int sel, int step,
                cudaStream_t s) {
    k_vec<T><<<grid, kTileThreads, 0, s>>>(d, items, op, sel, step);
}
template <typename T>
void launch_tvgrad(const Prob<T>* d, const Item* items, int grid, int src, int fuse,
                   int write_grad, int step, cudaStream_t s) {
    k_tvgrad<T><<<grid, kTileThreads, 0, s>>>(d, items, src, fuse, write_grad, step);
}
template <typename T>
void launch_trial(const Prob<T>* d, const Item* items, int grid, int ncand, cudaStream_t s) {
    if (ncand == kTrialsFirst) k_trial<T, kTrialsFirst><<<grid, kBackThreads, 0, s>>>(d, items);
    else k_trial<T, kTrials><<<grid, kBackThreads, 0, s>>>(d, items);
}
template <typename T>
void launch_sino_axpy(const Prob<T>* d, const Item* items, int grid, int step, cudaStream_t s) {
    k_sino_axpy<T><<<grid, kRayBlock, 0, s>>>(d, items, step);
}
template <typename T>
cudaError_t launch_filter(const Prob<T>* d, const Item* items, int grid, int max_nb, int src,
                          int dst, int mode, cudaStream_t s) {
    const size_t smem = filter_smem_bytes<typename Tr<T>::C>(max_nb);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_filter<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_filter<T><<<grid, kFilterThreads, smem, s>>>(d, items, src, dst, mode);
    return cudaSuccess;
}

#define SCG_INSTANTIATE(T)                                                                        \
    template void launch_project<T>(const Prob<T>*, const Item*, int, int, int, int, cudaStream_t); \
    template void launch_backproject<T>(const Prob<T>*, const Item*, int, int, int, int, int, int, \
                                        int, cudaStream_t);                                       \
    template void launch_vec<T>(const Prob<T>*, const Item*, int, int, int, int, cudaStream_t);     \
    template void launch_tvgrad<T>(const Prob<T>*, const Item*, int, int, int, int, int,          \
                                   cudaStream_t);                                                 \
    template void launch_trial<T>(const Prob<T>*, const Item*, int, int, cudaStream_t);                \
    template void launch_sino_axpy<T>(const Prob<T>*, const Item*, int, int, cudaStream_t);       \
    template cudaError_t launch_filter<T>(const Prob<T>*, const Item*, int, int, int, int, int,   \
                                          cudaStream_t);                                          \
    template void launch_sino_pairs<T>(const Prob<T>*, int, int, cudaStream_t);                   \
    template void launch_sino_comb<T>(const Prob<T>*, const Item*, int, int, int, cudaStream_t);    \
    template void launch_fgp<T>(const Prob<T>*, const Item*, int, int, double, int, cudaStream_t);  \
    template void launch_fgp2<T>(const Prob<T>*, const Item*, int, int, double, double, int, cudaStream_t); \
    template void launch_sino_norm<T>(const Prob<T>*, const Item*, int, int, int, cudaStream_t);    \
    template void launch_set_done<T>(const Prob<T>*, int, int, cudaStream_t);                     \
    template void launch_set_io<T>(Prob<T>*, const typename Tr<T>::S*, typename Tr<T>::S*,          \
                                   typename Tr<T>::S*, cudaStream_t);                            \
    template void launch_slots_done<T>(const Prob<T>*, const int*, int, int*, int, int, cudaStream_t); \
    template void launch_loop_cond_batch<T>(const Prob<T>*, BatchState*, cudaGraphConditionalHandle, \
                                            cudaStream_t);

SCG_INSTANTIATE(float)
SCG_INSTANTIATE(double)
SCG_INSTANTIATE(__half)
SCG_INSTANTIATE(__nv_bfloat16)

}  // namespace scg
