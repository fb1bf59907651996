// scg_device.cuh -- device-side data structures, the ray-pixel weight, the
// deterministic FP64 block reductions and the solver state machine shared by
// every kernel of libscg.
//
// Layout in HBM (one "problem" = one reconstruction):
//   image vectors      N*N, row-major, element type S: float or double, or
//                      half / bfloat16 storage with FP32 arithmetic
//                      (Tr<T> below gives S and the arithmetic type C)
//   projector views    two zero-padded copies of the image being projected, in
//                      "pair" layout (slot q of a line holds elements q and
//                      q+1, so the two pixels a ray meets in one strip are one
//                      aligned 8-byte load): row-major lines
//                      (view_rm[i*S + kPad + j]) for angles whose rays are
//                      walked row by row, column-major lines
//                      (view_cm[j*S + kPad + i]) for angles walked column by
//                      column, so the lanes of a warp (consecutive rays of a
//                      few adjacent angles, walking the same strip together)
//                      read a few short spans of one line.
//   sinogram views     [angle][kSPad + bin] rows of SB pairs with zero pads, so
//                      the backprojector's two candidate bins are one load and
//                      never need a bounds test (a clamped pair reads pads);
//                      a view holds v[a,b] * inv_m(a) (the angle's chord factor,
//                      applied once when the view is written).
//   partials           up to kSlots sums per work item, slot-major (slot k of
//                      item i at k * part_cap + i, so the final sum reads
//                      consecutive items), summed in a fixed order by the last
//                      item of a launch (no atomics on data).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "scg.h"

namespace scg {

constexpr int kPad = 2;          // zero elements on each side of an image-view line
constexpr int kSPad = 2;         // zero elements on each side of a sinogram-view row
constexpr int kSlots = 32;       // FP64 partial sums per work item (at most); stored slot-major
constexpr int kTrials = 31;      // TV trial candidates per pass (+1 baseline slot) ...
constexpr int kTrialsFirst = 3;  // ... except a step's first pass
// trial passes in a loop body for a budget of max_trials candidates per step
__host__ __device__ constexpr int trial_passes_for(int max_trials) {
    return max_trials <= kTrialsFirst ? 1 : 1 + (max_trials - kTrialsFirst + kTrials - 1) / kTrials;
}
constexpr int kTileW = 32;       // image tile width (pixels) = one warp
constexpr int kTileH = 8;        // image tile height
constexpr int kTileThreads = kTileW * kTileH;
constexpr int kBackThreads = 128;               // backprojector block: 32 x kBpTileH pixels ...
constexpr int kBpTileH32 = 32;                  // ... 8 per thread (FP32 arithmetic)
constexpr int kBpTileH64 = 8;                   // ... 2 per thread (FP64)
constexpr int kRayBlock = 128;   // rays per sinogram-row work item (axpy, pairs)
constexpr int kProjLog2 = 8;     // projector block: 2^8 threads = adjacent angles x consecutive
constexpr int kProjThreads = 1 << kProjLog2;   // rays (2^proj_shift rays of each angle; they read
constexpr int kProjShiftDefault = 6;           // nearly the same image spans): 4 x 64 by default
constexpr int kFilterThreads = 256; // filter block: two sinogram rows, one complex FFT pair
// filter length P (a power of two >= 2 n_bins) and the shared memory of its FFT
__host__ __device__ constexpr int filter_length_of(int nb) {
    int P = 1;
    while (P < 2 * nb) P *= 2;
    return P;
}
template <typename C>
// the row pair (P complex values) and the quarter twiddle table (max(P/4, 1))
__host__ __device__ constexpr size_t filter_smem_bytes(int nb) {
    return 2 * sizeof(C) * ((size_t)filter_length_of(nb) + (size_t)(filter_length_of(nb) / 4 > 0 ? filter_length_of(nb) / 4 : 1));
}
constexpr size_t kFilterSmemMax = 160 * 1024;   // largest FFT held in shared memory (FP32: n_bins <= 8192, FP64: 4096)

// Sinogram pair slots the gather stages per angle for one 32-pixel-wide tile
// (see k_backproject): 48 for FP32 pairs, 52 for 16-bit pairs.
template <typename S2> __host__ __device__ constexpr int band_slots() { return sizeof(S2) >= 8 ? 48 : 52; }
constexpr int kSinoMapBytes = 128;   // one TMA tensor map (CUtensorMap)

enum ImgBuf { IB_X = 0, IB_XH, IB_P, IB_H, IB_G, IB_Z, IB_TVG, IB_AUX, IB_COUNT };
enum SinoBuf { SB_R = 0, SB_Q, SB_W, SB_V, SB_COUNT };
// FISTA keeps x_k in kFistaX[k % 3] and its residual A x_k - y in kFistaQ[k % 3]
constexpr int kFistaX[3] = {IB_X, IB_XH, IB_P};
constexpr int kFistaQ[3] = {SB_Q, SB_W, SB_V};

// Per-angle constants (host computes them in FP64).  With m = max(|c|,|s|),
// n = min(|c|,|s|), the chord of a ray through a unit pixel whose centre is at
// signed detector distance d is T(d) = min(1/m, max(0, ((m+n)/2 - |d|)/(m n)))
// (for n = 0: 1, 1/2 on an edge, 0).  Two consequences are used:
//  * walking a ray along its driving axis (columns when |sin| >= |cos|), the
//    chord inside one column strip is exactly 1/m and lies in the two pixels
//    nearest the crossing c*, rows floor(c*) and floor(c*)+1; with
//    f = c* - floor(c*) the first gets u/m, the second (1-u)/m,
//    u = sat(h2 - f k2), k2 = m/n, h2 = (m+n)/(2n)   (n = 0: k2 = h2 = 1);
//    the FP32 walk carries c* in 32.32 fixed point (exact increments, no
//    FP64 anywhere in the FP32 kernels);
//  * gathering at a pixel whose centre projects to bin coordinate cb
//    (g = cb - floor(cb)), bins floor(cb) and floor(cb)+1 get
//    sat(hb0 - g kb)/m and sat(hb1 + g kb)/m,
//    kb = 1/n, hb0 = (m+n)/(2n), hb1 = ((m+n)/2 - 1)/n   (n = 0: 1, 1, 0).
template <typename T>
struct Angle {
    T c, s;        // cos, sin (exact 0/1 at theta = 0, pi/2)
    T inv_m;       // 1/m
    T k2, h2;      // forward weights
    T h2p;         // h2 + k2 (weight from a fraction f1 = f + 1 in [1, 2))
    T kb, hb0;     // gather weights
    T hb1;
    T slope;       // change of the crossing per step along the driving axis
    T inv_drive;   // 1/s (column-walked) or 1/c
    T c0_off;      // off_n * (e * inv_drive + 1), e = c (column-walked) or s
    T inv_slope;   // 1/slope (0 when slope = 0)
    int col_driven;
    double c_d, s_d;          // FP64 copies (FP64 kernels)
    double inv_d, c0_off_d, slope_d;
    long long c_fx, s_fx;     // 32.32 fixed point (FP32 kernels)
    int c23, s23;             // cos, sin in 9.23 fixed point (in-tile offsets of the gather)
    T hb0p, hb1p;             // hb0 + kb, hb1 - kb (gather weights from g1 = g + 1 in [1, 2))
    T m_w;                    // 1 / inv_m: undoes the chord factor of a sinogram view
    long long inv_fx, c0_off_fx, slope_fx;
};

// Work item of a launch over many problems (batched mode).  Single-problem
// launches pass items = nullptr and decode (u, v) from blockIdx.
struct Item {
    int prob;      // problem index
    int u, v;      // projector: angle, bin block; image: tile row, tile column; filter: row, block
    int local;     // index of this item among the problem's items of this kind
};

// Trace row fields (SCG_TRACE_FIELDS).
enum { TR_K = 0, TR_FTEST, TR_TV_BEFORE, TR_TV_AFTER, TR_TRIALS, TR_ACCEPTED, TR_ELL,
       TR_GAMMA, TR_ALPHA, TR_BETA, TR_MARGIN, TR_F_AFTER, TR_NF };

// Device-resident solver state: every scalar of Algorithms 1-14 lives here
// and is only ever written by the finalising block of a reduction.
struct DevState {
    double eps;
    double f_half;          // f at the point tested next: f(x_{k+1/2}) (S-variants), f(x_k) (CG)
    double pTh;             // p_{k-1}^T h_{k-1}
    double gTp;             // g_{k-1}^T p_{k-1} (S-CG-CD)
    double delta;           // CG/PCG delta_k
    double alpha, beta, num, gg;
    double tv_x, gnorm2, xnorm2;
    double gamma0, gamma0_rel, a;
    double coef;            // applied perturbation: x_{k+1/2} = x_k + coef * dTV(x_k)
    double trial_c0;        // coefficient of the first pending trial: -gamma0 a^ell / ||dTV||
    double a_ell;           // a^ell, kept by multiplication as ell advances
    union {
        double apow[kTrials];   // gamma rule: a^t, t = 0 .. kTrials-1 (set on the host); trial t: trial_c0 * apow[t]
        struct {                // FISTA and the Appendix rule, which take no gamma trials (sharing the
                                // table keeps the state, which every finalising block copies, its size)
            double eta0;        // Appendix rule: ||u_k|| = eta0 ||g_k||
            double c2;          // FISTA: c^2 = ||A||_2^2 (given, or the power iteration's estimate)
            double tk;          // FISTA: t_k of Eq. FISTA-u
            double lam;         // FISTA: lambda of the prox step lambda / c^2
        } ex;
    };
    double margin;
    double f_final, tv_final;
    long long ell;
    int k, iters, max_iter, done, status;
    int perturb, gamma_fixed, max_trials, trials, accepted;
    int in_init, variant, inner_stop, family;
    int bodies, max_bodies;  // loop bodies started by the device loop, and its hard cap
    int pass_cands;          // candidates of the trial pass being finalised
    int dev_error;           // set when a kernel's bounded wait on its own copies ran out (the solve
                             // then stops and reports SCG_ERR_CUDA); fills padding, no size change
};

enum Family { FAM_CG = 0, FAM_S_PR = 1, FAM_S_K = 2, FAM_FISTA = 3 };

// Loop bookkeeping of a batched solve (the problems' own states are DevState).
struct BatchState {
    int bodies, max_bodies, count, pad_;
};

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// Storage type S (and its pair S2) and arithmetic type C of a precision T:
// float and double compute in themselves; half and bfloat16 are storage
// formats whose values every kernel widens to FP32 on load and rounds to
// nearest on store (reductions stay double-float, scalars FP64).
template <typename T> struct Tr {
    using S = T;
    using S2 = typename Vec2<T>::type;
    using C = T;
};
template <> struct Tr<__half> {
    using S = __half;
    using S2 = __half2;
    using C = float;
};
template <> struct Tr<__nv_bfloat16> {
    using S = __nv_bfloat16;
    using S2 = __nv_bfloat162;
    using C = float;
};

__device__ __forceinline__ float to_c(float v) { return v; }
__device__ __forceinline__ double to_c(double v) { return v; }
__device__ __forceinline__ float to_c(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_c(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float2 to_c2(float2 v) { return v; }
__device__ __forceinline__ double2 to_c2(double2 v) { return v; }
__device__ __forceinline__ float2 to_c2(__half2 v) { return __half22float2(v); }
__device__ __forceinline__ float2 to_c2(__nv_bfloat162 v) { return __bfloat1622float2(v); }
template <typename S> __device__ __forceinline__ S to_s(typename Tr<S>::C v);
template <> __device__ __forceinline__ float to_s<float>(float v) { return v; }
template <> __device__ __forceinline__ double to_s<double>(double v) { return v; }
template <> __device__ __forceinline__ __half to_s<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 to_s<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
// v rounded to the storage format and widened back (identity for float/double)
template <typename T>
__device__ __forceinline__ typename Tr<T>::C rnd(typename Tr<T>::C v) {
    if constexpr (std::is_same<typename Tr<T>::S, typename Tr<T>::C>::value) return v;
    else return to_c(to_s<typename Tr<T>::S>(v));
}

template <typename T>
struct Prob {
    using elem_t = typename Tr<T>::S;     // storage element
    using pair_t = typename Tr<T>::S2;    // storage pair
    using calc_t = typename Tr<T>::C;     // arithmetic
    int n, na, nb;
    int S;                  // image-view line stride (elements)
    int SB;                 // sinogram-view row stride (elements)
    int cnt_ray, cnt_img, cnt_row;   // items per launch kind
    int cnt_proj, proj_blocks;       // projector items; bin blocks per angle group
    int proj_shift;                  // projector block = 2^(8-shift) angles x 2^shift rays
    int cnt_bp;                      // backprojector tiles (32 x kBpTileH32 or kBpTileH64)
    int bp_mirror;                   // the gather takes its mirror-paired path (FP32 arithmetic,
                                     // 64 | n, the scan's full angle set)
    int tiles_x;            // image tiles per row of tiles
    int ray_blocks;         // projector items per angle
    int filt_blocks;        // filter items per row pair (1)
    int P;                  // filter length (power of two >= 2 nb)
    calc_t off_n, off_b;    // (N-1)/2, (nb-1)/2
    calc_t y_scale;         // scale c of the solved system c A x ~ c y (a power of two; see Angle.inv_m)
    const Angle<calc_t>* ang;
    const elem_t* y;        // data [na][nb]
    elem_t* img[IB_COUNT];
    pair_t* sino[SB_COUNT]; // pair views of the sinogram-sized vectors
    pair_t* view_rm;
    pair_t* view_cm;
    const elem_t* user_in;  // caller's plain sinogram (operator entry points)
    elem_t* user_out;
    const calc_t* taps;     // filter tables: P factors gain c(w_k)/P, then P/2 twiddles exp(-2 pi i j/P)
    double* partials;
    unsigned* counter;
    DevState* st;
    double* trace;
    int trace_rows;
    int part_cap;           // items per slot of `partials` (slot-major: partials[k * part_cap + item])
    pair_t* dual[4];        // FISTA's TV prox: dual fields w_j (0, 1) and momentum points (2, 3), one
                            // (p, q) pair per interior term (i, j) at i*N + j
    const unsigned char* sino_map;   // SB_COUNT TMA tensor maps (128 bytes each): map q describes sino[q]
                                     // as na rows of SB pairs (FP32 / 16-bit storage; null for FP64)
};

// ---------------------------------------------------------------------------
// Rounding-explicit arithmetic helpers (used where the order of rounding
// matters: trial points and the applied perturbation must be identical).
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float tmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double tmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float tmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double tmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float tabs(float a) { return fabsf(a); }
__device__ __forceinline__ double tabs(double a) { return fabs(a); }
__device__ __forceinline__ float tfloor(float a) { return floorf(a); }
__device__ __forceinline__ double tfloor(double a) { return floor(a); }
__device__ __forceinline__ float tsqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double tsqrt(double a) { return sqrt(a); }

__device__ __forceinline__ float sat(float a) { return __saturatef(a); }
__device__ __forceinline__ double sat(double a) { return fmin(fmax(a, 0.0), 1.0); }

// floor(v) as value and integer without the conversion pipe: adding 1.5*2^23
// with round-toward-minus-infinity leaves floor(v) in the low mantissa bits
// (valid for |v| < 2^22; every caller stays below 2^14).
__device__ __forceinline__ float floor_split(float v, int& i) {
    const float t = __fadd_rd(v, 12582912.0f);
    i = __float_as_int(t) - 0x4B400000;
    return t - 12582912.0f;
}
__device__ __forceinline__ double floor_split(double v, int& i) {
    const double f = floor(v);
    i = (int)f;
    return f;
}

// Store element b of a pair-layout row (row points at the slot of element 0):
// slot b holds (e[b], e[b+1]), so e[b] is written twice.
template <typename T>
__device__ __forceinline__ void store_pair(typename Tr<T>::S2* row, int b, typename Tr<T>::C v) {
    using S = typename Tr<T>::S;
    S* e = reinterpret_cast<S*>(row);
    const S w = to_s<S>(v);
    e[2 * b] = w;
    e[2 * b - 1] = w;
}

// ---------------------------------------------------------------------------
// Reductions.  FP64 arithmetic is slow on this GPU, so the FP32 kernels carry
// their partial sums as double-float pairs (hi + lo, FP32 each): products are
// split exactly with an FMA, and sums use the error-free TwoSum, which keeps
// about 48 bits -- FP64-quality sums without FP64 instructions.  Only the
// finalising thread converts to double.  The FP64 kernels use doubles.
// Every sum runs in a fixed order, so results do not depend on scheduling.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_add(DF a, DF b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    const float lo = __fadd_rn(err, __fadd_rn(a.lo, b.lo));
    const float hi = __fadd_rn(s, lo);
    DF r;
    r.hi = hi;
    r.lo = __fsub_rn(lo, __fsub_rn(hi, s));
    return r;
}

template <typename T> struct AccOf;
template <> struct AccOf<float> { using type = DF; };
template <> struct AccOf<double> { using type = double; };
template <> struct AccOf<__half> { using type = DF; };
template <> struct AccOf<__nv_bfloat16> { using type = DF; };
template <typename T> using Acc = typename AccOf<T>::type;

__device__ __forceinline__ void acc_zero(DF& a) { a.hi = 0.f; a.lo = 0.f; }
__device__ __forceinline__ void acc_zero(double& a) { a = 0.0; }
// exact product of two FP32 values as a pair
__device__ __forceinline__ DF acc_prod(float a, float b) {
    DF r;
    r.hi = __fmul_rn(a, b);
    r.lo = __fmaf_rn(a, b, -r.hi);
    return r;
}
__device__ __forceinline__ double acc_prod(double a, double b) { return a * b; }
__device__ __forceinline__ DF acc_val(float a) { DF r; r.hi = a; r.lo = 0.f; return r; }
__device__ __forceinline__ double acc_val(double a) { return a; }
__device__ __forceinline__ DF acc_add(DF a, DF b) { return df_add(a, b); }
__device__ __forceinline__ double acc_add(double a, double b) { return a + b; }
__device__ __forceinline__ DF acc_shfl_down(DF a, int o) {
    DF r;
    r.hi = __shfl_down_sync(0xffffffffu, a.hi, o);
    r.lo = __shfl_down_sync(0xffffffffu, a.lo, o);
    return r;
}
__device__ __forceinline__ double acc_shfl_down(double a, int o) { return __shfl_down_sync(0xffffffffu, a, o); }
__device__ __forceinline__ double acc_to_double(DF a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ double acc_to_double(double a) { return a; }

// Warp-level step of a block sum.  Sums of non-negative terms (squares, TV
// terms) may take it in plain FP32: a 32-term tree sum of non-negative
// values is accurate to ~3e-7 relative, and those errors average out over the
// thousands of warps that the double-float stages then add exactly.  Signed
// dot products keep double-float throughout.
template <bool kPositive, typename A>
__device__ __forceinline__ A warp_sum(A v) {
    if constexpr (kPositive && std::is_same<A, DF>::value) {
        float h = v.hi + v.lo;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) h += __shfl_down_sync(0xffffffffu, h, o);
        A r;
        r.hi = h;
        r.lo = 0.f;
        return r;
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = acc_add(v, acc_shfl_down(v, o));
        return v;
    }
}

// Block sum of NS accumulators; the result is valid in thread 0.
template <typename A, int NS, bool kPositive = false>
__device__ __forceinline__ void block_sum(A (&v)[NS], A* smem /* >= 32*NS */) {
#pragma unroll
    for (int k = 0; k < NS; ++k) v[k] = warp_sum<kPositive>(v[k]);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NS; ++k) smem[warp * NS + k] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            if (lane < nwarps) v[k] = smem[lane * NS + k];
            else acc_zero(v[k]);
        }
#pragma unroll
        for (int k = 0; k < NS; ++k) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[k] = acc_add(v[k], acc_shfl_down(v[k], o));
        }
    }
}

template <typename T> __device__ void finalize(int step, const Prob<T>& P, DevState& st, const double* S);
template <typename T> __device__ __noinline__ void finalize_rare(int step, const Prob<T>& P, DevState& st, const double* S);

// The finalising block works on a shared-memory copy of the problem's state:
// the copy is loaded by the block's threads in parallel (one 8-byte word
// each), the state machine runs on it in one thread, and the block writes it
// back -- instead of one dependent global round trip per state field.
static_assert(sizeof(DevState) % 8 == 0, "state copied as 8-byte words");
static_assert(sizeof(DevState) == 496, "the state's size is part of the finalisers' register budget");
constexpr int kStateWords = (int)(sizeof(DevState) / 8);
// one word per thread: every kernel that finalises runs blocks of at least this many threads
static_assert(kStateWords <= kBackThreads && kStateWords <= kTileThreads && kStateWords <= kRayBlock &&
              kStateWords <= kProjThreads, "state words per finalising block");
struct StateCopy {
    unsigned long long w;
    __device__ __forceinline__ void load(const DevState* g) {
        if ((int)threadIdx.x < kStateWords) w = __ldcg(reinterpret_cast<const unsigned long long*>(g) + threadIdx.x);
    }
    __device__ __forceinline__ void to_smem(DevState& sst) const {
        if ((int)threadIdx.x < kStateWords) reinterpret_cast<unsigned long long*>(&sst)[threadIdx.x] = w;
    }
    __device__ __forceinline__ static void store(const DevState& sst, DevState* g) {
        if ((int)threadIdx.x < kStateWords)
            reinterpret_cast<unsigned long long*>(g)[threadIdx.x] = reinterpret_cast<const unsigned long long*>(&sst)[threadIdx.x];
    }
};

// One work item's arrival at the end of a launch: an acquire-release atomic
// increment at GPU scope.  Release: the partial sums this block wrote before
// it (by any of its threads, ordered before the calling thread by a block
// barrier) are visible to whoever observes the increment.  Acquire: the block
// that sees the count reach `total` sees every other item's partials (its
// other threads after a block barrier).  Returns true for that last item.
// (It takes the place of a sequentially consistent __threadfence in every
// block and in every thread of the last block.)
__device__ __forceinline__ bool arrive_last(unsigned* counter, unsigned total) {
    unsigned prev;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(prev) : "l"(counter) : "memory");
    return prev + 1u == total;
}

// Publish this item's partial sums; the block that completes the problem's
// last item sums all partials in item order and runs the step's finaliser.
// Must be called by every thread of the block (uniform control flow).
// Partials are stored as the accumulator type (8 bytes either way).
template <typename T, int NS, bool kPositive = false, bool kRare = false>
__device__ void reduce_and_finalize(Acc<T> (&v)[NS], const Prob<T>& P, int local, int total,
                                    int step) {
    using A = Acc<T>;
    __shared__ A red[32 * NS];
    __shared__ unsigned s_last;
    block_sum<A, NS, kPositive>(v, red);
    A* parts = reinterpret_cast<A*>(P.partials);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NS; ++k) parts[(size_t)k * P.part_cap + local] = v[k];
        s_last = arrive_last(P.counter, (unsigned)total);
    }
    __syncthreads();
    if (!s_last) return;
    StateCopy sc;
    sc.load(P.st);                                    // in flight during the sums below
    A acc[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) acc_zero(acc[k]);
#pragma unroll 4
    for (int it = threadIdx.x; it < total; it += blockDim.x) {      // loads of 4 items in flight
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            const A* src = parts + (size_t)k * P.part_cap + it;   // consecutive items: coalesced
            A x;
            if constexpr (sizeof(A) == 8 && !std::is_same<A, double>::value) {
                const float2 w = __ldcg(reinterpret_cast<const float2*>(src));
                x.hi = w.x;
                x.lo = w.y;
            } else {
                x = __ldcg(reinterpret_cast<const double*>(src));
            }
            acc[k] = acc_add(acc[k], x);
        }
    }
    block_sum<A, NS>(acc, red);
    __shared__ DevState sst;
    sc.to_smem(sst);
    __syncthreads();
    if (threadIdx.x == 0) {
        *P.counter = 0u;
        double S[NS < 4 ? 4 : NS];
#pragma unroll
        for (int k = 0; k < (NS < 4 ? 4 : NS); ++k) S[k] = k < NS ? acc_to_double(acc[k]) : 0.0;
        if constexpr (kRare) finalize_rare<T>(step, P, sst, S);
        else finalize<T>(step, P, sst, S);
    }
    __syncthreads();
    StateCopy::store(sst, P.st);
}

// ---------------------------------------------------------------------------
// Solver state machine.  Step codes name the reduction that just finished.
enum Step {
    FIN_NONE = 0,
    FIN_F,            // residual projection: f = S0/2 at the point just projected
    FIN_BETA,         // gradient backprojection (S-variants): S0 = g'^T h (or z'^T h), S1 = ||g'||^2,
                      // S2 = g'^T p, S3 = g'^T z' (S-PCG)
    FIN_NUM,          // new direction formed: S0 = g'^T p' (16-bit storage; FIN_BETA otherwise)
    FIN_ALPHA,        // h' backprojection: S0 = p'^T h'  ->  alpha = -g'^T p' / p'^T h'
    FIN_END,          // TV gradient of the new iterate: S0 = TV, S1 = ||dTV||^2, S2 = ||x||^2
    FIN_TRIAL,        // trial pass: S0..S(nc-1) = TV of the candidates, S(nc) = TV(x)
    FIN_CG_DELTA,     // CG(-K) start: S0 = ||g||^2, S1 = g^T z
    FIN_CG_ALPHA,     // CG-STEP: S0 = p^T h -> alpha = delta / p^T h
    FIN_CG_F,         // recursive residual: f = S0/2
    FIN_CG_BETA,      // CG-STEP: S0 = ||g'||^2, S1 = g'^T z' -> beta = delta'/delta
    FIN_CG_END,       // CG/PCG end of loop body (no sums)
    FIN_RESUME,       // resumed state: S0 = p^T h, S1 = g^T p
    FIN_TV,           // standalone TV: S0 -> trace slot 0
    FIN_FINAL_F,      // f of the output
    FIN_FINAL_TV,     // TV of the output
    FIN_POWER,        // power iteration: S0 = ||h||^2, S1 = p^T h with h = A^T A p (vector pass)
    FIN_POWER_NORM,   // power iteration: S0 = ||p||^2
    FIN_FISTA_F,      // FISTA: residual of x_k, S0 = ||A x_k - y||^2 -> stop test, t_{k+1}, beta_k
    FIN_ETA_SIZE,     // Appendix rule: S0 = ||g_k||^2 -> the perturbation's size
    FIN_PROX_END,     // proximal perturbation applied (no sums): fix gamma_0, l <- l+1, trace
    FIN_PERTURB_NEXT  // a later one of several perturbations per step: S0 = TV, S1 = ||dTV||^2,
                      // S2 = ||x||^2 of x_{k+1/2} so far -> that sub-step's set-up
};
// Steps at or after FIN_POWER are finalised by finalize_rare (see there).
constexpr int kFirstRareStep = FIN_POWER;

__device__ __forceinline__ bool finite_pos(double v) { return v > 0.0 && isfinite(v); }
// Step of the proximal perturbation x_{k+1/2} = prox_{lambda TV}(x_k) (the
// footnote to Eq. superiorized): lambda = gamma_0 a^l / ||dTV(x_k)||, the
// implicit counterpart of the gamma rule's step x_k + gamma v; gamma_0 as in
// the gamma rule (gamma0_rel ||x|| of the first perturbed image unless given).
// 0 when the subgradient is zero (x_k is then kept).
__device__ __forceinline__ double prox_lambda(const DevState& st) {
    if (!(st.gnorm2 > 0.0)) return 0.0;
    const double g0 = st.gamma_fixed ? st.gamma0 : st.gamma0_rel * sqrt(st.xnorm2);
    return g0 * st.a_ell / sqrt(st.gnorm2);
}

// Status of a stop at the loop test "while f > eps": f <= eps is success; a
// non-finite f (NaN data or arithmetic) is a breakdown, not a convergence.
__device__ __forceinline__ int stop_status(const DevState& st) {
    return st.f_half <= st.eps ? SCG_OK : SCG_ERR_BREAKDOWN;
}

template <typename T>
__device__ __forceinline__ double* trace_row(const Prob<T>& P, int it) {
    if (P.trace == nullptr || it < 0 || it >= P.trace_rows) return nullptr;
    return P.trace + (size_t)it * TR_NF;
}

// Finish a loop body: the algorithm's k <- k+1.
__device__ __forceinline__ void end_body(DevState& st) {
    st.k += 1;
    st.iters += 1;
}

// First pending trial coefficient -gamma0 a^ell / ||dTV||; trial t of the
// pass uses trial_c0 * a^t.
__device__ __forceinline__ void set_trial_coefs(DevState& st) {
    st.trial_c0 = -st.gamma0 * st.a_ell / sqrt(st.gnorm2);
}
// Top of the while loop: test f(x_{k-1/2}) > eps (f(x_k) for CG/PCG) and the
// iteration cap, open the trace row and prepare the perturbation of x_k.
template <typename T>
__device__ void top_of_loop(const Prob<T>& P, DevState& st) {
    if (st.done) return;
    if (!(st.f_half > st.eps)) { st.done = 1; st.status = stop_status(st); return; }
    if (st.iters >= st.max_iter) { st.done = 1; st.status = SCG_WARN_MAX_ITER; return; }
    double* row = trace_row(P, st.iters);
    if (row) {
        for (int q = 0; q < TR_NF; ++q) row[q] = 0.0;
        row[TR_K] = st.k;
        row[TR_FTEST] = st.f_half;
        row[TR_TV_BEFORE] = st.tv_x;
        row[TR_ACCEPTED] = -1.0;
        row[TR_MARGIN] = __longlong_as_double(0x7ff0000000000000LL);
    }
    st.trials = 0;
    st.margin = __longlong_as_double(0x7ff0000000000000LL);
    st.coef = 0.0;
    if (st.family != FAM_CG && st.perturb == SCG_PERTURB_GAMMA && st.gnorm2 > 0.0) {
        if (!st.gamma_fixed) {
            st.gamma0 = st.gamma0_rel * sqrt(st.xnorm2);
            st.gamma_fixed = 1;
        }
        st.accepted = 0;              // trials pending
        set_trial_coefs(st);
    } else {
        st.accepted = -1;             // no perturbation this k
        if (row) { row[TR_TV_AFTER] = st.tv_x; row[TR_ELL] = (double)st.ell; }
    }
}

__device__ __forceinline__ void breakdown(DevState& st) {
    st.done = 1;
    st.status = SCG_ERR_BREAKDOWN;
    end_body(st);
}


// Steps that only the power iteration, FISTA and the Appendix rule take,
// finalised by the vector and sinogram passes that sum them (never by the
// projector or the gather), so that the finaliser those kernels inline holds
// only the steps of Algorithms 1-14.
template <typename T>
__device__ __noinline__ void finalize_rare(int step, const Prob<T>& P, DevState& st, const double* S) {
    double* row = trace_row(P, st.iters);
    switch (step) {
    case FIN_ETA_SIZE: {
        // the Appendix rule's gradient at x_k:
        // u_k = eta0 ||g_k|| v_k with v_k = -dTV/||dTV|| (Eq. up bnd u_k); on
        // the scaled system c A x ~ c y, S0 = c^4 ||g_k||^2.  No TV test:
        // x_{k+1/2} = x_k + u_k.
        const double ys = (double)P.y_scale;
        const double un = st.ex.eta0 * sqrt(S[0]) / (ys * ys);
        // (the loop test left accepted = -1: no gamma trials under this rule)
        if (!st.done && st.family != FAM_CG && st.perturb == SCG_PERTURB_ETA && st.gnorm2 > 0.0) {
            st.coef = -un / sqrt(st.gnorm2);
            st.accepted = 1;
            if (row) {
                row[TR_ACCEPTED] = 1.0;
                row[TR_GAMMA] = un;
                row[TR_ELL] = (double)st.ell;
            }
        }
        break;
    }
    case FIN_PROX_END: {
        // x_{k+1/2} = prox_{lambda TV}(x_k) has been formed: a prox step cannot
        // raise TV, so there is no trial; l <- l+1 once per perturbed step.  The
        // TV of x_{k+1/2} is not computed here (the trace's TV-after field is NaN).
        if (!st.done && st.family != FAM_CG && st.perturb == SCG_PERTURB_PROX && st.gnorm2 > 0.0) {
            const double lam = prox_lambda(st);
            if (!st.gamma_fixed) {
                st.gamma0 = st.gamma0_rel * sqrt(st.xnorm2);
                st.gamma_fixed = 1;
            }
            st.ell += 1;
            st.a_ell *= st.a;
            st.accepted = 1;
            if (row) {
                row[TR_ACCEPTED] = 1.0;
                row[TR_GAMMA] = lam;
                row[TR_ELL] = (double)st.ell;
                row[TR_TV_AFTER] = __longlong_as_double(0x7ff8000000000000LL);
            }
        }
        break;
    }
    case FIN_PERTURB_NEXT:
        // several perturbations per step: a later sub-step starts from x_{k+1/2}
        // so far (copied into x's buffer) with its own subgradient and trial
        // budget, l running on; set up as at the top of the loop, without the
        // loop test.  The trace row keeps TV(x_k) and takes the last sub-step's
        // perturbation fields.
        st.tv_x = S[0];
        st.gnorm2 = S[1];
        st.xnorm2 = S[2];
        st.trials = 0;
        st.margin = __longlong_as_double(0x7ff0000000000000LL);
        st.coef = 0.0;
        if (row) {
            row[TR_TRIALS] = 0.0;
            row[TR_ACCEPTED] = -1.0;
            row[TR_GAMMA] = 0.0;
            row[TR_MARGIN] = st.margin;
        }
        if (st.family != FAM_CG && st.perturb == SCG_PERTURB_GAMMA && st.gnorm2 > 0.0) {
            st.accepted = 0;                                // trials pending
            set_trial_coefs(st);
        } else {
            st.accepted = -1;                               // (the prox rule's step follows)
            if (row) { row[TR_TV_AFTER] = st.tv_x; row[TR_ELL] = (double)st.ell; }
        }
        break;
    case FIN_POWER:
        st.ex.c2 = S[1] / st.xnorm2;                        // Rayleigh quotient of A^T A at p
        st.coef = 1.0 / sqrt(S[0]);
        break;
    case FIN_POWER_NORM:
        st.xnorm2 = S[0];
        break;
    case FIN_FISTA_F:
        st.f_half = 0.5 * S[0];                          // f(x_k)
        if (st.in_init) {
            st.in_init = 0;                              // x_0: t_1 = 1, u_1 = x_0
        } else {
            const double t1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * st.ex.tk * st.ex.tk));
            if (row) {
                row[TR_K] = st.iters + 1;
                row[TR_ALPHA] = st.ex.tk;
                row[TR_BETA] = (st.ex.tk - 1.0) / t1;
                row[TR_F_AFTER] = st.f_half;
            }
            st.beta = (st.ex.tk - 1.0) / t1;                // u_{k+1} = x_k + beta (x_k - x_{k-1})
            st.ex.tk = t1;
            st.iters += 1;
            st.k += 1;
        }
        if (!(st.f_half > st.eps)) { st.done = 1; st.status = stop_status(st); }
        else if (st.iters >= st.max_iter) { st.done = 1; st.status = SCG_WARN_MAX_ITER; }
        break;
    default:
        break;
    }
}

template <typename T>
__device__ void finalize(int step, const Prob<T>& P, DevState& st, const double* S) {
    double* row = trace_row(P, st.iters);
    switch (step) {
    case FIN_F:
        st.f_half = 0.5 * S[0];
        if (!st.in_init) {
            if (row) row[TR_F_AFTER] = st.f_half;
            // f(x_{k+1/2}) <= eps ends the loop at the next test; the rest of
            // this step only produces x_{k+1}, which is never used.
            if (!(st.f_half > st.eps)) { st.done = 1; st.status = stop_status(st); end_body(st); }
        }
        break;
    case FIN_BETA: {
        st.gg = S[1];
        if (st.in_init) {
            st.beta = 0.0;
        } else if (st.variant == SCG_S_CG_CD) {
            if (S[1] == 0.0) st.beta = 0.0;
            else if (!(st.gTp < 0.0) || !isfinite(st.gTp)) { breakdown(st); break; }
            else st.beta = -S[1] / st.gTp;               // beta = -||g'||^2 / g^T p
        } else {
            st.beta = S[0] / st.pTh;                     // beta = g'^T h / p^T h (z'^T h for S-PCG)
        }
        if (row && !st.in_init) row[TR_BETA] = st.beta;
        // g'^T p' of the direction formed next, p' = -d + beta p (d = g', or z'
        // for S-PCG): -g'^T d + beta g'^T p from this pass's sums, so forming p'
        // needs no reduction of its own.  (16-bit storage recomputes it from the
        // rounded p' in that pass: FIN_NUM.)
        const double gd = st.variant == SCG_S_PCG ? S[3] : S[1];
        st.num = -gd + st.beta * S[2];
        if (st.variant == SCG_S_CG_CD) st.gTp = st.num;
        break;
    }
    case FIN_NUM:
        st.num = S[0];                                   // g'^T p'
        if (st.variant == SCG_S_CG_CD) st.gTp = S[0];
        break;
    case FIN_ALPHA:
        if (finite_pos(S[0])) st.alpha = -st.num / S[0]; // alpha = -g'^T p' / p'^T h'
        else if (st.gg == 0.0) st.alpha = 0.0;
        else { breakdown(st); break; }
        st.pTh = S[0];
        if (row && !st.in_init) row[TR_ALPHA] = st.alpha;
        break;
    case FIN_END:
        st.tv_x = S[0];
        st.gnorm2 = S[1];
        st.xnorm2 = S[2];
        if (st.in_init) st.in_init = 0;
        else end_body(st);
        top_of_loop(P, st);
        break;
    case FIN_TRIAL: {
        const int nc = st.pass_cands;
        const double base = S[nc];
        int valid = st.max_trials - st.trials;
        if (valid > nc) valid = nc;
        int acc = -1;
        for (int t = 0; t < valid; ++t) {
            double rel = fabs(S[t] - base) / (base > 0.0 ? base : 1.0);
            if (rel < st.margin) st.margin = rel;
            if (S[t] <= base) { acc = t; break; }
        }
        if (acc >= 0) {
            st.coef = st.trial_c0 * st.apow[acc];       // the coefficient k_trial tested
            const double gamma = st.gamma0 * st.a_ell * st.apow[acc];
            st.a_ell = st.a_ell * st.apow[acc] * st.a;   // a^(ell + acc + 1)
            st.ell += acc + 1;
            st.trials += acc + 1;
            st.accepted = 1;
            if (row) {
                row[TR_TRIALS] = st.trials;
                row[TR_ACCEPTED] = 1.0;
                row[TR_GAMMA] = gamma;
                row[TR_TV_AFTER] = S[acc];
                row[TR_ELL] = (double)st.ell;
                row[TR_MARGIN] = st.margin;
            }
        } else {
            if (valid > 0) st.a_ell = st.a_ell * st.apow[valid - 1] * st.a;   // a^(ell + valid)
            st.ell += valid;
            st.trials += valid;
            if (st.trials >= st.max_trials) {
                st.accepted = 2;                         // gave up: x_{k+1/2} = x_k
                st.coef = 0.0;
                if (row) {
                    row[TR_TRIALS] = st.trials;
                    row[TR_ACCEPTED] = 0.0;
                    row[TR_TV_AFTER] = base;
                    row[TR_ELL] = (double)st.ell;
                    row[TR_MARGIN] = st.margin;
                }
            } else {
                set_trial_coefs(st);
            }
        }
        break;
    }
    case FIN_CG_DELTA:
        st.delta = (st.variant == SCG_PCG || st.variant == SCG_S_PCG_K) ? S[1] : S[0];
        st.inner_stop = 0;
        break;
    case FIN_CG_ALPHA:
        if (st.inner_stop) { st.alpha = 0.0; break; }
        if (finite_pos(S[0])) { st.alpha = st.delta / S[0]; }       // alpha = delta / p^T h
        else if (st.delta == 0.0) {
            st.alpha = 0.0;
            st.inner_stop = 1;
            if (st.family == FAM_CG) { st.done = 1; st.status = SCG_OK; }
        } else { breakdown(st); break; }
        if (row && st.family == FAM_CG) row[TR_ALPHA] = st.alpha;
        break;
    case FIN_CG_F:
        st.f_half = 0.5 * S[0];
        break;
    case FIN_CG_BETA: {
        if (st.inner_stop) { st.beta = 0.0; break; }
        double dn = (st.variant == SCG_PCG || st.variant == SCG_S_PCG_K) ? S[1] : S[0];
        st.beta = dn / st.delta;                         // beta = delta' / delta
        st.delta = dn;
        if (row && st.family == FAM_CG) row[TR_BETA] = st.beta;
        break;
    }
    case FIN_CG_END:
        if (st.in_init) st.in_init = 0;
        else end_body(st);
        top_of_loop(P, st);
        break;
    case FIN_RESUME:
        st.pTh = S[0];
        st.gTp = S[1];
        break;
    case FIN_TV:
        if (P.trace) P.trace[0] = S[0];
        break;
    case FIN_FINAL_F:
        st.f_final = 0.5 * S[0];
        break;
    case FIN_FINAL_TV:
        st.tv_final = S[0];
        break;
    default:
        break;
    }
}

}  // namespace scg
