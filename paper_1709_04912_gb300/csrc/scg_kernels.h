// scg_kernels.h -- host-side launchers of the kernels in kernels.cu.
#pragma once

#include "scg_device.cuh"

namespace scg {

enum ProjMode { PROJ_PLAIN = 0, PROJ_RESIDUAL = 1, PROJ_PLAIN_OUT = 2 };
enum FiltMode { FILT_VIEW = 0, FILT_PLAIN = 1, FILT_FBP = 2 };

enum VecOp {
    VEC_INIT = 0,          // X = XH = x0 (AUX or zeros); views
    VEC_VIEWS = 1,         // views of img[sel]
    VEC_PERTURB = 2,       // XH = X + coef * TVG; views
    VEC_FORM_P = 3,        // P = -img[sel] + beta P; views; S0 = G^T P
    VEC_FORM_P0 = 4,       // P = -img[sel]; views; S0 = G^T P
    VEC_FORM_P_NOVIEW = 5, // P = -img[sel] + beta P
    VEC_CG_UPDATE = 6,     // X = img[sel] + alpha P; G += alpha H; S0 = ||G||^2, S1 = G^T Z
    VEC_DOTS_RESUME = 7,   // S0 = P^T H, S1 = G^T P
    VEC_POWER_START = 8,   // P = start vector of the power iteration; views; S0 = ||P||^2
    VEC_NORMALIZE = 9,     // P = coef H; views; S0 = ||P||^2
    VEC_FISTA_B = 10,      // Z = u - G / c^2, u = img[c] + beta (img[c] - img[p]); sel = c | p << 4
    VEC_FGP_FINAL = 11,    // img[d] = Z - (lambda/c^2) L^T dual[w]; views; sel = d | w << 4 (w = 2: none)
    VEC_FISTA_OUT = 12,    // Z = user_out = x_k (buffer chosen by the device's k)
    VEC_POWER_DOTS = 13,   // S0 = ||H||^2, S1 = P^T H
    VEC_NORM_G = 14,       // S0 = ||G||^2
    VEC_COPY_HALF = 15     // X = XH: the next of several perturbations per step starts from x_{k+1/2}
};

template <typename T>
void launch_project(const Prob<T>* d, const Item* items, int grid, int dst, int mode, int step,
                    cudaStream_t s);
template <typename T>
void launch_backproject(const Prob<T>* d, const Item* items, int grid, int nrhs, int src0,
                        int src1, int dst0, int dst1, int step, cudaStream_t s);
template <typename T>
void launch_vec(const Prob<T>* d, const Item* items, int grid, int op, int sel, int step,
                cudaStream_t s);
template <typename T>
void launch_tvgrad(const Prob<T>* d, const Item* items, int grid, int src, int fuse,
                   int write_grad, int step, cudaStream_t s);
template <typename T>
void launch_trial(const Prob<T>* d, const Item* items, int grid, int ncand, cudaStream_t s);
template <typename T>
void launch_sino_axpy(const Prob<T>* d, const Item* items, int grid, int step, cudaStream_t s);
// mode: FILT_VIEW / FILT_PLAIN / FILT_FBP (see k_filter)
template <typename T>
cudaError_t launch_filter(const Prob<T>* d, const Item* items, int grid, int max_nb, int src,
                          int dst, int mode, cudaStream_t s);
template <typename T>
void launch_sino_pairs(const Prob<T>* d, int grid, int dst, cudaStream_t s);
template <typename T>
void launch_sino_comb(const Prob<T>* d, const Item* items, int grid, int cur, int prev, cudaStream_t s);
template <typename T>
void launch_fgp(const Prob<T>* d, const Item* items, int grid, int j, double beta, int mode, cudaStream_t s);
template <typename T>
void launch_fgp2(const Prob<T>* d, const Item* items, int grid, int p, double beta0, double beta1, int mode,
                 cudaStream_t s);
template <typename T>
void launch_sino_norm(const Prob<T>* d, const Item* items, int grid, int src, int step, cudaStream_t s);
void launch_loop_cond(DevState* st, cudaGraphConditionalHandle h, cudaStream_t s);
void launch_write_result(const DevState* st, scg_result* res, double s2, int cg_family, int base_launches,
                         int body_kernels, cudaStream_t s);
void noalloc_forget();   // scg_tv_static's cached scratch addresses (noalloc.cu)
template <typename T>
void launch_set_io(Prob<T>* d, const typename Tr<T>::S* in_sino, typename Tr<T>::S* out_sino,
                   typename Tr<T>::S* image, cudaStream_t s);
template <typename T>
void launch_set_done(const Prob<T>* d, int count, int value, cudaStream_t s);
template <typename T>
void launch_slots_done(const Prob<T>* d, const int* slots, int count, int* out, int set, int value,
                       cudaStream_t s);
template <typename T>
void launch_loop_cond_batch(const Prob<T>* d, BatchState* bs, cudaGraphConditionalHandle h, cudaStream_t s);

}  // namespace scg
