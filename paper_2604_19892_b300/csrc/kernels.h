// Launch wrappers of the device kernels (instantiated for R = double, float).
#pragma once
#include <cuda_runtime.h>

#include "dev.cuh"

namespace ipcb {

// exclusive prefix sum of n ints (out may alias in); tmp needs >= n/1024 + 2 ints
void scan_exclusive(const int* in, int* out, int n, int* tmp, cudaStream_t st);

// predictor x~ = x + h v + h^2 g_ext and x_start = x (Algorithm 1 input)
template <class R> void launch_predict(const Dev<R>& D, cudaStream_t st);
// x_try = x + a_v p with a_v = alpha_{d(v)} (mode 0), c * alpha_{b(v)}
// (mode 1, per body) or c (mode 2, uniform)
template <class R> void launch_trial_positions(const Dev<R>& D, int mode, double c, cudaStream_t st);
// E(x) and grad E(x) with the contact set C of x (Eq. 1); E accumulates into *E
template <class R> void launch_energy_grad(const Dev<R>& D, const double* x, const ContactBuf& C, R* g,
                                           double* E, cudaStream_t st);
// active contacts at x into C (ComputeConstraintSet); min distance into S->min_dist
template <class R> void launch_detect(const Dev<R>& D, const double* x, const ContactBuf& C, cudaStream_t st);
// RebuildMAS at x with contacts C: projected tet Hessians, level blocks,
// batched inversion, C_base snapshot
template <class R> void launch_restart(const Dev<R>& D, const double* x, const ContactBuf& C, cudaStream_t st);
// the batched inversion of the assembled blocks alone (part of launch_restart)
template <class R> void launch_invert(const Dev<R>& D, cudaStream_t st);
// picks the CTAs per SM of the persistent plain block apply by timing the
// candidates on this scene's blocks (zeroed first), sets D.apply_ctas and
// returns it (0 if timing failed: the default is used)
template <class R> int autotune_apply(Dev<R>& D, cudaStream_t st);
// classify C against C_base, per-subdomain top-K (Sec. 4.1.1)
template <class R> void launch_classify(const Dev<R>& D, const ContactBuf& C, cudaStream_t st);
// z = P g with optional Woodbury update (Eq. 7-8)
template <class R> void launch_precond(const Dev<R>& D, const R* g, R* z, const ContactBuf& C, bool woodbury,
                                       cudaStream_t st);
// the three parts of launch_precond: coarse restriction, block apply of all
// levels (with the Woodbury correction at level 0), prolongation
template <class R> void launch_restrict(const Dev<R>& D, const R* g, cudaStream_t st);
template <class R> void launch_blocks(const Dev<R>& D, const R* g, R* z, const ContactBuf& C, bool woodbury,
                                      cudaStream_t st);
template <class R> void launch_prolong(const Dev<R>& D, R* z, cudaStream_t st);
// reductions for the 2x2 system (supplement Eq. 13-19), r_k and |z|_inf
template <class R> void launch_forms(const Dev<R>& D, const ContactBuf& C, bool restart, cudaStream_t st);
// the two halves of launch_forms: packing z, p and zeroing the sums; the
// reduction kernel itself
template <class R> void launch_forms_prep(const Dev<R>& D, bool restart, cudaStream_t st);
template <class R> void launch_forms_main(const Dev<R>& D, const ContactBuf& C, bool restart, cudaStream_t st);
// (mu, nu) and p <- -mu z + nu p
template <class R> void launch_direction(const Dev<R>& D, bool restart, cudaStream_t st);
// per-subdomain step sizes for p at x with verification (supplement Sec. 3)
template <class R> void launch_ccd(const Dev<R>& D, cudaStream_t st);
// cached candidate pairs: build at x with margin delta; proximity and CCD
// over the listed pairs (same results as launch_detect / launch_ccd while
// every vertex stays within delta of the build positions)
template <class R> void launch_cand_build(const Dev<R>& D, const double* x, double delta, cudaStream_t st);
template <class R> void launch_detect_list(const Dev<R>& D, const double* x, const ContactBuf& C, cudaStream_t st);
// part 0: all; 1: the per-pair bounds only; 2: the verification only
template <class R> void launch_ccd_list(const Dev<R>& D, cudaStream_t st, int part = 0);
template <class R> void launch_global_alpha(const Dev<R>& D, cudaStream_t st);
// S->accepted = E_try <= E_k + tau (the rounding allowance of the energies)
template <class R> void launch_accept(const Dev<R>& D, cudaStream_t st);
// FMA throughput of the SIMT pipe for T (float or double) in TFLOP/s, from one
// launch of about target_ms on the current device; 0 on success
template <class T> int measure_fma_peak(double target_ms, double* tflops);
// H_base-only forms for evaluation entry points
template <class R> void launch_zero_scalars(const Dev<R>& D, cudaStream_t st);

}  // namespace ipcb
