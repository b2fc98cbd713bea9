/*
 * mlp_surrogate.h - C ABI of the learned surrogate for a B-spline orbital table.
 *
 * Not in arXiv:1611.02665 (which evaluates the spline only). A periodic
 * Fourier-feature MLP stands in for a large coefficient table: its inputs are
 * sin(2 pi k x_d), cos(2 pi k x_d) for k = 1..nfreq and the three fractional
 * coordinates (6*nfreq features, zero-padded to a multiple of 64), followed by
 * `layers` hidden layers of `hidden` SiLU units and a linear output of `nout`
 * orbital values. Weights and activations are bfloat16 with FP32
 * accumulation on the tensor cores (tcgen05, sm_103a); master weights and
 * Adam moments are FP32. Gradients and Laplacians of the orbitals come from
 * forward-mode propagation of (value, d/dx, d/dy, d/dz, Laplacian) through
 * the network: the Laplacian of a layer's pre-activation is W times the
 * previous layer's, and SiLU adds silu''(z) |grad z|^2 + silu'(z) lap z, so
 * one stream carries it. The plain spline (bspline_gb300.h) produces
 * the training targets and judges the surrogate's error.
 *
 * Conventions follow bspline_gb300.h: device pointers, asynchronous on
 * `stream`, status codes of type bspline_status, argument errors detected on
 * the host. Output layouts match the spline's: v[p*ld + n], g[(p*3+d)*ld + n],
 * l[p*ld + n]; ld must be a multiple of 4 and >= nout, output pointers 16-byte
 * aligned.
 */
#ifndef MLP_SURROGATE_H
#define MLP_SURROGATE_H

#include <stddef.h>

#include "bspline_gb300.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mlp_s *mlp_t;

/* nfreq 1..64, hidden a multiple of 128 (<= 4096), layers 1..6, nout a
 * multiple of 128 (<= 8192). Allocates parameters, gradients and Adam
 * moments on the current device; weights start at zero until mlp_init or
 * mlp_set_params. */
bspline_status mlp_create(int nfreq, int hidden, int layers, int nout, mlp_t *out);
bspline_status mlp_destroy(mlp_t m);

/* Number of FP32 parameters. Packing, layer by layer (layer 0 = first hidden,
 * layer `layers` = output): W[out][in] row-major, then b[out]. Layer 0's `in`
 * is the padded feature count (columns beyond 6*nfreq multiply zeros). */
size_t mlp_param_count(mlp_t m);
int mlp_feature_count(mlp_t m); /* padded input width */

/* Device status word of the surrogate: BSPLINE_OK, or BSPLINE_ERR_TIMEOUT if
 * a bounded wait inside one of its kernels ran out (a pipeline barrier) since
 * the last reset
 * (the first condition met is kept). Synchronises stream first; reset != 0
 * clears the word. */
bspline_status mlp_device_status(mlp_t m, void *stream, int reset);

/* Which GEMM kernel the network's layers run on: 0 = the library's choice
 * (one CTA per 128 x 256 or 128 x 128 tile), 1 = one CTA per tile, 2 = CTA
 * pairs on 256 x 256 tiles (tcgen05 cta_group::2 on clusters of two)
 * wherever the layer allows them (its width a multiple of 256 and no K
 * split), 3 = two CTAs per SM on 128 x 128 tiles (8 epilogue warps each, a
 * shallower operand ring) wherever the width is a multiple of 128. 0 and 1
 * give the same bits; 2 and 3 the same values up to FP32 summation order.
 * For tests and measurements; BSPLINE_ERR_ARG for another value. */
bspline_status mlp_set_gemm_kernel(mlp_t m, int kernel);

/* Uniform(-sqrt(6/in), sqrt(6/in)) / 2 weights, zero biases, from a 64-bit
 * seed; resets Adam. Synchronous. */
bspline_status mlp_init(mlp_t m, unsigned long long seed);
/* Host copies of the FP32 master parameters / last step's gradients. Synchronous. */
bspline_status mlp_get_params(mlp_t m, float *host, size_t count);
bspline_status mlp_set_params(mlp_t m, const float *host, size_t count);
bspline_status mlp_get_grads(mlp_t m, float *host, size_t count);

/* One Adam step on a batch: positions x,y,z (device double[batch]), targets
 * (device float [batch][ld_target], the spline's values), loss = mean squared
 * error over batch*nout values. batch: a positive multiple of 128. lr >= 0
 * (0 computes gradients without moving the weights). beta1 0.9, beta2 0.999,
 * eps 1e-8. loss_out (device float, may be NULL) receives the batch loss. */
bspline_status mlp_train_step(mlp_t m, int batch, const double *x, const double *y, const double *z,
                              const float *target, int ld_target, float lr, float *loss_out, void *stream);

/* One Adam step on values AND gradients (an optional gradient term of the
 * surrogate loss; not in the paper): the loss is
 *   mean over batch*nout of (v - target_v)^2
 *   + lambda * mean over batch*3*nout of (g - target_g)^2,
 * with the network's gradients g = d v / d x_d by forward-mode propagation
 * (each position is trained as 4 rows: its value and its three derivatives,
 * whose pre-activations carry no bias) and the loss gradient by reverse mode
 * through that propagation. target_v: device float [batch][ld_target];
 * target_g: device float [batch][3][ld_target] (the spline's VGL gradients).
 * batch: a positive multiple of 32; lambda >= 0 (0 gives the value loss on
 * the same rows); lr as for mlp_train_step. loss_out (device float, may be
 * NULL) receives the batch loss. Shares the training workspace, Adam state
 * and step counter with mlp_train_step. */
bspline_status mlp_train_step_vg(mlp_t m, int batch, const double *x, const double *y, const double *z,
                                 const float *target_v, const float *target_g, int ld_target, float lambda,
                                 float lr, float *loss_out, void *stream);

/* Orbital values at npos positions (device): v [npos][ld]. */
bspline_status mlp_eval_v(mlp_t m, int npos, const double *x, const double *y, const double *z, float *v,
                          int ld, void *stream);
/* Values, gradients and Laplacians by forward-mode propagation (device). */
bspline_status mlp_eval_vgl(mlp_t m, int npos, const double *x, const double *y, const double *z, float *v,
                            float *g, float *l, int ld, void *stream);

/* Weights + Adam state to a file: one JSON header line, then FP32 params,
 * first and second moments (little-endian). mlp_load requires matching
 * sizes. Synchronous. */
bspline_status mlp_save(mlp_t m, const char *path);
bspline_status mlp_load(mlp_t m, const char *path);

/* The tensor-core GEMM on its own, for testing: C[M][N] (float, ldc) =
 * A[M][K] . B[N][K]^T with A, B bfloat16 row-major (device). M >= 1,
 * N a multiple of 128, K a multiple of 64, ldc >= N and a multiple of 4.
 * splitk > 1 splits K over CTAs and sums with FP32 atomics (C is zeroed
 * first). */
bspline_status mlp_gemm_bf16(const void *A, const void *B, float *C, int M, int N, int K, int ldc, int splitk,
                             void *stream);

/* The same with the kernel chosen: kernel 0 = the library's choice (as
 * mlp_gemm_bf16), 1 = one CTA per 128 x 256 (or 128 x 128) tile, 2 = CTA
 * pairs on 256 x 256 tiles (tcgen05 cta_group::2 on clusters of two CTAs)
 * where N is a multiple of 256 and splitk is 1, else as 1, 3 = two CTAs
 * per SM on 128 x 128 tiles where N is a multiple of 128, else as 1. The
 * network's own GEMMs follow mlp_set_gemm_kernel. Errors as mlp_gemm_bf16,
 * and BSPLINE_ERR_ARG for another kernel value. */
bspline_status mlp_gemm_bf16_ex(const void *A, const void *B, float *C, int M, int N, int K, int ldc, int splitk,
                                int kernel, void *stream);

/* Tensor-pipe work of the last call of each kind, for reporting: dense
 * flops issued to tcgen05.mma per mlp_eval_v / mlp_eval_vgl / mlp_train_step
 * call at the given size (2*M*N*K summed over the GEMMs, padding included). */
double mlp_flops(mlp_t m, int what /* 0 eval_v, 1 eval_vgl, 2 train_step, 3 train_step_vg */, int n);

#ifdef __cplusplus
}
#endif

#endif /* MLP_SURROGATE_H */
