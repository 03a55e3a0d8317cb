/*
 * vp_fno.h -- C ABI of the Fourier-neural-operator surrogate in libvp.so.
 *
 * The paper has no learned component; this surrogate maps the normalised fundamental
 * on an N^3 focal box to the normalised harmonics 2..5 on the same box, and the plain
 * volume potential (vp.h) stays the reference for its error and the fallback.  The cascade
 * of Eq. 2.6 makes p_n homogeneous of degree n in p1, so with s = max |p1| the network
 * maps q1 = p1 / s (2 channels: Re, Im) to q_n = p_n / s^n (8 channels: Re, Im of
 * n = 2..5), and p_n = s^n q_n exactly undoes the scaling.
 *
 * Architecture (Fourier neural operator, L layers, width W, projection width H):
 *   h0 = phi(x) P + bP                                       (10 -> W)
 *   t_l = K_l(h_l) + h_l W_l + b_l,  h_{l+1} = GELU(t_l) for l < L-1, else t_l
 *   y = GELU(h_L Q1 + bQ1) Q2 + bQ2                          (W -> H -> 8)
 * phi(x) = (Re, Im of q^k, k = 1..5) with q = x0 + i x1: since p_n grows like p1^n times
 * a slowly varying envelope, the lift sees the powers of the normalised fundamental.
 * K_l: real 3-D DFT of each channel, keep kx in the lowest modes[0] (half non-negative,
 * half negative), ky likewise with modes[1], kz in [0, modes[2]); multiply every kept
 * mode by a complex W x W matrix R_l; inverse real DFT with the remaining modes zero
 * (the irfftn convention: 1/N^3, the kz = 0 imaginary part ignored).  GELU is
 * x (1 + erf(x / sqrt 2)) / 2.
 * Loss: (1/4) sum_n ||y_n - q_n||^2 / ||q_n||^2 (relative squared L2 per harmonic).
 *
 * Precision: parameters are kept as an FP32 master copy (`params`) and a BF16 copy
 * (`params_bf16`, same layout) used by the tensor-core GEMMs; activations are BF16,
 * every contraction over voxels accumulates in FP32 on BF16 tensor cores
 * (mma.sync m16n8k16); the truncated x/y transforms and the mode mixing run in FP32.
 *
 * Layouts: x is FP32 [N^3][2], targets and outputs FP32 [N^3][8], voxels x-major with z
 * fastest.  Parameters are one flat array; vp_fno_param_offsets gives the offsets of
 * P, bP, (R_l, W_l, b_l) for each layer, Q1, bQ1, Q2, bQ2 and the total count.
 * R_l is [mx][my][mz][W][W][2] (kept modes in kx-slot, ky-slot, kz order; slot j < m/2
 * is frequency j, else N - m + j; complex as Re, Im); W_l is [W][W] (in, out); P is
 * [10][W] (feature rows in phi's order); Q1 is [W][H]; Q2 is [H][8].
 * All pointers are device pointers; every call is asynchronous on `stream`.
 */
#ifndef VP_FNO_H
#define VP_FNO_H

#include "vp.h"

#ifdef __cplusplus
extern "C" {
#endif

#define VP_FNO_MAX_LAYERS 8
#define VP_FNO_POWERS 5                 /* powers of q in the input features */
#define VP_FNO_IN (2 * VP_FNO_POWERS)   /* input features per voxel          */

typedef struct vp_fno_desc {
    int n;          /* box voxels per axis, 4..256                         */
    int width;      /* W, 1..256                                           */
    int hidden;     /* H, 1..512                                           */
    int layers;     /* L, 1..VP_FNO_MAX_LAYERS                             */
    int modes[3];   /* mx, my (even, <= n), mz (1..n/2)                    */
} vp_fno_desc;

/* Number of parameters (FP32 entries), or -1 for an invalid descriptor. */
VP_API long long vp_fno_param_count(const vp_fno_desc* d);

/* Offsets (entries) of P, bP, then R_l, W_l, b_l for l = 0..L-1, then Q1, bQ1, Q2, bQ2,
 * then the total: 3 L + 7 values.  Errors: VP_ERR_ARG. */
VP_API int vp_fno_param_offsets(const vp_fno_desc* d, long long* offsets);

/* Bytes of device workspace one forward + backward needs (activations kept for the
 * backward pass), or -1 for an invalid descriptor. */
VP_API long long vp_fno_workspace_bytes(const vp_fno_desc* d);

/* Forward pass of one sample: y (FP32 [N^3][8], may be NULL) from x; keeps the
 * activations in ws for vp_fno_loss / vp_fno_backward.  Errors: VP_ERR_ARG, VP_ERR_CUDA. */
VP_API int vp_fno_forward(const vp_fno_desc* d, const float* params, const void* params_bf16, const float* x,
                          float* y, void* ws, vp_stream_t stream);

/* Inference: y (FP32 [N^3][8], required) from x, the same function as vp_fno_forward but
 * keeping no activations (vp_fno_loss / vp_fno_backward must not follow it) and with the
 * projection fused into one kernel.  ws as for vp_fno_forward.
 * Errors: VP_ERR_ARG, VP_ERR_CUDA. */
VP_API int vp_fno_infer(const vp_fno_desc* d, const float* params, const void* params_bf16, const float* x,
                        float* y, void* ws, vp_stream_t stream);

/* Loss of the last forward pass against target: sums8[n] = ||y_n - q_n||^2 and
 * sums8[4 + n] = ||q_n||^2, n = 0..3 (device FP32[8], may be NULL; the sums are also
 * kept in ws for vp_fno_backward).  Errors: VP_ERR_ARG, VP_ERR_CUDA. */
VP_API int vp_fno_loss(const vp_fno_desc* d, const float* target, float* sums8, void* ws, vp_stream_t stream);

/* Backward pass of the last forward / loss: ADDS the gradient of the loss to grads
 * (FP32, parameter layout; zero it before the first sample of a batch).
 * Errors: VP_ERR_ARG, VP_ERR_CUDA. */
VP_API int vp_fno_backward(const vp_fno_desc* d, const float* params, const void* params_bf16, const float* x,
                           const float* target, float* grads, void* ws, vp_stream_t stream);

/* One Adam step over n parameters: m, v moments, bias corrections c1 = 1 - b1^t,
 * c2 = 1 - b2^t, gradients scaled by grad_scale first; refreshes the BF16 copy.
 * Errors: VP_ERR_ARG, VP_ERR_CUDA. */
VP_API int vp_fno_adam(long long n, float* params, void* params_bf16, const float* grads, float* m, float* v,
                       float lr, float b1, float b2, float eps, float c1, float c2, float grad_scale,
                       vp_stream_t stream);

/* BF16 copy of n FP32 values (e.g. to refresh params_bf16).  Errors: VP_ERR_ARG, VP_ERR_CUDA. */
VP_API int vp_fno_to_bf16(long long n, const float* src, void* dst, vp_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* VP_FNO_H */
