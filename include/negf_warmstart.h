/*
 * negf_warmstart.h -- the learned initial guess of the lead surface Green's
 * function (part of libnegf.so; same context, stream and error conventions as
 * negf.h).
 *
 * The open-boundary term of the paper (Sec. II: the boundary self-energy "not
 * shown here") needs, per energy and lead, the surface Green's function g of a
 * semi-infinite periodic lead with onsite block H00 and hop H01:
 *     g = (a00 - a01 g a10)^{-1},  a00 = z - H00, a01 = -H01, a10 = -H01^H  (S = I).
 * negf_obc() solves it by decimation; given a guess g0 it first tries Newton steps
 * from g0 and keeps the result only if it passes the residual target and the
 * retarded-root test (see negf_obc in negf.h).  The functions below produce g0 with
 * a small network (no counterpart in the paper) and train it on pairs that
 * negf_obc() generates:
 *
 *   features  x = [sqrt(b) Re diag H00 | sqrt(b) Re H00[i<j] | sqrt(b) Im H00[i<j]
 *                  | sqrt(b) Re H01 | sqrt(b) Im H01 | E/3
 *                  | sin(w_m E), cos(w_m E) for m = 0..31, w_m = 2^(m/4)]
 *             (K0 = 3 b^2 + 65 values, upper triangles row-major, zero-padded to
 *             K0P = multiple of 128; the sine/cosine pairs are a Fourier encoding of
 *             the energy, which one BF16 feature would resolve only to ~1%)
 *   network   h1 = relu(W1 x + c1), h2 = relu(W2 h1 + c2), y = W3 h2 + c3
 *   output    g0 = y[0:b^2] + i y[b^2:2b^2]  (row-major b x b)
 *   loss      mean over the batch and the 2 b^2 outputs of (y - t)^2, t = [Re g | Im g]
 *   optimiser Adam with bias correction (beta1 0.9, beta2 0.999, eps 1e-8).
 *
 * Precision: BF16 operands on the tcgen05 tensor cores (features, weights, hidden
 * activations and back-propagated signals are rounded to BF16, round to nearest
 * even, where they enter a product), FP32 accumulation in tensor memory, FP32
 * master weights and optimiser state, FP64 loss.  The left lead of a device is the
 * same problem with H01 replaced by H01^H.
 *
 * Parameters live in one caller-owned FP32 device vector laid out as
 *   W1 [hidden][K0P], c1 [hidden], W2 [hidden][hidden], c2 [hidden],
 *   W3 [2b^2][hidden], c3 [2b^2]            (row-major; offsets in negf_mlp_dims),
 * with the Adam moments and the gradient in vectors of the same layout.
 * Requirements: b a multiple of 8 (so that 2 b^2 is a multiple of 128), hidden a
 * positive multiple of 128.  Samples are processed in row tiles of 128: buffers
 * sized by n are sized by NP = n rounded up to a multiple of 128.
 */
#ifndef NEGF_WARMSTART_H
#define NEGF_WARMSTART_H

#include "negf.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t b, hidden;        /* lead block size, hidden width                          */
  int32_t k0, k0p, nout;    /* 3b^2+65, k0 rounded up to 128, 2b^2                    */
  int64_t off_W1, off_c1, off_W2, off_c2, off_W3, off_c3;   /* element offsets        */
  int64_t n_params;         /* total FP32 parameters                                  */
} negf_mlp_dims;

/* Host only.  Fills `out` for leads of block size b and the given hidden width;
 * NEGF_ERR_ARG if b or hidden break the requirements above. */
negf_status negf_mlp_get_dims(int32_t b, int32_t hidden, negf_mlp_dims* out);

/* Feature rows of n samples: sample s takes lead lead[s] (H00/H01 = device
 * [nlead][b][b] complex128) at energy E[s] (device double).  X: device BF16
 * [NP][K0P], rows >= n written as zeros; lead: device int32 [n], each in
 * [0, nlead).  A row whose lead index is out of range is written as zeros and
 * NEGF_ERR_ARG is recorded in the context's error word (returned by
 * negf_ctx_sync).  The BF16 values are the features rounded once from FP64,
 * nearest even. */
negf_status negf_mlp_pack(negf_ctx* ctx, int32_t b, int32_t n, int32_t nlead, const void* H00,
                          const void* H01, const int32_t* lead, const double* E, void* X,
                          negf_stream stream);

/* Inference: g0[s] (device complex128 [n][b][b]) for the n feature rows of X
 * (device BF16 [NP][K0P], from negf_mlp_pack).  params: device FP32 [n_params]. */
negf_status negf_mlp_forward(negf_ctx* ctx, const negf_mlp_dims* dims, const float* params, int32_t n,
                             const void* X, void* g0, negf_stream stream);

/* One training step on a batch of n samples: forward, loss, backward, and (when
 * `update` != 0) the Adam update with step index `step` (>= 1) and learning rate lr.
 *   params, adam_m, adam_v : device FP32 [n_params], updated in place
 *   grad                   : device FP32 [n_params], out: the gradient of the loss
 *                            at the incoming parameters
 *   rows                   : device int32 [n] or NULL.  NULL: the batch is rows 0..n-1
 *                            of X and g_target.  Otherwise batch row r is sample rows[r]
 *                            of a larger set (a minibatch; each index in [0, n_set))
 *   X                      : device BF16 [NP][K0P] features (NP from n, or from n_set
 *                            when rows is given)
 *   g_target               : device complex128 targets (surface functions), [n][b][b]
 *                            or [n_set][b][b] when rows is given
 *   loss                   : device double [1], out: the loss at the incoming parameters
 * An index outside [0, n_set) makes that row contribute nothing and records
 * NEGF_ERR_ARG in the context's error word.  The context workspace holds the
 * activations (negf_mlp_workspace_bytes). */
negf_status negf_mlp_train_step(negf_ctx* ctx, const negf_mlp_dims* dims, float* params, float* adam_m,
                                float* adam_v, float* grad, int32_t step, float lr, int32_t n,
                                const int32_t* rows, int32_t n_set, const void* X, const void* g_target,
                                double* loss, int32_t update, negf_stream stream);

/* Host only.  Workspace bytes negf_mlp_train_step / negf_mlp_forward need for n
 * samples (the context must have been created with at least this much). */
size_t negf_mlp_workspace_bytes(const negf_mlp_dims* dims, int32_t n);

#ifdef __cplusplus
}
#endif

#endif /* NEGF_WARMSTART_H */
