/*
 * lee_mlp.h -- the learned non-reflecting boundary (library addition; the paper treats periodic
 * domains only, Sec. 2.2, and leaves boundaries to future work, Sec. 10).
 *
 * At each edge cell of an open 2D five-velocity grid one population enters from outside.  A small
 * network predicts it from the post-collision populations of the 3-cell strip along the inward
 * normal:
 *   h      = the 15 values g_i / f*_i of the strip (depth 0, 1, 2; per depth the velocities in the
 *            canonical order rest, inward, outward, tangential+, tangential-, i.e. the edge is
 *            rotated onto the left edge by a proper rotation; for 16-bit storage the stored
 *            values S g_i / f*_i are used as they are),
 *   s      = max(rms(h), 1e-30),  x = (h / s, 0)  (16 values),
 *   y      = W3 GELU(W2 GELU(W1 x + b1) + b2) + b3,   GELU(z) = z (1 + erf(z / sqrt 2)) / 2,
 *   g_in   = a s y f*_in   (a s y for 16-bit storage, in stored units).  The factor a <= 1 is
 *            the passivity bound of each group of 16 consecutive border rows (rows ordered x = 0,
 *            x = nx - 1, y = 0, y = ny - 1, then along the edge): a = min(1, sqrt(sum h_out^2 /
 *            sum (s y)^2)) over the group, h_out the outward population leaving through the same
 *            cell (strip slot 2 at depth 0).  The edge then never adds weighted energy
 *            sum g^2 / f*, so with tau >= 1/2 the step is L2-stable for any network weights.
 * Sizes 16 -> 64 -> 64 -> 1.  The GEMMs run on the tensor cores (mma.sync m16n8k16, BF16 inputs,
 * FP32 accumulation): weights and every layer input are rounded to BF16, biases stay FP32.
 *
 * Parameter vector (FP32, LEE_MLP_NPARAM values, row-major out x in):
 *   W1[64][16], b1[64], W2[64][64], b2[64], W3[1][64], b3[1]
 * (column 15 of W1 multiplies the zero pad).
 *
 * All device pointers below must be valid on the network's stream; calls are asynchronous unless
 * they read or write host memory.
 */
#ifndef LEE_MLP_H
#define LEE_MLP_H

#include <stdint.h>

#include "lee_batch.h"
#include "lee_lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

#define LEE_MLP_NPARAM 5313
#define LEE_MLP_IN 16

typedef struct lee_mlp lee_mlp; /* parameters (FP32 master + BF16 copies), Adam state, gradients */

/* Creates a network on the current device from host parameters (NULL: all zero). */
lee_status lee_mlp_create(const float *params, void *cuda_stream, lee_mlp **out);

/* Copies the FP32 master parameters to / from host memory (synchronous). */
lee_status lee_mlp_get_params(lee_mlp *m, float *params);
lee_status lee_mlp_set_params(lee_mlp *m, const float *params);

/* Inference: y[rows] = network(x[rows][16]); x, y device FP32. */
lee_status lee_mlp_forward(lee_mlp *m, const float *x, int64_t rows, float *y);

/* Loss and gradient of L = mean_r (y_r - t_r)^2 over x[rows][16], t[rows] (device FP32).  The
 * backward pass multiplies BF16 operands on the tensor cores like the forward pass (the
 * back-propagated dz2, dz1 are rounded to BF16 before their GEMMs); per-block partial gradients
 * are summed in a fixed order, so the result is deterministic.  grad: device [NPARAM] or NULL
 * (the gradient is kept for lee_mlp_adam_step either way); loss: device [1] or NULL. */
lee_status lee_mlp_loss_grad(lee_mlp *m, const float *x, const float *t, int64_t rows, float *grad, float *loss);

/* One Adam step (Kingma & Ba, bias-corrected) on the FP32 master parameters with the kept
 * gradient; refreshes the BF16 copies. */
lee_status lee_mlp_adam_step(lee_mlp *m, float lr, float beta1, float beta2, float eps);

/* Network inputs and training targets from a batch of domains that share one geometry: for each
 * domain and each cell on the border of region (x0, y0, nx, ny) -- edges in the order x = x0,
 * x = x0 + nx - 1, y = y0, y = y0 + ny - 1, cells along each edge in increasing coordinate --
 * writes x[r][16] (see above), t[r] = (g*_in at the cell just outside the region) / (f*_in s)
 * and s[r] (s may be NULL).  Rows r = d * 2 (nx + ny) + (edge offset) + k.  The region must lie
 * at least one cell inside every domain and be at least 3 cells wide.  Device outputs. */
lee_status lee_batch_edge_samples(lee_batch *b, int64_t x0, int64_t y0, int64_t nx, int64_t ny, float *x, float *t,
                                  float *s);

/* The same inputs for the edges of a single open grid (the whole grid is the region), from a
 * solver handle's current state; t is not produced (the entering populations are unknown). */
lee_status lee_lbm_edge_inputs(lee_lbm *h, float *x, float *s);

lee_status lee_mlp_destroy(lee_mlp *m);

#ifdef __cplusplus
}
#endif

#endif /* LEE_MLP_H */
