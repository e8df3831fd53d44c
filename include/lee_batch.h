/*
 * lee_batch.h -- many independent periodic 2D domains advanced together (library addition; the
 * paper treats one periodic domain at a time).  Every domain runs the same LBE update scheme of
 * Sec. 6 as lee_lbm_step, on its own grid and with its own relaxation time; one kernel launch
 * advances all domains by one time step, and lee_batch_step can replay those launches from a
 * CUDA graph.  Per domain the result is bit for bit the one lee_lbm_step gives.
 *
 * Conventions are those of lee_lbm.h (layouts, post-collision state, status codes, poisoning).
 * Domain d's cells are indexed x + nx_d * y.
 */
#ifndef LEE_BATCH_H
#define LEE_BATCH_H

#include <stdint.h>

#include "lee_lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int64_t nx, ny; /* extents of the domain (>= 1) */
    double tau;     /* its BGK relaxation time, >= 1/2 */
} lee_batch_domain;

typedef enum {
    LEE_BATCH_GRAPH = 0,      /* one batched launch per step, replayed from a captured CUDA graph */
    LEE_BATCH_LAUNCH = 1,     /* one batched launch per step, launched directly                   */
    LEE_BATCH_SEQUENTIAL = 2  /* one single-domain launch per domain per step (the plain form)    */
} lee_batch_mode;

typedef struct lee_batch lee_batch;

/* Creates a batch of `count` (1 .. 65535) periodic domains of a 2D velocity set (LEE_D2Q5 or
 * LEE_D2Q5_DIATOMIC) with FP32 or FP64 storage.  All populations share one pair of device
 * buffers; each domain starts at the rest state.  cuda_stream: stream to run on (NULL = legacy
 * default stream).  Returns LEE_ERR_UNSUPPORTED for other sets or storages. */
lee_status lee_batch_create(int32_t set, int32_t storage, const lee_batch_domain *domains, int32_t count,
                            void *cuda_stream, lee_batch **out);

/* Equilibrium initial state of domain d (Sec. 7): fields rho[cells_d], u[2][cells_d],
 * theta[cells_d] in FP64, host (on_device = 0, synchronous) or device memory. */
lee_status lee_batch_init_fields(lee_batch *b, int32_t d, const double *rho, const double *u, const double *theta,
                                 int32_t on_device);

/* Advances every domain n >= 0 steps (Sec. 6).  mode: lee_batch_mode.  The first GRAPH or
 * LAUNCH call runs the autotuner unless lee_batch_set_tuning fixed the launch shape.  In GRAPH
 * mode a run of up to 4096 steps is one launch of a graph holding all its steps (captured on
 * first use of that length and parity, then cached); longer runs replay a 100-step graph.  With
 * FP32 storage and every nx a multiple of 4, GRAPH and LAUNCH modes advance several steps per
 * launch (the intermediate states kept in shared memory; tiles of 128 columns), with the count,
 * tile rows and tile order the autotuner picks (lee_batch_tune_shape; LEE_TB_STEPS=1..4 in the
 * environment at create time fixes the count), bit-identical to single steps. */
lee_status lee_batch_step(lee_batch *b, int64_t n, int32_t mode);

/* Per-cell moments of domain d (as lee_lbm_moments).  NULL outputs are skipped. */
lee_status lee_batch_moments(lee_batch *b, int32_t d, double *rho, double *u, double *theta, int32_t on_device);

/* FP64 global sums of domain d, out[6] (as lee_lbm_reduce). */
lee_status lee_batch_reduce(lee_batch *b, int32_t d, double *out, int32_t on_device);

/* Post-collision populations of domain d as FP64 g[5][cells_d] (library velocity order). */
lee_status lee_batch_get_populations(lee_batch *b, int32_t d, double *g, int32_t on_device);

/* Launch shape of a batch: the one-step batched kernel (threads per block, cells per thread) and
 * the fused multi-step kernel (steps per launch; tiles of 128 columns x tile_rows rows; dispatch
 * order 0 = tiles with the most rows first, 1 = domain by domain).  steps_per_launch = 1 means
 * every step runs the one-step kernel.  us_per_step: the tuner's measurement of one time step of
 * the whole batch with this shape (0 when the shape was set by hand). */
typedef struct {
    int32_t threads, cells_per_thread;
    int32_t steps_per_launch, tile_rows, tile_order;
    float us_per_step;
} lee_batch_shape;

/* Autotuner: times every candidate shape for a few launches on the batch itself (CUDA events on
 * its stream) and keeps the one with the least time per step:
 *   one-step kernel: threads per block {128, 256, 512} x cells per thread {V/2, V}
 *     (V = 16 bytes / storage size);
 *   fused kernel (FP32 storage, every nx a multiple of 4): steps per launch {2, 3, 4} (only the
 *     count LEE_TB_STEPS fixed at create time, if set) x tile rows {32, 48, 64, 96, 128} x both
 *     tile orders; it is kept only if it beats the one-step kernel per step.
 * Every shape gives the same bits.  Tuning writes only the idle buffer, so the state does not
 * change.  Results are cached per (set, storage, domain list) for the process, and in the text
 * file named by the environment variable LEE_AUTOTUNE_CACHE when it is set.  lee_batch_tune
 * reports the one-step part (either pointer may be NULL), lee_batch_tune_shape all of it. */
lee_status lee_batch_tune(lee_batch *b, int32_t *threads, int32_t *cells_per_thread);
lee_status lee_batch_tune_shape(lee_batch *b, lee_batch_shape *out);

/* Fixes the whole launch shape instead of tuning: threads and cells_per_thread as for
 * lee_batch_set_tuning; steps_per_launch 1, or 2..4 where the fused kernel applies, with
 * tile_rows a multiple of 4 in 4..1024 and tile_order 0 or 1.  LEE_ERR_INVALID_ARGUMENT
 * otherwise. */
lee_status lee_batch_set_shape(lee_batch *b, const lee_batch_shape *shape);

/* Fixes the launch shape instead of tuning (threads in {128, 256, 512}; cells_per_thread must
 * divide every nx_d and be one of the tuner's candidates). */
lee_status lee_batch_set_tuning(lee_batch *b, int32_t threads, int32_t cells_per_thread);

/* Total number of cells over all domains. */
lee_status lee_batch_cells(lee_batch *b, int64_t *cells);

/* Blocks until the batch's stream is idle. */
lee_status lee_batch_sync(lee_batch *b);

/* Last error message (never NULL for a non-NULL batch). */
const char *lee_batch_last_error(lee_batch *b);

/* Frees the batch, its graphs and its device memory.  NULL-safe. */
lee_status lee_batch_destroy(lee_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* LEE_BATCH_H */
