// handles.cuh -- the opaque handle types of the C ABI, shared by the translation units that
// implement them (lee_lbm.cu, batch.cu, mlp.cu).
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/lee_batch.h"
#include "../../include/lee_lbm.h"
#include "ops.cuh"

struct lee_lbm {
    lee_lbm_config cfg{};
    const lee::SetOps *ops = nullptr;
    int device = 0;
    int D = 0, Q = 0;
    long long cells = 0, pitch = 0;
    size_t elem = 0;
    void *buf[2] = {nullptr, nullptr};
    int cur = 0;
    double *fields = nullptr;  // (D + 2) * cells FP64 staging for host fields
    double *pops64 = nullptr;  // Q * cells FP64 staging for host populations
    double *partial = nullptr;
    int nblocks = 0;
    double *red_out = nullptr;
    unsigned int *maxbits = nullptr;
    cudaStream_t st = nullptr;
    long long steps = 0;
    double scale = 1.0;
    bool poisoned = false;
    std::string err;
    // learned boundary: entering populations [4][ghost_L] in the arithmetic type, and the
    // network's packed BF16 weights (MlpDev layout, mlp.cuh)
    void *ghost = nullptr;
    int ghost_L = 0;
    void *mlp = nullptr;
    bool mlp_ready = false;
    // captured step graphs keyed by (starting parity, number of steps), even lengths only, and
    // the stream they are captured on
    std::map<std::pair<int, long long>, cudaGraphExec_t> exec;
    cudaStream_t cap = nullptr;
    // learned edge: the slots of the four corner cells in the one-launch step
    // (k_learned_step); with LEE_LEARNED_STREAMS=1 at create time the step runs as the network
    // and the border cells on `side` while the interior runs on the handle's stream instead
    unsigned long long *corner = nullptr;
    bool learned_streams = false;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // time steps fused per launch on periodic 2D FP32 grids (temporal blocking): 4 by default;
    // LEE_TB_STEPS=1..4 in the environment at create time overrides it, and LEE_SINGLE_STEP=1
    // sets 1 (for comparisons between the one-, two-, three- and four-step kernels)
    int tb_steps = 4;
    bool tb_env = false;  // tb_steps came from LEE_TB_STEPS
    // set by LEE_FORCE_SCALAR=1 at create time: one cell per thread in every step kernel, and one
    // step per launch (for comparisons of the vector and packed paths against the scalar one)
    bool force_scalar = false;
    // LEE_BFP_CELLS=4 or 8 at create time: cells per lane of the BFP16 one-step kernel (0: default)
    int bfp_cells = 0;
    // 3D two-step tile: LEE_T3_TMA=1 at create time picks the TMA-fed kernel (0 or -1, unset: the
    // register-fed one); the TMA-fed kernel records a timed-out stage wait in
    // wait_host (page-locked, mapped; wait_dev is its device address), read after synchronisations
    int t3_tma = -1;
    unsigned *wait_host = nullptr, *wait_dev = nullptr;
    // LEE_BC_SLAB: nl owned planes of `plane` cells along the cut (last) axis, with one halo plane
    // before and after them in every velocity array (the state copies start one plane in, see
    // state()); the four halo messages send_lo, send_hi, recv_lo, recv_hi of `crossing` planes each
    bool slab = false;
    long long plane = 0;
    int nl = 0, crossing = 0;
    void *halo[4] = {nullptr, nullptr, nullptr, nullptr};
};

namespace lee {
// Every CUDA status the handles check passes through here.  Normally it returns e unchanged; after
// lee_test_inject_cuda_error(n) the (n+1)-th successful call checked from then on is reported as
// cudaErrorUnknown instead (once), so that tests can drive a handle into its failure path from the
// host without any real GPU error.
cudaError_t checked(cudaError_t e);
using BatchedFn = cudaError_t (*)(const void *, void *, const void *, const unsigned short *, int, int, cudaStream_t);
using BatchedTbFn = cudaError_t (*)(const void *, void *, const void *, const void *, int, cudaStream_t);
}

struct lee_batch {
    int set = 0, storage = 0, count = 0, Q = 0;
    const lee::SetOps *ops = nullptr;
    size_t elem = 0;
    int device = 0;
    std::vector<lee_batch_domain> doms;
    std::vector<long long> offset, pitch, cells;
    long long total_elems = 0, total_cells = 0, max_cells = 0;
    void *buf[2] = {nullptr, nullptr};
    int cur = 0;
    cudaStream_t st = nullptr, cap = nullptr;
    // launch shape
    bool tuned = false;
    int threads = 0, V = 0, nblocks = 0;
    void *d_doms = nullptr;
    unsigned short *d_table = nullptr;
    size_t d_doms_cap = 0, d_table_cap = 0;
    lee::BatchedFn fn = nullptr;
    // time steps per launch: 1, or 2..4 fused (FP32, every nx % 4 == 0) with per-domain tiles and
    // a block table
    int unit = 1;
    void *d_tb = nullptr;
    void *d_tb_tiles = nullptr;  // int3 (domain, x0, y0) per block, in the tile order below
    size_t d_tb_cap = 0, d_tb_tiles_cap = 0;
    int tb_blocks = 0;
    lee::BatchedTbFn tb_fn = nullptr;
    // fused launch shape: tile rows (a multiple of 4) and dispatch order (0: tiles with the most
    // rows first, 1: domain by domain, row-major); fuse_ok: every domain can take a fused kernel;
    // unit_fixed: steps per launch fixed by the environment at create time (0: the tuner picks)
    int tile_rows = 64, tile_order = 0;
    bool fuse_ok = false;
    int unit_fixed = 0;
    float tuned_us_per_step = 0.f;
    // captured graphs, keyed by (starting parity, number of steps); every graph has an even
    // number of steps, so replaying it leaves the buffer parity unchanged
    static constexpr int kMaxGraphSteps = 4096;
    static constexpr int kChunkSteps = 100;
    std::map<std::pair<int, long long>, cudaGraphExec_t> exec;
    // aux
    double *fields = nullptr, *pops64 = nullptr, *partial = nullptr, *red_out = nullptr;
    int red_blocks = 0;
    bool poisoned = false;
    std::string err;
};
