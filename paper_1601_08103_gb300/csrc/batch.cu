// batch.cu -- many periodic 2D domains per launch (include/lee_batch.h): descriptors, the
// block -> domain table, the autotuner, CUDA-graph replay and the sequential baseline.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/lee_batch.h"
#include "handles.cuh"
#include "set_impl.cuh"

namespace lee {
SetConsts consts_for(int set, double scale);
void fold_coefficients(int set, bool scaled, double omega, double M[4][4], double N[4][4]);

template <class S, class T, int V>
cudaError_t launch_batched(const void *src, void *dst, const void *doms, const unsigned short *table, int nblocks,
                           int threads, cudaStream_t st) {
    using C = typename Store<T>::C;
    k_stream_collide_batched<S, T, V><<<nblocks, threads, 0, st>>>(
        static_cast<const T *>(src), static_cast<T *>(dst), static_cast<const BatchDomain<C> *>(doms), table);
    return cudaGetLastError();
}

template <class S, class T>
BatchedFn batched_fn(int V) {
    switch (V) {
    case 1: return &launch_batched<S, T, 1>;
    case 2: return &launch_batched<S, T, 2>;
    case 4: if constexpr (sizeof(T) <= 4) return &launch_batched<S, T, 4>; else return nullptr;
    default: return nullptr;
    }
}

template <class S>
cudaError_t launch_batched_2step(const void *src, void *dst, const void *doms, const void *tiles, int nblocks,
                                 cudaStream_t st) {
    k_stream_collide_2step_batched<S><<<nblocks, 128, tb_smem_bytes<S>(), st>>>(
        static_cast<const float *>(src), static_cast<float *>(dst), static_cast<const TbDomain *>(doms),
        static_cast<const int3 *>(tiles));
    return cudaGetLastError();
}

template <class S, int K>
cudaError_t launch_batched_kstep(const void *src, void *dst, const void *doms, const void *tiles, int nblocks,
                                 cudaStream_t st) {
    k_stream_collide_kstep_batched<S, K><<<nblocks, kTbkThreads, tbk_smem_bytes<S, K>(), st>>>(
        static_cast<const float *>(src), static_cast<float *>(dst), static_cast<const TbDomain *>(doms),
        static_cast<const int3 *>(tiles));
    return cudaGetLastError();
}

// Sets the shared-memory attribute of the batched multi-step kernel fusing `unit` steps on the
// current device (outside any stream capture) and returns its launcher.
template <class S>
cudaError_t prepare_batched_tb(int unit, lee::BatchedTbFn *fn) {
    cudaError_t e = cudaErrorInvalidValue;
    if (unit == 2) {
        e = cudaFuncSetAttribute(k_stream_collide_2step_batched<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 tb_smem_bytes<S>());
        *fn = &launch_batched_2step<S>;
    } else if (unit == 3) {
        e = cudaFuncSetAttribute(k_stream_collide_kstep_batched<S, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 tbk_smem_bytes<S, 3>());
        *fn = &launch_batched_kstep<S, 3>;
    } else if (unit == 4) {
        e = cudaFuncSetAttribute(k_stream_collide_kstep_batched<S, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 tbk_smem_bytes<S, 4>());
        *fn = &launch_batched_kstep<S, 4>;
    }
    return e;
}

BatchedFn pick_batched(int set, int storage, int V) {
    if (set == LEE_D2Q5) return storage == LEE_STORE_F32 ? batched_fn<D2Q5, float>(V) : batched_fn<D2Q5, double>(V);
    if (set == LEE_D2Q5_DIATOMIC)
        return storage == LEE_STORE_F32 ? batched_fn<D2Q5Di, float>(V) : batched_fn<D2Q5Di, double>(V);
    return nullptr;
}

}  // namespace lee

using namespace lee;


namespace {

lee_status bfail(lee_batch *b, lee_status s, const std::string &m) {
    if (b) {
        b->err = m;
        if (s == LEE_ERR_CUDA) b->poisoned = true;
    }
    return s;
}

#define BCK(b, call, what)                                                                       \
    do {                                                                                         \
        cudaError_t e_ = lee::checked(call);                                                     \
        if (e_ != cudaSuccess)                                                                   \
            return bfail((b), e_ == cudaErrorMemoryAllocation ? LEE_ERR_OUT_OF_MEMORY : LEE_ERR_CUDA, \
                         std::string(what) + ": " + cudaGetErrorString(e_));                      \
    } while (0)

lee_status benter(lee_batch *b) {
    if (!b) return LEE_ERR_INVALID_ARGUMENT;
    if (b->poisoned) return LEE_ERR_POISONED;
    cudaError_t e = lee::checked(cudaSetDevice(b->device));
    if (e != cudaSuccess) return bfail(b, LEE_ERR_CUDA, "cudaSetDevice");
    return LEE_OK;
}

void drop_graphs(lee_batch *b) {
    for (auto &kv : b->exec)
        if (kv.second) cudaGraphExecDestroy(kv.second);
    b->exec.clear();
}

void *dom_ptr(lee_batch *b, int which, int d) { return static_cast<char *>(b->buf[which]) + b->elem * b->offset[d]; }

// Per-domain descriptors and the block table for a launch shape.
template <class C>
lee_status build_shape_t(lee_batch *b, int threads, int V) {
    std::vector<BatchDomain<C>> hd(b->count);
    std::vector<unsigned short> table;
    int block = 0;
    for (int d = 0; d < b->count; ++d) {
        BatchDomain<C> &D = hd[d];
        D.gd.nx = (int)b->doms[d].nx;
        D.gd.ny = (int)b->doms[d].ny;
        D.gd.nz = 1;
        D.gd.nxc = (int)(b->doms[d].nx / V);
        D.gd.nchunks = (long long)D.gd.nxc * D.gd.ny;
        D.gd.pitch = b->pitch[d];
        double M[4][4], N[4][4];
        const double omega = omega_for(b->storage, b->doms[d].tau);
        fold_coefficients(b->set, false, omega, M, N);
        D.cf = make_coef<C>(omega, M, N);
        D.offset = b->offset[d];
        D.first_block = block;
        const long long nb = (D.gd.nchunks + threads - 1) / threads;
        for (long long k = 0; k < nb; ++k) table.push_back((unsigned short)d);
        block += (int)nb;
    }
    const size_t dbytes = sizeof(BatchDomain<C>) * hd.size(), tbytes = sizeof(unsigned short) * table.size();
    if (dbytes > b->d_doms_cap) {
        cudaFree(b->d_doms);
        b->d_doms = nullptr;
        BCK(b, cudaMalloc(&b->d_doms, dbytes), "cudaMalloc(domains)");
        b->d_doms_cap = dbytes;
    }
    if (tbytes > b->d_table_cap) {
        cudaFree(b->d_table);
        b->d_table = nullptr;
        BCK(b, cudaMalloc(&b->d_table, tbytes), "cudaMalloc(block table)");
        b->d_table_cap = tbytes;
    }
    BCK(b, cudaMemcpyAsync(b->d_doms, hd.data(), dbytes, cudaMemcpyHostToDevice, b->st), "H2D domains");
    BCK(b, cudaMemcpyAsync(b->d_table, table.data(), tbytes, cudaMemcpyHostToDevice, b->st), "H2D block table");
    BCK(b, cudaStreamSynchronize(b->st), "sync");
    b->threads = threads;
    b->V = V;
    b->nblocks = block;
    b->fn = pick_batched(b->set, b->storage, V);
    drop_graphs(b);
    return b->fn ? LEE_OK : bfail(b, LEE_ERR_UNSUPPORTED, "no batched kernel for this shape");
}

lee_status build_shape(lee_batch *b, int threads, int V) {
    return b->storage == LEE_STORE_F32 ? build_shape_t<float>(b, threads, V) : build_shape_t<double>(b, threads, V);
}

lee_status launch_one(lee_batch *b, int src_which, cudaStream_t st) {
    BCK(b, b->fn(b->buf[src_which], b->buf[src_which ^ 1], b->d_doms, b->d_table, b->nblocks, b->threads, st),
        "batched launch");
    return LEE_OK;
}

int full_vec(int storage) { return storage == LEE_STORE_F32 ? 4 : 2; }

// Tile rows of the fused kernel before tuning (on the 96-domain workload, hand-swept with the
// four-step kernel: 64 rows 374 GLUPS, 48-80 rows 360-366, 128 rows 367, 256 rows 359).
constexpr int kBatchTileRows = 64;

// Multi-step tiles of 128 columns x `rows` rows (fewer for short domains), in dispatch order
// `order`: 0 = tiles with the most rows first, so that the block scheduler balances the uneven
// domains; 1 = domain by domain, rows then columns.  Every shape gives the same bits.
lee_status build_tb(lee_batch *b, int unit, int rows, int order) {
    cudaError_t e = b->set == LEE_D2Q5 ? prepare_batched_tb<D2Q5>(unit, &b->tb_fn)
                                       : prepare_batched_tb<D2Q5Di>(unit, &b->tb_fn);
    if (e != cudaSuccess) return bfail(b, LEE_ERR_CUDA, std::string("multi-step prepare: ") + cudaGetErrorString(e));
    std::vector<TbDomain> hd(b->count);
    struct Tile {
        int rows, d, x0, y0;
    };
    std::vector<Tile> tiles;
    for (int d = 0; d < b->count; ++d) {
        TbDomain &D = hd[d];
        D.nx = (int)b->doms[d].nx;
        D.ny = (int)b->doms[d].ny;
        int H = rows;
        const int ny4 = (D.ny + 3) / 4 * 4;
        if (H > ny4) H = ny4;
        D.H = H;
        D.pitch = b->pitch[d];
        D.offset = b->offset[d];
        double M[4][4], N[4][4];
        const double omega = omega_for(b->storage, b->doms[d].tau);
        fold_coefficients(b->set, false, omega, M, N);
        D.cf = make_coef<float>(omega, M, N);
        for (int y0 = 0; y0 < D.ny; y0 += H)
            for (int x0 = 0; x0 < D.nx; x0 += kTbW) tiles.push_back({std::min(H, D.ny - y0), d, x0, y0});
    }
    if (order == 0)
        std::stable_sort(tiles.begin(), tiles.end(), [](const Tile &p, const Tile &q) { return p.rows > q.rows; });
    std::vector<int3> ht(tiles.size());
    for (size_t k = 0; k < tiles.size(); ++k) ht[k] = make_int3(tiles[k].d, tiles[k].x0, tiles[k].y0);
    const size_t db = sizeof(TbDomain) * hd.size(), tb = sizeof(int3) * ht.size();
    if (db > b->d_tb_cap) {
        cudaFree(b->d_tb);
        b->d_tb = nullptr;
        BCK(b, cudaMalloc(&b->d_tb, db), "cudaMalloc(multi-step domains)");
        b->d_tb_cap = db;
    }
    if (tb > b->d_tb_tiles_cap) {
        cudaFree(b->d_tb_tiles);
        b->d_tb_tiles = nullptr;
        BCK(b, cudaMalloc(&b->d_tb_tiles, tb), "cudaMalloc(multi-step tiles)");
        b->d_tb_tiles_cap = tb;
    }
    BCK(b, cudaMemcpyAsync(b->d_tb, hd.data(), db, cudaMemcpyHostToDevice, b->st), "H2D");
    BCK(b, cudaMemcpyAsync(b->d_tb_tiles, ht.data(), tb, cudaMemcpyHostToDevice, b->st), "H2D");
    BCK(b, cudaStreamSynchronize(b->st), "sync");
    b->tb_blocks = (int)ht.size();
    b->unit = unit;
    b->tile_rows = rows;
    b->tile_order = order;
    drop_graphs(b);
    return LEE_OK;
}

// A shape of both kernels: one-step (threads, cells per thread) and fused (steps per launch,
// tile rows, tile order; steps 1 = no fused kernel).
struct BatchShape {
    int threads, V, unit, rows, order;
    float us;  // measured time per step (0 if set by hand)
};

lee_status apply_shape(lee_batch *b, const BatchShape &sh) {
    lee_status s = build_shape(b, sh.threads, sh.V);
    if (s != LEE_OK) return s;
    if (sh.unit > 1) return build_tb(b, sh.unit, sh.rows, sh.order);
    b->unit = 1;
    drop_graphs(b);
    return LEE_OK;
}

std::mutex g_cache_mutex;
std::map<std::string, BatchShape> g_cache;

std::string cache_key(const lee_batch *b) {
    unsigned long long h = 1469598103934665603ULL;  // FNV-1a over the domain extents
    for (const auto &d : b->doms) {
        const long long v[2] = {d.nx, d.ny};
        for (long long x : v)
            for (int k = 0; k < 8; ++k) {
                h ^= (unsigned long long)((x >> (8 * k)) & 0xff);
                h *= 1099511628211ULL;
            }
    }
    std::ostringstream o;
    o << "batch2/set" << b->set << "/st" << b->storage << "/n" << b->count << "/c" << b->total_cells << "/u"
      << b->unit_fixed << "/h" << std::hex << h;
    return o.str();
}

bool cache_lookup(const std::string &key, BatchShape *sh) {
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
        *sh = it->second;
        return true;
    }
    const char *path = std::getenv("LEE_AUTOTUNE_CACHE");
    if (!path || !*path) return false;
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char k[512];
    BatchShape v{};
    bool found = false;
    while (std::fscanf(f, "%511s %d %d %d %d %d %f", k, &v.threads, &v.V, &v.unit, &v.rows, &v.order, &v.us) == 7) {
        if (key == k) {
            *sh = v;
            found = true;
        }
    }
    std::fclose(f);
    if (found) g_cache[key] = *sh;
    return found;
}

void cache_store(const std::string &key, const BatchShape &sh) {
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    g_cache[key] = sh;
    const char *path = std::getenv("LEE_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    if (FILE *f = std::fopen(path, "a")) {
        std::fprintf(f, "%s %d %d %d %d %d %.4f\n", key.c_str(), sh.threads, sh.V, sh.unit, sh.rows, sh.order, sh.us);
        std::fclose(f);
    }
}

// Candidates of the fused kernel's tile rows (multiples of 4, the rows a block's four row warps
// advance per iteration).
constexpr int kTuneRows[] = {32, 48, 64, 96, 128};

// The autotuner: times every candidate shape on the batch itself with CUDA events and keeps the
// one with the least time per step of the whole batch.
//   one-step kernel: threads per block {128, 256, 512} x cells per thread {V/2, V} (10 launches);
//   fused kernel (FP32, every nx % 4 == 0): steps per launch {2, 3, 4} (or the one fixed by
//   LEE_TB_STEPS) x tile rows kTuneRows x tile order {largest first, domain by domain} (6
//   launches each, after 2 untimed ones).
// The one-step shape is kept in any case (it runs the steps a fused launch cannot take); the fused
// shape only if it beats the one-step kernel.  Every tuning launch reads the current buffer and
// writes the idle one, so the state does not change; every candidate gives the same bits.
lee_status tune(lee_batch *b) {
    const std::string key = cache_key(b);
    BatchShape best{};
    if (cache_lookup(key, &best)) {
        lee_status s = apply_shape(b, best);
        if (s == LEE_OK) {
            b->tuned = true;
            b->tuned_us_per_step = best.us;
        }
        return s;
    }
    const int vf = full_vec(b->storage);
    const int cand_v[2] = {vf / 2, vf};
    const int cand_t[3] = {128, 256, 512};
    float best_us = 1e30f;
    cudaEvent_t e0, e1;
    BCK(b, cudaEventCreate(&e0), "event");
    BCK(b, cudaEventCreate(&e1), "event");
    auto timed = [&](int launches, bool fused, float *us) -> lee_status {
        lee_status s = LEE_OK;
        auto one = [&]() -> lee_status {
            if (fused) {
                BCK(b, b->tb_fn(b->buf[b->cur], b->buf[b->cur ^ 1], b->d_tb, b->d_tb_tiles, b->tb_blocks, b->st),
                    "tuning launch");
                return LEE_OK;
            }
            return launch_one(b, b->cur, b->st);
        };
        for (int w = 0; w < 2; ++w)
            if ((s = one()) != LEE_OK) return s;
        BCK(b, cudaEventRecord(e0, b->st), "event");
        for (int r = 0; r < launches; ++r)
            if ((s = one()) != LEE_OK) return s;
        BCK(b, cudaEventRecord(e1, b->st), "event");
        BCK(b, cudaEventSynchronize(e1), "event sync");
        float ms = 0.f;
        BCK(b, cudaEventElapsedTime(&ms, e0, e1), "elapsed");
        *us = ms * 1e3f / (float)launches;
        return LEE_OK;
    };
    for (int vi = 0; vi < 2; ++vi) {
        const int V = cand_v[vi];
        bool ok = true;
        for (const auto &d : b->doms) ok = ok && (d.nx % V == 0);
        if (!ok) continue;
        for (int ti = 0; ti < 3; ++ti) {
            lee_status s = build_shape(b, cand_t[ti], V);
            if (s != LEE_OK) return s;
            float us = 0.f;
            if ((s = timed(10, false, &us)) != LEE_OK) return s;
            if (us < best_us) {
                best_us = us;
                best = BatchShape{cand_t[ti], V, 1, 64, 0, us};
            }
        }
    }
    if (best.threads == 0) return bfail(b, LEE_ERR_UNSUPPORTED, "no launch shape divides every nx");
    if (b->fuse_ok && b->unit_fixed != 1) {
        const BatchShape one = best;
        for (int unit = 2; unit <= 4; ++unit) {
            if (b->unit_fixed > 1 && unit != b->unit_fixed) continue;
            for (int rows : kTuneRows)
                for (int order = 0; order < 2; ++order) {
                    lee_status s = build_tb(b, unit, rows, order);
                    if (s != LEE_OK) return s;
                    float us = 0.f;
                    if ((s = timed(6, true, &us)) != LEE_OK) return s;
                    if (us / unit < best_us) {
                        best_us = us / unit;
                        best = BatchShape{one.threads, one.V, unit, rows, order, us / unit};
                    }
                }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    lee_status s = apply_shape(b, best);
    if (s != LEE_OK) return s;
    cache_store(key, best);
    b->tuned_us_per_step = best_us;
    b->tuned = true;
    return LEE_OK;
}

// One launch of the step unit (b->unit fused steps, or one step) reading buffer src_which and
// writing the other one.
cudaError_t launch_unit(lee_batch *b, int src_which, cudaStream_t st) {
    if (b->unit > 1) return b->tb_fn(b->buf[src_which], b->buf[src_which ^ 1], b->d_tb, b->d_tb_tiles, b->tb_blocks, st);
    return b->fn(b->buf[src_which], b->buf[src_which ^ 1], b->d_doms, b->d_table, b->nblocks, b->threads, st);
}

lee_status ensure_graph(lee_batch *b, int parity, long long steps, cudaGraphExec_t *out) {
    auto it = b->exec.find({parity, steps});
    if (it != b->exec.end()) {
        *out = it->second;
        return LEE_OK;
    }
    cudaGraph_t g = nullptr;
    BCK(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    int w = parity;
    const int unit = b->unit;
    for (long long k = 0; k < steps / unit; ++k) {
        cudaError_t e = launch_unit(b, w, b->cap);
        if (e != cudaSuccess) {
            cudaStreamEndCapture(b->cap, &g);
            if (g) cudaGraphDestroy(g);
            return bfail(b, LEE_ERR_CUDA, std::string("capture launch: ") + cudaGetErrorString(e));
        }
        w ^= 1;
    }
    BCK(b, cudaStreamEndCapture(b->cap, &g), "end capture");
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    BCK(b, e, "graph instantiate");
    b->exec[{parity, steps}] = ex;
    *out = ex;
    return LEE_OK;
}

lee_status ensure_aux(lee_batch *b) {
    if (b->fields) return LEE_OK;
    BCK(b, cudaMalloc(&b->fields, sizeof(double) * 4 * (size_t)b->max_cells), "cudaMalloc(fields)");
    BCK(b, cudaMalloc(&b->pops64, sizeof(double) * (size_t)b->Q * (size_t)b->max_cells), "cudaMalloc(pops64)");
    return LEE_OK;
}

}  // namespace

extern "C" {

lee_status lee_batch_create(int32_t set, int32_t storage, const lee_batch_domain *domains, int32_t count,
                            void *cuda_stream, lee_batch **out) {
    if (!out) return LEE_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    if (!domains || count < 1 || count > 65535) return LEE_ERR_INVALID_ARGUMENT;
    if (set != LEE_D2Q5 && set != LEE_D2Q5_DIATOMIC) return LEE_ERR_UNSUPPORTED;
    if (storage != LEE_STORE_F32 && storage != LEE_STORE_F64) return LEE_ERR_UNSUPPORTED;
    long long total = 0, maxc = 0;
    for (int d = 0; d < count; ++d) {
        const lee_batch_domain &D = domains[d];
        if (D.nx < 1 || D.ny < 1 || D.nx > (1 << 30) || D.ny > (1 << 30)) return LEE_ERR_INVALID_ARGUMENT;
        if (!(D.tau == D.tau) || D.tau > 1e300) return LEE_ERR_INVALID_ARGUMENT;
        if (D.tau < 0.5) return LEE_ERR_UNSTABLE_TAU;
        const long long c = D.nx * D.ny;
        if (c >= (1LL << 31)) return LEE_ERR_INVALID_ARGUMENT;
        total += c;
        maxc = std::max(maxc, c);
    }
    lee_batch *b = new (std::nothrow) lee_batch();
    if (!b) return LEE_ERR_OUT_OF_MEMORY;
    b->set = set;
    b->storage = storage;
    b->count = count;
    b->ops = set_ops(set);
    b->Q = b->ops->Q;
    b->elem = storage == LEE_STORE_F32 ? 4 : 8;
    b->doms.assign(domains, domains + count);
    long long off = 0;
    for (int d = 0; d < count; ++d) {
        const long long c = domains[d].nx * domains[d].ny;
        const long long p = (c + 63) / 64 * 64;
        b->offset.push_back(off);
        b->pitch.push_back(p);
        b->cells.push_back(c);
        off += p * b->Q;
    }
    b->total_elems = off;
    b->total_cells = total;
    b->max_cells = maxc;
    b->st = static_cast<cudaStream_t>(cuda_stream);
    b->red_blocks = aux_blocks(maxc, kReduceThreads);
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&b->buf[0], b->elem * (size_t)off);
    if (e == cudaSuccess) e = cudaMalloc(&b->buf[1], b->elem * (size_t)off);
    if (e == cudaSuccess) e = cudaMalloc(&b->partial, sizeof(double) * kReduceMax * (size_t)b->red_blocks);
    if (e == cudaSuccess) e = cudaMalloc(&b->red_out, sizeof(double) * kReduceMax);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->buf[0], 0, b->elem * (size_t)off, b->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->buf[1], 0, b->elem * (size_t)off, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) {
        lee_status s = e == cudaErrorMemoryAllocation ? LEE_ERR_OUT_OF_MEMORY : LEE_ERR_CUDA;
        lee_batch_destroy(b);
        cudaGetLastError();
        return s;
    }
    // time steps fused per launch: 4, or LEE_TB_STEPS=1..4 / LEE_SINGLE_STEP=1 at create time
    int unit = 4;
    if (const char *ev = std::getenv("LEE_TB_STEPS")) {
        if (ev[0] >= '1' && ev[0] <= '4' && ev[1] == 0) unit = ev[0] - '0';
    }
    if (const char *ev = std::getenv("LEE_SINGLE_STEP")) {
        if (ev[0] == '1') unit = 1;
    }
    bool fuse_ok = storage == LEE_STORE_F32;
    for (int d = 0; d < count; ++d) fuse_ok = fuse_ok && domains[d].nx % 4 == 0 && domains[d].ny >= 3;
    b->fuse_ok = fuse_ok;
    b->unit_fixed = (std::getenv("LEE_TB_STEPS") || std::getenv("LEE_SINGLE_STEP")) ? unit : 0;
    if (fuse_ok && unit > 1) {  // the shape before tuning: the given step count, 64-row tiles
        lee_status s2 = build_tb(b, unit, kBatchTileRows, 0);
        if (s2 != LEE_OK) {
            lee_batch_destroy(b);
            cudaGetLastError();
            return s2;
        }
    }
    *out = b;
    return LEE_OK;
}

lee_status lee_batch_init_fields(lee_batch *b, int32_t d, const double *rho, const double *u, const double *theta,
                                 int32_t on_device) {
    lee_status s = benter(b);
    if (s != LEE_OK) return s;
    if (d < 0 || d >= b->count || !rho || !u || !theta) return bfail(b, LEE_ERR_INVALID_ARGUMENT, "init_fields: bad args");
    const long long c = b->cells[d];
    const double *dr = rho, *du = u, *dt = theta;
    if (!on_device) {
        if ((s = ensure_aux(b)) != LEE_OK) return s;
        const size_t n = sizeof(double) * (size_t)c;
        BCK(b, cudaMemcpyAsync(b->fields, rho, n, cudaMemcpyHostToDevice, b->st), "H2D rho");
        BCK(b, cudaMemcpyAsync(b->fields + c, u, 2 * n, cudaMemcpyHostToDevice, b->st), "H2D u");
        BCK(b, cudaMemcpyAsync(b->fields + 3 * c, theta, n, cudaMemcpyHostToDevice, b->st), "H2D theta");
        dr = b->fields;
        du = b->fields + c;
        dt = b->fields + 3 * c;
    }
    BCK(b, b->ops->init(b->storage, dr, du, dt, dom_ptr(b, b->cur, d), c, b->pitch[d], consts_for(b->set, 1.0), b->st),
        "init kernel");
    if (!on_device) BCK(b, cudaStreamSynchronize(b->st), "sync");
    return LEE_OK;
}

lee_status lee_batch_step(lee_batch *b, int64_t n, int32_t mode) {
    lee_status s = benter(b);
    if (s != LEE_OK) return s;
    if (n < 0 || mode < LEE_BATCH_GRAPH || mode > LEE_BATCH_SEQUENTIAL)
        return bfail(b, LEE_ERR_INVALID_ARGUMENT, "step: bad n or mode");
    if (mode == LEE_BATCH_SEQUENTIAL) {
        StepLaunch L{};
        L.storage = b->storage;
        L.nz = 1;
        L.open = false;
        L.stream = b->st;
        for (int64_t t = 0; t < n; ++t) {
            for (int d = 0; d < b->count; ++d) {
                L.src = dom_ptr(b, b->cur, d);
                L.dst = dom_ptr(b, b->cur ^ 1, d);
                L.nx = (int)b->doms[d].nx;
                L.ny = (int)b->doms[d].ny;
                L.pitch = b->pitch[d];
                L.omega = omega_for(b->storage, b->doms[d].tau);
                fold_coefficients(b->set, false, L.omega, L.coefM, L.coefN);
                BCK(b, b->ops->step(L), "sequential launch");
            }
            b->cur ^= 1;
        }
        return LEE_OK;
    }
    if (!b->tuned && (s = tune(b)) != LEE_OK) return s;
    const int unit = b->unit;
    int64_t units = n / unit;
    if (mode == LEE_BATCH_GRAPH) {
        // up to kMaxGraphSteps steps: one graph of all of them (one launch of the whole run);
        // longer runs: replays of a kChunkSteps graph.  Graphs hold an even number of launches.
        const long long gunits = units * unit <= lee_batch::kMaxGraphSteps ? (units & ~1LL)
                                                                           : (lee_batch::kChunkSteps / unit) & ~1LL;
        while (gunits > 0 && units >= gunits) {
            cudaGraphExec_t ex = nullptr;
            if ((s = ensure_graph(b, b->cur, gunits * unit, &ex)) != LEE_OK) return s;
            BCK(b, cudaGraphLaunch(ex, b->st), "graph launch");  // even number of launches: parity kept
            units -= gunits;
        }
    }
    for (; units > 0; --units) {
        BCK(b, launch_unit(b, b->cur, b->st), "batched launch");
        b->cur ^= 1;
    }
    for (int64_t left = n % unit; left > 0; --left) {
        if ((s = launch_one(b, b->cur, b->st)) != LEE_OK) return s;
        b->cur ^= 1;
    }
    return LEE_OK;
}

lee_status lee_batch_moments(lee_batch *b, int32_t d, double *rho, double *u, double *theta, int32_t on_device) {
    lee_status s = benter(b);
    if (s != LEE_OK) return s;
    if (d < 0 || d >= b->count) return bfail(b, LEE_ERR_INVALID_ARGUMENT, "moments: bad domain");
    const long long c = b->cells[d];
    const SetConsts k = consts_for(b->set, 1.0);
    if (on_device) {
        BCK(b, b->ops->moments(b->storage, dom_ptr(b, b->cur, d), c, b->pitch[d], k, rho, u, theta, b->st), "moments");
        return LEE_OK;
    }
    if ((s = ensure_aux(b)) != LEE_OK) return s;
    BCK(b, b->ops->moments(b->storage, dom_ptr(b, b->cur, d), c, b->pitch[d], k, b->fields, b->fields + c,
                           b->fields + 3 * c, b->st),
        "moments");
    const size_t nb = sizeof(double) * (size_t)c;
    if (rho) BCK(b, cudaMemcpyAsync(rho, b->fields, nb, cudaMemcpyDeviceToHost, b->st), "D2H rho");
    if (u) BCK(b, cudaMemcpyAsync(u, b->fields + c, 2 * nb, cudaMemcpyDeviceToHost, b->st), "D2H u");
    if (theta) BCK(b, cudaMemcpyAsync(theta, b->fields + 3 * c, nb, cudaMemcpyDeviceToHost, b->st), "D2H theta");
    BCK(b, cudaStreamSynchronize(b->st), "sync");
    return LEE_OK;
}

lee_status lee_batch_reduce(lee_batch *b, int32_t d, double *out, int32_t on_device) {
    lee_status s = benter(b);
    if (s != LEE_OK) return s;
    if (d < 0 || d >= b->count || !out) return bfail(b, LEE_ERR_INVALID_ARGUMENT, "reduce: bad args");
    const long long c = b->cells[d];
    const int nblocks = aux_blocks(c, kReduceThreads);
    const SetConsts k = consts_for(b->set, 1.0);
    BCK(b, b->ops->reduce_partial(b->storage, dom_ptr(b, b->cur, d), c, b->pitch[d], k, b->partial, nblocks, b->st),
        "reduce_partial");
    double *dst = on_device ? out : b->red_out;
    const ReduceCombine rc = make_reduce_combine(b->ops, k, false);
    k_reduce_final<<<1, 32 * rc.nraw, 0, b->st>>>(b->partial, nblocks, rc, dst);
    BCK(b, cudaGetLastError(), "reduce_final");
    if (!on_device) {
        BCK(b, cudaMemcpyAsync(out, b->red_out, sizeof(double) * 6, cudaMemcpyDeviceToHost, b->st), "D2H reduce");
        BCK(b, cudaStreamSynchronize(b->st), "sync");
    }
    return LEE_OK;
}

lee_status lee_batch_get_populations(lee_batch *b, int32_t d, double *g, int32_t on_device) {
    lee_status s = benter(b);
    if (s != LEE_OK) return s;
    if (d < 0 || d >= b->count || !g) return bfail(b, LEE_ERR_INVALID_ARGUMENT, "get_populations: bad args");
    const long long c = b->cells[d];
    double *dst = g;
    if (!on_device) {
        if ((s = ensure_aux(b)) != LEE_OK) return s;
        dst = b->pops64;
    }
    BCK(b, b->ops->export_f64(b->storage, dom_ptr(b, b->cur, d), c, b->pitch[d], consts_for(b->set, 1.0), dst, b->st),
        "export");
    if (!on_device) {
        BCK(b, cudaMemcpyAsync(g, dst, sizeof(double) * (size_t)b->Q * c, cudaMemcpyDeviceToHost, b->st), "D2H g");
        BCK(b, cudaStreamSynchronize(b->st), "sync");
    }
    return LEE_OK;
}

lee_status lee_batch_tune(lee_batch *b, int32_t *threads, int32_t *cells_per_thread) {
    lee_status s = benter(b);
    if (s != LEE_OK) return s;
    if (!b->tuned && (s = tune(b)) != LEE_OK) return s;
    if (threads) *threads = b->threads;
    if (cells_per_thread) *cells_per_thread = b->V;
    return LEE_OK;
}

lee_status lee_batch_tune_shape(lee_batch *b, lee_batch_shape *out) {
    lee_status s = benter(b);
    if (s != LEE_OK) return s;
    if (!out) return bfail(b, LEE_ERR_INVALID_ARGUMENT, "tune_shape: NULL out");
    if (!b->tuned && (s = tune(b)) != LEE_OK) return s;
    out->threads = b->threads;
    out->cells_per_thread = b->V;
    out->steps_per_launch = b->unit;
    out->tile_rows = b->unit > 1 ? b->tile_rows : 0;
    out->tile_order = b->unit > 1 ? b->tile_order : 0;
    out->us_per_step = b->tuned_us_per_step;
    return LEE_OK;
}

lee_status lee_batch_set_shape(lee_batch *b, const lee_batch_shape *shape) {
    lee_status s = benter(b);
    if (s != LEE_OK) return s;
    if (!shape) return bfail(b, LEE_ERR_INVALID_ARGUMENT, "set_shape: NULL shape");
    const int vf = full_vec(b->storage);
    const BatchShape sh{shape->threads, shape->cells_per_thread, shape->steps_per_launch, shape->tile_rows,
                        shape->tile_order, 0.f};
    if ((sh.threads != 128 && sh.threads != 256 && sh.threads != 512) || (sh.V != vf && sh.V != vf / 2))
        return bfail(b, LEE_ERR_INVALID_ARGUMENT, "set_shape: not a candidate one-step shape");
    for (const auto &d : b->doms)
        if (d.nx % sh.V) return bfail(b, LEE_ERR_INVALID_ARGUMENT, "set_shape: width does not divide nx");
    if (sh.unit < 1 || sh.unit > 4 || (sh.unit > 1 && !b->fuse_ok))
        return bfail(b, LEE_ERR_INVALID_ARGUMENT, "set_shape: no fused kernel with that step count here");
    if (sh.unit > 1 && (sh.rows < 4 || sh.rows > 1024 || sh.rows % 4 != 0 || sh.order < 0 || sh.order > 1))
        return bfail(b, LEE_ERR_INVALID_ARGUMENT, "set_shape: tile rows must be a multiple of 4 in 4..1024, order 0 or 1");
    if ((s = apply_shape(b, sh)) != LEE_OK) return s;
    b->tuned_us_per_step = 0.f;
    b->tuned = true;
    return LEE_OK;
}

lee_status lee_batch_set_tuning(lee_batch *b, int32_t threads, int32_t cells_per_thread) {
    lee_status s = benter(b);
    if (s != LEE_OK) return s;
    const int vf = full_vec(b->storage);
    if ((threads != 128 && threads != 256 && threads != 512) ||
        (cells_per_thread != vf && cells_per_thread != vf / 2))
        return bfail(b, LEE_ERR_INVALID_ARGUMENT, "set_tuning: not a candidate shape");
    for (const auto &d : b->doms)
        if (d.nx % cells_per_thread) return bfail(b, LEE_ERR_INVALID_ARGUMENT, "set_tuning: width does not divide nx");
    if ((s = build_shape(b, threads, cells_per_thread)) != LEE_OK) return s;
    b->tuned = true;
    return LEE_OK;
}

lee_status lee_batch_cells(lee_batch *b, int64_t *cells) {
    if (!b || !cells) return LEE_ERR_INVALID_ARGUMENT;
    *cells = b->total_cells;
    return LEE_OK;
}

lee_status lee_batch_sync(lee_batch *b) {
    lee_status s = benter(b);
    if (s != LEE_OK) return s;
    BCK(b, cudaStreamSynchronize(b->st), "sync");
    return LEE_OK;
}

const char *lee_batch_last_error(lee_batch *b) { return b ? b->err.c_str() : "NULL batch"; }

lee_status lee_batch_destroy(lee_batch *b) {
    if (!b) return LEE_OK;
    cudaSetDevice(b->device);
    if (b->st) cudaStreamSynchronize(b->st);
    drop_graphs(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    cudaFree(b->buf[0]);
    cudaFree(b->buf[1]);
    cudaFree(b->d_doms);
    cudaFree(b->d_table);
    cudaFree(b->d_tb);
    cudaFree(b->d_tb_tiles);
    cudaFree(b->fields);
    cudaFree(b->pops64);
    cudaFree(b->partial);
    cudaFree(b->red_out);
    delete b;
    cudaGetLastError();
    return LEE_OK;
}

}  // extern "C"
