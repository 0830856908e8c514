// k_batch.cu -- many 2-D grids of uneven size and mixed stencils in one
// persistent launch (the batched form), optionally replayed from a CUDA graph.
//
// Work list: one item per (grid, tile, sweep), ordered sweep-major (all
// sweep-0 items of every grid, then all sweep-1 items, ...).  CTAs pull items
// from a global atomic counter.  An item of sweep s > 0 of grid g waits until
// every tile of sweep s-1 of g has been counted done (bounded spin); because
// every item it waits for has a smaller index and was therefore already
// taken by a running CTA, the wait always ends without any co-residency
// assumption.  Each item stages its tile grown by t*r (L2-coherent loads:
// other CTAs of the same launch produced the data), runs the grid's t
// sub-steps on CUDA cores in shared memory (the same temporal blocking as
// cu2d_sweep) and writes the tile.  Sweep-0 items also copy the halo cells
// nearest to their tile from `in` to the grid's output and ping-pong buffers.
// On a wait that runs out, the CTA sets the abort word and every CTA leaves.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "cu_kernels.cuh"
#include "launch.h"

namespace gbs {
namespace bt {

constexpr int kThreads = 256;
constexpr int kMaxR = 3;
constexpr int kMaxK = (2 * kMaxR + 1) * (2 * kMaxR + 1);

struct GridDev {
    const void *in;
    void *out;
    void *pp;          // ping-pong buffer (null if the run is one sweep)
    int64_t ey, ex;    // stored extents
    int kind;          // shape * 4 + r
    int t, nsweeps, rem;  // fusion depth, sweeps, last sweep depth (0 = t)
    int ntiles, ntx, by, bx;
    int woff;          // offset of the weights in the weight table
    int doff;          // offset of this grid's per-sweep done counters
};

struct Item {
    int g, tile, s, pad;
};

struct Ctl {
    int head;   // next work item
    int abort;  // set when a dependency wait ran out
    int never;  // a counter nothing increments (test hook: an unmet dependency)
    int pad;
};

constexpr unsigned long long kWaitCycles = 2ull << 30;  // ~1 s at 2 GHz

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <typename T>
__device__ __forceinline__ T ld_l2(const T *p)
{
    return __ldcg(p);
}

// One item: tile `tile` of grid G, sweep s (depth t_s) from src to dst.
template <typename T, int SHAPE, int R, int V>
__device__ void run_item(const GridDev &G, const T *__restrict__ wg, const T *src_g, T *dst_g, int tile, int s,
                         int ts, unsigned char *smem)
{
    constexpr int KT = cu::Taps<SHAPE, 2, R>::K;
    T w[KT];
#pragma unroll
    for (int k = 0; k < KT; ++k) w[k] = wg[k];
    const int BY = G.by, BX = G.bx;
    const int H = BY + 2 * ts * R, W = BX + 2 * ts * R, P = W;  // W is even
    T *bufA = reinterpret_cast<T *>(smem);
    T *bufB = bufA + (size_t)H * W;
    const int tby = tile / G.ntx, tbx = tile % G.ntx;
    const int64_t Ey = G.ey, Ex = G.ex, ny = Ey - 2 * R, nx = Ex - 2 * R;
    const int64_t Y0 = R + (int64_t)tby * BY - (int64_t)ts * R;
    const int64_t X0 = R + (int64_t)tbx * BX - (int64_t)ts * R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;

    for (int y = warp; y < H; y += nwarps) {
        const int64_t gy = Y0 + y;
        const bool rowok = gy >= 0 && gy < Ey;
        for (int x = lane; x < W; x += 32) {
            const int64_t gx = X0 + x;
            bufA[y * P + x] = (rowok && gx >= 0 && gx < Ex) ? ld_l2(src_g + gy * Ex + gx) : T(0);
        }
    }
    __syncthreads();
    if (s == 0) {
        // halo cells whose nearest interior point lies in this tile
        T *outp = reinterpret_cast<T *>(G.out);
        T *ppp = reinterpret_cast<T *>(G.pp);
        for (int i = threadIdx.x; i < H * W; i += blockDim.x) {
            const int y = i / W, x = i % W;
            const int64_t gy = Y0 + y, gx = X0 + x;
            if (gy < 0 || gy >= Ey || gx < 0 || gx >= Ex) continue;
            if (gy >= R && gy < Ey - R && gx >= R && gx < Ex - R) continue;  // interior
            const int64_t iy = min(max(gy - R, (int64_t)0), ny - 1), ix = min(max(gx - R, (int64_t)0), nx - 1);
            if (iy / BY != tby || ix / BX != tbx) continue;
            outp[gy * Ex + gx] = bufA[y * P + x];
            if (ppp) ppp[gy * Ex + gx] = bufA[y * P + x];
        }
    }

    T *src = bufA, *dst = bufB;
    for (int sub = 1; sub <= ts; ++sub) {
        const int lo = sub * R;
        const int hiY = H - sub * R, hiX = W - sub * R;
        const int cw = hiX - lo, ch = hiY - lo;
        const int strips = (ch + V - 1) / V;
        const bool last = sub == ts;
        if constexpr (sizeof(T) == 4) {
            struct {
                float w[KT];
            } wrs;
#pragma unroll
            for (int k = 0; k < KT; ++k) wrs.w[k] = w[k];
            const bool all_int = Y0 + lo >= R && Y0 + hiY <= Ey - R && X0 + lo >= R && X0 + hiX <= Ex - R;
            if (((lo - R) & 1) == 0)
                cu::f32_substep<SHAPE, R, 0>(src, dst, dst_g, wrs, P, H, lo, hiY, hiX, Y0, X0, Ey, Ex, last,
                                                all_int, 0);
            else
                cu::f32_substep<SHAPE, R, 1>(src, dst, dst_g, wrs, P, H, lo, hiY, hiX, Y0, X0, Ey, Ex, last,
                                                all_int, 0);
            __syncthreads();
            T *tmp = src;
            src = dst;
            dst = tmp;
            continue;
        }
        for (int item = threadIdx.x; item < cw * strips; item += blockDim.x) {
            const int x = lo + item % cw;
            const int y0 = lo + (item / cw) * V;
            T acc[V];
#pragma unroll
            for (int j = 0; j < V; ++j) acc[j] = T(0);
#pragma unroll
            for (int q = 0; q < V + 2 * R; ++q) {
                const int yy = y0 - R + q;
                if (yy < H) {
                    const T *row = src + yy * P + x;
                    T v[2 * R + 1];
#pragma unroll
                    for (int c = 0; c < 2 * R + 1; ++c) v[c] = row[c - R];
#pragma unroll
                    for (int j = 0; j < V; ++j) {
                        const int oy = q - R - j;
                        if (oy >= -R && oy <= R) {
#pragma unroll
                            for (int ox = -R; ox <= R; ++ox) {
                                const int k = cu::tap_index<SHAPE, 2, R>(0, oy, ox);
                                if (k >= 0) acc[j] = fma(w[k], v[ox + R], acc[j]);
                            }
                        }
                    }
                }
            }
            const int64_t gx = X0 + x;
            const bool colint = gx >= R && gx < Ex - R;
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const int y = y0 + j;
                if (y < hiY) {
                    const int64_t gy = Y0 + y;
                    const bool interior = colint && gy >= R && gy < Ey - R;
                    if (last) {
                        if (interior) dst_g[gy * Ex + gx] = acc[j];
                    } else {
                        dst[y * P + x] = interior ? acc[j] : src[y * P + x];
                    }
                }
            }
        }
        __syncthreads();
        T *tmp = src;
        src = dst;
        dst = tmp;
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    batch_sweeps(const GridDev *__restrict__ grids, const Item *__restrict__ items, int nitems,
                 const T *__restrict__ wtab, int *done, Ctl *ctl, unsigned long long wait_cycles, int block_sweep)
{
    constexpr int V = sizeof(T) == 8 ? 4 : 8;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_idx, s_go;
    for (;;) {
        if (threadIdx.x == 0) {
            s_idx = *(volatile int *)&ctl->abort ? nitems : atomicAdd(&ctl->head, 1);
            s_go = 1;
        }
        __syncthreads();
        const int idx = s_idx;
        if (idx >= nitems) break;
        const Item it = items[idx];
        const GridDev G = grids[it.g];
        if (it.s > 0 && threadIdx.x == 0) {
            const int *dep = it.s == block_sweep ? &ctl->never : done + G.doff + it.s - 1;
            const unsigned long long t0 = clock64();
            while (ld_acquire(dep) < G.ntiles) {
                if (clock64() - t0 > wait_cycles || *(volatile int *)&ctl->abort) {
                    atomicExch(&ctl->abort, 1);
                    s_go = 0;
                    break;
                }
            }
        }
        __syncthreads();
        if (!s_go) break;
        const int ts = (it.s == G.nsweeps - 1 && G.rem) ? G.rem : G.t;
        const T *src = it.s == 0 ? reinterpret_cast<const T *>(G.in)
                                 : reinterpret_cast<const T *>(((G.nsweeps - it.s) % 2 == 0) ? G.out : G.pp);
        T *dst = reinterpret_cast<T *>(((G.nsweeps - 1 - it.s) % 2 == 0) ? G.out : G.pp);
        const T *wg = wtab + G.woff;
        switch (G.kind) {
        case 0 * 4 + 1: run_item<T, 0, 1, V>(G, wg, src, dst, it.tile, it.s, ts, smem); break;
        case 0 * 4 + 2: run_item<T, 0, 2, V>(G, wg, src, dst, it.tile, it.s, ts, smem); break;
        case 0 * 4 + 3: run_item<T, 0, 3, V>(G, wg, src, dst, it.tile, it.s, ts, smem); break;
        case 1 * 4 + 1: run_item<T, 1, 1, V>(G, wg, src, dst, it.tile, it.s, ts, smem); break;
        case 1 * 4 + 2: run_item<T, 1, 2, V>(G, wg, src, dst, it.tile, it.s, ts, smem); break;
        case 1 * 4 + 3: run_item<T, 1, 3, V>(G, wg, src, dst, it.tile, it.s, ts, smem); break;
        default: break;
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(done + G.doff + it.s, 1);
    }
}

}  // namespace bt

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct BatchGridHost {
    Plan plan;  // pattern, weights, path, precision, t and tile
    // CUDA-core grids run as work items of the persistent kernel; a grid on a
    // tensor-core path runs as the plan's own sweeps after it, on the same
    // stream (and inside the same graph)
    bool on_cu() const { return plan.path == STENCIL_PATH_CUDA_CORE; }
};

struct BatchCache {
    std::vector<const void *> ins;
    std::vector<void *> outs;
    int64_t steps = -1;
    size_t kernel_nodes = 1;
    void *ws = nullptr;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
};

}  // namespace gbs

struct stencil_batch {
    stencil_dtype dtype = STENCIL_F32;
    std::vector<gbs::BatchGridHost> grids;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    size_t ctl_off = 0;  // control word of the last run
    bool ran = false;
    unsigned long long wait_cycles = gbs::bt::kWaitCycles;  // bounded dependency wait
    int block_sweep = -1;  // test hook: sweep whose items wait on a counter nothing increments
    int precision = STENCIL_PREC_NATIVE;  // forms the autotuner may use for FP32 grids
    gbs::BatchCache cache;
};

namespace gbs {
namespace {

// Shared memory of one work item (a staging and a work buffer of the tile
// grown by t r), and the budget every item of a batch keeps to: the launch
// takes the largest item's size, and three CTAs per SM need <= ~74 KB each.
constexpr size_t kBatchItemSmem = 74 * 1024;

size_t batch_item_smem(int by, int bx, int t, int r, size_t es)
{
    return (size_t)(by + 2 * t * r) * (bx + 2 * t * r) * es * 2;
}

struct Layout {
    size_t grids_off, items_off, w_off, done_off, ctl_off, pp_off, total;
    int nitems, ndone;
    bool too_many;  // more work items than an int indexes: the run is refused
    std::vector<size_t> pp_of;  // per grid: offset of its ping-pong buffer (or SIZE_MAX)
};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int64_t sweeps_of(const Plan &p, int64_t steps) { return steps / p.t + (steps % p.t ? 1 : 0); }

int64_t ntiles_of(const Plan &p)
{
    return ((p.dims[1] + p.tile[1] - 1) / p.tile[1]) * ((p.dims[2] + p.tile[2] - 1) / p.tile[2]);
}

Layout layout_of(const stencil_batch &b, int64_t steps)
{
    Layout L{};
    const size_t es = b.dtype == STENCIL_F64 ? 8 : 4;
    int64_t nitems = 0, ndone = 0, nw = 0;
    for (auto &g : b.grids) {
        const int64_t ns = steps > 0 ? sweeps_of(g.plan, steps) : 0;
        if (g.on_cu()) nitems += ntiles_of(g.plan) * ns;
        ndone += ns;
        nw += g.plan.pat.K;
    }
    L.too_many = nitems > 0x7fffffff || ndone > 0x7fffffff;  // the device tables index with int
    L.nitems = L.too_many ? 0 : (int)nitems;
    L.ndone = L.too_many ? 0 : (int)ndone;
    size_t off = 0;
    L.grids_off = off;
    off = align_up(off + sizeof(bt::GridDev) * b.grids.size(), 256);
    L.items_off = off;
    off = align_up(off + sizeof(bt::Item) * (size_t)nitems, 256);
    L.w_off = off;
    off = align_up(off + es * (size_t)nw, 256);
    L.done_off = off;
    off = align_up(off + sizeof(int) * (size_t)std::max<int64_t>(ndone, 1), 256);
    L.ctl_off = off;
    off = align_up(off + sizeof(bt::Ctl), 256);
    L.pp_off = off;
    for (auto &g : b.grids) {
        const int64_t ns = steps > 0 ? sweeps_of(g.plan, steps) : 0;
        if (ns > 1) {
            L.pp_of.push_back(off);
            off = align_up(off + g.plan.grid_bytes(), 256);
        } else {
            L.pp_of.push_back(SIZE_MAX);
        }
    }
    L.total = off;
    return L;
}

// Grids on a tensor-core path: each runs its plan's sweeps (ping-pong
// through its buffer in the workspace).
stencil_status launch_tc_grids(stencil_batch *b, const Layout &L, const void *const *ins, void *const *outs,
                               int64_t steps, cudaStream_t st)
{
    for (size_t i = 0; i < b->grids.size(); i++) {
        BatchGridHost &g = b->grids[i];
        if (g.on_cu()) continue;
        void *pp = L.pp_of[i] == SIZE_MAX ? nullptr : (char *)b->ws + L.pp_of[i];
        stencil_status s = run_sweeps(g.plan, ins[i], outs[i], pp, pp ? g.plan.grid_bytes() : 0, steps, st);
        if (s != STENCIL_OK) return s;
    }
    return STENCIL_OK;
}

stencil_status launch_batch(stencil_batch *b, const Layout &L, const void *const *ins, void *const *outs,
                            int64_t steps, cudaStream_t st, bool count)
{
    char *ws = (char *)b->ws;
    cudaError_t e = cudaMemsetAsync(ws + L.done_off, 0, L.ctl_off - L.done_off + sizeof(bt::Ctl), st);
    if (e != cudaSuccess) return cuda_fail(e, "batch: clearing the counters");
    b->ctl_off = L.ctl_off;
    b->ran = true;
    if (L.nitems == 0) return launch_tc_grids(b, L, ins, outs, steps, st);
    size_t smem = 0;
    const size_t es = b->dtype == STENCIL_F64 ? 8 : 4;
    for (auto &g : b->grids) {
        if (!g.on_cu()) continue;
        const int R = g.plan.pat.r, t = g.plan.t;
        smem = std::max(smem, batch_item_smem(g.plan.tile[1], g.plan.tile[2], t, R, es));
    }
    const void *fn = b->dtype == STENCIL_F64 ? (const void *)bt::batch_sweeps<double> : (const void *)bt::batch_sweeps<float>;
    stencil_status s = ensure_smem(fn, smem);
    if (s != STENCIL_OK) return s;
    int occ = 0, dev = 0, sms = 0;
    s = occupancy(fn, bt::kThreads, smem, &occ);
    if (s != STENCIL_OK) return s;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)std::min<int64_t>(L.nitems, (int64_t)std::max(1, occ) * sms);
    const bt::GridDev *gd = (const bt::GridDev *)(ws + L.grids_off);
    const bt::Item *items = (const bt::Item *)(ws + L.items_off);
    int *done = (int *)(ws + L.done_off);
    bt::Ctl *ctl = (bt::Ctl *)(ws + L.ctl_off);
    if (b->dtype == STENCIL_F64)
        bt::batch_sweeps<double><<<grid, bt::kThreads, smem, st>>>(gd, items, L.nitems, (const double *)(ws + L.w_off),
                                                                   done, ctl, b->wait_cycles, b->block_sweep);
    else
        bt::batch_sweeps<float><<<grid, bt::kThreads, smem, st>>>(gd, items, L.nitems, (const float *)(ws + L.w_off),
                                                                  done, ctl, b->wait_cycles, b->block_sweep);
    if (count) note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "batch_sweeps launch");
    return launch_tc_grids(b, L, ins, outs, steps, st);
}

// Host tables for one run: grid descriptors with this run's pointers, the
// sweep-major work list and the weights, uploaded into the workspace.
stencil_status upload_tables(stencil_batch *b, const Layout &L, const void *const *ins, void *const *outs,
                             int64_t steps, cudaStream_t st)
{
    const size_t es = b->dtype == STENCIL_F64 ? 8 : 4;
    std::vector<unsigned char> host(L.done_off, 0);
    bt::GridDev *gd = (bt::GridDev *)(host.data() + L.grids_off);
    bt::Item *items = (bt::Item *)(host.data() + L.items_off);
    unsigned char *w = host.data() + L.w_off;
    int woff = 0, doff = 0, maxs = 0;
    for (size_t i = 0; i < b->grids.size(); i++) {
        const Plan &p = b->grids[i].plan;
        bt::GridDev &g = gd[i];
        g.in = ins[i];
        g.out = outs[i];
        g.pp = L.pp_of[i] == SIZE_MAX ? nullptr : (char *)b->ws + L.pp_of[i];
        g.ey = p.ext[1];
        g.ex = p.ext[2];
        g.kind = p.pat.shape * 4 + p.pat.r;
        g.t = p.t;
        g.nsweeps = b->grids[i].on_cu() ? (int)sweeps_of(p, steps) : 0;  // tensor-core grids have no items
        g.rem = (int)(steps % p.t);
        g.by = p.tile[1];
        g.bx = p.tile[2];
        g.ntx = (int)((p.dims[2] + g.bx - 1) / g.bx);
        g.ntiles = (int)ntiles_of(p);
        g.woff = woff;
        g.doff = doff;
        for (int k = 0; k < p.pat.K; k++) {
            if (es == 8) ((double *)w)[woff + k] = p.w[k];
            else ((float *)w)[woff + k] = (float)p.w[k];
        }
        woff += p.pat.K;
        doff += g.nsweeps;
        maxs = std::max(maxs, g.nsweeps);
    }
    int n = 0;
    for (int s = 0; s < maxs; s++)
        for (size_t i = 0; i < b->grids.size(); i++)
            if (s < gd[i].nsweeps)
                for (int tl = 0; tl < gd[i].ntiles; tl++) items[n++] = bt::Item{(int)i, tl, s, 0};
    cudaError_t e = cudaMemcpyAsync(b->ws, host.data(), host.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host table is released on return
    return e == cudaSuccess ? STENCIL_OK : cuda_fail(e, "batch: uploading the tables");
}

stencil_status check_run_args(stencil_batch *b, const void *const *ins, void *const *outs, int64_t steps,
                              Layout *L)
{
    if (!b || !ins || !outs) return fail(STENCIL_ERR_INVALID_ARG, "stencil_batch_run: null argument");
    if (steps < 0) return fail(STENCIL_ERR_INVALID_ARG, "stencil_batch_run: steps < 0");
    for (size_t i = 0; i < b->grids.size(); i++) {
        if (!ins[i] || !outs[i] || ins[i] == outs[i])
            return fail(STENCIL_ERR_INVALID_ARG, "stencil_batch_run: grid " + std::to_string(i) +
                                                     ": null or identical in/out");
    }
    *L = layout_of(*b, steps);
    if (L->too_many)
        return fail(STENCIL_ERR_UNSUPPORTED, "stencil_batch_run: more than 2^31 - 1 work items; split the batch");
    if (!b->ws || b->ws_bytes < L->total)
        return fail(STENCIL_ERR_OOM, "stencil_batch_run: workspace smaller than stencil_batch_workspace_bytes");
    return STENCIL_OK;
}

// One staging + one work buffer per work item: the CUDA-core default tile,
// halved until the grown tile pair fits the per-item budget.
void batch_tile(Plan *p)
{
    int tile[3];
    cu_default_tile(*p, p->t, tile);
    for (;;) {
        const size_t bytes = batch_item_smem(tile[1], tile[2], p->t, p->pat.r, p->elem_bytes());
        if (bytes <= kBatchItemSmem || (tile[1] <= 16 && tile[2] <= 16)) break;
        if (tile[2] >= tile[1]) tile[2] /= 2; else tile[1] /= 2;
    }
    for (int k = 0; k < 3; k++) p->tile[k] = tile[k];
    p->info.tile[0] = tile[0];
    p->info.tile[1] = tile[1];
    p->info.tile[2] = tile[2];
}

void drop_graph(BatchCache &c)
{
    if (c.exec) cudaGraphExecDestroy(c.exec);
    if (c.graph) cudaGraphDestroy(c.graph);
    c.exec = nullptr;
    c.graph = nullptr;
    c.steps = -1;
}

}  // namespace
}  // namespace gbs

using namespace gbs;

extern "C" {

stencil_status stencil_batch_create(stencil_batch **batch, int n, const stencil_grid_desc *grids, stencil_dtype dtype,
                                    int t)
try {
    if (!batch) return fail(STENCIL_ERR_INVALID_ARG, "stencil_batch_create: batch is null");
    *batch = nullptr;
    if (n < 1 || !grids) return fail(STENCIL_ERR_INVALID_ARG, "stencil_batch_create: need n >= 1 grids");
    if (dtype != STENCIL_F64 && dtype != STENCIL_F32)
        return fail(STENCIL_ERR_INVALID_ARG, "stencil_batch_create: dtype must be F64 or F32");
    if (t < 0 || t > kMaxT) return fail(STENCIL_ERR_INVALID_ARG, "stencil_batch_create: t must be 0..16");
    auto *b = new (std::nothrow) stencil_batch;
    if (!b) return fail(STENCIL_ERR_OOM, "stencil_batch_create: host allocation");
    b->dtype = dtype;
    for (int i = 0; i < n; i++) {
        const stencil_grid_desc &d = grids[i];
        if (d.r < 1 || d.r > bt::kMaxR || (d.shape != STENCIL_BOX && d.shape != STENCIL_STAR)) {
            delete b;
            return fail(STENCIL_ERR_UNSUPPORTED, "stencil_batch_create: grid " + std::to_string(i) +
                                                     ": the batched form takes box/star with r = 1..3");
        }
        int64_t dims[2] = {d.ny, d.nx};
        stencil_plan *p = nullptr;
        stencil_status s = stencil_plan_create(&p, (stencil_shape)d.shape, 2, d.r, d.weights, dtype, dims, t);
        if (s == STENCIL_OK) s = stencil_plan_set_option(p, "path", "cuda_core");
        if (s != STENCIL_OK) {
            stencil_plan_destroy(p);
            delete b;
            return s;
        }
        BatchGridHost g;
        g.plan = p->p;
        stencil_plan_destroy(p);
        batch_tile(&g.plan);
        b->grids.push_back(std::move(g));
    }
    *batch = b;
    return STENCIL_OK;
} catch (...) {
    return gbs::abi_exception("stencil_batch_create");
}

size_t stencil_batch_workspace_bytes(const stencil_batch *batch, int64_t steps)
try {
    if (!batch || steps < 0) return 0;
    return layout_of(*batch, steps).total;
} catch (...) {
    gbs::abi_exception("stencil_batch_workspace_bytes");
    return 0;
}

stencil_status stencil_batch_set_workspace(stencil_batch *batch, void *dev_ptr, size_t bytes)
try {
    if (!batch) return fail(STENCIL_ERR_INVALID_ARG, "stencil_batch_set_workspace: batch is null");
    if (!dev_ptr && bytes) return fail(STENCIL_ERR_INVALID_ARG, "stencil_batch_set_workspace: null with bytes > 0");
    if (dev_ptr != batch->ws) drop_graph(batch->cache);
    batch->ws = dev_ptr;
    batch->ws_bytes = dev_ptr ? bytes : 0;
    return STENCIL_OK;
} catch (...) {
    return gbs::abi_exception("stencil_batch_set_workspace");
}

stencil_status stencil_batch_info(const stencil_batch *batch, int i, stencil_info *info)
try {
    if (!batch || !info || i < 0 || i >= (int)batch->grids.size())
        return fail(STENCIL_ERR_INVALID_ARG, "stencil_batch_info: bad argument");
    *info = batch->grids[i].plan.info;
    for (int k = 0; k < 3; k++) info->tile[k] = batch->grids[i].plan.tile[k];
    return STENCIL_OK;
} catch (...) {
    return gbs::abi_exception("stencil_batch_info");
}

stencil_status stencil_batch_run(stencil_batch *batch, const void *const *ins, void *const *outs, int64_t steps,
                                 stencil_stream_t stream)
try {
    Layout L;
    stencil_status s = check_run_args(batch, ins, outs, steps, &L);
    if (s != STENCIL_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if (steps == 0) {
        for (size_t i = 0; i < batch->grids.size(); i++) {
            cudaError_t e = cudaMemcpyAsync(outs[i], ins[i], batch->grids[i].plan.grid_bytes(),
                                            cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return cuda_fail(e, "stencil_batch_run: copy");
        }
        return STENCIL_OK;
    }
    drop_graph(batch->cache);  // the tables are about to change
    s = upload_tables(batch, L, ins, outs, steps, st);
    if (s != STENCIL_OK) return s;
    return launch_batch(batch, L, ins, outs, steps, st, true);
} catch (...) {
    return gbs::abi_exception("stencil_batch_run");
}

stencil_status stencil_batch_run_graph(stencil_batch *batch, const void *const *ins, void *const *outs, int64_t steps,
                                       stencil_stream_t stream)
try {
    Layout L;
    stencil_status s = check_run_args(batch, ins, outs, steps, &L);
    if (s != STENCIL_OK) return s;
    if (!stream) return fail(STENCIL_ERR_INVALID_ARG, "stencil_batch_run_graph: needs a non-default stream");
    if (steps == 0) return stencil_batch_run(batch, ins, outs, 0, stream);
    cudaStream_t st = (cudaStream_t)stream;
    BatchCache &c = batch->cache;
    const size_t n = batch->grids.size();
    const bool same = c.exec && c.steps == steps && c.ws == batch->ws && c.stream == st &&
                      std::equal(c.ins.begin(), c.ins.end(), ins) && std::equal(c.outs.begin(), c.outs.end(), outs);
    if (!same) {
        drop_graph(c);
        s = upload_tables(batch, L, ins, outs, steps, st);
        if (s != STENCIL_OK) return s;
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "stencil_batch_run_graph: begin capture");
        s = launch_batch(batch, L, ins, outs, steps, st, false);  // counted at each replay
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(st, &g);
        if (s != STENCIL_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e != cudaSuccess) return cuda_fail(e, "stencil_batch_run_graph: end capture");
        e = cudaGraphInstantiate(&c.exec, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            return cuda_fail(e, "stencil_batch_run_graph: instantiate");
        }
        c.graph = g;
        size_t nn = 0;
        c.kernel_nodes = 0;
        if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
            std::vector<cudaGraphNode_t> nodes(nn);
            if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
                for (auto nd : nodes) {
                    cudaGraphNodeType ty;
                    if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel)
                        c.kernel_nodes++;
                }
        }
        c.ins.assign(ins, ins + n);
        c.outs.assign(outs, outs + n);
        c.steps = steps;
        c.ws = batch->ws;
        c.stream = st;
    }
    cudaError_t e = cudaGraphLaunch(c.exec, st);
    if (e != cudaSuccess) return cuda_fail(e, "stencil_batch_run_graph: launch");
    note_launch(c.kernel_nodes);
    return STENCIL_OK;
} catch (...) {
    return gbs::abi_exception("stencil_batch_run_graph");
}

stencil_status stencil_batch_status(stencil_batch *batch, stencil_stream_t stream)
try {
    if (!batch) return fail(STENCIL_ERR_INVALID_ARG, "stencil_batch_status: batch is null");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "stencil_batch_status: stream");
    if (!batch->ran || !batch->ws) return STENCIL_OK;
    bt::Ctl ctl{};
    e = cudaMemcpy(&ctl, (char *)batch->ws + batch->ctl_off, sizeof(ctl), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "stencil_batch_status: reading the control word");
    if (ctl.abort) return fail(STENCIL_ERR_TIMEOUT, "stencil_batch: a dependency wait ran out; outputs incomplete");
    return STENCIL_OK;
} catch (...) {
    return gbs::abi_exception("stencil_batch_status");
}

stencil_status stencil_batch_set_option(stencil_batch *batch, const char *key, const char *value)
try {
    if (!batch || !key || !value) return fail(STENCIL_ERR_INVALID_ARG, "stencil_batch_set_option: null argument");
    const std::string ks(key), vs(value);
    if (ks == "precision") {
        int pr;
        if (vs == "native") pr = STENCIL_PREC_NATIVE;
        else if (vs == "tf32") pr = STENCIL_PREC_TF32;
        else if (vs == "tf32x3") pr = STENCIL_PREC_TF32X3;
        else if (vs == "bf16x3") pr = STENCIL_PREC_BF16X3;
        else if (vs == "any") pr = STENCIL_PREC_ANY;
        else return fail(STENCIL_ERR_INVALID_ARG, "batch precision must be native|tf32|tf32x3|bf16x3|any");
        if (batch->dtype == STENCIL_F64 && pr != STENCIL_PREC_NATIVE)
            return fail(STENCIL_ERR_UNSUPPORTED, "batch precision: FP64 grids compute natively");
        batch->precision = pr;
        return STENCIL_OK;
    }
    if (ks == "path") {
        // every grid on this path (its model-chosen form and t)
        int path;
        if (vs == "auto") path = STENCIL_PATH_AUTO;
        else if (vs == "cuda_core") path = STENCIL_PATH_CUDA_CORE;
        else if (vs == "tensor_core") path = STENCIL_PATH_TENSOR_CORE;
        else if (vs == "sparse_tensor_core") path = STENCIL_PATH_SPARSE_TENSOR_CORE;
        else return fail(STENCIL_ERR_INVALID_ARG, "batch path must be auto|cuda_core|tensor_core|sparse_tensor_core");
        std::vector<Plan> plans;
        for (auto &g : batch->grids) {
            Plan q = g.plan;
            q.req_path = path;
            q.req_precision = path == STENCIL_PATH_CUDA_CORE ? STENCIL_PREC_NATIVE : batch->precision;
            q.req_tile[0] = q.req_tile[1] = q.req_tile[2] = 0;
            stencil_status s = dispatch(&q);
            if (s != STENCIL_OK) return s;
            if (q.path == STENCIL_PATH_CUDA_CORE) batch_tile(&q);
            plans.push_back(q);
        }
        for (size_t i = 0; i < plans.size(); i++) batch->grids[i].plan = plans[i];
        drop_graph(batch->cache);
        return STENCIL_OK;
    }
    char *end = nullptr;
    const long long v = std::strtoll(value, &end, 10);
    if (!*value || *end) return fail(STENCIL_ERR_INVALID_ARG, "stencil_batch_set_option: value must be an integer");
    const std::string k(key);
    if (k == "wait_cycles") {
        if (v < 1) return fail(STENCIL_ERR_INVALID_ARG, "wait_cycles must be >= 1");
        batch->wait_cycles = (unsigned long long)v;
    } else if (k == "debug_block_sweep") {
        if (v < -1 || v == 0) return fail(STENCIL_ERR_INVALID_ARG, "debug_block_sweep must be -1 or >= 1");
        batch->block_sweep = (int)v;
    } else {
        return fail(STENCIL_ERR_INVALID_ARG, "unknown batch option '" + k + "'");
    }
    drop_graph(batch->cache);
    return STENCIL_OK;
} catch (...) {
    return gbs::abi_exception("stencil_batch_set_option");
}

// Autotuner of the batched form.  Grids are grouped into shape classes
// (stencil shape and radius, and size class c: interior points in
// [4^(6+c), 4^(7+c)), i.e. sides around 64 * 2^c).  For each class the
// candidates -- CUDA-core work items with t = 1..4 and tiles from 16 x 64 to
// 128 x 128, and, where the batch precision allows and the grids are large,
// the dense and sparse tensor-core paths with t = 1..4 -- are ranked by the
// model (the dispatcher's prediction for the class's first grid); the
// model's best kTunePerPath of each path plus the current choice are
// measured on a batch made of the class's grids alone (CUDA events on
// `stream`, after one untimed run), and the fastest becomes the choice of
// every grid of the class.
static const int kTuneTiles[][2] = {{16, 64}, {32, 64}, {32, 128}, {64, 64}, {64, 128}, {128, 128}};
constexpr int kTunePerPath = 4;

static int size_class(const Plan &p)
{
    const double pts = (double)p.dims[1] * (double)p.dims[2];
    int c = (int)std::floor(std::log2(std::max(pts, 1.0)) / 2.0) - 6;
    return std::min(6, std::max(0, c));
}

stencil_status stencil_batch_autotune(stencil_batch *batch, const void *const *ins, void *const *outs, int64_t steps,
                                      int reps, stencil_stream_t stream, stencil_batch_tune_result *results,
                                      int max_results, int *n_results)
try {
    if (n_results) *n_results = 0;
    if (steps < 1 || reps < 1) return fail(STENCIL_ERR_INVALID_ARG, "stencil_batch_autotune: steps and reps >= 1");
    Layout L0;
    stencil_status s = check_run_args(batch, ins, outs, steps, &L0);
    if (s != STENCIL_OK) return s;
    drop_graph(batch->cache);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t es = batch->dtype == STENCIL_F64 ? 8 : 4;
    std::map<long, std::vector<int>> classes;
    for (size_t i = 0; i < batch->grids.size(); i++) {
        const Plan &p = batch->grids[i].plan;
        classes[(long)p.pat.shape * 10000 + p.pat.r * 100 + size_class(p)].push_back((int)i);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return fail(STENCIL_ERR_CUDA, "stencil_batch_autotune: cudaEventCreate");
    }
    struct Cand {
        int path, prec, t, ty, tx;
        double model, measured;
    };
    int nres = 0, cls = 0;
    for (auto &kv : classes) {
        const std::vector<int> &members = kv.second;
        const Plan &base = batch->grids[members[0]].plan;
        const int r = base.pat.r, sc = size_class(base);
        int64_t maxy = 0, maxx = 0;
        double pts = 0;
        for (int i : members) {
            maxy = std::max(maxy, batch->grids[i].plan.dims[1]);
            maxx = std::max(maxx, batch->grids[i].plan.dims[2]);
            pts += (double)batch->grids[i].plan.dims[1] * (double)batch->grids[i].plan.dims[2];
        }
        // configure plan q for a candidate; false if no kernel takes it
        auto configure = [&](Plan *q, const Cand &c) {
            q->req_path = c.path;
            q->req_precision = c.prec;
            q->req_t = c.t;
            q->req_tile[0] = q->req_tile[1] = q->req_tile[2] = 0;
            if (c.path == STENCIL_PATH_CUDA_CORE) {
                q->req_tile[0] = 1;
                q->req_tile[1] = c.ty;
                q->req_tile[2] = c.tx;
            }
            return dispatch(q) == STENCIL_OK;
        };
        std::vector<Cand> cands;
        for (int t = 1; t <= 4; t++)
            for (auto &tl : kTuneTiles) {
                const int ty = tl[0], tx = tl[1];
                if (batch_item_smem(ty, tx, t, r, es) > kBatchItemSmem) continue;
                if (ty > 2 * std::max<int64_t>(16, maxy) || tx > 2 * std::max<int64_t>(64, maxx)) continue;
                Cand c{STENCIL_PATH_CUDA_CORE, STENCIL_PREC_NATIVE, t, ty, tx, 0, 0};
                Plan q = base;
                if (configure(&q, c)) {
                    c.model = q.info.predicted_gstencils;
                    cands.push_back(c);
                }
            }
        const bool tc_ok = batch->dtype == STENCIL_F64 || batch->precision != STENCIL_PREC_NATIVE;
        if (tc_ok && sc >= 3) {
            std::vector<int> precs;
            if (batch->dtype == STENCIL_F64) precs = {STENCIL_PREC_NATIVE};
            else if (batch->precision == STENCIL_PREC_ANY) precs = {STENCIL_PREC_TF32, STENCIL_PREC_TF32X3, STENCIL_PREC_BF16X3};
            else precs = {batch->precision};
            for (int path : {STENCIL_PATH_TENSOR_CORE, STENCIL_PATH_SPARSE_TENSOR_CORE})
                for (int pr : precs)
                    for (int t = 1; t <= 4 && t * r <= 12; t++) {
                        Cand c{path, pr, t, 0, 0, 0, 0};
                        Plan q = base;
                        if (configure(&q, c)) {
                            c.model = q.info.predicted_gstencils;
                            c.ty = q.tile[1];
                            c.tx = q.tile[2];
                            cands.push_back(c);
                        }
                    }
        }
        std::stable_sort(cands.begin(), cands.end(), [](const Cand &a, const Cand &b) { return a.model > b.model; });
        {
            // the model's best kTunePerPath of each path
            std::vector<Cand> keep;
            int taken[4] = {0, 0, 0, 0};
            for (auto &c : cands)
                if (taken[c.path]++ < kTunePerPath) keep.push_back(c);
            cands.swap(keep);
        }
        // the current choice is always among the measured
        {
            Cand cur{base.path, base.precision, base.t, base.tile[1], base.tile[2], base.info.predicted_gstencils, 0};
            bool have = false;
            for (auto &c : cands)
                have |= c.path == cur.path && c.prec == cur.prec && c.t == cur.t &&
                        (c.path != STENCIL_PATH_CUDA_CORE || (c.ty == cur.ty && c.tx == cur.tx));
            if (!have) cands.push_back(cur);
        }
        int best = -1;
        std::vector<Plan> best_plans;
        for (size_t ci = 0; ci < cands.size(); ci++) {
            Cand &c = cands[ci];
            stencil_batch sub;
            sub.dtype = batch->dtype;
            sub.ws = batch->ws;
            sub.ws_bytes = batch->ws_bytes;
            sub.wait_cycles = batch->wait_cycles;
            std::vector<const void *> sin;
            std::vector<void *> sout;
            bool ok = true;
            for (int i : members) {
                BatchGridHost g = batch->grids[i];
                ok = ok && configure(&g.plan, c);
                sub.grids.push_back(g);
                sin.push_back(ins[i]);
                sout.push_back(outs[i]);
            }
            if (!ok) continue;
            const Layout Ls = layout_of(sub, steps);
            if (Ls.too_many || Ls.total > sub.ws_bytes) continue;  // too large for the caller's workspace
            s = upload_tables(&sub, Ls, sin.data(), sout.data(), steps, st);
            if (s == STENCIL_OK) s = launch_batch(&sub, Ls, sin.data(), sout.data(), steps, st, true);
            if (s == STENCIL_OK && cudaEventRecord(e0, st) != cudaSuccess) s = fail(STENCIL_ERR_CUDA, "event");
            for (int k = 0; k < reps && s == STENCIL_OK; k++)
                s = launch_batch(&sub, Ls, sin.data(), sout.data(), steps, st, true);
            if (s == STENCIL_OK && cudaEventRecord(e1, st) != cudaSuccess) s = fail(STENCIL_ERR_CUDA, "event");
            if (s != STENCIL_OK) break;
            cudaError_t e = cudaEventSynchronize(e1);
            float ms = 0;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                s = cuda_fail(e, "stencil_batch_autotune: timing");
                break;
            }
            bt::Ctl ctl{};
            e = cudaMemcpy(&ctl, (char *)sub.ws + Ls.ctl_off, sizeof(ctl), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) {
                s = cuda_fail(e, "stencil_batch_autotune: control word");
                break;
            }
            if (ctl.abort) {
                s = fail(STENCIL_ERR_TIMEOUT, "stencil_batch_autotune: a dependency wait ran out");
                break;
            }
            c.measured = pts * (double)steps * reps / (ms * 1e-3) / 1e9;
            if (best < 0 || c.measured > cands[best].measured) {
                best = (int)ci;
                best_plans.clear();
                for (auto &g : sub.grids) best_plans.push_back(g.plan);
            }
        }
        if (s != STENCIL_OK) break;
        if (best >= 0)
            for (size_t k = 0; k < members.size(); k++) batch->grids[members[k]].plan = best_plans[k];
        for (size_t ci = 0; ci < cands.size(); ci++) {
            if (results && nres < max_results) {
                stencil_batch_tune_result &o = results[nres];
                o.cls = cls;
                o.shape = base.pat.shape;
                o.r = r;
                o.size_class = sc;
                o.ngrids = (int)members.size();
                o.path = cands[ci].path;
                o.precision = cands[ci].prec;
                o.t = cands[ci].t;
                o.tile_y = cands[ci].ty;
                o.tile_x = cands[ci].tx;
                o.model_gstencils = cands[ci].model;
                o.measured_gstencils = cands[ci].measured;
                o.chosen = (int)ci == best;
            }
            nres++;
        }
        cls++;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    batch->ran = false;
    if (n_results) *n_results = nres;
    return s;
} catch (...) {
    return gbs::abi_exception("stencil_batch_autotune");
}

void stencil_batch_destroy(stencil_batch *batch)
try {
    if (!batch) return;
    drop_graph(batch->cache);
    delete batch;
} catch (...) {
    gbs::abi_exception("stencil_batch_destroy");
}

}  // extern "C"
