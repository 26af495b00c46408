// Batched super time stepping: many independent conduction problems of uneven sizes and stage
// counts advanced in one persistent, CUDA-graph-launched kernel, plus the autotuner that picks
// its tile schedule.
//
// Work items are (problem p, level L, tile t); level 1 is y0 = F(u), level 2 the fused stages
// 1+2, level L >= 3 stage L.  Items are ordered level-major across problems, and a block
// claims the next item with an atomic counter.  Before working on (p, L, t) it waits until
// all tiles of (p, L-1) are done; those items have lower indices, so they were claimed earlier
// by blocks that are running, and the wait cannot deadlock whatever the number of resident
// blocks.  Each wait is bounded: on timeout the kernel raises an error flag and stops claiming.
// Operands produced inside the launch are read through L2 (PolF32CG on the register tile).
// Problems whose arrays tensor maps can describe march their 32 x 8 tiles through the same TMA
// ring as the one-problem kernel (tma_march_tile), with the problem's tensor maps in global
// memory; a block acquires a level's completion, then orders its later TMA reads after it with
// a proxy fence.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

#include "epilogues.cuh"
#include "launch.h"
#include "march.cuh"
#include "march_tma.cuh"
#include "sts_coeffs.h"

namespace pb {

struct BatchProblem {
    CompGrid cg;               // offset 0, tiles / chunks for this problem's tile variant
    const Coef4<float>* coef;
    float* u;
    float* y0;
    float* buf[3];
    unsigned int* done;        // done[L] = finished tiles of level L (L = 1..s)
    int s;
    int tiles;                 // tiles per level
    int variant;               // 0: 32 x 8 tiles, 1: 16 x 16 tiles
    int coef_off;              // first level-coefficient record of this problem
    const CUtensorMap* maps;   // kMaps tensor maps of the TMA ring (variant 0), or null
};

// Tensor maps of one problem: halo boxes of the fields a level marches (u, y0, buf[0..2]), point
// boxes of the same arrays (epilogue operands), and the records.
enum { kMapField = 0, kMapCen = 5, kMapCoef = 10, kMaps = 11 };
using BatchTma3 = TmaLayout<PolF32, 3, PlainField<PolF32>>;   // the largest ring layout an item uses

struct BatchSeg { long long begin; int p; int level; };

// level-2 record: {a1, cy, cf, -}; level L >= 3 record: {mu, nu, mdt, ydt}; each float64
// coefficient as a float pair (the double-float stage recurrence of the float32 policy)
struct LevelCoef { float a, b, c, d, al, bl, cl, dl; };

static LevelCoef level_coef(double a, double b, double c, double d) {
    auto lo = [](double x) { return (float)(x - (double)(float)x); };
    return LevelCoef{(float)a, (float)b, (float)c, (float)d, lo(a), lo(b), lo(c), lo(d)};
}

namespace {

constexpr unsigned kSpinLimit = 1u << 26;

template <int TXv, int TYv>
__device__ TileIdx tile_of(const CompGrid& cg, int t) {
    const int tr = t % cg.tiles_r;
    t /= cg.tiles_r;
    const int tt = t % cg.tiles_t;
    const int ch = t / cg.tiles_t;
    TileIdx ti;
    ti.comp = 0;
    ti.i0 = tr * TXv;
    ti.j0 = tt * TYv;
    ti.k0 = ch * cg.kchunk;
    ti.k1 = min(ti.k0 + cg.kchunk, cg.np);
    return ti;
}

union BatchSmem {
    TileSmem<PolF32CG, 32, 8> a;
    TileSmem<PolF32CG, 16, 16> b;
};

// dynamic shared memory of a batch block: the register tiles or the largest TMA ring (+ alignment)
constexpr int kBatchSmem = (int)sizeof(BatchSmem) > BatchTma3::TOTAL + 128 ? (int)sizeof(BatchSmem) : BatchTma3::TOTAL + 128;

// Array index a (0 u, 1 y0, 2..4 buf[0..2]) of the maps
__device__ __forceinline__ TmaRefs batch_refs(const CUtensorMap* M, int field, int c0, int c1, int c2) {
    return TmaRefs{{M + kMapField + field, nullptr, nullptr},
                   M + kMapCoef,
                   {c0 >= 0 ? M + kMapCen + c0 : nullptr, c1 >= 0 ? M + kMapCen + c1 : nullptr,
                    c2 >= 0 ? M + kMapCen + c2 : nullptr}};
}

// One work item through the TMA ring (32 x 8 tiles); the same epilogues as run_item, on the
// one-problem kernel's policy, so a problem's stages equal its one-problem TMA launches bit for
// bit.  Returns false when a copy never landed.
__device__ bool run_item_tma(const BatchProblem& pr, int L, int t, const LevelCoef* lc, unsigned char* smem, int tid,
                             int* err) {
    using P = PolF32;
    const TileIdx ti = tile_of<32, 8>(pr.cg, t);
    const bool last = L == pr.s;
    const CUtensorMap* M = pr.maps;
    const PlainField<P> fld{};
    if (L == 1) {
        EpiF<P, false, false> ep{pr.y0, nullptr, 0.f, nullptr, nullptr};
        ep.init();
        return tma_march_tile<P>(pr.cg, ti, batch_refs(M, 0, -1, -1, -1), ep, fld, err, smem, tid);
    }
    if (L == 2) {
        const LevelCoef c = lc[pr.coef_off + 2];
        if (last) {
            EpiStage2<P, true> ep{pr.u, nullptr, pr.u, c.a, c.b, c.c, nullptr, c.al, c.bl, c.cl};
            return tma_march_tile<P>(pr.cg, ti, batch_refs(M, 1, 0, -1, -1), ep, fld, err, smem, tid);
        }
        EpiStage2<P, false> ep{nullptr, pr.buf[0], pr.buf[1], c.a, c.b, c.c, nullptr, c.al, c.bl, c.cl};
        return tma_march_tile<P>(pr.cg, ti, batch_refs(M, 1, -1, -1, -1), ep, fld, err, smem, tid);
    }
    const LevelCoef c = lc[pr.coef_off + L];
    const int bm1 = (L - 2) % 3, bm2 = (L - 3) % 3;        // buffers of d_{L-1}, d_{L-2}
    if (last) {
        EpiStage<P, true, true> ep{pr.buf[bm2], pr.y0, pr.u, pr.u, c.a, c.b, c.c, c.d, nullptr, c.al, c.bl, c.cl, c.dl};
        return tma_march_tile<P>(pr.cg, ti, batch_refs(M, 2 + bm1, 1, 2 + bm2, 0), ep, fld, err, smem, tid);
    }
    EpiStage<P, true, false> ep{pr.buf[bm2], pr.y0, nullptr, pr.buf[(L - 1) % 3], c.a, c.b, c.c, c.d, nullptr, c.al, c.bl,
                                c.cl, c.dl};
    return tma_march_tile<P>(pr.cg, ti, batch_refs(M, 2 + bm1, 1, 2 + bm2, -1), ep, fld, err, smem, tid);
}

template <int TXv, int TYv>
__device__ void run_item(const BatchProblem& pr, int L, int t, const LevelCoef* lc, TileSmem<PolF32CG, TXv, TYv>& sm,
                         int tid) {
    using P = PolF32CG;
    const TileIdx ti = tile_of<TXv, TYv>(pr.cg, t);
    const bool last = L == pr.s;
    if (L == 1) {
        EpiF<P, false, false> ep{pr.y0, nullptr, 0.f, nullptr, nullptr};
        ep.init();
        tc_tile<P, TXv, TYv>(pr.cg, ti, pr.coef, LoadState<P>{pr.u}, ep, tid, sm);
    } else if (L == 2) {
        const LevelCoef c = lc[pr.coef_off + 2];
        if (last) {
            EpiStage2<P, true> ep{pr.u, nullptr, pr.u, c.a, c.b, c.c, nullptr, c.al, c.bl, c.cl};
            tc_tile<P, TXv, TYv>(pr.cg, ti, pr.coef, LoadState<P>{pr.y0}, ep, tid, sm);
        } else {
            EpiStage2<P, false> ep{nullptr, pr.buf[0], pr.buf[1], c.a, c.b, c.c, nullptr, c.al, c.bl, c.cl};
            tc_tile<P, TXv, TYv>(pr.cg, ti, pr.coef, LoadState<P>{pr.y0}, ep, tid, sm);
        }
    } else {
        const LevelCoef c = lc[pr.coef_off + L];
        const float* dkm1 = pr.buf[(L - 2) % 3];
        const float* dkm2 = pr.buf[(L - 3) % 3];
        if (last) {
            EpiStage<P, true, true> ep{dkm2, pr.y0, pr.u, pr.u, c.a, c.b, c.c, c.d, nullptr, c.al, c.bl, c.cl, c.dl};
            tc_tile<P, TXv, TYv>(pr.cg, ti, pr.coef, LoadState<P>{dkm1}, ep, tid, sm);
        } else {
            EpiStage<P, true, false> ep{dkm2, pr.y0, nullptr, pr.buf[(L - 1) % 3], c.a, c.b, c.c, c.d, nullptr, c.al, c.bl,
                                        c.cl, c.dl};
            tc_tile<P, TXv, TYv>(pr.cg, ti, pr.coef, LoadState<P>{dkm1}, ep, tid, sm);
        }
    }
}

// 5 resident blocks per SM (48 registers; the spills are in the item dispatch, outside the
// per-plane loop): one kernel carries every epilogue, and without the cap it takes 80 registers
// and only 3 blocks fit on an SM
__global__ void __launch_bounds__(NTHREADS, 5)
batch_kernel(const BatchProblem* __restrict__ probs, const BatchSeg* __restrict__ segs, int nsegs, long long total,
             const LevelCoef* __restrict__ lc, unsigned long long* next, int* err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    BatchSmem& sm = *reinterpret_cast<BatchSmem*>(smem);
    __shared__ long long item;
    __shared__ int stop;
    const int tid = threadIdx.x;
    for (;;) {
        __syncthreads();
        if (tid == 0) {
            item = (long long)atomicAdd(next, 1ull);
            stop = 0;
        }
        __syncthreads();
        const long long it = item;
        if (it >= total) return;
        // the segment holding item `it` (segments are sorted by begin)
        int lo = 0, hi = nsegs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (segs[mid].begin <= it) lo = mid; else hi = mid - 1;
        }
        const BatchSeg sg = segs[lo];
        const BatchProblem& pr = probs[sg.p];
        const int L = sg.level;
        if (L >= 2 && tid == 0) {
            unsigned spins = 0;
            while (atomicAdd(&pr.done[L - 1], 0u) < (unsigned)pr.tiles) {
                if (++spins > kSpinLimit || *((volatile int*)err)) {
                    atomicExch(err, 1);
                    stop = 1;
                    break;
                }
                __nanosleep(64);
            }
            __threadfence();
        }
        // the TMA reads of this item (issued by thread 0) come after what it acquired above
        if (tid == 0 && pr.maps) fence_proxy_async_global();
        __syncthreads();
        if (stop) return;
        const int t = (int)(it - sg.begin);
        if (pr.maps) {
            if (!run_item_tma(pr, L, t, lc, smem, tid, err)) return;
        } else if (pr.variant == 0) {
            run_item<32, 8>(pr, L, t, lc, sm.a, tid);
        } else {
            run_item<16, 16>(pr, L, t, lc, sm.b, tid);
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            fence_proxy_async_global();
            atomicAdd(&pr.done[L], 1u);
        }
    }
}

template <typename T>
void grow(T*& d, size_t& cap, size_t need) {
    if (need <= cap) return;
    if (d) cudaFree(d);
    d = nullptr;
    cap = 0;
    void* p = nullptr;
    if (cudaMalloc(&p, need * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        throw Error{PB_ENOMEM, "batch table allocation failed"};
    }
    d = static_cast<T*>(p);
    cap = need;
}

template <typename T>
void grow_host(T*& h, size_t& cap, size_t need) {
    if (need <= cap) return;
    if (h) cudaFreeHost(h);
    h = nullptr;
    cap = 0;
    void* p = nullptr;
    if (cudaMallocHost(&p, need * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        throw Error{PB_ENOMEM, "pinned batch table allocation failed"};
    }
    h = static_cast<T*>(p);
    cap = need;
}

}  // namespace
}  // namespace pb

using namespace pb;

struct pb_batch {
    std::vector<pb_ctx*> ctxs;
    pb_tune tune{};
    cudaStream_t stream = nullptr;        // the batch's own stream (capturable)
    cudaStream_t user = nullptr;          // the contexts' stream
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int sm_count = 0;
    // device tables
    BatchProblem* d_probs = nullptr; size_t cap_probs = 0;
    BatchSeg* d_segs = nullptr; size_t cap_segs = 0;
    LevelCoef* d_lc = nullptr; size_t cap_lc = 0;
    CUtensorMap* d_maps = nullptr; size_t cap_maps = 0;
    unsigned int* d_done = nullptr; size_t cap_done = 0;
    unsigned long long* d_next = nullptr;
    int* d_err = nullptr;
    // pinned mirrors
    BatchProblem* h_probs = nullptr; size_t hcap_probs = 0;
    BatchSeg* h_segs = nullptr; size_t hcap_segs = 0;
    LevelCoef* h_lc = nullptr; size_t hcap_lc = 0;
    CUtensorMap* h_maps = nullptr; size_t hcap_maps = 0;
    int* h_err = nullptr;
    // the captured launch and the structure it was captured for
    cudaGraphExec_t exec = nullptr;
    std::vector<long long> key;
    long long launches = 0;
    std::string err;
};

namespace {

thread_local std::string g_batch_error;

void free_batch(pb_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->stream) cudaStreamDestroy(b->stream);
    void* d[] = {b->d_probs, b->d_segs, b->d_lc, b->d_done, b->d_next, b->d_err, b->d_maps};
    for (void* p : d)
        if (p) cudaFree(p);
    void* h[] = {b->h_probs, b->h_segs, b->h_lc, b->h_err, b->h_maps};
    for (void* p : h)
        if (p) cudaFreeHost(p);
}

template <class F>
int bguard(pb_batch* b, F&& f) {
    try {
        f();
        if (b) b->err.clear();
        return PB_OK;
    } catch (const Error& e) {
        if (b) b->err = e.msg; else g_batch_error = e.msg;
        return e.code;
    } catch (const std::bad_alloc&) {
        if (b) b->err = "host allocation failed"; else g_batch_error = "host allocation failed";
        return PB_ENOMEM;
    }
}

// Builds the tables for one advance call; returns the structure key (sizes, stages, tiling).
std::vector<long long> build_tables(pb_batch* b, void* const* u, const double* dts, int scheme,
                                    long long& total, int& nsegs, std::vector<int>& stages) {
    const int n = (int)b->ctxs.size();
    std::vector<BatchProblem> probs(n);
    stages.assign(n, 0);
    size_t lc_total = 0, done_total = 0;
    int max_s = 0;
    std::vector<double> r_of(n);
    for (int p = 0; p < n; ++p) {
        const Ctx& c = b->ctxs[p]->c;
        const double r = dts[p] / c.dt_e;
        r_of[p] = r;
        if (!(dts[p] >= 0.0) || std::isinf(dts[p]) || !(r >= 0.0) || std::isinf(r) || r > 1e11)
            throw Error{PB_EINVAL, "dt must be finite, >= 0 and below 1e11 dt_E"};
        const long long s = scheme == PB_RKG2 ? stages_rkg2(r) : stages_rkl2(r);
        if (s > kMaxStages) throw Error{PB_EINVAL, "stage count above 2^20"};
        stages[p] = (int)s;
        max_s = std::max(max_s, stages[p]);
        lc_total += stages[p] + 1;
        done_total += stages[p] + 1;
    }
    grow(b->d_lc, b->cap_lc, lc_total);
    grow_host(b->h_lc, b->hcap_lc, lc_total);
    grow(b->d_maps, b->cap_maps, (size_t)n * kMaps);
    grow_host(b->h_maps, b->hcap_maps, (size_t)n * kMaps);
    grow(b->d_done, b->cap_done, done_total);
    std::vector<long long> key;
    key.push_back(b->tune.kchunk);
    key.push_back(b->tune.blocks_per_sm);
    key.push_back(b->tune.small_tiles);
    size_t lc_off = 0, done_off = 0;
    for (int p = 0; p < n; ++p) {
        const Ctx& c = b->ctxs[p]->c;
        BatchProblem& pr = probs[p];
        const int variant = (b->tune.small_tiles && c.nr <= 16) ? 1 : 0;
        const int txv = variant ? 16 : 32, tyv = variant ? 16 : 8;
        pr.cg = CompGrid{};
        pr.cg.nr = c.nr; pr.cg.nt = c.nt; pr.cg.np = c.np;
        pr.cg.tiles_r = (c.nr + txv - 1) / txv;
        pr.cg.tiles_t = (c.nt + tyv - 1) / tyv;
        pr.cg.kchunk = std::max(1, std::min(b->tune.kchunk, c.np));
        pr.cg.nchunk = (c.np + pr.cg.kchunk - 1) / pr.cg.kchunk;
        pr.cg.offset = 0;
        pr.coef = static_cast<const Coef4<float>*>(c.coef);
        pr.u = static_cast<float*>(u[p]);
        pr.y0 = static_cast<float*>(c.y0);
        for (int a = 0; a < 3; ++a) pr.buf[a] = static_cast<float*>(c.buf[a]);
        pr.done = b->d_done + done_off;
        pr.s = stages[p];
        pr.tiles = pr.cg.tiles_r * pr.cg.tiles_t * pr.cg.nchunk;
        pr.variant = variant;
        pr.coef_off = (int)lc_off;
        // the TMA ring for the 32 x 8 tiles when every array can be described by a tensor map
        pr.maps = nullptr;
        if (variant == 0 && c.use_tma) {
            CUtensorMap* hm = b->h_maps + (size_t)p * kMaps;
            const void* arr[5] = {pr.u, pr.y0, pr.buf[0], pr.buf[1], pr.buf[2]};
            bool ok = tma_coef_map(&hm[kMapCoef], pr.coef, 4, c.nr, c.nt, c.np, BatchTma3::CBX, TY + 1);
            for (int a = 0; ok && a < 5; ++a)
                ok = tma_state_map(&hm[kMapField + a], arr[a], 4, c.nr, c.nt, c.np, BatchTma3::BXW, TY + 2) &&
                     tma_state_map(&hm[kMapCen + a], arr[a], 4, c.nr, c.nt, c.np, TX, TY);
            if (ok) pr.maps = b->d_maps + (size_t)p * kMaps;
        }
        Sts co;
        make_sts(scheme, r_of[p], co);
        const std::vector<double>&mu = co.mu, &nu = co.nu, &mut = co.mut, &gt = co.gt;
        const double dt = dts[p];
        const double a1 = mut[1] * dt;
        LevelCoef* L = b->h_lc + lc_off;
        L[0] = L[1] = level_coef(0, 0, 0, 0);
        const double ydt2 = (mut[2] + gt[2]) * dt;
        L[2] = level_coef(a1, mu[2] * a1 + ydt2, mut[2] * dt * a1, 0.0);
        for (int k = 3; k <= pr.s; ++k) L[k] = level_coef(mu[k], nu[k], mut[k] * dt, (mut[k] + gt[k]) * dt);
        lc_off += pr.s + 1;
        done_off += pr.s + 1;
        key.push_back(pr.s);
        key.push_back(pr.tiles);
    }
    // level-major item order
    std::vector<BatchSeg> segs;
    total = 0;
    for (int L = 1; L <= max_s; ++L)
        for (int p = 0; p < n; ++p)
            if (probs[p].s >= L) {
                segs.push_back(BatchSeg{total, p, L});
                total += probs[p].tiles;
            }
    nsegs = (int)segs.size();
    grow(b->d_probs, b->cap_probs, (size_t)n);
    grow_host(b->h_probs, b->hcap_probs, (size_t)n);
    grow(b->d_segs, b->cap_segs, segs.size());
    grow_host(b->h_segs, b->hcap_segs, segs.size());
    std::memcpy(b->h_probs, probs.data(), n * sizeof(BatchProblem));
    std::memcpy(b->h_segs, segs.data(), segs.size() * sizeof(BatchSeg));
    key.push_back((long long)done_total);
    // the captured copies read these buffers: a reallocation needs a new capture
    for (const void* ptr : {(const void*)b->h_probs, (const void*)b->h_segs, (const void*)b->h_lc, (const void*)b->d_probs,
                            (const void*)b->d_segs, (const void*)b->d_lc, (const void*)b->d_done,
                            (const void*)b->h_maps, (const void*)b->d_maps})
        key.push_back(reinterpret_cast<long long>(ptr));
    return key;
}

void launch(pb_batch* b, void* const* u, const double* dts, int scheme, std::vector<int>& stages) {
    long long total = 0;
    int nsegs = 0;
    std::vector<long long> key = build_tables(b, u, dts, scheme, total, nsegs, stages);
    const int n = (int)b->ctxs.size();
    size_t lc_total = 0, done_total = 0;
    for (int s : stages) { lc_total += s + 1; done_total += s + 1; }
    if (b->exec && key != b->key) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (!b->exec) {
        // once per process (a function-local static: thread-safe initialisation), before capture
        static const cudaError_t attr =
            cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kBatchSmem);
        PB_CUDA_TRY(attr);
        // capture: copy the tables, clear the counters, run the persistent kernel
        cudaGraph_t graph = nullptr;
        PB_CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        cudaMemcpyAsync(b->d_probs, b->h_probs, n * sizeof(BatchProblem), cudaMemcpyHostToDevice, b->stream);
        cudaMemcpyAsync(b->d_segs, b->h_segs, nsegs * sizeof(BatchSeg), cudaMemcpyHostToDevice, b->stream);
        cudaMemcpyAsync(b->d_lc, b->h_lc, lc_total * sizeof(LevelCoef), cudaMemcpyHostToDevice, b->stream);
        cudaMemcpyAsync(b->d_maps, b->h_maps, n * kMaps * sizeof(CUtensorMap), cudaMemcpyHostToDevice, b->stream);
        cudaMemsetAsync(b->d_done, 0, done_total * sizeof(unsigned int), b->stream);
        cudaMemsetAsync(b->d_next, 0, sizeof(unsigned long long), b->stream);
        const int grid = std::max(1, b->tune.blocks_per_sm) * b->sm_count;
        batch_kernel<<<grid, NTHREADS, kBatchSmem, b->stream>>>(b->d_probs, b->d_segs, nsegs, total, b->d_lc,
                                                                b->d_next, b->d_err);
        const cudaError_t le = cudaGetLastError();
        const cudaError_t ce = cudaStreamEndCapture(b->stream, &graph);
        if (le != cudaSuccess || ce != cudaSuccess)
            throw Error{PB_ECUDA, std::string("batch capture: ") + cudaGetErrorString(le != cudaSuccess ? le : ce)};
        const cudaError_t ie = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) throw Error{PB_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie)};
        b->key = key;
    }
    // order the launch after prior work on the contexts' stream, and that stream after it
    PB_CUDA_TRY(cudaEventRecord(b->ev_in, b->user));
    PB_CUDA_TRY(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
    PB_CUDA_TRY(cudaGraphLaunch(b->exec, b->stream));
    PB_CUDA_TRY(cudaEventRecord(b->ev_out, b->stream));
    PB_CUDA_TRY(cudaStreamWaitEvent(b->user, b->ev_out, 0));
    b->launches += 1;
}

void finish(pb_batch* b) {
    PB_CUDA_TRY(cudaMemcpyAsync(b->h_err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    PB_CUDA_TRY(cudaStreamSynchronize(b->stream));
    if (*b->h_err) {
        *b->h_err = 0;
        cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream);
        cudaStreamSynchronize(b->stream);
        throw Error{PB_ETIMEOUT, "a batched work item waited too long for its previous level"};
    }
}

}  // namespace

extern "C" {

void pb_tune_init(pb_tune* t) {
    if (!t) return;
    t->kchunk = 16;
    t->blocks_per_sm = 4;
    t->small_tiles = 1;
}

int pb_batch_create(pb_ctx* const* ctxs, int32_t n, const pb_tune* tune, pb_batch** out) {
    return bguard(nullptr, [&] {
        if (!ctxs || n <= 0 || !out) throw Error{PB_EINVAL, "need n > 0 contexts"};
        *out = nullptr;
        for (int p = 0; p < n; ++p) {
            if (!ctxs[p]) throw Error{PB_EINVAL, "null context"};
            const Ctx& c = ctxs[p]->c;
            if (c.kind != PB_TC_ANISO || c.prec != PB_FP32)
                throw Error{PB_ENOTSUP, "the batched launch takes float32 conduction contexts"};
            if (c.stream != ctxs[0]->c.stream) throw Error{PB_EINVAL, "contexts must share one stream"};
        }
        pb_batch* b = new pb_batch();
        try {
            b->ctxs.assign(ctxs, ctxs + n);
            pb_tune_init(&b->tune);
            if (tune) b->tune = *tune;
            if (b->tune.kchunk <= 0 || b->tune.blocks_per_sm <= 0) throw Error{PB_EINVAL, "bad tune"};
            b->user = ctxs[0]->c.stream;
            PB_CUDA_TRY(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
            PB_CUDA_TRY(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
            PB_CUDA_TRY(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
            b->sm_count = ctxs[0]->c.sm_count;
            PB_CUDA_TRY(cudaMalloc(&b->d_next, sizeof(unsigned long long)));
            PB_CUDA_TRY(cudaMalloc(&b->d_err, sizeof(int)));
            PB_CUDA_TRY(cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream));
            PB_CUDA_TRY(cudaMallocHost(&b->h_err, sizeof(int)));
            *b->h_err = 0;
        } catch (...) {
            free_batch(b);
            delete b;
            throw;
        }
        *out = b;
    });
}

int pb_batch_destroy(pb_batch* b) {
    if (!b) return PB_OK;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    delete b;
    return PB_OK;
}

const char* pb_batch_last_error(const pb_batch* b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

int pb_batch_rkl2_advance(pb_batch* b, void* const* u_devs, const double* dts, int32_t scheme, pb_stats* per_problem) {
    if (!b) return PB_EINVAL;
    return bguard(b, [&] {
        if (!u_devs || !dts) throw Error{PB_EINVAL, "null argument"};
        if (scheme != PB_RKL2 && scheme != PB_RKG2) throw Error{PB_EINVAL, "unknown scheme"};
        for (size_t p = 0; p < b->ctxs.size(); ++p)
            if (!u_devs[p]) throw Error{PB_EINVAL, "null state pointer"};
        std::vector<int> stages;
        launch(b, u_devs, dts, scheme, stages);
        finish(b);
        if (per_problem)
            for (size_t p = 0; p < b->ctxs.size(); ++p) {
                pb_stats& s = per_problem[p];
                const int cap = s.cycle_capacity;
                double* dc = s.dt_cycle;
                int32_t* wc = s.work_cycle;
                double* pc = s.dt_ptl_cycle;
                int64_t* kc = s.k_cycle;
                std::memset(&s, 0, sizeof(s));
                s.cycle_capacity = cap;
                s.dt_cycle = dc; s.work_cycle = wc; s.dt_ptl_cycle = pc; s.k_cycle = kc;
                s.cycles = 1;
                s.status_cycle = -1;
                s.total_stages = stages[p];
                s.dt_explicit = b->ctxs[p]->c.dt_e;
                s.last_dt_ptl = std::numeric_limits<double>::quiet_NaN();
                s.fmax = std::numeric_limits<double>::quiet_NaN();
                s.k_index = -1;
                s.final_rel_residual = std::numeric_limits<double>::quiet_NaN();
                if (cap > 0) {
                    if (dc) dc[0] = dts[p];
                    if (wc) wc[0] = stages[p];
                    if (pc) pc[0] = std::numeric_limits<double>::quiet_NaN();
                    if (kc) kc[0] = -1;
                }
            }
    });
}

int pb_autotune(pb_batch* b, void* const* u_devs, const double* dts, int32_t scheme, pb_tune* out, double* best_ms) {
    if (!b) return PB_EINVAL;
    return bguard(b, [&] {
        if (!u_devs || !dts || !out) throw Error{PB_EINVAL, "null argument"};
        const int n = (int)b->ctxs.size();
        // the candidates run on scratch copies so the caller's states are not advanced
        std::vector<void*> work(n, nullptr), save(n, nullptr);
        std::vector<size_t> bytes(n);
        struct Free {
            std::vector<void*>& a; std::vector<void*>& b;
            ~Free() { for (void* p : a) if (p) cudaFree(p); for (void* p : b) if (p) cudaFree(p); }
        } guard{work, save};
        PB_CUDA_TRY(cudaEventRecord(b->ev_in, b->user));
        PB_CUDA_TRY(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
        for (int p = 0; p < n; ++p) {
            bytes[p] = (size_t)b->ctxs[p]->c.n * sizeof(float);
            PB_CUDA_TRY(cudaMalloc(&work[p], bytes[p]));
            PB_CUDA_TRY(cudaMalloc(&save[p], bytes[p]));
            PB_CUDA_TRY(cudaMemcpyAsync(save[p], u_devs[p], bytes[p], cudaMemcpyDeviceToDevice, b->stream));
        }
        cudaEvent_t e0, e1;
        PB_CUDA_TRY(cudaEventCreate(&e0));
        PB_CUDA_TRY(cudaEventCreate(&e1));
        const pb_tune keep = b->tune;
        pb_tune best = keep;
        double best_t = 1e300;
        const int kchunks[] = {4, 8, 16, 32, 64};
        const int bpsm[] = {2, 4, 6, 8};
        try {
            for (int small = 0; small <= 1; ++small)
                for (int kc : kchunks)
                    for (int bp : bpsm) {
                        b->tune = pb_tune{kc, bp, small};
                        std::vector<int> stages;
                        double t = 0.0;
                        for (int rep = 0; rep < 3; ++rep) {
                            for (int p = 0; p < n; ++p)
                                PB_CUDA_TRY(cudaMemcpyAsync(work[p], save[p], bytes[p], cudaMemcpyDeviceToDevice, b->stream));
                            PB_CUDA_TRY(cudaEventRecord(e0, b->stream));
                            launch(b, work.data(), dts, scheme, stages);
                            PB_CUDA_TRY(cudaEventRecord(e1, b->stream));
                            finish(b);
                            float ms = 0.f;
                            PB_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
                            if (rep > 0) t += ms;   // the first repetition captures the graph
                        }
                        t /= 2.0;
                        if (t < best_t) { best_t = t; best = b->tune; }
                    }
        } catch (...) {
            b->tune = keep;
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            throw;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        b->tune = best;
        if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
        *out = best;
        if (best_ms) *best_ms = best_t;
    });
}

}  // extern "C"
