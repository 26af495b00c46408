// pb_ptl_noalloc: the PTL evaluation (F = L u, argmax |F|, Eq. 5) for callers that cannot
// allocate device memory.  It needs no context: the caller passes the operator's packed
// coefficient records, the state and the output array for F.  The only scratch -- the per-block
// arg-max partials, the non-finite flag and the result record -- lives in one file-scope device
// array of fixed size, shared by every call on a device.
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "epilogues.cuh"
#include "march.cuh"

namespace pb {
namespace {

constexpr size_t kScratchBytes = 1u << 20;           // 1 MiB per device that loads the library
constexpr size_t kResultOff = 0;                      // PtlResult (48 bytes)
constexpr size_t kFlagOff = 64;                       // non-finite flag (int)
constexpr size_t kPartOff = 256;                      // ArgMax partials (16 bytes per block)
constexpr int kMaxBlocks = (int)((kScratchBytes - kPartOff) / sizeof(ArgMax));
constexpr int kMaxDevices = 64;
static_assert(sizeof(PtlResult) <= kFlagOff - kResultOff, "the result record overlaps the flag");

static __device__ __align__(256) unsigned char g_ptl_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};   // id of the context the address belongs to

PFN_cuCtxGetCurrent_v4000 g_ctx_current = nullptr;
PFN_cuCtxGetId_v12000 g_ctx_id = nullptr;
std::once_flag g_once;

void resolve_driver() {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuCtxGetCurrent", &fn, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        g_ctx_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(fn);
    fn = nullptr;
    if (cudaGetDriverEntryPoint("cuCtxGetId", &fn, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        g_ctx_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(fn);
    cudaGetLastError();
}

// Unique id of the current context (0 if unknown): a device reset tears the primary context
// down, the library's module is loaded again in the new one and the array may move.
unsigned long long current_ctx_id() {
    std::call_once(g_once, resolve_driver);
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!g_ctx_current || !g_ctx_id || g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx || g_ctx_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of the scratch array on the current device, looked up on the first call in a
// context (the symbol's host-side name is only a stand-in and must never be handed to a kernel).
int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return PB_ECUDA;
    }
    const unsigned long long ctx = current_ctx_id();
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev] || ctx == 0 || g_scratch_ctx[dev] != ctx) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_ptl_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return PB_ECUDA;
        }
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = current_ctx_id();   // the lookup made the device's context current
    }
    *out = g_scratch_addr[dev];
    return PB_OK;
}

// The same tile decomposition as a context's, capped so the partials fit the scratch array.
bool make_grid(int kind, int nr, int nt, int np, int sm_count, MarchGrid& g, long long& n) {
    g = MarchGrid{};
    g.ncomp = kind == PB_TC_ANISO ? 1 : 3;
    int dims[3][3];
    if (kind == PB_TC_ANISO) {
        dims[0][0] = nr; dims[0][1] = nt; dims[0][2] = np;
    } else {
        dims[0][0] = nr - 1; dims[0][1] = nt; dims[0][2] = np;
        dims[1][0] = nr; dims[1][1] = nt - 1; dims[1][2] = np;
        dims[2][0] = nr; dims[2][1] = nt; dims[2][2] = np;
    }
    long long tiles = 0;
    for (int a = 0; a < g.ncomp; ++a)
        tiles += (long long)((dims[a][0] + TX - 1) / TX) * ((dims[a][1] + TY - 1) / TY);
    if (tiles > kMaxBlocks) return false;
    const long long target = (long long)sm_count * 16;
    long long nchunk = std::max(1LL, (target + tiles - 1) / tiles);
    nchunk = std::min(nchunk, (long long)std::max(1, np / 4));
    nchunk = std::min(nchunk, (long long)kMaxBlocks / tiles);
    const int kchunk = (int)((np + nchunk - 1) / nchunk);
    const int nch = (np + kchunk - 1) / kchunk;
    long long off = 0;
    int blocks = 0;
    for (int a = 0; a < g.ncomp; ++a) {
        CompGrid& c = g.c[a];
        c.nr = dims[a][0]; c.nt = dims[a][1]; c.np = dims[a][2];
        c.tiles_r = (c.nr + TX - 1) / TX;
        c.tiles_t = (c.nt + TY - 1) / TY;
        c.kchunk = kchunk;
        c.nchunk = nch;
        c.offset = off;
        c.block_begin = blocks;
        off += (long long)c.nr * c.nt * c.np;
        blocks += c.tiles_r * c.tiles_t * nch;
    }
    g.nblocks = blocks;
    n = off;
    return blocks <= kMaxBlocks;
}

// P: the policy (records P::C, F written as P::S); the state is read as the caller's type P::U
template <class P>
int run(const MarchGrid& g, int kind, const void* rec, const void* u, void* F, unsigned char* scratch,
        cudaStream_t s) {
    using S = typename P::S;
    using C = typename P::C;
    using U = typename P::U;
    using Ld = LoadStateT<P, U>;
    ArgMax* part = reinterpret_cast<ArgMax*>(scratch + kPartOff);
    int* flag = reinterpret_cast<int*>(scratch + kFlagOff);
    PtlResult* res = reinterpret_cast<PtlResult*>(scratch + kResultOff);
    // the flag is the only scratch word that must start at zero; the partials and the result
    // are written in full by every call
    if (cudaMemsetAsync(flag, 0, sizeof(int), s) != cudaSuccess) return PB_ECUDA;
    EpiF<P, true, false> ep{static_cast<S*>(F), nullptr, typename P::A(0), part, flag};
    const Ld ld{static_cast<const U*>(u)};
    const Coef4<C>* cf = static_cast<const Coef4<C>*>(rec);
    if (kind == PB_TC_ANISO)
        tc_march<P, Ld, EpiF<P, true, false>><<<g.nblocks, dim3(TX, TY), 0, s>>>(g, cf, ld, ep);
    else
        visc_march<P, Ld, EpiF<P, true, false>><<<g.nblocks, dim3(TX, TY), 0, s>>>(g, cf, ld, ep);
    ptl_finalize_kernel<P, U><<<1, kFinalizeThreads, 0, s>>>(g, static_cast<const U*>(u), static_cast<const S*>(F), part,
                                               g.nblocks, res, flag);
    return cudaGetLastError() == cudaSuccess ? PB_OK : PB_ECUDA;
}

}  // namespace
}  // namespace pb

using namespace pb;

extern "C" PB_API int pb_ptl_noalloc(int32_t kind, int32_t n_r, int32_t n_theta, int32_t n_phi,
                                     int32_t precision, const void* records, const void* u, void* F,
                                     double* dt_ptl, int64_t* k_index, double* fmax, void* stream) {
    if ((kind != PB_TC_ANISO && kind != PB_VISC_ISO) || n_r < 2 || n_theta < 2 || n_phi < 3)
        return PB_EINVAL;
    if (precision != PB_FP64 && precision != PB_FP32 && precision != PB_BF16_STORE) return PB_EINVAL;
    if (!records || !u || !F || u == F) return PB_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return PB_ECUDA;
    }
    MarchGrid g;
    long long n = 0;
    if (!make_grid(kind, n_r, n_theta, n_phi, sms, g, n)) return PB_EINVAL;   // beyond the scratch size
    void* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != PB_OK) return rc;
    unsigned char* sp = static_cast<unsigned char*>(scratch);
    switch (precision) {
        case PB_FP64: rc = run<PolF64>(g, kind, records, u, F, sp, s); break;
        case PB_FP32: rc = run<PolF32>(g, kind, records, u, F, sp, s); break;
        default: rc = run<PolB16>(g, kind, records, u, F, sp, s); break;
    }
    if (rc != PB_OK) {
        cudaGetLastError();
        return rc;
    }
    PtlResult r;
    if (cudaMemcpyAsync(&r, sp + kResultOff, sizeof(r), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return PB_ECUDA;
    }
    if (r.nonfinite) return PB_ENONFINITE;
    if (dt_ptl) *dt_ptl = r.dt_ptl;
    if (k_index) *k_index = r.k;
    if (fmax) *fmax = r.fmax;
    return PB_OK;
}
