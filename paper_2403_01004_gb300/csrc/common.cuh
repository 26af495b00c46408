// Shared definitions of libparabolic's CUDA translation units: precision policies, the packed
// coefficient record, grid descriptors, reductions and the context.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/parabolic.h"
#include "prof.h"

namespace pb {

// ---- precision policies -----------------------------------------------------------------
// S: storage of the working state and the stage values (y0, the stage increments); C: coefficient
// records; A: stencil arithmetic; E: the stage recurrence (the update of the stored stage values
// from A-precision F); U: the caller's state arrays (S, or bfloat16 held in a float32 working
// copy during a call).  DF: the float32 stage recurrence runs in double-float arithmetic (see
// DfAcc), so the only rounding a stage adds is the store of its result.
// CG: operands may have been written earlier in the same launch (the batched persistent kernel),
// so they are read through L2 (ld.global.cg) instead of the non-coherent read-only path.
struct PolF64 { using S = double; using C = double; using A = double; using E = double; using U = double;
                static constexpr int id = PB_FP64; static constexpr bool CG = false; static constexpr bool DF = false; };
struct PolF32 { using S = float; using C = float; using A = float; using E = float; using U = float;
                static constexpr int id = PB_FP32; static constexpr bool CG = false; static constexpr bool DF = true; };
// bfloat16 storage with float32 accumulation: the operator records (the largest stream of every
// pass) and the caller's state are bfloat16; the stage values and the state between the cycles
// of a call are float32, where rounding would otherwise accumulate over the stages
struct PolB16 { using S = float; using C = __nv_bfloat16; using A = float; using E = float; using U = __nv_bfloat16;
                static constexpr int id = PB_BF16_STORE; static constexpr bool CG = false; static constexpr bool DF = true; };
// float64 storage and recurrence, float32 records and stencil (GB300: float64 arithmetic is
// scarce, bandwidth is not; the stage recurrence is where storage rounding accumulates)
struct PolF64S { using S = double; using C = float; using A = float; using E = double; using U = double;
                 static constexpr int id = PB_FP64_STORE; static constexpr bool CG = false; static constexpr bool DF = false; };
struct PolF32CG : PolF32 { static constexpr bool CG = true; };

template <typename T> __host__ __device__ __forceinline__ float to_f(T v);
template <> __host__ __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <typename A, typename T> __device__ __forceinline__ A cvt(T v) { return (A)v; }
template <> __device__ __forceinline__ float cvt<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ double cvt<double, __nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
template <> __device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16, float>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16, double>(double v) { return __float2bfloat16_rn((float)v); }

// Read-only load of a state element through the non-coherent path.
template <typename T> __device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }
template <> __device__ __forceinline__ __nv_bfloat16 ldg<__nv_bfloat16>(const __nv_bfloat16* p) {
    unsigned short s = __ldg(reinterpret_cast<const unsigned short*>(p));
    return __ushort_as_bfloat16(s);
}

template <typename T> __device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }
template <> __device__ __forceinline__ __nv_bfloat16 ldcg<__nv_bfloat16>(const __nv_bfloat16* p) {
    unsigned short s = __ldcg(reinterpret_cast<const unsigned short*>(p));
    return __ushort_as_bfloat16(s);
}
// Load of a state operand under policy P (read-only path, or L2 for in-launch producers).
template <class P, typename T> __device__ __forceinline__ T ldx(const T* p) { return P::CG ? ldcg(p) : ldg(p); }

// Packed 4-word coefficient record stored at every grid point [i,j,k]:
//   conduction: {ahat_r, ahat_t, ahat_p} of corner [i,j,k] and the cell weight w of cell [i,j,k]
//   viscosity : {c_r, c_t, c_p} of the +1 faces of point [i,j,k] and its weight w
template <typename T> struct alignas(4 * sizeof(T)) Coef4 { T a, b, c, w; };

template <typename A, typename T> __device__ __forceinline__ Coef4<A> load_coef(const Coef4<T>* p);
template <> __device__ __forceinline__ Coef4<double> load_coef<double, double>(const Coef4<double>* p) {
    const double2* q = reinterpret_cast<const double2*>(p);
    double2 x = __ldg(q), y = __ldg(q + 1);
    return Coef4<double>{x.x, x.y, y.x, y.y};
}
template <> __device__ __forceinline__ Coef4<float> load_coef<float, float>(const Coef4<float>* p) {
    float4 x = __ldg(reinterpret_cast<const float4*>(p));
    return Coef4<float>{x.x, x.y, x.z, x.w};
}
// bfloat16 record: one 8-byte load; a bfloat16 is the upper half of the float with the same value
template <> __device__ __forceinline__ Coef4<float> load_coef<float, __nv_bfloat16>(const Coef4<__nv_bfloat16>* p) {
    const uint2 x = __ldg(reinterpret_cast<const uint2*>(p));
    return Coef4<float>{__uint_as_float(x.x << 16), __uint_as_float(x.x & 0xffff0000u), __uint_as_float(x.y << 16),
                        __uint_as_float(x.y & 0xffff0000u)};
}
// One word of a record (a neighbour's face coefficient)
template <typename A, typename C> __device__ __forceinline__ A coef_word(const C* p) { return cvt<A>(ldg(p)); }

// float64 set-up value into the record precision (one rounding)
template <typename C> __device__ __forceinline__ C to_rec(double v) { return (C)v; }
template <> __device__ __forceinline__ __nv_bfloat16 to_rec<__nv_bfloat16>(double v) { return __double2bfloat16(v); }

// ---- grid descriptors ----------------------------------------------------------------------
// Stencil tiles: TX cells along r (a full warp, coalesced) x TY cells along theta; each block
// marches through a chunk of consecutive phi planes.
constexpr int TX = 32;
constexpr int TY = 8;
constexpr int NTHREADS = TX * TY;

struct CompGrid {          // one scalar field (a conduction state or one velocity component)
    int nr, nt, np;
    int tiles_r, tiles_t, kchunk, nchunk;
    int64_t offset;        // element offset of this component in the state / coefficient arrays
    int block_begin;       // first block index of this component in a march launch
    int periodic;          // r and theta wrap as phi does (the periodic box)
};

struct MarchGrid {
    int ncomp;
    CompGrid c[3];
    int nblocks;
};

// ---- device-side scalar state ----------------------------------------------------------------
struct ArgMax { double v; long long i; };

struct PtlResult {
    double dt_ptl;         // Eq. 5 at k = argmax |F|
    double fmax;
    long long k;
    int nonfinite;
    int pad;
    double dt_full;        // Eq. 4 over every pair of face neighbours (NaN when not evaluated)
    long long key_full;    // its pair (i, i + e_d) as 3 i + d, -1 when none qualifies
};

struct PcgScalars {
    double rz, rr, bb, pq, alpha, beta, tol2;
    long long iter, max_iter, fixed;
    int done;       // 1 converged / finished, 2 breakdown or non-finite, 3 iteration cap
    int first;
    double dt;
};

// ---- context ------------------------------------------------------------------------------
struct Ctx {
    int kind = 0, prec = 0;
    int elem = 8;
    cudaStream_t stream = nullptr;
    int nr = 0, nt = 0, np = 0;
    int geometry = 0;              // pb_geometry
    MarchGrid grid{};
    int64_t n = 0;                 // state length
    double dt_e = 0.0;
    // device workspace
    void* coef = nullptr;          // Coef4<C>[n], 4th word w (super time stepping, apply, PTL)
    void* coef_be = nullptr;       // Coef4<C>[n], 4th word M = 1/w (Backward Euler system)
    Coef4<double>* coef64 = nullptr;  // float64 record (kept for refinement / diagnostics)
    void* adiag = nullptr;         // diag(A) in C precision [n]
    int welem = 8;                 // element size of the working state and stage values (sizeof S)
    void* y0 = nullptr;            // working-precision scratch [n]
    void* buf[3] = {nullptr, nullptr, nullptr};
    void* work = nullptr;          // float32 working state of a bfloat16-storage context [n]
    // PCG vectors (S precision)
    void* r = nullptr; void* p[2] = {nullptr, nullptr}; void* q = nullptr; void* dinv = nullptr;
    // reductions
    void* partials = nullptr;      // max(nblocks, reduce blocks) * 32 bytes
    int partial_cap = 0;
    unsigned int* counter = nullptr;
    PtlResult* d_ptl = nullptr;
    PcgScalars* d_pcg = nullptr;
    double* d_scalar = nullptr;    // misc scalar (dt_E)
    int* d_flag = nullptr;         // non-finite flag
    int* d_err = nullptr;          // set by a kernel whose bounded wait ran out
    int* h_err = nullptr;          // pinned mirror
    bool use_tma = true;
    // pinned host mirrors
    PtlResult* h_ptl = nullptr;
    PcgScalars* h_pcg = nullptr;
    double* h_scalar = nullptr;
    // persistent set-up workspace (coefficient updates allocate nothing)
    double* s64 = nullptr;         // float64 scratch [n]: kappa, then diag(A)
    double* arow = nullptr;        // sum_j |A_ij| per row (float64) [n]: the Chebyshev bound
    void* cheb[3] = {nullptr, nullptr, nullptr};   // Chebyshev preconditioner: z and the y ring
    double* geo[16] = {};          // device copies of the face / point coordinate arrays
    Prof prof;
    struct Ctx* shadow = nullptr;  // float32 shadow for mixed-precision BE (float64 contexts)
    void* spec = nullptr;          // second working-state buffer of speculated floor cycles [n]
    cudaEvent_t ev_ptl = nullptr;  // recorded after a PTL result's copy to the host
    std::string err;
    int sm_count = 0;
};

struct Error {
    int code;
    std::string msg;
};

}  // namespace pb

struct pb_ctx { pb::Ctx c; };

// Status helpers for host code.
#define PB_CUDA_TRY(expr)                                                                     \
    do {                                                                                      \
        cudaError_t e__ = (expr);                                                             \
        if (e__ != cudaSuccess)                                                               \
            throw pb::Error{PB_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e__)};   \
    } while (0)
