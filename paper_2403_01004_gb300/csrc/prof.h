// Per-kernel-class launch counting and (optional) CUDA-event timing on the context's stream,
// with the algorithmic bytes each launch must move.  Launch counts are always kept; timing is
// switched on by pb_profile_enable and harvested whenever the host synchronises.
#pragma once

#include <cuda_runtime.h>

#include <vector>

namespace pb {

enum KClass {
    K_APPLY = 0,      // F = L u
    K_PTL_PASS,       // y0 = L u with the PTL arg-max partials
    K_Y0_D1,          // y0 = L u fused with the stage-1 increment d1 = a y0
    K_PTL_FINAL,      // Eq. 5 at argmax |F|
    K_STAGE1,         // d1 = a y0
    K_STAGE,          // STS stage k >= 2
    K_PCG_INIT,
    K_PCG_SPMV,
    K_PCG_UPDATE,
    K_SETUP,
    K_PCG32_SPMV,     // float32 inner solves of mixed-precision Backward Euler
    K_PCG32_UPDATE,
    K_PCG32_REFINE,   // their right-hand-side set-up and the float64 correction x += d
    K_PTL_FULL,       // Eq. 4 over every pair of face neighbours
    K_PCG_CHEB,       // the Chebyshev preconditioner's stencil passes
    K_NCLASS
};

inline const char* kclass_name(int k) {
    static const char* names[K_NCLASS] = {"apply", "ptl_pass", "y0_stage1", "ptl_finalize", "stage1", "stage",
                                          "pcg_init", "pcg_spmv", "pcg_update", "setup",
                                          "pcg32_spmv", "pcg32_update", "pcg32_refine", "ptl_full", "pcg_cheb"};
    return names[k];
}

struct Prof {
    bool on = false;
    long long launches[K_NCLASS] = {};
    double ms[K_NCLASS] = {};
    double bytes[K_NCLASS] = {};
    long long timed[K_NCLASS] = {};
    struct Pending { int cls; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;

    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    // Accumulates the durations of completed launches (called after a stream synchronisation).
    void harvest() {
        for (const Pending& p : pending) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
                ms[p.cls] += t;
                timed[p.cls] += 1;
            } else {
                cudaGetLastError();
            }
            pool.push_back(p.a);
            pool.push_back(p.b);
        }
        pending.clear();
    }
    void reset() {
        for (int k = 0; k < K_NCLASS; ++k) { launches[k] = 0; ms[k] = 0.0; bytes[k] = 0.0; timed[k] = 0; }
    }
    // Moves the totals of class `from` of another (harvested) record into class `to` of this one.
    void absorb(Prof& o, int from, int to) {
        launches[to] += o.launches[from];
        ms[to] += o.ms[from];
        bytes[to] += o.bytes[from];
        timed[to] += o.timed[from];
        o.launches[from] = 0; o.ms[from] = 0.0; o.bytes[from] = 0.0; o.timed[from] = 0;
    }
    void release() {
        harvest();
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
        pool.clear();
    }
};

// RAII bracket around one launch of class `cls` moving `bytes` algorithmic bytes.
struct KScope {
    Prof& p;
    cudaStream_t s;
    int cls;
    cudaEvent_t b = nullptr;
    KScope(Prof& prof, cudaStream_t stream, int k, double bytes) : p(prof), s(stream), cls(k) {
        p.launches[k] += 1;
        p.bytes[k] += bytes;
        if (p.on) {
            cudaEvent_t a = p.get();
            b = p.get();
            cudaEventRecord(a, s);
            p.pending.push_back(Prof::Pending{k, a, b});
        }
    }
    ~KScope() {
        if (b) cudaEventRecord(b, s);
    }
};

}  // namespace pb
