// Mixed-precision Backward Euler for float64 contexts: iterative refinement around float32 PCG.
//
// Outer loop (float64): r = b - S x from the current x (the float64 set-up kernel of PCG), stop
// when r.r <= rtol^2 b.b.  Inner solve (float32): S d = r by the same point-Jacobi PCG kernels on
// a float32 shadow of the context (records and vectors), from d = 0 to a relative residual
// inner_rtol; then x += d in float64.  Each refinement reduces the float64 residual by about
// inner_rtol, so a few refinements reach the float64 tolerance while the iterations run at
// float32 bandwidth and arithmetic.
#include <cmath>
#include <cstring>

#include "epilogues.cuh"
#include "launch.h"

namespace pb {
namespace {

// r32 = rhs, d = 0, D^-1 = 1/(M - dt diag A) and the sums <r, D^-1 r>, <r, r>, <rhs, rhs>;
// the last block initialises the scalar state of the inner solve.
__global__ void __launch_bounds__(256)
init_rhs_kernel(long long n, const double* rhs, const Coef4<float>* rec_be, const float* adiag, double dt, float* r,
                float* dinv, float* d, PcgScalars* sc, double* part, unsigned int* counter) {
    double acc[3] = {0.0, 0.0, 0.0};
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const float rs = (float)rhs[t];
        const float ds = 1.0f / (rec_be[t].w - (float)dt * adiag[t]);
        r[t] = rs;
        dinv[t] = ds;
        d[t] = 0.0f;
        const double z = (double)(ds * rs);
        acc[0] += (double)rs * z;
        acc[1] += (double)rs * (double)rs;
        acc[2] += rhs[t] * rhs[t];
    }
    block_sum<3>(acc);
    if (threadIdx.x == 0) {
        part[blockIdx.x * 4 + 0] = acc[0];
        part[blockIdx.x * 4 + 1] = acc[1];
        part[blockIdx.x * 4 + 2] = acc[2];
    }
    if (last_block(counter, gridDim.x)) {
        double v[3];
        sum_partials<3>(part, gridDim.x, 4, v);
        if (threadIdx.x == 0) {
            sc->rz = v[0];
            sc->rr = v[1];
            sc->bb = v[2];
            sc->iter = 0;
            sc->first = 1;
            sc->beta = 0.0;
            sc->alpha = 0.0;
            int done = 0;
            if (!(v[0] == v[0]) || !(v[1] == v[1])) done = 2;
            else if (v[1] <= sc->tol2 * v[2]) done = 1;
            sc->done = done;
            *counter = 0u;
        }
    }
}

__global__ void add_correction_kernel(long long n, double* x, const float* d) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        x[t] += (double)d[t];
}

void* dalloc(size_t bytes) {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        throw Error{PB_ENOMEM, "mixed-precision workspace allocation failed"};
    }
    return p;
}

}  // namespace

// Builds (once) the float32 shadow of a float64 context: records, diag(A), PCG vectors and the
// reduction state of the inner solves.
Ctx& mixed_shadow(Ctx& c) {
    if (c.shadow) return *c.shadow;
    Ctx* s = new Ctx();
    try {
        s->kind = c.kind;
        s->prec = PB_FP32;
        s->elem = 4;
        s->stream = c.stream;
        s->nr = c.nr; s->nt = c.nt; s->np = c.np;
        s->grid = c.grid;
        s->n = c.n;
        s->dt_e = c.dt_e;
        s->sm_count = c.sm_count;
        s->use_tma = c.use_tma;
        s->d_err = c.d_err;                          // shared: the parent's sync reports a timeout
        const size_t n = (size_t)c.n;
        s->coef = dalloc(n * sizeof(Coef4<float>));
        s->coef_be = dalloc(n * sizeof(Coef4<float>));
        s->adiag = dalloc(n * sizeof(float));
        s->r = dalloc(n * sizeof(float));
        s->p[0] = dalloc(n * sizeof(float));
        s->p[1] = dalloc(n * sizeof(float));
        s->q = dalloc(n * sizeof(float));
        s->dinv = dalloc(n * sizeof(float));
        s->y0 = dalloc(n * sizeof(float));           // the correction d
        s->partial_cap = c.partial_cap;
        s->partials = dalloc((size_t)c.partial_cap * 32);
        s->counter = static_cast<unsigned int*>(dalloc(sizeof(unsigned int)));
        s->d_pcg = static_cast<PcgScalars*>(dalloc(sizeof(PcgScalars)));
        PB_CUDA_TRY(cudaMemsetAsync(s->counter, 0, sizeof(unsigned int), c.stream));
        PB_CUDA_TRY(cudaMallocHost(&s->h_pcg, sizeof(PcgScalars)));
        // float32 copies of the float64 records (w and M = 1/w variants) and of diag(A)
        ops_f32()->store_coefs(*s, c.coef64, static_cast<const double*>(c.adiag));
        PB_CUDA_TRY(cudaStreamSynchronize(c.stream));
    } catch (...) {
        free_shadow(s);
        throw;
    }
    c.shadow = s;
    return *s;
}

void free_shadow(Ctx* s) {
    if (!s) return;
    void* p[] = {s->coef, s->coef_be, s->adiag, s->r, s->p[0], s->p[1], s->q, s->dinv, s->y0, s->partials,
                 s->counter, s->d_pcg};
    for (void* q : p)
        if (q) cudaFree(q);
    if (s->h_pcg) cudaFreeHost(s->h_pcg);
    s->prof.release();
    delete s;
}

// One refinement's inner solve: S d = r (c.r, float64) to relative residual inner_rtol with at
// most max_iter float32 PCG iterations, then x += d.  Returns the inner iterations; sets
// *status to 0 (ok), 2 (non-finite) or 3 (cap reached, which the outer loop tolerates).
long long mixed_inner(Ctx& c, void* x, double dt, double inner_rtol, long long max_iter, int check_every, int* status) {
    Ctx& s = mixed_shadow(c);
    PcgScalars& h = *s.h_pcg;
    std::memset(&h, 0, sizeof(h));
    h.tol2 = inner_rtol * inner_rtol;
    h.max_iter = max_iter;
    h.fixed = 0;
    h.dt = dt;
    PB_CUDA_TRY(cudaMemcpyAsync(s.d_pcg, &h, sizeof(h), cudaMemcpyHostToDevice, s.stream));
    const int blocks = reduce_blocks(s);
    s.prof.on = c.prof.on;
    {
    KScope ks(s.prof, s.stream, K_PCG32_REFINE, (double)s.n * (8 + 16 + 4 + 3 * 4));
    init_rhs_kernel<<<blocks, 256, 0, s.stream>>>(s.n, static_cast<const double*>(c.r),
                                                   static_cast<const Coef4<float>*>(s.coef_be),
                                                   static_cast<const float*>(s.adiag), dt, static_cast<float*>(s.r),
                                                   static_cast<float*>(s.dinv), static_cast<float*>(s.y0), s.d_pcg,
                                                   static_cast<double*>(s.partials), s.counter);
    PB_CUDA_TRY(cudaGetLastError());
    }
    int parity = 0;
    Ops* ops = ops_f32();
    for (;;) {
        PB_CUDA_TRY(cudaMemcpyAsync(s.h_pcg, s.d_pcg, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s.stream));
        PB_CUDA_TRY(cudaStreamSynchronize(s.stream));
        if (s.h_pcg->done) break;
        for (int m = 0; m < check_every; ++m) {
            ops->pcg_iter(s, s.y0, parity, dt);
            parity ^= 1;
        }
    }
    const PcgScalars r = *s.h_pcg;
    *status = r.done == 1 ? 0 : r.done;
    if (r.done != 2) {
        KScope ks(s.prof, s.stream, K_PCG32_REFINE, (double)s.n * (8 + 4 + 8));
        add_correction_kernel<<<reduce_blocks(c), 256, 0, c.stream>>>(c.n, static_cast<double*>(x),
                                                                      static_cast<const float*>(s.y0));
        PB_CUDA_TRY(cudaGetLastError());
    }
    PB_CUDA_TRY(cudaStreamSynchronize(s.stream));
    s.prof.harvest();
    c.prof.absorb(s.prof, K_PCG_SPMV, K_PCG32_SPMV);
    c.prof.absorb(s.prof, K_PCG_UPDATE, K_PCG32_UPDATE);
    c.prof.absorb(s.prof, K_PCG32_REFINE, K_PCG32_REFINE);
    return r.iter;
}

}  // namespace pb
