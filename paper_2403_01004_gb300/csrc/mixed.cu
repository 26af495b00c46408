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

#include "dfloat.cuh"
#include "epilogues.cuh"
#include "launch.h"
#include "march.cuh"

namespace pb {


// float64 storage, double-float records and stencil arithmetic: the conduction residual of
// mixed-precision Backward Euler (the kernel templates of the march take it as a policy)
struct PolDF { using S = double; using C = dfloat; using A = dfloat; using E = double; using U = double;
               static constexpr int id = PB_FP64; static constexpr bool CG = false; static constexpr bool DF = false; };

// float64 -> double-float by integer operations on the bits (no float64 arithmetic, which GB300
// issues at a small fraction of its float32 rate): hi = the value rounded to the nearest float,
// lo = the remainder (an integer of at most 29 bits times 2^(e-52)) rounded to float, so hi + lo
// carries 48 significant bits.  Values outside 2^-70 <= |v| < 2^126 (and zero, non-finite) take
// the float64 route.
__device__ __forceinline__ dfloat split_double(double v) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((bits >> 52) & 0x7FF) - 1023;
    if (e < -70 || e > 125) {
        const float h = __double2float_rn(v);
        return dfloat(h, __double2float_rn(v - (double)h));
    }
    const unsigned long long m = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);   // 53-bit significand
    unsigned long long top = m >> 29;                                         // the leading 24 bits
    const long long rem = (long long)(m & ((1ull << 29) - 1));
    const bool up = rem > (1ll << 28) || (rem == (1ll << 28) && (top & 1ull));
    const long long r = up ? rem - (1ll << 29) : rem;                          // |r| <= 2^28
    top += up ? 1ull : 0ull;                                                  // 2^24 carries into the exponent
    const unsigned int sign = (unsigned int)(bits >> 63) << 31;
    const float hi = __uint_as_float(sign | (((unsigned int)(e + 127) << 23) + (unsigned int)(top - (1ull << 23))));
    const float scale = __uint_as_float((unsigned int)(e - 52 + 127) << 23);  // 2^(e-52)
    const float lo = __fmul_rn(__int2float_rn((int)(sign ? -r : r)), scale);   // |r| <= 2^28
    return dfloat(hi, lo);
}

// float64 -> float rounded to nearest (ties to even) by integer operations on the bits; results
// outside the normal float range (and zero, non-finite values) take the conversion instruction
__device__ __forceinline__ float narrow(double v) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((bits >> 52) & 0x7FF) - 1023;
    if (e < -126 || e > 126) return __double2float_rn(v);
    const unsigned long long m = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    unsigned long long top = m >> 29;
    const unsigned long long rem = m & ((1ull << 29) - 1);
    if (rem > (1ull << 28) || (rem == (1ull << 28) && (top & 1ull))) ++top;   // 2^24 carries into the exponent
    const unsigned int sign = (unsigned int)(bits >> 63) << 31;
    return __uint_as_float(sign | (((unsigned int)(e + 127) << 23) + (unsigned int)(top - (1ull << 23))));
}

// float -> float64 by integer operations on the bits (exact; zero, subnormal and non-finite
// values take the conversion instruction, which GB300 issues on its float64 pipes)
__device__ __forceinline__ double widen(float f) {
    const unsigned int b = __float_as_uint(f);
    const unsigned int ex = (b >> 23) & 0xFFu;
    if (ex == 0u || ex == 0xFFu) return (double)f;
    const unsigned long long w = ((unsigned long long)(b >> 31) << 63) | ((unsigned long long)(ex + 896u) << 52) |
                                 ((unsigned long long)(b & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)w);
}

template <> __device__ __forceinline__ dfloat cvt<dfloat, double>(double v) { return split_double(v); }
template <> __device__ __forceinline__ Coef4<dfloat> load_coef<dfloat, dfloat>(const Coef4<dfloat>* p) {
    const float4* q = reinterpret_cast<const float4*>(p);
    const float4 x = __ldg(q), y = __ldg(q + 1);
    return Coef4<dfloat>{dfloat(x.x, x.y), dfloat(x.z, x.w), dfloat(y.x, y.y), dfloat(y.z, y.w)};
}

namespace {

// r = b - S x = M (u^n - x) + dt A x for the outer test of mixed-precision BE, in double-float
// (x, u^n split by integer operations, A x from the double-float march), and the sums <r, r>,
// <b, b> over the leading floats (the stopping test needs a few digits of them, and a stop is
// confirmed on the float64 residual); the last block writes the outer scalar state (as the
// float64 set-up pass does, without D^-1 and <r, D^-1 r>, which the float32 inner solves form
// themselves).  r is stored as its leading float (the inner solve's right-hand side is float32).
struct EpiResidualDF {
    struct Pre { double un; };
    const double* un;
    double* r;
    dfloat dt;
    PcgScalars* sc;
    double* part;
    unsigned int* counter;
    int nblocks;
    DfAcc acc[2];      // <r, r> and <b, b> of this thread, in double-float on the float32 pipes
    __device__ void init() { acc[0] = DfAcc{0.f, 0.f}; acc[1] = DfAcc{0.f, 0.f}; }
    __device__ bool skip() const { return false; }
    __device__ Pre prefetch(long long idx) const { return Pre{__ldg(un + idx)}; }
    // x: the marched field at this point, split exactly as its halo copies are
    __device__ void apply(long long idx, dfloat Au, dfloat m, dfloat x, const Pre& p) {
        const dfloat und = split_double(p.un);
        const dfloat rv = m * (und - x) + dt * Au;
        r[idx] = widen(rv.hi);
        const dfloat b = m * und;
        acc[0].add(rv.hi, 0.f, rv.hi);
        acc[1].add(b.hi, 0.f, b.hi);
    }
    __device__ void finish() {
        double v[2] = {(double)acc[0].s + (double)acc[0].e, (double)acc[1].s + (double)acc[1].e};
        block_sum<2>(v);
        const int tid = threadIdx.x + blockDim.x * threadIdx.y;
        if (tid == 0) {
            part[blockIdx.x * 4 + 0] = v[0];
            part[blockIdx.x * 4 + 1] = v[1];
        }
        if (last_block(counter, nblocks)) {
            double v[2];
            sum_partials<2>(part, nblocks, 4, v);
            if (tid == 0) {
                sc->rz = 0.0;
                sc->rr = v[0];
                sc->bb = v[1];
                sc->iter = 0;
                sc->first = 1;
                sc->beta = 0.0;
                sc->alpha = 0.0;
                int done = 0;
                if (!(v[0] == v[0]) || !(v[1] == v[1])) done = 2;
                else if (v[0] <= sc->tol2 * v[1]) done = 1;
                sc->done = done;
                *counter = 0u;
            }
        }
    }
};

// The double-float march (the conduction tile of the one-problem kernel) with the register
// budget of 3 resident blocks per SM.
template <bool PER>
__global__ void __launch_bounds__(NTHREADS, 3)
residual_df_kernel(MarchGrid g, const Coef4<dfloat>* __restrict__ coef, LoadState<PolDF> ld, EpiResidualDF ep) {
    ep.init();
    const TileIdx t = decode_tile(g);
    __shared__ TileSmem<PolDF, TX, TY> sm;
    tc_tile<PolDF, TX, TY, LoadState<PolDF>, EpiResidualDF, PER>(g.c[0], t, coef, ld, ep, threadIdx.x + TX * threadIdx.y, sm);
    ep.finish();
}

// double-float copies of the float64 Backward Euler records (4th word M = 1/w)
__global__ void records_df_kernel(long long n, const Coef4<double>* rec, Coef4<dfloat>* out) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const Coef4<double> c = rec[t];
        out[t] = Coef4<dfloat>{cvt<dfloat>(c.a), cvt<dfloat>(c.b), cvt<dfloat>(c.c), cvt<dfloat>(c.w)};
    }
}

// r32 = rhs, d = 0, D^-1 = 1/(M - dt diag A) and the sums <r, D^-1 r>, <r, r>, <rhs, rhs>;
// the last block initialises the scalar state of the inner solve.
__global__ void __launch_bounds__(256)
init_rhs_kernel(long long n, const double* rhs, const Coef4<float>* rec_be, const float* adiag, double dt, float* r,
                float* dinv, float* d, PcgScalars* sc, double* part, unsigned int* counter) {
    // the sums in double-float on the float32 pipes (GB300 issues float64 at a small fraction of
    // the float32 rate); <rhs, rhs> from the leading float of rhs (the inner test needs a few digits)
    DfAcc a[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    const float dtf = (float)dt;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const float rs = narrow(rhs[t]);
        const float ds = 1.0f / (rec_be[t].w - dtf * adiag[t]);
        r[t] = rs;
        dinv[t] = ds;
        d[t] = 0.0f;
        a[0].add(rs, 0.f, ds * rs);
        a[1].add(rs, 0.f, rs);
    }
    a[2] = a[1];
    double acc[3];
    for (int k = 0; k < 3; ++k) acc[k] = (double)a[k].s + (double)a[k].e;
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

__global__ void to_float_kernel(long long n, const double* x, float* y) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        y[t] = narrow(x[t]);
}

__global__ void add_correction_kernel(long long n, double* x, const float* d) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        x[t] += widen(d[t]);
}

// The shadow's records from the context's current float64 ones: float32 records (w and M = 1/w
// variants), float32 diag(A), and the double-float Backward Euler records.
void refresh_shadow(Ctx& c, Ctx& s) {
    s.dt_e = c.dt_e;
    ops_f32()->store_coefs(s, c.coef64, static_cast<const double*>(c.adiag));
    if (s.coef64) {
        records_df_kernel<<<reduce_blocks(c), 256, 0, c.stream>>>(c.n, static_cast<const Coef4<double>*>(c.coef_be),
                                                                  reinterpret_cast<Coef4<dfloat>*>(s.coef64));
        PB_CUDA_TRY(cudaGetLastError());
    }
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
        s->welem = 4;
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
        // the shadow's float64-record slot holds the double-float Backward Euler records of the
        // conduction residual (the same 32-byte stride)
        if (c.kind == PB_TC_ANISO) s->coef64 = static_cast<Coef4<double>*>(dalloc(n * sizeof(Coef4<dfloat>)));
        refresh_shadow(c, *s);
        PB_CUDA_TRY(cudaStreamSynchronize(c.stream));
    } catch (...) {
        free_shadow(s);
        throw;
    }
    c.shadow = s;
    return *s;
}

// The PTL pass of a mixed-precision Backward Euler cycle on a float32 view of the state (as the
// float32 super-time-stepping path takes it): F = L u in float32 on the shadow's records, the
// arg-max compared in float, Eq. 5 from the float values; the result lands in the context's
// mapped PTL record.  GB300 runs the float64 pass on its thin float64 pipes.
void mixed_ptl(Ctx& c, const void* u, bool full) {
    Ctx& s = mixed_shadow(c);
    s.d_flag = c.d_flag;
    s.d_ptl = c.d_ptl;
    float* u32 = static_cast<float*>(s.r);       // free until the solve's set-up
    {
        KScope ks(c.prof, c.stream, K_PCG32_REFINE, (double)c.n * (8 + 4));
        to_float_kernel<<<reduce_blocks(c), 256, 0, c.stream>>>(c.n, static_cast<const double*>(u), u32);
        PB_CUDA_TRY(cudaGetLastError());
    }
    Ops* ops = ops_f32();
    s.prof.on = c.prof.on;
    ops->y0_pass(s, u32, s.y0, true, nullptr, 0.0);
    ops->ptl_finalize(s, u32, s.y0);
    if (full) ops->ptl_full(s, u32, s.y0);
    PB_CUDA_TRY(cudaStreamSynchronize(s.stream));
    s.prof.harvest();
    c.prof.absorb(s.prof, K_PTL_PASS, K_PTL_PASS);
    c.prof.absorb(s.prof, K_PTL_FINAL, K_PTL_FINAL);
    c.prof.absorb(s.prof, K_PTL_FULL, K_PTL_FULL);
}

// Rewrites the shadow's records after every coefficient update (parabolic_update).
void mixed_refresh(Ctx& c) {
    if (c.shadow) refresh_shadow(c, *c.shadow);
}

// The outer residual of mixed-precision BE for conduction: r = b - S x (b = M u^n) into c.r
// (float64) with <r, r>, <b, b> and the outer stopping decision in c.d_pcg, by the double-float
// march over the double-float records.
void mixed_residual(Ctx& c, const void* x, const void* un, double dt) {
    Ctx& s = mixed_shadow(c);
    if (!s.coef64) throw Error{PB_ENOTSUP, "the double-float residual is built for conduction"};
    const Coef4<dfloat>* rec = reinterpret_cast<const Coef4<dfloat>*>(s.coef64);
    const float dth = (float)dt;
    EpiResidualDF ep{static_cast<const double*>(un), static_cast<double*>(c.r), dfloat(dth, (float)(dt - (double)dth)),
                     c.d_pcg, static_cast<double*>(c.partials), c.counter, c.grid.nblocks, {}};
    const LoadState<PolDF> ld{static_cast<const double*>(x)};
    KScope ks(c.prof, c.stream, K_PCG_INIT, (double)c.n * (8 + 8 + 32 + 8));   // x, u^n, records; r
    if (c.grid.c[0].periodic)
        residual_df_kernel<true><<<c.grid.nblocks, dim3(TX, TY), 0, c.stream>>>(c.grid, rec, ld, ep);
    else
        residual_df_kernel<false><<<c.grid.nblocks, dim3(TX, TY), 0, c.stream>>>(c.grid, rec, ld, ep);
    PB_CUDA_TRY(cudaGetLastError());
}

void free_shadow(Ctx* s) {
    if (!s) return;
    void* p[] = {s->coef, s->coef_be, s->adiag, s->r, s->p[0], s->p[1], s->q, s->dinv, s->y0, s->partials,
                 s->counter, s->d_pcg, s->coef64, s->cheb[0], s->cheb[1], s->cheb[2]};
    for (void* q : p)
        if (q) cudaFree(q);
    if (s->h_pcg) cudaFreeHost(s->h_pcg);
    s->prof.release();
    delete s;
}

// One refinement's inner solve: S d = r (c.r, float64) to relative residual inner_rtol with at
// most max_iter float32 PCG iterations, then x += d.  Returns the inner iterations; sets
// *status to 0 (ok), 2 (non-finite) or 3 (cap reached, which the outer loop tolerates).
long long mixed_inner(Ctx& c, void* x, double dt, double inner_rtol, long long max_iter, int check_every, int* status,
                      const ChebPlan* plan) {
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
    if (plan) ops->pcg_precond(s, *plan, dt);      // z_0 = P r_0 (Chebyshev inner solves)
    for (;;) {
        PB_CUDA_TRY(cudaMemcpyAsync(s.h_pcg, s.d_pcg, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s.stream));
        PB_CUDA_TRY(cudaStreamSynchronize(s.stream));
        if (s.h_pcg->done) break;
        for (int m = 0; m < check_every; ++m) {
            if (plan) ops->pcg_iter_poly(s, s.y0, parity, dt, *plan);
            else ops->pcg_iter(s, s.y0, parity, dt);
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
    c.prof.absorb(s.prof, K_PCG_CHEB, K_PCG_CHEB);
    return r.iter;
}

}  // namespace pb
