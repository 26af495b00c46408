// Loaders and epilogues fused into the march kernels, and the element-wise / finishing kernels
// of the cycle loop (PTL evaluation, STS stage 1, PCG update).
#pragma once

#include <climits>

#include "common.cuh"
#include "dfloat.cuh"
#include "march.cuh"
#include "reduce.cuh"

namespace pb {

struct NoPre {};

// ---- loaders -------------------------------------------------------------------------------
// A state stored in type T (the caller's bfloat16 array of a bfloat16-storage policy)
template <class P, typename T>
struct LoadStateT {
    const T* u;
    __device__ void init() {}
    __device__ typename P::A operator()(long long idx) const { return cvt<typename P::A>(ldg(u + idx)); }
};

template <class P>
struct LoadState {
    const typename P::S* u;
    __device__ void init() {}
    __device__ typename P::A operator()(long long idx) const { return cvt<typename P::A>(ldx<P>(u + idx)); }
};

// PCG search direction p = z + beta p_old with z = D^-1 r, formed on the fly (halo included).
template <class P>
struct LoadPcgP {
    using A = typename P::A;
    using S = typename P::S;
    const S* r;
    const S* dinv;
    const S* pold;
    const PcgScalars* sc;
    A beta;
    int first;
    __device__ void init() {
        beta = (A)sc->beta;
        first = sc->first;
    }
    __device__ A operator()(long long idx) const {
        // z is rounded to the state precision exactly as the dot <r, z> sees it
        const A z = cvt<A>(cvt<S>(cvt<A>(ldg(dinv + idx)) * cvt<A>(ldg(r + idx))));
        return first ? z : z + beta * cvt<A>(ldg(pold + idx));
    }
};

// Order key of a non-negative value: its bit pattern as a signed integer orders like the value,
// and Inf and NaN sort above every finite value (-1 is below every key).
template <typename A> struct MagKey;
template <> struct MagKey<float> {
    using K = int;
    __device__ static K of(float v) { return __float_as_int(v); }
    __device__ static float value(K k) { return __int_as_float(k); }
};
template <> struct MagKey<double> {
    using K = long long;
    __device__ static K of(double v) { return __double_as_longlong(v); }
    __device__ static double value(K k) { return __longlong_as_double(k); }
};

// ---- epilogues -----------------------------------------------------------------------------
// F = w A u (stored), optionally the stage-1 increment d1 = a F (STS stage 1, see EpiStage)
// and the block arg-max of |F|.
template <class P, bool ARGMAX, bool U1>
struct EpiF {
    using A = typename P::A;
    using S = typename P::S;
    using K = typename MagKey<A>::K;
    using Pre = NoPre;
    S* F;
    S* u1;
    A a;
    ArgMax* part;
    int* nonfinite;
    // running max |F| of this thread as an order key of the arithmetic-precision value (the stored
    // F converts exactly, so the decision equals a float64 comparison); one integer compare per
    // point, non-finite values win it and are reported once at the end
    K bk;
    long long bi;
    float al = 0.f;                  // low part of a (double-float policies)
    static constexpr int NC = 0;     // point operands delivered by the TMA kernel
    __device__ void init() { bk = K(-1); bi = LLONG_MAX; }
    __device__ bool skip() const { return false; }
    __device__ Pre prefetch(long long) const { return {}; }
    using E = typename P::E;
    __device__ void apply_c(long long idx, A Au, A w, E center, E, E, E) { apply(idx, Au, w, (A)center, Pre{}); }
    __device__ void apply(long long idx, A Au, A w, A center, const Pre&) {
        const A f = w * Au;
        const S fs = cvt<S>(f);
        F[idx] = fs;
        if constexpr (U1) {
            if constexpr (P::DF) u1[idx] = cvt<S>(df_scale(a, al, f));
            else u1[idx] = cvt<S>(a * f);
        }
        if (ARGMAX) {
            const K key = MagKey<A>::of(fabs(cvt<A>(fs)));
            if (key > bk) { bk = key; bi = idx; }    // a thread visits its indices in rising order
        }
    }
    __device__ void finish() {
        if (!ARGMAX) return;
        const A bv = bk < 0 ? A(-1) : MagKey<A>::value(bk);
        if (bk >= 0 && !isfinite(bv)) atomicOr(nonfinite, 1);
        double v = (double)bv;
        long long i = bi;
        block_argmax(v, i);
        if (threadIdx.x == 0 && threadIdx.y == 0) part[blockIdx.x] = ArgMax{v, i};
    }
};

// STS stage k >= 2 (Appendix A) in increment form.  With the frozen (linear) operator,
// F(u_0 + d) = y_0 + F(d), so the stage recurrence for d_k = u_k - u_0 reads
//   d_k = mu d_{k-1} + nu d_{k-2} + mut dt F(d_{k-1}) + (mut + gt) dt y_0,   d_0 = 0,
// which is algebraically the stage update u_k = mu u_{k-1} + nu u_{k-2} + (1-mu-nu) u_0
// + mut dt F(u_{k-1}) + gt dt y_0; it drops the u_0 read from every stage but the last and
// keeps stored stage values small (the rounding of reduced-precision storage acts on d, not u).
// The last stage writes u_s = u_0 + d_s over u_0 in place (each point is read before it is
// written, by the same thread).  Under a double-float policy (P::DF) the increment's right-hand
// side is summed in double-float with the float64 coefficients split into float pairs, so the
// stage adds one rounding, the store's (float32 arithmetic would add several, at the magnitude
// of the largest term: in the stiff modes mdt F and ydt y_0 nearly cancel); the last stage then
// adds the increment to u_0 in float, one more rounding per cycle.
template <class P, bool KM2, bool LAST>
struct EpiStage {
    using A = typename P::A;
    using S = typename P::S;
    using E = typename P::E;
    // E wider than A: the register-path kernels hand over d_{k-1} in A, so its stored value is
    // reloaded (the TMA kernel hands it over exactly)
    static constexpr bool kExact = sizeof(E) > sizeof(A);
    struct Pre { E dkm2, y0, u0, dkm1; };
    const S* dkm2;
    const S* y0;
    const S* u0;
    S* out;
    E mu, nu, mdt, ydt;
    const S* dkm1;
    float mul = 0.f, nul = 0.f, mdtl = 0.f, ydtl = 0.f;   // low parts of the coefficients (P::DF)
    // point operands of the TMA kernel, in this order: y0, d_{k-2} (KM2), u0 (LAST)
    static constexpr int NC = 1 + (KM2 ? 1 : 0) + (LAST ? 1 : 0);
    __device__ void apply_c(long long idx, A Au, A w, E d1, E c0, E c1, E c2) {
        update(idx, Au, w, d1, KM2 ? c1 : E(0), c0, LAST ? (KM2 ? c2 : c1) : E(0));
    }
    __device__ void init() {}
    __device__ bool skip() const { return false; }
    __device__ Pre prefetch(long long idx) const {
        return Pre{KM2 ? cvt<E>(ldx<P>(dkm2 + idx)) : E(0), cvt<E>(ldx<P>(y0 + idx)), LAST ? cvt<E>(u0[idx]) : E(0),
                   kExact ? cvt<E>(ldx<P>(dkm1 + idx)) : E(0)};
    }
    __device__ void apply(long long idx, A Au, A w, A d1, const Pre& p) {
        update(idx, Au, w, kExact ? p.dkm1 : (E)d1, p.dkm2, p.y0, p.u0);
    }
    __device__ void update(long long idx, A Au, A w, E d1, E d2, E y, E u) {
        if constexpr (P::DF) {
            DfAcc acc;
            acc.set(mu, mul, d1);
            if (KM2) acc.add(nu, nul, d2);
            acc.add(mdt, mdtl, __fmul_rn(w, Au));
            acc.add(ydt, ydtl, y);
            // the last stage adds the increment to u_0 once: one more rounding per cycle, not per stage
            out[idx] = cvt<S>(LAST ? __fadd_rn(u, acc.value()) : acc.value());
        } else {
            const E d = mu * d1 + nu * d2 + mdt * (E)(w * Au) + ydt * y;
            out[idx] = cvt<S>(LAST ? u + d : d);
        }
    }
    __device__ void finish() {}
};

// STS stage 2 fused with stage 1.  The march runs on y0 itself: with d1 = a y0 and the linear
// operator, F(d1) = a F(y0), so
//   d2 = mu_2 d1 + mut_2 dt F(d1) + (mut_2 + gt_2) dt y0 = (mu_2 a + ydt) y0 + (mdt a) F(y0),
// and d1 is written (for stage 3) only when s > 2; when s = 2 this is the last stage and
// u0 + d2 is written over u0.
template <class P, bool LAST>
struct EpiStage2 {
    using A = typename P::A;
    using S = typename P::S;
    using E = typename P::E;
    static constexpr bool kExact = sizeof(E) > sizeof(A);
    struct Pre { E u0, y; };
    const S* u0;
    S* d1;
    S* out;
    E a, cy, cf;       // a = mut_1 dt, cy = mu_2 a + ydt, cf = mdt a
    const S* y0;       // the marched field, reloaded exactly when E is wider than A
    float al = 0.f, cyl = 0.f, cfl = 0.f;   // low parts of the coefficients (P::DF)
    static constexpr int NC = LAST ? 1 : 0;
    __device__ void init() {}
    __device__ bool skip() const { return false; }
    __device__ Pre prefetch(long long idx) const {
        return Pre{LAST ? cvt<E>(u0[idx]) : E(0), kExact ? cvt<E>(ldx<P>(y0 + idx)) : E(0)};
    }
    __device__ void apply_c(long long idx, A Au, A w, E y, E c0, E, E) { update(idx, Au, w, y, c0); }
    __device__ void apply(long long idx, A Au, A w, A y, const Pre& p) { update(idx, Au, w, kExact ? p.y : (E)y, p.u0); }
    __device__ void update(long long idx, A Au, A w, E y, E u) {
        if constexpr (P::DF) {
            // two terms: the product cy y split exactly (FMA error term), cf F added to it by one
            // fused multiply-add, so the two nearly cancelling terms of the stiff modes are summed
            // exactly and d2 is rounded at its own magnitude (the error terms, coefficients' low
            // parts included, added after)
            const float F = __fmul_rn(w, Au);
            const float p = __fmul_rn(cy, y);
            const float err = __fmaf_rn(cfl, F, __fmaf_rn(cyl, y, __fmaf_rn(cy, y, -p)));
            const float d2 = __fadd_rn(__fmaf_rn(cf, F, p), err);
            if (LAST) {
                out[idx] = cvt<S>(__fadd_rn(u, d2));
            } else {
                d1[idx] = cvt<S>(df_scale(a, al, y));
                out[idx] = cvt<S>(d2);
            }
        } else {
            const E d2 = cy * y + cf * (E)(w * Au);
            if (LAST) {
                out[idx] = cvt<S>(u + d2);
            } else {
                d1[idx] = cvt<S>(a * y);
                out[idx] = cvt<S>(d2);
            }
        }
    }
    __device__ void finish() {}
};

// PCG set-up on the system S x = b, S = M - dt A, b = M u^n (the record's 4th word is M = 1/w):
//   r = b - S x = M (u^n - x) + dt A x,  D^-1 = 1/(M - dt diag A),  and the sums <r, D^-1 r>,
//   <r, r>, <b, b>; the last block initialises the scalar state.  FULL = false forms r, <r, r> and
//   <b, b> only (<r, D^-1 r> = 0): the outer residual of an iterative refinement, which needs no
//   D^-1 (and skips its division, costly in float64 on GB300).
template <class P, bool FULL = true>
struct EpiPcgInit {
    using A = typename P::A;
    using S = typename P::S;
    using C = typename P::C;
    struct Pre { A un, ad; };
    const S* un;
    S* r;
    S* dinv;
    const C* adiag;
    PcgScalars* sc;
    double* part;
    unsigned int* counter;
    int nblocks;
    A dt;
    double acc[3];
    __device__ void init() { acc[0] = acc[1] = acc[2] = 0.0; }
    __device__ bool skip() const { return false; }
    __device__ Pre prefetch(long long idx) const { return Pre{cvt<A>(un[idx]), FULL ? (A)__ldg(adiag + idx) : A(0)}; }
    __device__ void apply(long long idx, A Au, A m, A x, const Pre& p) {
        const S rs = cvt<S>(m * (p.un - x) + dt * Au);
        r[idx] = rs;
        const double rd = (double)cvt<A>(rs);
        const double b = (double)(m * p.un);
        if constexpr (FULL) {
            const S ds = cvt<S>(A(1) / (m - dt * p.ad));
            dinv[idx] = ds;
            const double z = (double)cvt<A>(cvt<S>(cvt<A>(ds) * cvt<A>(rs)));
            acc[0] += rd * z;
        }
        acc[1] += rd * rd;
        acc[2] += b * b;
    }
    __device__ void finish() {
        block_sum<3>(acc);
        const int tid = threadIdx.x + blockDim.x * threadIdx.y;
        if (tid == 0) {
            part[blockIdx.x * 4 + 0] = acc[0];
            part[blockIdx.x * 4 + 1] = acc[1];
            part[blockIdx.x * 4 + 2] = acc[2];
        }
        if (last_block(counter, nblocks)) {
            double v[3];
            sum_partials<3>(part, nblocks, 4, v);
            if (tid == 0) {
                sc->rz = v[0];
                sc->rr = v[1];
                sc->bb = v[2];
                sc->iter = 0;
                sc->first = 1;
                sc->beta = 0.0;
                sc->alpha = 0.0;
                const long long limit = sc->fixed > 0 ? sc->fixed : sc->max_iter;
                int done = 0;
                if (!(v[0] == v[0]) || !(v[1] == v[1]) || !(v[2] == v[2])) done = 2;
                else if (sc->fixed == 0 && v[1] <= sc->tol2 * v[2]) done = 1;
                else if (limit == 0) done = 3;
                sc->done = done;
                *counter = 0u;
            }
        }
    }
};

// PCG SpMV: p (from the loader) is stored, q = S p = M p - dt A p, and <p, q> gives alpha.
template <class P>
struct EpiPcgSpmv {
    using A = typename P::A;
    using S = typename P::S;
    using Pre = NoPre;
    S* pout;
    S* q;
    PcgScalars* sc;
    double* part;
    unsigned int* counter;
    int nblocks;
    A dt;
    int done;
    DotAcc<A> acc;
    static constexpr int NC = 0;     // point operands delivered by the TMA kernel
    __device__ void init() {
        acc.init();
        done = sc->done;
    }
    __device__ bool skip() const { return done != 0; }
    __device__ Pre prefetch(long long) const { return {}; }
    using E = typename P::E;
    __device__ void apply_c(long long idx, A Au, A m, E pv, E, E, E) { apply(idx, Au, m, (A)pv, Pre{}); }
    __device__ void apply(long long idx, A Au, A m, A pv, const Pre&) {
        const S ps = cvt<S>(pv);
        const S qs = cvt<S>(m * pv - dt * Au);
        pout[idx] = ps;
        q[idx] = qs;
        acc.add(cvt<A>(ps), cvt<A>(qs));
    }
    __device__ void finish() {
        double v0[1] = {acc.value()};
        block_sum<1>(v0);
        const int tid = threadIdx.x + blockDim.x * threadIdx.y;
        if (tid == 0) part[blockIdx.x * 4] = v0[0];
        if (last_block(counter, nblocks)) {
            double v[1];
            sum_partials<1>(part, nblocks, 4, v);
            if (tid == 0) {
                const double pq = v[0];
                sc->pq = pq;
                if (!(pq > 0.0) || !(pq <= 1.79769313486231570e308)) sc->done = 2;
                else sc->alpha = sc->rz / pq;
                *counter = 0u;
            }
        }
    }
};

// ---- element-wise kernels ------------------------------------------------------------------
// d1 = a y0 (STS stage-1 increment when the cycle length is known only after the PTL pass).
template <class P>
__global__ void stage1_kernel(long long n, const typename P::S* y0, typename P::S* d1, typename P::A a) {
    using A = typename P::A;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        d1[t] = cvt<typename P::S>(a * cvt<A>(y0[t]));
}

// Block partials of <r, z> and <r, r>; the last block applies the stopping test (r.r <= rtol^2 b.b
// after the update) and forms beta.
__device__ inline void pcg_update_finish(double (&acc)[2], PcgScalars* sc, double* part, unsigned int* counter) {
    block_sum<2>(acc);
    if (threadIdx.x == 0) {
        part[blockIdx.x * 4 + 0] = acc[0];
        part[blockIdx.x * 4 + 1] = acc[1];
    }
    if (last_block(counter, gridDim.x)) {
        double v[2];
        sum_partials<2>(part, gridDim.x, 4, v);
        if (threadIdx.x == 0) {
            const double rz = v[0], rr = v[1];
            sc->rr = rr;
            sc->iter += 1;
            int done = 0;
            if (!(rr == rr) || !(rz == rz)) done = 2;
            else if (sc->fixed > 0) done = sc->iter >= sc->fixed ? 1 : 0;
            else if (rr <= sc->tol2 * sc->bb) done = 1;
            else if (sc->iter >= sc->max_iter) done = 3;
            if (!done) {
                sc->beta = rz / sc->rz;
                sc->rz = rz;
                sc->first = 0;
            }
            sc->done = done;
            *counter = 0u;
        }
    }
}

// PCG update: x += alpha p, r -= alpha q, z = D^-1 r, sums <r, z> and <r, r>.
template <class P>
__global__ void __launch_bounds__(256)
pcg_update_kernel(long long n, typename P::S* x, typename P::S* r, const typename P::S* p,
                  const typename P::S* q, const typename P::S* dinv, PcgScalars* sc,
                  double* part, unsigned int* counter) {
    using A = typename P::A;
    using S = typename P::S;
    if (sc->done) return;
    const A alpha = (A)sc->alpha;
    double acc[2] = {0.0, 0.0};
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        x[t] = cvt<S>(cvt<A>(x[t]) + alpha * cvt<A>(p[t]));
        const S rs = cvt<S>(cvt<A>(r[t]) - alpha * cvt<A>(q[t]));
        r[t] = rs;
        const A ra = cvt<A>(rs);
        const double z = (double)cvt<A>(cvt<S>(cvt<A>(dinv[t]) * ra));
        acc[0] += (double)ra * z;
        acc[1] += (double)ra * (double)ra;
    }
    pcg_update_finish(acc, sc, part, counter);
}

// The same update for float32 state, four points per step through 16-byte accesses (all five
// arrays 16-byte aligned).  The dot products sum each group of four in float and add the group
// sums in double: GB300 issues float64 arithmetic at a small fraction of its float32 rate, and
// double arithmetic on every point would bound this pass instead of HBM.
static __global__ void __launch_bounds__(256)
pcg_update_f32x4_kernel(long long n, float* x, float* r, const float* p, const float* q, const float* dinv,
                        PcgScalars* sc, double* part, unsigned int* counter) {
    if (sc->done) return;
    const float alpha = (float)sc->alpha;
    double acc[2] = {0.0, 0.0};
    const long long n4 = n >> 2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (long long t = t0; t < n4; t += stride) {
        float4 xv = reinterpret_cast<const float4*>(x)[t];
        float4 rv = reinterpret_cast<const float4*>(r)[t];
        const float4 pv = __ldg(reinterpret_cast<const float4*>(p) + t);
        const float4 qv = __ldg(reinterpret_cast<const float4*>(q) + t);
        const float4 dv = __ldg(reinterpret_cast<const float4*>(dinv) + t);
        xv.x += alpha * pv.x; xv.y += alpha * pv.y; xv.z += alpha * pv.z; xv.w += alpha * pv.w;
        rv.x -= alpha * qv.x; rv.y -= alpha * qv.y; rv.z -= alpha * qv.z; rv.w -= alpha * qv.w;
        reinterpret_cast<float4*>(x)[t] = xv;
        reinterpret_cast<float4*>(r)[t] = rv;
        const float rz = rv.x * (dv.x * rv.x) + rv.y * (dv.y * rv.y) + rv.z * (dv.z * rv.z) + rv.w * (dv.w * rv.w);
        const float rr = rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w;
        acc[0] += (double)rz;
        acc[1] += (double)rr;
    }
    const long long tt = 4 * n4 + t0;          // the last n mod 4 points
    if (tt < n) {
        x[tt] += alpha * p[tt];
        const float rs = r[tt] - alpha * q[tt];
        r[tt] = rs;
        acc[0] += (double)(rs * (dinv[tt] * rs));
        acc[1] += (double)(rs * rs);
    }
    pcg_update_finish(acc, sc, part, counter);
}

// PTL (Eq. 5) at k = argmax |F| over the block partials; one block of up to kFinalizeThreads
// (a march launch leaves thousands of partials: more threads shorten each one's chain of loads).
constexpr int kFinalizeThreads = 1024;

template <class P, typename UT = typename P::S>
__global__ void __launch_bounds__(kFinalizeThreads)
ptl_finalize_kernel(MarchGrid g, const UT* u, const typename P::S* F,
                    const ArgMax* part, int nparts, PtlResult* res, const int* nonfinite) {
    using A = typename P::A;
    double v = -1.0;
    long long i = LLONG_MAX;
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
        const ArgMax m = part[b];
        argmax_merge(v, i, m.v, m.i);
    }
    block_argmax(v, i);
    if (threadIdx.x >= 32) return;
    // warp 0 holds the arg-max; Eq. 5 at k: lane a < nn takes neighbour a, so the six pairs of
    // dependent loads are in flight together, and a warp min gives the smallest bound
    const int lane = threadIdx.x;
    double best = 1.0 / 0.0;
    if (i >= 0 && i != LLONG_MAX) {
        int comp = 0;
        for (int c = 1; c < g.ncomp; ++c)
            if (i >= g.c[c].offset) comp = c;
        const CompGrid& cg = g.c[comp];
        const long long loc = i - cg.offset;
        const long long plane = (long long)cg.nr * cg.nt;
        const int kk = (int)(loc / plane);
        const long long rem = loc - (long long)kk * plane;
        const int jj = (int)(rem / cg.nr);
        const int ii = (int)(rem - (long long)jj * cg.nr);
        long long nb[6];
        int nn = 0;
        const bool per = cg.periodic != 0;        // the box: r and theta neighbours wrap
        if (ii > 0) nb[nn++] = i - 1;
        else if (per) nb[nn++] = i + cg.nr - 1;
        if (ii < cg.nr - 1) nb[nn++] = i + 1;
        else if (per) nb[nn++] = i - (cg.nr - 1);
        if (jj > 0) nb[nn++] = i - cg.nr;
        else if (per) nb[nn++] = i + (long long)(cg.nt - 1) * cg.nr;
        if (jj < cg.nt - 1) nb[nn++] = i + cg.nr;
        else if (per) nb[nn++] = i - (long long)(cg.nt - 1) * cg.nr;
        nb[nn++] = cg.offset + (long long)((kk + cg.np - 1) % cg.np) * plane + rem;
        nb[nn++] = cg.offset + (long long)((kk + 1) % cg.np) * plane + rem;
        if (lane < nn) {
            long long j = nb[0];
#pragma unroll
            for (int a = 1; a < 6; ++a)
                if (lane == a) j = nb[a];
            const double uk = (double)cvt<A>(u[i]), fk = (double)cvt<A>(F[i]);
            const double du = uk - (double)cvt<A>(u[j]);
            const double df = fk - (double)cvt<A>(F[j]);
            if (du != 0.0 && df != 0.0 && du * df < 0.0) best = -du / df;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
    }
    if (lane != 0) return;
    PtlResult out;
    out.nonfinite = *nonfinite;
    out.fmax = v;
    out.k = i;
    out.dt_ptl = best;
    out.pad = 0;
    out.dt_full = __longlong_as_double(0x7ff8000000000000LL);
    out.key_full = -1;
    *res = out;
}

// Eq. 4 over every pair of face neighbours (i, i + e_d) of one component, d = 0 (r), 1 (theta),
// 2 (phi, periodic; r and theta wrap too on the periodic box), without the F_max localisation of Eq. 5: a pair with du = u_i - u_j != 0,
// dF = F_i - F_j != 0 and du dF < 0 bounds dt by -du/dF (arithmetic precision).  Each block
// leaves the smallest bound and, among equal bounds, the smallest key 3 i + d, as an ArgMax of
// -bound (-inf when no pair qualifies).
template <typename A> struct Eps;
template <> struct Eps<float> { static constexpr float value = 1.1920929e-7f; };
template <> struct Eps<double> { static constexpr double value = 2.220446049250313e-16; };

template <class P>
__global__ void __launch_bounds__(256)
ptl_full_kernel(MarchGrid g, long long n, const typename P::S* u, const typename P::S* F, ArgMax* part) {
    using A = typename P::A;
    A best = A(0);
    long long key = LLONG_MAX;
    // rows of constant (component, phi, theta): a warp walks a row along r (coalesced), so the
    // flat index is decoded once per row instead of once per point
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const long long w0 = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    long long rows_before = 0;
    for (int c = 0; c < g.ncomp; ++c) {
        const CompGrid& cg = g.c[c];
        const long long plane = (long long)cg.nr * cg.nt;
        const long long rows = (long long)cg.nt * cg.np;
        // this warp's first row of the component in the global row sequence
        long long r = w0 - rows_before;
        if (r < 0) r += ((-r + warps - 1) / warps) * warps;
        for (; r < rows; r += warps) {
            const int kk = (int)(r / cg.nt);
            const int j = (int)(r - (long long)kk * cg.nt);
            const long long row = cg.offset + (long long)kk * plane + (long long)j * cg.nr;
            const long long up_t = j + 1 < cg.nt ? (long long)cg.nr : (cg.periodic ? -(long long)(cg.nt - 1) * cg.nr : 0);
            const long long up_p = kk + 1 < cg.np ? plane : -(long long)(cg.np - 1) * plane;
            for (int i = lane; i < cg.nr; i += 32) {
                const long long t = row + i;
                const A ut = cvt<A>(u[t]), ft = cvt<A>(F[t]);
                auto pair = [&](long long q, int d) {
                    const A du = ut - cvt<A>(u[q]);
                    const A df = ft - cvt<A>(F[q]);
                    if (du != A(0) && df != A(0) && du * df < A(0)) {
                        // b = |du| / |dF| can only reach `best` if |du| <= best |dF| (1 + 4 eps):
                        // a multiply rules out most pairs before the (exact) division
                        if (key != LLONG_MAX && fabs(du) > best * fabs(df) * (A(1) + A(4) * Eps<A>::value)) return;
                        const A b = -du / df;
                        const long long kq = 3 * t + d;
                        if (key == LLONG_MAX || b < best || (b == best && kq < key)) {
                            best = b;
                            key = kq;
                        }
                    }
                };
                if (i + 1 < cg.nr) pair(t + 1, 0);
                else if (cg.periodic) pair(t - (cg.nr - 1), 0);
                if (up_t != 0) pair(t + up_t, 1);
                pair(t + up_p, 2);
            }
        }
        rows_before += rows;
    }
    (void)n;
    double v = key == LLONG_MAX ? -(1.0 / 0.0) : -(double)best;
    block_argmax(v, key);
    if (threadIdx.x == 0) part[blockIdx.x] = ArgMax{v, key};
}

// One block: the smallest bound over the partials of ptl_full_kernel into res->dt_full / key_full.
static __global__ void __launch_bounds__(kFinalizeThreads)
ptl_full_finalize_kernel(const ArgMax* part, int nparts, PtlResult* res) {
    double v = -(1.0 / 0.0);
    long long i = LLONG_MAX;
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
        const ArgMax m = part[b];
        argmax_merge(v, i, m.v, m.i);
    }
    block_argmax(v, i);
    if (threadIdx.x != 0) return;
    const bool none = i == LLONG_MAX;
    res->dt_full = none ? 1.0 / 0.0 : -v;
    res->key_full = none ? -1 : i;
}

}  // namespace pb
