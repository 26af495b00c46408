// Polynomial (Chebyshev) preconditioning of the Backward Euler PCG: the GPU form of the
// stronger preconditioner that Sec. 3.1 calls PC2.  PC2 is an incomplete factorisation, whose
// triangular solves are sequential; the preconditioner here is instead z = p(D^-1 S) D^-1 r, the
// Chebyshev acceleration of point-Jacobi over [a, b] (a bound of the spectrum of D^-1 S), built
// from the same fused stencil passes as the PCG product.
//
// With theta = (a + b)/2, delta = (b - a)/2, sigma = theta/delta, rho_0 = 1/sigma:
//   y_0 = 0,  y_1 = D^-1 r / theta,
//   y_{j+1} = y_j + rho_j rho_{j-1} (y_j - y_{j-1}) + (2 rho_j / delta) D^-1 (r - S y_j),
//   rho_j = 1/(2 sigma - rho_{j-1}),  j = 1 .. m-1,   z = y_m,
// so 1 - lambda p(lambda) = T_m((theta - lambda)/delta) / T_m(sigma) on the eigenvalues lambda of
// D^-1 S: z is exact to within that factor on [a, b], and P = p(D^-1 S) D^-1 is symmetric
// positive definite when b bounds the spectrum (p > 0 there).  A degree-m application costs m - 1
// stencil passes (y_1 is formed on the fly inside the first).  Per PCG iteration: the product
// q = S p with p = z + beta p_old, the update of x and r (||r||^2 for the stopping test), then the
// m - 1 passes, the last of which sums <r, z> and forms beta.
#pragma once

#include "epilogues.cuh"
#include "march_tma.cuh"

namespace pb {

// y_1 = D^-1 r / theta, rounded to the state precision (the same value wherever it is formed)
template <class P>
__device__ __forceinline__ typename P::A cheb_y1(typename P::A dinv, typename P::A r, typename P::A inv_theta) {
    using A = typename P::A;
    return cvt<A>(cvt<typename P::S>((dinv * r) * inv_theta));
}

// ---- fields of the first pass (y_1 on the fly) and of the product (p = z + beta p_old) --------
template <class P>
struct LoadChebY1 {
    using A = typename P::A;
    using S = typename P::S;
    const S* r;
    const S* dinv;
    A inv_theta;
    __device__ void init() {}
    __device__ A operator()(long long idx) const { return cheb_y1<P>(cvt<A>(ldg(dinv + idx)), cvt<A>(ldg(r + idx)), inv_theta); }
};

template <class P>
struct ChebY1Field {
    using A = typename P::A;
    using S = typename P::S;
    static constexpr int NF = 2;
    static constexpr bool CENTER_RAW = false;
    using FT = S;
    A inv_theta;
    __device__ void init() {}
    __device__ void combine(unsigned char* base, int pitch, int n, S* dst) const {
        const S* r = reinterpret_cast<const S*>(base);
        const S* di = reinterpret_cast<const S*>(base + pitch);
        for (int e = threadIdx.x + TX * threadIdx.y; e < n; e += NTHREADS)
            dst[e] = cvt<S>(cheb_y1<P>(cvt<A>(di[e]), cvt<A>(r[e]), inv_theta));
    }
};

template <class P>
struct LoadPolyP {
    using A = typename P::A;
    using S = typename P::S;
    const S* z;
    const S* pold;
    const PcgScalars* sc;
    A beta;
    int first;
    __device__ void init() {
        beta = (A)sc->beta;
        first = sc->first;
    }
    __device__ A operator()(long long idx) const {
        const A zv = cvt<A>(ldg(z + idx));
        return first ? zv : cvt<A>(cvt<S>(zv + beta * cvt<A>(ldg(pold + idx))));
    }
};

template <class P>
struct PolyPField {
    using A = typename P::A;
    using S = typename P::S;
    static constexpr int NF = 2;
    static constexpr bool CENTER_RAW = false;
    using FT = S;
    const PcgScalars* sc;
    A beta;
    int first;
    __device__ void init() {
        beta = (A)sc->beta;
        first = sc->first;
    }
    __device__ void combine(unsigned char* base, int pitch, int n, S* dst) const {
        const S* z = reinterpret_cast<const S*>(base);
        const S* po = reinterpret_cast<const S*>(base + pitch);
        for (int e = threadIdx.x + TX * threadIdx.y; e < n; e += NTHREADS)
            dst[e] = first ? z[e] : cvt<S>(cvt<A>(z[e]) + beta * cvt<A>(po[e]));
    }
};

// ---- one Chebyshev pass ---------------------------------------------------------------------------
// KIND 1: the first pass (the marched field is y_1, y_0 = 0); 2: the second (y_{j-1} = y_1, formed
// from r and D^-1); 3: later passes (y_{j-1} read).  Point operands: r, D^-1 (and y_{j-1}, KIND 3).
// The record's 4th word is M (the Backward Euler records), so S y = M y - dt A y.
template <class P, int KIND, bool LAST>
struct EpiCheb {
    using A = typename P::A;
    using S = typename P::S;
    using E = typename P::E;
    struct Pre { A r, dinv, yp; };
    const S* r;
    const S* dinv;
    const S* yprev;
    S* out;
    A dt, c1, c2, inv_theta;
    PcgScalars* sc;
    double* part;
    unsigned int* counter;
    int nblocks;
    int done;
    DotAcc<A> acc;
    static constexpr int NC = KIND == 3 ? 3 : 2;
    __device__ void init() {
        acc.init();
        done = sc->done;
    }
    __device__ bool skip() const { return done != 0; }
    __device__ Pre prefetch(long long idx) const {
        return Pre{cvt<A>(ldg(r + idx)), cvt<A>(ldg(dinv + idx)), KIND == 3 ? cvt<A>(ldg(yprev + idx)) : A(0)};
    }
    __device__ void apply_c(long long idx, A Au, A m, E y, E c0, E cd, E cp) { update(idx, Au, m, (A)y, (A)c0, (A)cd, (A)cp); }
    __device__ void apply(long long idx, A Au, A m, A y, const Pre& p) { update(idx, Au, m, y, p.r, p.dinv, p.yp); }
    __device__ void update(long long idx, A Au, A m, A y, A rv, A dv, A yp_stored) {
        const A yp = KIND == 1 ? A(0) : (KIND == 2 ? cheb_y1<P>(dv, rv, inv_theta) : yp_stored);
        const A sy = m * y - dt * Au;
        const S ys = cvt<S>(y + c1 * (y - yp) + c2 * (dv * (rv - sy)));
        out[idx] = ys;
        if (LAST) acc.add(rv, cvt<A>(ys));
    }
    __device__ void finish() {
        if (!LAST) return;
        double v0[1] = {acc.value()};
        block_sum<1>(v0);
        const int tid = threadIdx.x + blockDim.x * threadIdx.y;
        if (tid == 0) part[blockIdx.x * 4] = v0[0];
        if (last_block(counter, nblocks)) {
            double v[1];
            sum_partials<1>(part, nblocks, 4, v);
            if (tid == 0) {
                const double rz = v[0];
                if (!(rz == rz) || !(rz <= 1.79769313486231570e308)) {
                    sc->done = 2;
                } else {
                    if (!sc->first) sc->beta = rz / sc->rz;
                    sc->rz = rz;
                }
                *counter = 0u;
            }
        }
    }
};

// ---- the update of a polynomially preconditioned iteration ------------------------------------
// x += alpha p, r -= alpha q and <r, r>; the last block applies the stopping test (beta and <r, z>
// come from the preconditioner's last pass).
__device__ inline void pcg_update_poly_finish(double (&acc)[1], PcgScalars* sc, double* part, unsigned int* counter) {
    block_sum<1>(acc);
    if (threadIdx.x == 0) part[blockIdx.x * 4] = acc[0];
    if (last_block(counter, gridDim.x)) {
        double v[1];
        sum_partials<1>(part, gridDim.x, 4, v);
        if (threadIdx.x == 0) {
            const double rr = v[0];
            sc->rr = rr;
            sc->iter += 1;
            int done = 0;
            if (!(rr == rr)) done = 2;
            else if (sc->fixed > 0) done = sc->iter >= sc->fixed ? 1 : 0;
            else if (rr <= sc->tol2 * sc->bb) done = 1;
            else if (sc->iter >= sc->max_iter) done = 3;
            if (!done) sc->first = 0;
            sc->done = done;
            *counter = 0u;
        }
    }
}

template <class P>
__global__ void __launch_bounds__(256)
pcg_update_poly_kernel(long long n, typename P::S* x, typename P::S* r, const typename P::S* p, const typename P::S* q,
                       PcgScalars* sc, double* part, unsigned int* counter) {
    using A = typename P::A;
    using S = typename P::S;
    if (sc->done) return;
    const A alpha = (A)sc->alpha;
    double acc[1] = {0.0};
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        x[t] = cvt<S>(cvt<A>(x[t]) + alpha * cvt<A>(p[t]));
        const S rs = cvt<S>(cvt<A>(r[t]) - alpha * cvt<A>(q[t]));
        r[t] = rs;
        const A ra = cvt<A>(rs);
        acc[0] += (double)ra * (double)ra;
    }
    pcg_update_poly_finish(acc, sc, part, counter);
}

// float32 state, four points per step (16-byte accesses); each group of four squares is summed in
// float and the group sums in double (as pcg_update_f32x4_kernel)
static __global__ void __launch_bounds__(256)
pcg_update_poly_f32x4_kernel(long long n, float* x, float* r, const float* p, const float* q, PcgScalars* sc,
                             double* part, unsigned int* counter) {
    if (sc->done) return;
    const float alpha = (float)sc->alpha;
    double acc[1] = {0.0};
    const long long n4 = n >> 2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (long long t = t0; t < n4; t += stride) {
        float4 xv = reinterpret_cast<const float4*>(x)[t];
        float4 rv = reinterpret_cast<const float4*>(r)[t];
        const float4 pv = __ldg(reinterpret_cast<const float4*>(p) + t);
        const float4 qv = __ldg(reinterpret_cast<const float4*>(q) + t);
        xv.x += alpha * pv.x; xv.y += alpha * pv.y; xv.z += alpha * pv.z; xv.w += alpha * pv.w;
        rv.x -= alpha * qv.x; rv.y -= alpha * qv.y; rv.z -= alpha * qv.z; rv.w -= alpha * qv.w;
        reinterpret_cast<float4*>(x)[t] = xv;
        reinterpret_cast<float4*>(r)[t] = rv;
        acc[0] += (double)(rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w);
    }
    const long long tt = 4 * n4 + t0;
    if (tt < n) {
        x[tt] += alpha * p[tt];
        const float rs = r[tt] - alpha * q[tt];
        r[tt] = rs;
        acc[0] += (double)(rs * rs);
    }
    pcg_update_poly_finish(acc, sc, part, counter);
}

// Upper bound of the spectrum of D^-1 S for a cycle of length dt: Gershgorin,
// max_i (M_i + dt sum_j |A_ij|) / (M_i - dt A_ii), block maxima into part.
template <class P>
__global__ void __launch_bounds__(256)
cheb_bound_kernel(long long n, const Coef4<double>* rec64, const typename P::C* adiag, const double* arow, double dt,
                  double* part) {
    double m = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const double M = 1.0 / rec64[t].w;
        const double d = M - dt * (double)cvt<double>(adiag[t]);
        m = fmax(m, (M + dt * arow[t]) / d);
    }
    m = warp_max(m);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = red[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) x = fmax(x, red[w]);
        part[blockIdx.x] = x;
    }
}

// One block of 256 threads: the maximum of the partials into *out.
static __global__ void __launch_bounds__(256) max_partials_kernel(const double* part, int n, double* out) {
    double m = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) m = fmax(m, part[b]);
    m = warp_max(m);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = red[0];
        for (int w = 1; w < 8; ++w) x = fmax(x, red[w]);
        *out = x;
    }
}

}  // namespace pb
