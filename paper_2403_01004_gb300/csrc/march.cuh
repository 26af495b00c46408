// The two flux-form stencils (Eq. 2), written as phi-marching tile kernels.
//
// A block owns a TX x TY tile of (r, theta) points and walks a chunk of consecutive phi planes.
// Per plane it stages the input field (with a one-point halo) in shared memory, forms the
// stencil A u for its points and hands (A u, w, u_center) to an epilogue that fuses whatever
// the caller needs (an STS stage update, y0 = F(u) with the PTL arg-max, a PCG SpMV, ...).
// The input field comes from a loader, so fused element-wise producers (p = z + beta p in PCG)
// are evaluated on the fly for the halo as well.
//
// Conduction (27-point corner scheme).  Corner c = (i+1/2, j+1/2, k+1/2) carries the record
// ahat_c; its field-aligned gradient is s_c = ahat_c . D_c with D_c,x the sum of the four cell
// differences straddling c along x, and its flux Q_c = ahat_c s_c.  A cell at position
// p in {0,1}^3 inside corner c receives -sigma(p) . Q_c, sigma = 2p - 1.  Writing
//   E0 = Qr+Qt+Qp, E1 = Qr+Qt-Qp, E2 = Qr-Qt+Qp, E3 = Qr-Qt-Qp
// per corner, the eight corner contributions of cell (i,j,k) are
//   (A u) = -[E0(i-1,j-1,k-1) - E0(i,j,k) + E1(i-1,j-1,k) - E1(i,j,k-1)
//             + E2(i-1,j,k-1) - E2(i,j-1,k) + E3(i-1,j,k) - E3(i,j-1,k-1)].
// Corners outside the interior carry ahat = 0 (zero-flux boundaries).
//
// Viscosity (7-point): (A u)_i = sum over the six faces of c_f (u_nbr - u_i), the record of
// point i holding the coefficients of its +r, +theta, +phi faces.
#pragma once

#include "common.cuh"
#include "reduce.cuh"

namespace pb {

__device__ __forceinline__ int wrap_phi(int k, int np) {
    k %= np;
    return k < 0 ? k + np : k;
}

// Decodes blockIdx.x into (component, tile origin, phi chunk).
struct TileIdx { int comp, i0, j0, k0, k1; };

__device__ __forceinline__ TileIdx decode_tile(const MarchGrid& g) {
    int b = blockIdx.x;
    int comp = 0;
    if (g.ncomp > 1 && b >= g.c[1].block_begin) comp = 1;
    if (g.ncomp > 2 && b >= g.c[2].block_begin) comp = 2;
    const CompGrid& c = g.c[comp];
    b -= c.block_begin;
    const int tr = b % c.tiles_r; b /= c.tiles_r;
    const int tt = b % c.tiles_t;
    const int ch = b / c.tiles_t;
    TileIdx t;
    t.comp = comp;
    t.i0 = tr * TX;
    t.j0 = tt * TY;
    t.k0 = ch * c.kchunk;
    t.k1 = min(t.k0 + c.kchunk, c.np);
    return t;
}

template <typename A> struct Quad { A e0, e1, e2, e3; };

// ---------------------------------------------------------------------------------------------
// Conduction march over one tile of TXv x TYv points (r, theta) and phi planes [k0, k1), run by a
// block of at least TXv x TYv threads (tid = linear thread index; extra threads only help with
// the halo and the extra corners).  Shared by the one-problem kernel below and the batched
// persistent kernel.
// Loader: A operator()(long long idx) const   (idx valid);   void init();
// Epi: init(), skip(), Pre prefetch(idx), apply(idx, Au, w, center, pre), finish()
// ---------------------------------------------------------------------------------------------
template <class P, int TXv, int TYv>
struct TileSmem {
    typename P::A cell[2][TYv + 2][TXv + 2];
    Quad<typename P::A> corn[2][TYv + 1][TXv + 1];
};

template <class P, int TXv, int TYv, class Load, class Epi, bool PER = false>
__device__ __forceinline__ void tc_tile(const CompGrid& cg, const TileIdx& t, const Coef4<typename P::C>* __restrict__ coef,
                                        const Load& ld, Epi& ep, int tid, TileSmem<P, TXv, TYv>& sm) {
    using A = typename P::A;
    auto& cell = sm.cell;
    auto& corn = sm.corn;

    const int nr = cg.nr, nt = cg.nt, np = cg.np;
    const long long plane = (long long)nr * nt;
    const int tx = tid % TXv, ty = tid / TXv;
    const bool inb = tid < TXv * TYv;          // a point of the tile
    const int i = t.i0 + tx, j = t.j0 + ty;
    const bool own = inb && (i < nr) && (j < nt);

    // halo slot handled by thread `tid` (2 (TXv + 2) + 2 TYv halo cells)
    int hi = -1, hj = -1;
    if (tid < 2 * (TXv + 2)) {
        hi = tid % (TXv + 2);
        hj = tid < TXv + 2 ? 0 : TYv + 1;
    } else if (tid < 2 * (TXv + 2) + 2 * TYv) {
        const int q = tid - 2 * (TXv + 2);
        hi = q < TYv ? 0 : TXv + 1;
        hj = 1 + (q % TYv);
    }
    // extra corner handled by thread `tid` (the TYv + 1 + TXv corners on the low-r / low-theta edges)
    int xci = -1, xcj = -1;
    if (tid < TYv + 1) { xci = 0; xcj = tid; }
    else if (tid < TYv + 1 + TXv) { xci = tid - TYv; xcj = 0; }

    // points outside the r / theta range: zero on the shell (their corners carry no flux), the
    // wrapped point on the periodic box (PER)
    auto fetch = [&](int gi, int gj, int kk) -> A {
        if (gi < 0 || gi >= nr || gj < 0 || gj >= nt) {
            if (!PER) return A(0);
            gi = wrap_phi(gi, nr);
            gj = wrap_phi(gj, nt);
        }
        return ld(cg.offset + (long long)wrap_phi(kk, np) * plane + (long long)gj * nr + gi);
    };
    auto fetch_coef = [&](int ci, int cj, int kk) -> Coef4<A> {
        int gi = t.i0 - 1 + ci, gj = t.j0 - 1 + cj;
        if (gi < 0 || gi >= nr || gj < 0 || gj >= nt) {
            if (!PER) return Coef4<A>{A(0), A(0), A(0), A(0)};
            gi = wrap_phi(gi, nr);
            gj = wrap_phi(gj, nt);
        }
        return load_coef<A, typename P::C>(coef + cg.offset + (long long)wrap_phi(kk, np) * plane + (long long)gj * nr + gi);
    };
    // Corner (ci, cj) of the (TXv+1) x (TYv+1) corner grid from cell planes `pa` (k) and `pb` (k+1).
    auto corner = [&](int cbuf, int pa, int pb, int ci, int cj, const Coef4<A>& c) {
        const A u000 = cell[pa][cj][ci], u100 = cell[pa][cj][ci + 1];
        const A u010 = cell[pa][cj + 1][ci], u110 = cell[pa][cj + 1][ci + 1];
        const A u001 = cell[pb][cj][ci], u101 = cell[pb][cj][ci + 1];
        const A u011 = cell[pb][cj + 1][ci], u111 = cell[pb][cj + 1][ci + 1];
        const A P00 = u001 + u000, M00 = u001 - u000;
        const A P10 = u101 + u100, M10 = u101 - u100;
        const A P01 = u011 + u010, M01 = u011 - u010;
        const A P11 = u111 + u110, M11 = u111 - u110;
        const A X = P11 - P00, Y = P10 - P01;
        const A Dr = X + Y, Dt = X - Y, Dp = (M00 + M01) + (M10 + M11);
        const A s = c.a * Dr + c.b * Dt + c.c * Dp;
        const A Qr = c.a * s, Qt = c.b * s, Qp = c.c * s;
        const A t1 = Qr + Qt, t2 = Qr - Qt;
        corn[cbuf][cj][ci] = Quad<A>{t1 + Qp, t1 - Qp, t2 + Qp, t2 - Qp};
    };

    // prologue: cell planes k0-1, k0 and corner plane k0-1 into shared memory
    if (inb) {
        cell[0][ty + 1][tx + 1] = fetch(i, j, t.k0 - 1);
        cell[1][ty + 1][tx + 1] = fetch(i, j, t.k0);
    }
    if (hi >= 0) {
        cell[0][hj][hi] = fetch(t.i0 - 1 + hi, t.j0 - 1 + hj, t.k0 - 1);
        cell[1][hj][hi] = fetch(t.i0 - 1 + hi, t.j0 - 1 + hj, t.k0);
    }
    {
        Coef4<A> c0{A(0), A(0), A(0), A(0)}, c1{A(0), A(0), A(0), A(0)};
        if (inb) c0 = fetch_coef(tx + 1, ty + 1, t.k0 - 1);
        if (xci >= 0) c1 = fetch_coef(xci, xcj, t.k0 - 1);
        __syncthreads();
        if (inb) corner(0, 0, 1, tx + 1, ty + 1, c0);
        if (xci >= 0) corner(0, 0, 1, xci, xcj, c1);
    }
    // register prefetch of the next plane: cell plane k+1, corner records of plane k, epilogue
    // operands of plane k
    A nu_own = inb ? fetch(i, j, t.k0 + 1) : A(0);
    A nu_halo = hi >= 0 ? fetch(t.i0 - 1 + hi, t.j0 - 1 + hj, t.k0 + 1) : A(0);
    Coef4<A> nc_own{A(0), A(0), A(0), A(0)};
    if (inb) nc_own = fetch_coef(tx + 1, ty + 1, t.k0);
    Coef4<A> nc_x{A(0), A(0), A(0), A(0)};
    if (xci >= 0) nc_x = fetch_coef(xci, xcj, t.k0);
    typename Epi::Pre npre{};
    if (own) npre = ep.prefetch(cg.offset + (long long)t.k0 * plane + (long long)j * nr + i);
    __syncthreads();

    int cb = 1;   // cell buffer holding plane k
    int kb = 0;   // corner buffer holding corner plane k-1
    for (int k = t.k0; k < t.k1; ++k) {
        const long long idx = cg.offset + (long long)k * plane + (long long)j * nr + i;
        if (inb) cell[cb ^ 1][ty + 1][tx + 1] = nu_own;
        if (hi >= 0) cell[cb ^ 1][hj][hi] = nu_halo;
        const Coef4<A> c_own = nc_own, c_x = nc_x;
        const typename Epi::Pre pre = npre;
        if (k + 1 < t.k1) {
            if (inb) nu_own = fetch(i, j, k + 2);
            if (hi >= 0) nu_halo = fetch(t.i0 - 1 + hi, t.j0 - 1 + hj, k + 2);
            if (inb) nc_own = fetch_coef(tx + 1, ty + 1, k + 1);
            if (xci >= 0) nc_x = fetch_coef(xci, xcj, k + 1);
            if (own) npre = ep.prefetch(idx + plane);
        }
        __syncthreads();
        if (inb) corner(kb ^ 1, cb, cb ^ 1, tx + 1, ty + 1, c_own);
        if (xci >= 0) corner(kb ^ 1, cb, cb ^ 1, xci, xcj, c_x);
        const A center = inb ? cell[cb][ty + 1][tx + 1] : A(0);
        __syncthreads();
        if (own) {
            const Quad<A>(&Cp)[TYv + 1][TXv + 1] = corn[kb];       // corner plane k-1
            const Quad<A>(&Cc)[TYv + 1][TXv + 1] = corn[kb ^ 1];   // corner plane k
            const A sum = (Cp[ty][tx].e0 - Cc[ty + 1][tx + 1].e0) + (Cc[ty][tx].e1 - Cp[ty + 1][tx + 1].e1)
                        + (Cp[ty + 1][tx].e2 - Cc[ty][tx + 1].e2) + (Cc[ty + 1][tx].e3 - Cp[ty][tx + 1].e3);
            ep.apply(idx, -sum, c_own.w, center, pre);
        }
        cb ^= 1;
        kb ^= 1;
    }
}

// One-problem conduction march kernel (the register-prefetch path).
template <class P, class Load, class Epi, bool PER = false>
__global__ void __launch_bounds__(NTHREADS)
tc_march(MarchGrid g, const Coef4<typename P::C>* __restrict__ coef, Load ld_in, Epi ep_in) {
    Epi ep = ep_in;
    ep.init();
    if (ep.skip()) return;
    Load ld = ld_in;
    ld.init();
    const TileIdx t = decode_tile(g);
    __shared__ TileSmem<P, TX, TY> sm;
    tc_tile<P, TX, TY, Load, Epi, PER>(g.c[0], t, coef, ld, ep, threadIdx.x + TX * threadIdx.y, sm);
    ep.finish();
}

// ---------------------------------------------------------------------------------------------
// Viscosity march kernel (all three components in one launch).  The 7-point stencil reuses
// little in a tile, so there is no shared-memory staging and no barrier: each thread walks its
// (r, theta) column along phi keeping planes k-1, k, k+1 of its own point in registers, reads
// the four in-plane neighbours (other threads' points, served by L1 / L2) and prefetches the
// next plane's operands one iteration ahead.
// ---------------------------------------------------------------------------------------------
template <class P, class Load, class Epi, bool PER>
__device__ __forceinline__ void visc_march_body(const MarchGrid& g, const Coef4<typename P::C>* __restrict__ coef,
                                                const Load& ld_in, const Epi& ep_in) {
    using A = typename P::A;
    using C = typename P::C;

    Epi ep = ep_in;
    ep.init();
    if (ep.skip()) return;
    Load ld = ld_in;
    ld.init();

    const TileIdx t = decode_tile(g);
    const CompGrid& cg = g.c[t.comp];
    const int nr = cg.nr, nt = cg.nt, np = cg.np;
    const long long plane = (long long)nr * nt;
    const int i = t.i0 + threadIdx.x, j = t.j0 + threadIdx.y;
    const bool own = (i < nr) && (j < nt);
    if (own) {
        // in-plane neighbours: absent past the r / theta ends of the shell, wrapped on the box (PER)
        const bool rm = i > 0 || PER, rp = i < nr - 1 || PER, tm = j > 0 || PER, tp = j < nt - 1 || PER;
        const int orm = PER && i == 0 ? nr - 1 : -1, orp = PER && i == nr - 1 ? -(nr - 1) : 1;
        const int otm = PER && j == 0 ? (nt - 1) * nr : -nr, otp = PER && j == nt - 1 ? -(nt - 1) * nr : nr;
        const long long col = cg.offset + (long long)j * nr + i;
        auto at = [&](int kk) -> long long {
            kk = kk < 0 ? kk + np : (kk >= np ? kk - np : kk);
            return col + (long long)kk * plane;
        };
        // in-plane operands of one phi plane (the point's own value travels separately)
        struct Plane { A urm, urp, utm, utp, crm, ctm; Coef4<A> c; };
        auto fetch = [&](long long idx) -> Plane {
            Plane q;
            q.urm = rm ? ld(idx + orm) : A(0);
            q.urp = rp ? ld(idx + orp) : A(0);
            q.utm = tm ? ld(idx + otm) : A(0);
            q.utp = tp ? ld(idx + otp) : A(0);
            q.c = load_coef<A, C>(coef + idx);
            q.crm = rm ? (A)__ldg(&coef[idx + orm].a) : A(0);
            q.ctm = tm ? (A)__ldg(&coef[idx + otm].b) : A(0);
            return q;
        };
        A ukm = ld(at(t.k0 - 1));
        A cpm = (A)__ldg(&coef[at(t.k0 - 1)].c);
        long long idx = at(t.k0);
        A uk = ld(idx);
        Plane cur = fetch(idx);
        A ukp = ld(at(t.k0 + 1));
        typename Epi::Pre pre = ep.prefetch(idx);
        for (int k = t.k0; k < t.k1; ++k) {
            Plane nxt{};
            A ukpp = A(0);
            typename Epi::Pre npre{};
            const long long idn = at(k + 1);
            if (k + 1 < t.k1) {
                nxt = fetch(idn);
                ukpp = ld(at(k + 2));
                npre = ep.prefetch(idn);
            }
            const A Au = cur.c.a * (cur.urp - uk) + cur.crm * (cur.urm - uk) + cur.c.b * (cur.utp - uk)
                       + cur.ctm * (cur.utm - uk) + cur.c.c * (ukp - uk) + cpm * (ukm - uk);
            ep.apply(idx, Au, cur.c.w, uk, pre);
            ukm = uk;
            uk = ukp;
            ukp = ukpp;
            cpm = cur.c.c;
            cur = nxt;
            pre = npre;
            idx = idn;
        }
    }
    ep.finish();
}

template <class P, class Load, class Epi, bool PER = false>
__global__ void __launch_bounds__(NTHREADS)
visc_march(MarchGrid g, const Coef4<typename P::C>* __restrict__ coef, Load ld, Epi ep) {
    visc_march_body<P, Load, Epi, PER>(g, coef, ld, ep);
}

// The same march with the register budget of 5 resident blocks per SM (48 registers): used where
// that fits without spilling and the extra block hides memory latency (the float32 PTL pass).
template <class P, class Load, class Epi, bool PER = false>
__global__ void __launch_bounds__(NTHREADS, 5)
visc_march_5(MarchGrid g, const Coef4<typename P::C>* __restrict__ coef, Load ld, Epi ep) {
    visc_march_body<P, Load, Epi, PER>(g, coef, ld, ep);
}

}  // namespace pb
