// Conduction march kernel with a TMA pipeline (the production path on sm_103a).
//
// Same stencil and epilogues as tc_march (march.cuh), but every global operand of a phi plane --
// the input field with its halo, the corner records and the epilogue's point operands -- arrives
// by cp.async.bulk.tensor into a ring of D shared-memory slots, tracked by one mbarrier per slot.
// One elected thread keeps D-1 planes of loads in flight; out-of-range halo points (r_min,
// r_max, the poles) come back as zeros from the TMA bounds handling, and phi wraps by issuing
// the wrapped plane index.  The x (r) box origin is rounded down by HX points so that its byte
// offset is 16-byte aligned.
//
// Slot q of a block holds plane k0 - 1 + q; iteration k (plane k) needs slots k-k0+1 (plane k:
// field, corners k+1/2, point operands) and k-k0+2 (plane k+1: field).  Every wait is bounded:
// if a copy never lands the block records the failure in *err, waits (bounded) for its other
// copies and returns.
//
// The field is either one array (PlainField) or, for the PCG product, assembled per plane from
// several arrays (PcgField): once a slot has landed the block forms the field on the whole halo
// box into a buffer of that slot that only ordinary stores write, so the TMA destinations are
// never written by the threads.
#pragma once

#include <type_traits>

#include "march.cuh"
#include "tma.cuh"

namespace pb {

template <typename S> struct HaloPad { static constexpr int value = 16 / (int)sizeof(S); };

constexpr int kSlots = 3;

__host__ __device__ constexpr int align128(int b) { return (b + 127) & ~127; }

// The field of the conduction product: one array read as it is.
template <class P>
struct PlainField {
    static constexpr int NF = 1;
    static constexpr bool CENTER_RAW = true;     // the centre comes from the landed array
    using FT = typename P::S;                    // element type the stencil reads
    __device__ void init() {}
    __device__ void combine(unsigned char*, int, int, FT*) const {}
};

// One array stored wider than the stencil arithmetic (float64 storage, float32 stencil): the
// halo box is converted once per plane instead of once per corner that reads it.
template <class P>
struct ConvField {
    using A = typename P::A;
    using S = typename P::S;
    static constexpr int NF = 1;
    static constexpr bool CENTER_RAW = true;
    using FT = A;
    __device__ void init() {}
    __device__ void combine(unsigned char* base, int, int n, A* dst) const {
        const S* f = reinterpret_cast<const S*>(base);
        for (int e = threadIdx.x + TX * threadIdx.y; e < n; e += NTHREADS) dst[e] = cvt<A>(f[e]);
    }
};

// The PCG search direction p = z + beta p_old with z = D^-1 r rounded to the state precision,
// formed from the arrays r, D^-1 and p_old exactly as the register path does (Sec. 3.1 PCG).
template <class P>
struct PcgField {
    using A = typename P::A;
    using S = typename P::S;
    static constexpr int NF = 3;
    static constexpr bool CENTER_RAW = false;    // the centre is the assembled p
    using FT = S;
    const PcgScalars* sc;
    A beta;
    int first;
    __device__ void init() {
        beta = (A)sc->beta;
        first = sc->first;
    }
    // src: NF arrays of n points, each at `pitch` bytes from the previous; dst: n points
    __device__ void combine(unsigned char* base, int pitch, int n, S* dst) const {
        const S* r = reinterpret_cast<const S*>(base);
        const S* di = reinterpret_cast<const S*>(base + pitch);
        const S* po = reinterpret_cast<const S*>(base + 2 * pitch);
        for (int e = threadIdx.x + TX * threadIdx.y; e < n; e += NTHREADS) {
            const A z = cvt<A>(cvt<S>(cvt<A>(di[e]) * cvt<A>(r[e])));
            dst[e] = cvt<S>(first ? z : z + beta * cvt<A>(po[e]));
        }
    }
};

template <class P, int NC, class Field = PlainField<P>>
struct TmaLayout {
    using S = typename P::S;
    using C = typename P::C;
    using A = typename P::A;
    static constexpr int NF = Field::NF;
    // a buffer of the assembled / converted field when the stencil does not read the landed array
    static constexpr bool ASSEMBLED = NF > 1 || !std::is_same<typename Field::FT, S>::value;
    static constexpr int HX = HaloPad<S>::value;
    static constexpr int BXW = TX + 2 * HX;                              // halo box width (points)
    static constexpr int U_BYTES = (TY + 2) * BXW * (int)sizeof(S);
    static constexpr int U_PITCH = align128(U_BYTES);
    static constexpr int F_BYTES = (TY + 2) * BXW * (int)sizeof(typename Field::FT);
    // records: a 4-D box of 4 words x (TX + 1) x (TY + 1) corners; bfloat16 records (8 bytes, a
    // 4-word row of 8 bytes is below TMA's 16-byte minimum) travel as one 8-byte element each in a
    // 3-D box whose x origin is rounded down by one record (16-byte aligned) and whose width
    // TX + 2 keeps the row a multiple of 16 bytes
    static constexpr bool CPACK = sizeof(C) == 2;
    static constexpr int CBX = CPACK ? TX + 2 : TX + 1;    // records per landed row
    static constexpr int CSHIFT = CPACK ? 1 : 0;           // landed position of corner ci is ci + CSHIFT
    static constexpr int C_BYTES = (TY + 1) * CBX * 4 * (int)sizeof(C);
    static constexpr int E_BYTES = TY * TX * (int)sizeof(S);
    static constexpr int U_OFF = 0;
    static constexpr int C_OFF = NF * U_PITCH;
    static constexpr int E_OFF = C_OFF + align128(C_BYTES);
    static constexpr int P_OFF = E_OFF + NC * align128(E_BYTES);         // assembled field
    static constexpr int FIELD_OFF = ASSEMBLED ? P_OFF : U_OFF;
    static constexpr int SLOT = P_OFF + (ASSEMBLED ? align128(F_BYTES) : 0);
    static constexpr int TX_BYTES = NF * U_BYTES + C_BYTES + NC * E_BYTES;   // bytes a slot's copies deliver
    static constexpr int CW = TX + 2;                                    // corner row pitch
    static constexpr int CORN_OFF = kSlots * SLOT;
    static constexpr int CORN_BYTES = 4 * (TY + 1) * CW * (int)sizeof(A);   // one corner plane
    static constexpr int BAR_OFF = align128(CORN_OFF + CORN_BYTES);
    static constexpr int TOTAL = BAR_OFF + kSlots * 8 + 16;
};

// The march of one tile t: planes [t.k0, t.k1) of its (r, theta) tile, every epilogue call made.
// Returns false when a copy never landed (the block has recorded it in *err, drained its other
// copies and must stop).  smem: the block's 128-byte-aligned TMA layout; tid: the linear thread
// index (TX x TY threads).  The mbarriers are initialised on entry and invalidated on exit, so a
// persistent block can march tile after tile.
template <class P, class Epi, class Field>
__device__ __forceinline__ bool tma_march_tile(const CompGrid& cg, const TileIdx& t, const TmaRefs& m, Epi& ep,
                                               const Field& fld, int* err, unsigned char* smem, int tid) {
    using S = typename P::S;
    using C = typename P::C;
    using A = typename P::A;
    using L = TmaLayout<P, Epi::NC, Field>;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
    int* abort_flag = reinterpret_cast<int*>(smem + L::BAR_OFF + kSlots * 8);
    A* corn = reinterpret_cast<A*>(smem + L::CORN_OFF);

    const int nr = cg.nr, nt = cg.nt, np = cg.np;
    const long long plane = (long long)nr * nt;
    const int tx = tid % TX, ty = tid / TX;
    const int i = t.i0 + tx, j = t.j0 + ty;
    const bool own = (i < nr) && (j < nt);
    const int nplanes = t.k1 - t.k0 + 2;       // planes k0-1 .. k1

    int xci = -1, xcj = -1;                    // extra corner of this thread (low-r / low-theta edge)
    if (tid < TY + 1) { xci = 0; xcj = tid; }
    else if (tid < TY + 1 + TX) { xci = tid - TY; xcj = 0; }

    auto slot = [&](int q) -> unsigned char* { return smem + (q % kSlots) * L::SLOT; };
    auto issue = [&](int q) {
        unsigned char* s = slot(q);
        uint64_t* bar = bars + (q % kSlots);
        int z = t.k0 - 1 + q;
        z = z < 0 ? z + np : (z >= np ? z - np : z);
        mbar_expect_tx(bar, L::TX_BYTES);
#pragma unroll
        for (int f = 0; f < Field::NF; ++f) tma_load_3d(s + L::U_OFF + f * L::U_PITCH, m.halo[f], t.i0 - L::HX, t.j0 - 1, z, bar);
        if constexpr (L::CPACK) tma_load_3d(s + L::C_OFF, m.coef, t.i0 - 2, t.j0 - 1, z, bar);
        else tma_load_4d(s + L::C_OFF, m.coef, 0, t.i0 - 1, t.j0 - 1, z, bar);
#pragma unroll
        for (int a = 0; a < Epi::NC; ++a) tma_load_3d(s + L::E_OFF + a * align128(L::E_BYTES), m.cen[a], t.i0, t.j0, z, bar);
    };
    // all threads wait for slot q; returns false (in every thread) if the copy never landed
    auto wait = [&](int q) -> bool {
        if (!mbar_wait(bars + (q % kSlots), (q / kSlots) & 1)) *abort_flag = 1;
        __syncthreads();
        if (*abort_flag != 0) return false;
        if constexpr (L::ASSEMBLED) {
            fld.combine(slot(q) + L::U_OFF, L::U_PITCH, (TY + 2) * L::BXW,
                        reinterpret_cast<typename Field::FT*>(slot(q) + L::P_OFF));
            __syncthreads();
        }
        return true;
    };
    auto bail = [&](int issued, int waited) {
        if (tid == 0) {
            atomicExch(err, 1);
            for (int q = waited; q < issued; ++q) mbar_wait(bars + (q % kSlots), (q / kSlots) & 1);
            for (int b = 0; b < kSlots; ++b) mbar_inval(bars + b);
        }
        __syncthreads();
    };
    using FT = typename Field::FT;
    auto field = [&](int q) -> const FT* { return reinterpret_cast<const FT*>(slot(q) + L::FIELD_OFF); };
    // corner (ci, cj) of plane z = k0-1+q from the field of planes z (f0) and z+1 (f1) and the
    // records of slot q (cr0)
    auto corner = [&](const FT* f0, const FT* f1, const C* cr0, int ci, int cj) -> A {
        const C* cr = cr0 + 4 * (cj * L::CBX + ci + L::CSHIFT);
        const A ca = cvt<A>(cr[0]), cb = cvt<A>(cr[1]), cc = cvt<A>(cr[2]), cw = cvt<A>(cr[3]);
        const int o = cj * L::BXW + ci - 1 + L::HX;
        const A u000 = cvt<A>(f0[o]), u100 = cvt<A>(f0[o + 1]);
        const A u010 = cvt<A>(f0[o + L::BXW]), u110 = cvt<A>(f0[o + L::BXW + 1]);
        const A u001 = cvt<A>(f1[o]), u101 = cvt<A>(f1[o + 1]);
        const A u011 = cvt<A>(f1[o + L::BXW]), u111 = cvt<A>(f1[o + L::BXW + 1]);
        const A P00 = u001 + u000, M00 = u001 - u000;
        const A P10 = u101 + u100, M10 = u101 - u100;
        const A P01 = u011 + u010, M01 = u011 - u010;
        const A P11 = u111 + u110, M11 = u111 - u110;
        const A X = P11 - P00, Y = P10 - P01;
        const A Dr = X + Y, Dt = X - Y, Dp = (M00 + M01) + (M10 + M11);
        const A s = ca * Dr + cb * Dt + cc * Dp;
        const A Qr = ca * s, Qt = cb * s, Qp = cc * s;
        const A t1 = Qr + Qt, t2 = Qr - Qt;
        A* cp = corn + cj * L::CW + ci;
        cp[0 * (TY + 1) * L::CW] = t1 + Qp;
        cp[1 * (TY + 1) * L::CW] = t1 - Qp;
        cp[2 * (TY + 1) * L::CW] = t2 + Qp;
        cp[3 * (TY + 1) * L::CW] = t2 - Qp;
        return cw;
    };

    if (tid == 0) {
        *abort_flag = 0;
        for (int b = 0; b < kSlots; ++b) mbar_init(bars + b, 1);
        fence_mbar_init();
    }
    __syncthreads();
    int issued = 0;
    if (tid == 0)
        for (; issued < kSlots && issued < nplanes; ++issued) issue(issued);
    issued = min(kSlots, nplanes);

    auto recs = [&](int q) -> const C* { return reinterpret_cast<const C*>(slot(q) + L::C_OFF); };
    // corner plane k0-1 from slots 0 and 1
    if (!wait(0) || !wait(1)) { bail(issued, 0); return false; }
    corner(field(0), field(1), recs(0), tx + 1, ty + 1);
    if (xci >= 0) corner(field(0), field(1), recs(0), xci, xcj);
    __syncthreads();
    if (tid == 0 && issued < nplanes) issue(issued);
    if (issued < nplanes) ++issued;

    // One corner plane lives in shared memory at a time: the entries of plane k-1/2 that the
    // cell of plane k needs (its four low-phi corners) are kept in registers (e0..e3) from the
    // iteration that read plane k-1/2 as its high-phi side; the barrier inside wait() orders
    // those reads before the next plane's corners overwrite the buffer.
    constexpr int EP = (TY + 1) * L::CW;          // stride between the four quad entries
    const A* cb = corn + ty * L::CW + tx;
    A e0 = A(0), e1 = A(0), e2 = A(0), e3 = A(0);
    if (own) {
        e0 = cb[0 * EP]; e1 = cb[1 * EP + L::CW + 1]; e2 = cb[2 * EP + L::CW]; e3 = cb[3 * EP + 1];
    }
    for (int k = t.k0; k < t.k1; ++k) {
        const int q = k - t.k0 + 1;
        if (!wait(q + 1)) { bail(issued, q + 1); return false; }
        const FT* f0 = field(q);
        const FT* f1 = field(q + 1);
        const C* cr0 = recs(q);
        const A w = corner(f0, f1, cr0, tx + 1, ty + 1);
        if (xci >= 0) corner(f0, f1, cr0, xci, xcj);
        // the centre and the point operands go to the epilogue at the stage-recurrence precision E
        using R = typename P::E;
        const R center = Field::CENTER_RAW
                             ? cvt<R>(reinterpret_cast<const S*>(slot(q) + L::U_OFF)[(ty + 1) * L::BXW + tx + L::HX])
                             : cvt<R>(reinterpret_cast<const typename Field::FT*>(slot(q) + L::FIELD_OFF)[(ty + 1) * L::BXW + tx + L::HX]);
        auto cen = [&](int a) -> R {
            return a < Epi::NC ? cvt<R>(reinterpret_cast<const S*>(slot(q) + L::E_OFF + a * align128(L::E_BYTES))[ty * TX + tx])
                               : R(0);
        };
        const R c0 = cen(0), c1 = cen(1), c2 = cen(2);
        __syncthreads();
        // slot q is no longer read: refill it with plane k0-1+q+kSlots
        if (tid == 0 && issued < nplanes) issue(issued);
        if (issued < nplanes) ++issued;
        if (own) {
            // the eight corners of the cell: planes k-1/2 (registers) and k+1/2 (the buffer)
            const A sum = (e0 - cb[0 * EP + L::CW + 1]) + (cb[1 * EP] - e1) + (e2 - cb[2 * EP + 1]) + (cb[3 * EP + L::CW] - e3);
            e0 = cb[0 * EP]; e1 = cb[1 * EP + L::CW + 1]; e2 = cb[2 * EP + L::CW]; e3 = cb[3 * EP + 1];
            const long long idx = cg.offset + (long long)k * plane + (long long)j * nr + i;
            ep.apply_c(idx, -sum, w, center, c0, c1, c2);
        }
    }
    // every copy issued has been waited for (the last iteration waited for the last plane)
    if (tid == 0)
        for (int b = 0; b < kSlots; ++b) mbar_inval(bars + b);
    return true;
}

template <class P, class Epi, class Field = PlainField<P>>
__global__ void __launch_bounds__(NTHREADS)
tc_march_tma(MarchGrid g, const __grid_constant__ TmaMaps maps, Epi ep_in, int* err, Field fld = Field{}) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations are kept 128-byte aligned (the launch adds 128 bytes of slack)
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    Epi ep = ep_in;
    ep.init();
    if (ep.skip()) return;
    fld.init();
    const TmaRefs m{{&maps.halo[0], &maps.halo[1], &maps.halo[2]}, &maps.coef, {&maps.cen[0], &maps.cen[1], &maps.cen[2]}};
    if (!tma_march_tile<P>(g.c[0], decode_tile(g), m, ep, fld, err, smem, threadIdx.x + TX * threadIdx.y)) return;
    ep.finish();
}

}  // namespace pb
