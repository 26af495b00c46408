// Launchers for one precision policy P; included by ops_f64.cu / ops_f32.cu / ops_b16.cu.
#pragma once

#include <cstdint>
#include <type_traits>

#include "cheb.cuh"
#include "epilogues.cuh"
#include "launch.h"
#include "march.cuh"
#include "march_tma.cuh"

namespace pb {

// Epilogues whose viscosity march runs with the 5-blocks-per-SM register budget (checked free of
// spills with -Xptxas -v): the float32 PTL pass.
template <class Epi> struct ViscCapped { static constexpr bool value = false; };
template <bool U1> struct ViscCapped<EpiF<PolF32, true, U1>> { static constexpr bool value = true; };

// Element-wise conversion between the caller's state type and the working precision.
template <typename From, typename To>
__global__ void convert_kernel(long long n, const From* in, To* out) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        out[t] = cvt<To>(ldg(in + t));
}

template <class P>
class OpsImpl : public Ops {
    using S = typename P::S;
    using C = typename P::C;
    using A = typename P::A;
    using E = typename P::E;
    using U = typename P::U;

    template <class Load, class Epi>
    static void march(Ctx& c, const void* coef, const Load& ld, const Epi& ep) {
        dim3 block(TX, TY);
        const Coef4<C>* cf = static_cast<const Coef4<C>*>(coef);
        const bool box = c.grid.c[0].periodic != 0;
        if (c.kind == PB_TC_ANISO) {
            if (box) tc_march<P, Load, Epi, true><<<c.grid.nblocks, block, 0, c.stream>>>(c.grid, cf, ld, ep);
            else tc_march<P, Load, Epi><<<c.grid.nblocks, block, 0, c.stream>>>(c.grid, cf, ld, ep);
        } else if constexpr (ViscCapped<Epi>::value) {
            if (box) visc_march_5<P, Load, Epi, true><<<c.grid.nblocks, block, 0, c.stream>>>(c.grid, cf, ld, ep);
            else visc_march_5<P, Load, Epi><<<c.grid.nblocks, block, 0, c.stream>>>(c.grid, cf, ld, ep);
        } else {
            if (box) visc_march<P, Load, Epi, true><<<c.grid.nblocks, block, 0, c.stream>>>(c.grid, cf, ld, ep);
            else visc_march<P, Load, Epi><<<c.grid.nblocks, block, 0, c.stream>>>(c.grid, cf, ld, ep);
        }
        PB_CUDA_TRY(cudaGetLastError());
    }

    // Conduction march on a plain state field through the TMA kernel when every array can be
    // described by a tensor map; otherwise the register-prefetch kernel.
    // float64 storage with a float32 stencil converts the halo box once per plane
    using StateField = typename std::conditional<(sizeof(S) > sizeof(A)), ConvField<P>, PlainField<P>>::type;

    template <class Epi>
    static void march_state(Ctx& c, const void* field, const void* const* cen, const Epi& ep) {
        if (c.kind == PB_TC_ANISO && c.use_tma) {
            using L = TmaLayout<P, Epi::NC, StateField>;
            const CompGrid& g = c.grid.c[0];
            TmaMaps maps;
            bool ok = tma_state_map(&maps.halo[0], field, sizeof(S), g.nr, g.nt, g.np, L::BXW, TY + 2) &&
                      tma_coef_map(&maps.coef, c.coef, sizeof(C), g.nr, g.nt, g.np, L::CBX, TY + 1);
            for (int a = 0; ok && a < Epi::NC; ++a)
                ok = tma_state_map(&maps.cen[a], cen[a], sizeof(S), g.nr, g.nt, g.np, TX, TY);
            if (ok) {
                const int smem = L::TOTAL + 128;
                // once per kernel instantiation (a function-local static: thread-safe initialisation)
                static const cudaError_t attr = cudaFuncSetAttribute(tc_march_tma<P, Epi, StateField>,
                                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
                PB_CUDA_TRY(attr);
                tc_march_tma<P, Epi, StateField><<<c.grid.nblocks, dim3(TX, TY), smem, c.stream>>>(c.grid, maps, ep, c.d_err);
                PB_CUDA_TRY(cudaGetLastError());
                return;
            }
        }
        march(c, c.coef, LoadState<P>{static_cast<const S*>(field)}, ep);
    }

    // PCG product q = S p through the TMA kernel, p assembled on chip from r, D^-1 and p_old;
    // false when the arrays cannot be described by tensor maps (the caller then uses tc_march).
    static bool pcg_spmv_tma(Ctx& c, const S* pold, const EpiPcgSpmv<P>& ep) {
        if (c.kind != PB_TC_ANISO || !c.use_tma) return false;
        using Fld = PcgField<P>;
        using L = TmaLayout<P, 0, Fld>;
        const CompGrid& g = c.grid.c[0];
        TmaMaps maps;
        const void* f[3] = {c.r, c.dinv, pold};
        bool ok = tma_coef_map(&maps.coef, c.coef_be, sizeof(C), g.nr, g.nt, g.np, L::CBX, TY + 1);
        for (int a = 0; ok && a < 3; ++a) ok = tma_state_map(&maps.halo[a], f[a], sizeof(S), g.nr, g.nt, g.np, L::BXW, TY + 2);
        if (!ok) return false;
        const int smem = L::TOTAL + 128;
        static const cudaError_t attr = cudaFuncSetAttribute(tc_march_tma<P, EpiPcgSpmv<P>, Fld>,
                                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        PB_CUDA_TRY(attr);
        tc_march_tma<P, EpiPcgSpmv<P>, Fld><<<c.grid.nblocks, dim3(TX, TY), smem, c.stream>>>(c.grid, maps, ep, c.d_err,
                                                                                             Fld{c.d_pcg, A(0), 0});
        PB_CUDA_TRY(cudaGetLastError());
        return true;
    }

    // low part of a float64 coefficient under a double-float policy (x = (float)x + lo), else 0
    static float lo_part(double x) { return P::DF ? (float)(x - (double)(float)x) : 0.f; }

    // A conduction march through the TMA kernel on field Fld (its NF arrays) with the epilogue's
    // point operands; false when an array cannot be described by a tensor map.
    template <class Epi, class Fld>
    static bool tma_march(Ctx& c, const void* coef, const void* const* fields, const void* const* cen, const Epi& ep,
                          const Fld& fld) {
        if (c.kind != PB_TC_ANISO || !c.use_tma) return false;
        using L = TmaLayout<P, Epi::NC, Fld>;
        const CompGrid& g = c.grid.c[0];
        TmaMaps maps;
        bool ok = tma_coef_map(&maps.coef, coef, sizeof(C), g.nr, g.nt, g.np, L::CBX, TY + 1);
        for (int a = 0; ok && a < Fld::NF; ++a) ok = tma_state_map(&maps.halo[a], fields[a], sizeof(S), g.nr, g.nt, g.np, L::BXW, TY + 2);
        for (int a = 0; ok && a < Epi::NC; ++a) ok = tma_state_map(&maps.cen[a], cen[a], sizeof(S), g.nr, g.nt, g.np, TX, TY);
        if (!ok) return false;
        const int smem = L::TOTAL + 128;
        static const cudaError_t attr = cudaFuncSetAttribute(tc_march_tma<P, Epi, Fld>,
                                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        PB_CUDA_TRY(attr);
        tc_march_tma<P, Epi, Fld><<<c.grid.nblocks, dim3(TX, TY), smem, c.stream>>>(c.grid, maps, ep, c.d_err, fld);
        PB_CUDA_TRY(cudaGetLastError());
        return true;
    }

    static void* ensure_cheb(Ctx& c, int i) {
        if (!c.cheb[i]) {
            void* p = nullptr;
            if (cudaMalloc(&p, (size_t)c.n * sizeof(S)) != cudaSuccess) {
                cudaGetLastError();
                throw Error{PB_ENOMEM, "cudaMalloc of a Chebyshev vector failed"};
            }
            c.cheb[i] = p;
        }
        return c.cheb[i];
    }

    // Chebyshev pass j (1 .. m-1) of the preconditioner
    template <int KIND, bool LAST>
    static void cheb_pass(Ctx& c, const ChebPlan& pl, int j, double dt) {
        S* r = static_cast<S*>(c.r);
        S* dinv = static_cast<S*>(c.dinv);
        S* out = static_cast<S*>(LAST ? c.cheb[0] : c.cheb[1 + (j + 1) % 2]);
        const S* y = static_cast<const S*>(c.cheb[1 + j % 2]);          // y_j (j >= 2)
        const S* yprev = static_cast<const S*>(c.cheb[1 + (j - 1) % 2]);   // y_{j-1} (j >= 3)
        EpiCheb<P, KIND, LAST> ep{r, dinv, KIND == 3 ? yprev : nullptr, out, (A)dt, (A)pl.c1[j], (A)pl.c2[j],
                                  (A)pl.inv_theta, c.d_pcg, static_cast<double*>(c.partials), c.counter,
                                  c.grid.nblocks, 0, {}};
        const void* cen[3] = {r, dinv, yprev};
        KScope ks(c.prof, c.stream, K_PCG_CHEB, nb(c, KIND == 1 ? 3 : (KIND == 2 ? 4 : 5), 4));
        if constexpr (KIND == 1) {
            const void* f[2] = {r, dinv};
            if (!tma_march(c, c.coef_be, f, cen, ep, ChebY1Field<P>{(A)pl.inv_theta}))
                march(c, c.coef_be, LoadChebY1<P>{r, dinv, (A)pl.inv_theta}, ep);
        } else {
            const void* f[1] = {y};
            if (!tma_march(c, c.coef_be, f, cen, ep, PlainField<P>{}))
                march(c, c.coef_be, LoadState<P>{y}, ep);
        }
    }

public:
    double cheb_bound(Ctx& c, double dt) override {
        const int blocks = reduce_blocks(c);
        cheb_bound_kernel<P><<<blocks, 256, 0, c.stream>>>(c.n, c.coef64, static_cast<const C*>(c.adiag), c.arow, dt,
                                                           static_cast<double*>(c.partials));
        max_partials_kernel<<<1, 256, 0, c.stream>>>(static_cast<const double*>(c.partials), blocks, c.d_scalar);
        PB_CUDA_TRY(cudaGetLastError());
        PB_CUDA_TRY(cudaMemcpyAsync(c.h_scalar, c.d_scalar, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
        PB_CUDA_TRY(cudaStreamSynchronize(c.stream));
        return *c.h_scalar;
    }

    void pcg_precond(Ctx& c, const ChebPlan& pl, double dt) override {
        for (int i = 0; i < 3; ++i) ensure_cheb(c, i);
        const int m = pl.m;
        for (int j = 1; j < m; ++j) {
            const bool last = j == m - 1;
            if (j == 1) last ? cheb_pass<1, true>(c, pl, j, dt) : cheb_pass<1, false>(c, pl, j, dt);
            else if (j == 2) last ? cheb_pass<2, true>(c, pl, j, dt) : cheb_pass<2, false>(c, pl, j, dt);
            else last ? cheb_pass<3, true>(c, pl, j, dt) : cheb_pass<3, false>(c, pl, j, dt);
        }
    }

    void pcg_iter_poly(Ctx& c, void* x, int parity, double dt, const ChebPlan& pl) override {
        S* pold = static_cast<S*>(c.p[parity]);
        S* pnew = static_cast<S*>(c.p[parity ^ 1]);
        const S* z = static_cast<const S*>(c.cheb[0]);
        EpiPcgSpmv<P> ep{pnew, static_cast<S*>(c.q), c.d_pcg, static_cast<double*>(c.partials), c.counter,
                         c.grid.nblocks, (A)dt};
        {
            KScope ks(c.prof, c.stream, K_PCG_SPMV, nb(c, 4, 4));
            const void* f[2] = {z, pold};
            if (!tma_march(c, c.coef_be, f, nullptr, ep, PolyPField<P>{c.d_pcg, A(0), 0}))
                march(c, c.coef_be, LoadPolyP<P>{z, pold, c.d_pcg, A(0), 0}, ep);
        }
        {
            const int blocks = reduce_blocks(c);
            KScope ks(c.prof, c.stream, K_PCG_UPDATE, nb(c, 6, 0));
            bool vec = false;
            if constexpr (std::is_same<S, float>::value && std::is_same<A, float>::value) {
                const uintptr_t a = reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(c.r) |
                                    reinterpret_cast<uintptr_t>(pnew) | reinterpret_cast<uintptr_t>(c.q);
                if ((a & 15) == 0) {
                    pcg_update_poly_f32x4_kernel<<<blocks, 256, 0, c.stream>>>(
                        c.n, static_cast<float*>(x), static_cast<float*>(c.r), pnew, static_cast<const float*>(c.q), c.d_pcg,
                        static_cast<double*>(c.partials), c.counter);
                    vec = true;
                }
            }
            if (!vec)
                pcg_update_poly_kernel<P><<<blocks, 256, 0, c.stream>>>(c.n, static_cast<S*>(x), static_cast<S*>(c.r), pnew,
                                                                        static_cast<const S*>(c.q), c.d_pcg,
                                                                        static_cast<double*>(c.partials), c.counter);
            PB_CUDA_TRY(cudaGetLastError());
        }
        pcg_precond(c, pl, dt);
    }

    bool supports_pcg() const override { return P::id == PB_FP64 || P::id == PB_FP32; }

    static double nb(const Ctx& c, double s_words, double c_words) {
        return (double)c.n * (s_words * sizeof(S) + c_words * sizeof(C));
    }

    void apply(Ctx& c, const void* u, void* F) override {
        KScope ks(c.prof, c.stream, K_APPLY, nb(c, 2, 4));
        EpiF<P, false, false> ep{static_cast<S*>(F), nullptr, A(0), nullptr, nullptr};
        march_state(c, u, nullptr, ep);
    }

    void y0_pass(Ctx& c, const void* u, void* y0, bool argmax, void* u1, double a) override {
        ArgMax* part = static_cast<ArgMax*>(c.partials);
        if (argmax) {
            PB_CUDA_TRY(cudaMemsetAsync(c.d_flag, 0, sizeof(int), c.stream));
            KScope ks(c.prof, c.stream, K_PTL_PASS, nb(c, u1 ? 3 : 2, 4));
            if (u1) {
                EpiF<P, true, true> ep{static_cast<S*>(y0), static_cast<S*>(u1), (A)a, part, c.d_flag};
                ep.al = lo_part(a);
                march_state(c, u, nullptr, ep);
            } else {
                EpiF<P, true, false> ep{static_cast<S*>(y0), nullptr, A(0), part, c.d_flag};
                march_state(c, u, nullptr, ep);
            }
        } else if (u1) {
            KScope ks(c.prof, c.stream, K_Y0_D1, nb(c, 3, 4));
            EpiF<P, false, true> ep{static_cast<S*>(y0), static_cast<S*>(u1), (A)a, nullptr, nullptr};
            ep.al = lo_part(a);
            march_state(c, u, nullptr, ep);
        } else {
            apply(c, u, y0);
        }
    }

    void ptl_finalize(Ctx& c, const void* u, const void* F) override {
        KScope ks(c.prof, c.stream, K_PTL_FINAL, (double)c.grid.nblocks * sizeof(ArgMax));
        ptl_finalize_kernel<P><<<1, kFinalizeThreads, 0, c.stream>>>(c.grid, static_cast<const S*>(u), static_cast<const S*>(F),
                                                        static_cast<const ArgMax*>(c.partials), c.grid.nblocks,
                                                        c.d_ptl, c.d_flag);
        PB_CUDA_TRY(cudaGetLastError());
    }

    void ptl_full(Ctx& c, const void* u, const void* F) override {
        const int blocks = reduce_blocks(c);
        {
            KScope ks(c.prof, c.stream, K_PTL_FULL, nb(c, 2, 0));
            ptl_full_kernel<P><<<blocks, 256, 0, c.stream>>>(c.grid, c.n, static_cast<const S*>(u),
                                                             static_cast<const S*>(F), static_cast<ArgMax*>(c.partials));
            PB_CUDA_TRY(cudaGetLastError());
        }
        ptl_full_finalize_kernel<<<1, kFinalizeThreads, 0, c.stream>>>(static_cast<const ArgMax*>(c.partials), blocks, c.d_ptl);
        PB_CUDA_TRY(cudaGetLastError());
    }

    void stage1(Ctx& c, const void* y0, void* d1, double a) override {
        const int blocks = reduce_blocks(c);
        KScope ks(c.prof, c.stream, K_STAGE1, nb(c, 2, 0));
        stage1_kernel<P><<<blocks, 256, 0, c.stream>>>(c.n, static_cast<const S*>(y0), static_cast<S*>(d1), (A)a);
        PB_CUDA_TRY(cudaGetLastError());
    }

    template <bool LAST>
    void stage2_t(Ctx& c, const void* y0, void* d1, const void* u0, void* out, double a1, const StageCoef& k) {
        KScope ks(c.prof, c.stream, K_STAGE, nb(c, 3, 4));
        const double cy = k.mu * a1 + k.ydt, cf = k.mdt * a1;
        EpiStage2<P, LAST> ep{static_cast<const S*>(u0), static_cast<S*>(d1), static_cast<S*>(out), (E)a1,
                              (E)cy, (E)cf, static_cast<const S*>(y0)};
        ep.al = lo_part(a1);
        ep.cyl = lo_part(cy);
        ep.cfl = lo_part(cf);
        const void* cen[1] = {u0};
        march_state(c, y0, cen, ep);
    }

    void stage2(Ctx& c, const void* y0, void* d1, const void* u0, void* out, double a1, const StageCoef& k) override {
        if (u0) stage2_t<true>(c, y0, d1, u0, out, a1, k);
        else stage2_t<false>(c, y0, d1, u0, out, a1, k);
    }

    template <bool KM2, bool LAST>
    void stage_t(Ctx& c, const void* dkm1, const void* dkm2, const void* u0, const void* y0, void* out,
                 const StageCoef& k) {
        EpiStage<P, KM2, LAST> ep{static_cast<const S*>(dkm2), static_cast<const S*>(y0), static_cast<const S*>(u0),
                                  static_cast<S*>(out), (E)k.mu, (E)k.nu, (E)k.mdt, (E)k.ydt,
                                  static_cast<const S*>(dkm1)};
        ep.mul = lo_part(k.mu);
        ep.nul = lo_part(k.nu);
        ep.mdtl = lo_part(k.mdt);
        ep.ydtl = lo_part(k.ydt);
        KScope ks(c.prof, c.stream, K_STAGE, nb(c, 3 + (KM2 ? 1 : 0) + (LAST ? 1 : 0), 4));
        const void* cen[3];
        int n = 0;
        cen[n++] = y0;
        if (KM2) cen[n++] = dkm2;
        if (LAST) cen[n++] = u0;
        march_state(c, dkm1, cen, ep);
    }

    void stage(Ctx& c, const void* dkm1, const void* dkm2, const void* u0, const void* y0, void* out,
               const StageCoef& k) override {
        if (dkm2) {
            if (u0) stage_t<true, true>(c, dkm1, dkm2, u0, y0, out, k);
            else stage_t<true, false>(c, dkm1, dkm2, u0, y0, out, k);
        } else {
            if (u0) stage_t<false, true>(c, dkm1, dkm2, u0, y0, out, k);
            else stage_t<false, false>(c, dkm1, dkm2, u0, y0, out, k);
        }
    }

    void pcg_init(Ctx& c, const void* x, const void* un, double dt) override {
        KScope ks(c.prof, c.stream, K_PCG_INIT, nb(c, 4, 5));
        EpiPcgInit<P> ep{static_cast<const S*>(un), static_cast<S*>(c.r), static_cast<S*>(c.dinv),
                         static_cast<const C*>(c.adiag), c.d_pcg, static_cast<double*>(c.partials),
                         c.counter, c.grid.nblocks, (A)dt};
        march(c, c.coef_be, LoadState<P>{static_cast<const S*>(x)}, ep);
    }

    void pcg_residual(Ctx& c, const void* x, const void* un, double dt) override {
        KScope ks(c.prof, c.stream, K_PCG_INIT, nb(c, 3, 4));
        EpiPcgInit<P, false> ep{static_cast<const S*>(un), static_cast<S*>(c.r), nullptr, nullptr, c.d_pcg,
                                static_cast<double*>(c.partials), c.counter, c.grid.nblocks, (A)dt};
        march(c, c.coef_be, LoadState<P>{static_cast<const S*>(x)}, ep);
    }

    void pcg_iter(Ctx& c, void* x, int parity, double dt) override {
        S* pold = static_cast<S*>(c.p[parity]);
        S* pnew = static_cast<S*>(c.p[parity ^ 1]);
        LoadPcgP<P> ld{static_cast<const S*>(c.r), static_cast<const S*>(c.dinv), pold, c.d_pcg, A(0), 0};
        EpiPcgSpmv<P> ep{pnew, static_cast<S*>(c.q), c.d_pcg, static_cast<double*>(c.partials), c.counter,
                         c.grid.nblocks, (A)dt};
        {
            KScope ks(c.prof, c.stream, K_PCG_SPMV, nb(c, 5, 4));
            if (!pcg_spmv_tma(c, pold, ep)) march(c, c.coef_be, ld, ep);
        }
        const int blocks = reduce_blocks(c);
        KScope ks(c.prof, c.stream, K_PCG_UPDATE, nb(c, 7, 0));
        bool vec = false;
        if constexpr (std::is_same<S, float>::value && std::is_same<A, float>::value) {
            const uintptr_t a = reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(c.r) |
                                reinterpret_cast<uintptr_t>(pnew) | reinterpret_cast<uintptr_t>(c.q) |
                                reinterpret_cast<uintptr_t>(c.dinv);
            if ((a & 15) == 0) {
                pcg_update_f32x4_kernel<<<blocks, 256, 0, c.stream>>>(
                    c.n, static_cast<float*>(x), static_cast<float*>(c.r), pnew, static_cast<const float*>(c.q),
                    static_cast<const float*>(c.dinv), c.d_pcg, static_cast<double*>(c.partials), c.counter);
                vec = true;
            }
        }
        if (!vec)
            pcg_update_kernel<P><<<blocks, 256, 0, c.stream>>>(c.n, static_cast<S*>(x), static_cast<S*>(c.r), pnew,
                                                               static_cast<const S*>(c.q), static_cast<const S*>(c.dinv),
                                                               c.d_pcg, static_cast<double*>(c.partials), c.counter);
        PB_CUDA_TRY(cudaGetLastError());
    }

    void* enter(Ctx& c, const void* u) override {
        if constexpr (std::is_same<U, S>::value) {
            return const_cast<void*>(u);
        } else {
            convert_kernel<U, S><<<reduce_blocks(c), 256, 0, c.stream>>>(c.n, static_cast<const U*>(u), static_cast<S*>(c.work));
            PB_CUDA_TRY(cudaGetLastError());
            return c.work;
        }
    }

    void leave(Ctx& c, const void* w, void* u) override {
        if constexpr (std::is_same<U, S>::value) {
            if (w != u) PB_CUDA_TRY(cudaMemcpyAsync(u, w, (size_t)c.n * sizeof(S), cudaMemcpyDeviceToDevice, c.stream));
        } else {
            convert_kernel<S, U><<<reduce_blocks(c), 256, 0, c.stream>>>(c.n, static_cast<const S*>(w), static_cast<U*>(u));
            PB_CUDA_TRY(cudaGetLastError());
        }
    }

    void to_f64(Ctx& c, const void* w, double* out) override {
        convert_kernel<S, double><<<reduce_blocks(c), 256, 0, c.stream>>>(c.n, static_cast<const S*>(w), out);
        PB_CUDA_TRY(cudaGetLastError());
    }

    void store_coefs(Ctx& c, const Coef4<double>* rec, const double* adiag) override;
};

template <class P>
__global__ void store_coefs_kernel(long long n, const Coef4<double>* rec, const double* adiag,
                                   Coef4<typename P::C>* out, Coef4<typename P::C>* out_be,
                                   typename P::C* adiag_out) {
    using C = typename P::C;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const Coef4<double> r = rec[t];
        out[t] = Coef4<C>{to_rec<C>(r.a), to_rec<C>(r.b), to_rec<C>(r.c), to_rec<C>(r.w)};
        // the Backward Euler record carries the mass M = 1/w instead of w
        out_be[t] = Coef4<C>{to_rec<C>(r.a), to_rec<C>(r.b), to_rec<C>(r.c), to_rec<C>(1.0 / r.w)};
        adiag_out[t] = to_rec<C>(adiag[t]);
    }
}

template <class P>
void OpsImpl<P>::store_coefs(Ctx& c, const Coef4<double>* rec, const double* adiag) {
    store_coefs_kernel<P><<<reduce_blocks(c), 256, 0, c.stream>>>(c.n, rec, adiag, static_cast<Coef4<C>*>(c.coef),
                                                                  static_cast<Coef4<C>*>(c.coef_be),
                                                                  static_cast<C*>(c.adiag));
    PB_CUDA_TRY(cudaGetLastError());
}

}  // namespace pb
