// Host-side kernel launchers, one implementation per precision policy (see ops_*.cu).
#pragma once

#include "common.cuh"

namespace pb {

// d_k = mu d_{k-1} + nu d_{k-2} + mdt F(d_{k-1}) + ydt y0   (increment form, see EpiStage)
struct StageCoef { double mu, nu, mdt, ydt; };

// The Chebyshev preconditioner of one Backward Euler cycle (see cheb.cuh): degree m, 1/theta, and
// the coefficients c1[j] = rho_j rho_{j-1}, c2[j] = 2 rho_j / delta of passes j = 1 .. m-1.
struct ChebPlan {
    int m = 0;
    double inv_theta = 0.0;
    double c1[32] = {}, c2[32] = {};
};

class Ops {
public:
    virtual ~Ops() {}
    // F = L u over the whole state
    virtual void apply(Ctx& c, const void* u, void* F) = 0;
    // y0 = L u, with the PTL arg-max partials (argmax = true) or the fused stage-1 increment
    // d1 = a y0 (d1 != nullptr)
    virtual void y0_pass(Ctx& c, const void* u, void* y0, bool argmax, void* d1, double a) = 0;
    // Eq. 5 at argmax |F|; result in c.d_ptl
    virtual void ptl_finalize(Ctx& c, const void* u, const void* F) = 0;
    // Eq. 4 over every pair of face neighbours of (u, F = L u) into c.d_ptl->dt_full / key_full
    virtual void ptl_full(Ctx& c, const void* u, const void* F) = 0;
    // d1 = a y0
    virtual void stage1(Ctx& c, const void* y0, void* d1, double a) = 0;
    // stages 1 and 2 fused (EpiStage2): from y0, writes d1 (when u0 == nullptr) and d2 into out,
    // or u0 + d2 into out when u0 != nullptr (s = 2)
    virtual void stage2(Ctx& c, const void* y0, void* d1, const void* u0, void* out, double a1,
                        const StageCoef& k) = 0;
    // one STS stage k >= 2 on increments; dkm2 == nullptr means d_{k-2} = 0 (k = 2); u0 !=
    // nullptr marks the last stage, which writes u0 + d_s into out
    virtual void stage(Ctx& c, const void* dkm1, const void* dkm2, const void* u0, const void* y0,
                       void* out, const StageCoef& k) = 0;
    // PCG: set-up from x (in place) and u^n; one SpMV + update iteration
    virtual void pcg_init(Ctx& c, const void* x, const void* un, double dt) = 0;
    // r = b - S x with <r, r>, <b, b> and the stopping decision only (no D^-1, no <r, D^-1 r>):
    // the outer residual of mixed-precision Backward Euler
    virtual void pcg_residual(Ctx& c, const void* x, const void* un, double dt) = 0;
    virtual void pcg_iter(Ctx& c, void* x, int parity, double dt) = 0;
    // Chebyshev-preconditioned PCG: the bound b of the spectrum of D^-1 S for step dt (host
    // value); z = P r with <r, z> and beta; one iteration (product, update, preconditioner)
    virtual double cheb_bound(Ctx& c, double dt) = 0;
    virtual void pcg_precond(Ctx& c, const ChebPlan& pl, double dt) = 0;
    virtual void pcg_iter_poly(Ctx& c, void* x, int parity, double dt, const ChebPlan& pl) = 0;
    // The state the kernels work on: the caller's array itself, or, under bfloat16 storage, the
    // context's float32 working copy (c.work) filled from it
    virtual void* enter(Ctx& c, const void* u) = 0;
    // Hands a working state back to the caller's array u (a conversion under bfloat16 storage,
    // otherwise a copy when the two differ)
    virtual void leave(Ctx& c, const void* work, void* u) = 0;
    // converts the float64 coefficient records into the context's storage precision
    virtual void store_coefs(Ctx& c, const Coef4<double>* rec, const double* adiag) = 0;
    // a working state widened to float64 (the lagged temperature of a per-cycle coefficient update)
    virtual void to_f64(Ctx& c, const void* work, double* out) = 0;
    virtual bool supports_pcg() const = 0;
};

Ops* ops_f64();
Ops* ops_f32();
Ops* ops_b16();
Ops* ops_f64s();   // PolF64S: float64 storage and recurrence, float32 stencil

// set-up kernels (float64), see setup.cu.  setup_tc / setup_visc leave diag(A) in c.s64.
void setup_geometry(Ctx& c, const pb_grid& g);
// clamp: kappa = max(T0, 0)^{5/2} (T0 may be c.s64 itself)
void setup_tc(Ctx& c, const pb_operator& op, Coef4<double>* rec, double* dt_e, bool clamp = false);
void setup_visc(Ctx& c, const pb_operator& op, Coef4<double>* rec, double* dt_e);

int reduce_blocks(const Ctx& c);   // grid size of the element-wise reduction kernels

// mixed-precision Backward Euler (mixed.cu)
Ctx& mixed_shadow(Ctx& c);
void mixed_refresh(Ctx& c);            // the shadow's records from the current float64 ones
void mixed_residual(Ctx& c, const void* x, const void* un, double dt);   // conduction, double-float
void free_shadow(Ctx* s);
void mixed_ptl(Ctx& c, const void* u, bool full);    // the PTL pass on a float32 view (result in c.h_ptl)
// plan: Chebyshev-preconditioned inner solves (nullptr: point-Jacobi)
long long mixed_inner(Ctx& c, void* x, double dt, double inner_rtol, long long max_iter, int check_every, int* status,
                      const ChebPlan* plan = nullptr);

}  // namespace pb
