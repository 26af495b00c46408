// C ABI of libparabolic: context set-up, the PTL cycle loop (Sec. 2) around the super-time-
// stepping stage loop (Appendix A) or Backward Euler + PCG (Sec. 3.1), and the host-side
// float64 super-time-stepping coefficients.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <string>
#include <vector>

#include "launch.h"
#include "sts_coeffs.h"

namespace pb {
namespace {

thread_local std::string g_setup_error;

Ops* ops_of(const Ctx& c) {
    switch (c.prec) {
        case PB_FP64: return ops_f64();
        case PB_FP32: return ops_f32();
        case PB_FP64_STORE: return ops_f64s();
        default: return ops_b16();
    }
}

// ---- allocation helpers --------------------------------------------------------------------
void* dmalloc(size_t bytes) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error{PB_ENOMEM, std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e)};
    }
    return p;
}

void build_grid(Ctx& c) {
    MarchGrid& g = c.grid;
    g.ncomp = c.kind == PB_TC_ANISO ? 1 : 3;
    const bool box = c.geometry == PB_CARTESIAN_PERIODIC;
    int dims[3][3];
    if (c.kind == PB_TC_ANISO || box) {
        for (int a = 0; a < g.ncomp; ++a) {
            dims[a][0] = c.nr; dims[a][1] = c.nt; dims[a][2] = c.np;
        }
    } else {
        dims[0][0] = c.nr - 1; dims[0][1] = c.nt; dims[0][2] = c.np;
        dims[1][0] = c.nr; dims[1][1] = c.nt - 1; dims[1][2] = c.np;
        dims[2][0] = c.nr; dims[2][1] = c.nt; dims[2][2] = c.np;
    }
    long long tiles_total = 0;
    for (int a = 0; a < g.ncomp; ++a)
        tiles_total += (long long)((dims[a][0] + TX - 1) / TX) * ((dims[a][1] + TY - 1) / TY);
    // enough phi chunks for ~16 resident tiles per SM, each chunk at least 4 planes long
    const long long target = (long long)std::max(1, c.sm_count) * 16;
    int nchunk = (int)std::max(1LL, (target + tiles_total - 1) / tiles_total);
    nchunk = std::min(nchunk, std::max(1, c.np / 4));
    const int kchunk = (c.np + nchunk - 1) / nchunk;
    nchunk = (c.np + kchunk - 1) / kchunk;
    int64_t off = 0;
    int blocks = 0;
    for (int a = 0; a < g.ncomp; ++a) {
        CompGrid& cg = g.c[a];
        cg.nr = dims[a][0]; cg.nt = dims[a][1]; cg.np = dims[a][2];
        cg.tiles_r = (cg.nr + TX - 1) / TX;
        cg.tiles_t = (cg.nt + TY - 1) / TY;
        cg.kchunk = kchunk;
        cg.nchunk = nchunk;
        cg.offset = off;
        cg.block_begin = blocks;
        cg.periodic = box ? 1 : 0;
        off += (int64_t)cg.nr * cg.nt * cg.np;
        blocks += cg.tiles_r * cg.tiles_t * nchunk;
    }
    g.nblocks = blocks;
    c.n = off;
}

void free_ctx(Ctx& c) {
    cudaStreamSynchronize(c.stream);
    c.prof.release();
    free_shadow(c.shadow);
    c.shadow = nullptr;
    void* ptrs[] = {c.coef, c.coef_be, c.coef64, c.adiag, c.y0, c.buf[0], c.buf[1], c.buf[2], c.r, c.p[0],
                    c.p[1], c.q, c.dinv, c.partials, c.counter, c.d_pcg, c.d_scalar, c.d_flag, c.d_err,
                    c.spec, c.work};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c.s64) cudaFree(c.s64);
    if (c.arow) cudaFree(c.arow);
    for (void* p : c.cheb)
        if (p) cudaFree(p);
    for (double* p : c.geo)
        if (p) cudaFree(p);
    if (c.h_ptl) cudaFreeHost(c.h_ptl);
    if (c.h_pcg) cudaFreeHost(c.h_pcg);
    if (c.h_scalar) cudaFreeHost(c.h_scalar);
    if (c.h_err) cudaFreeHost(c.h_err);
    if (c.ev_ptl) cudaEventDestroy(c.ev_ptl);
}

// Second state buffer for speculated cycles, and the event the host waits on for a PTL result.
void* ensure_spec(Ctx& c) {
    if (!c.spec) c.spec = dmalloc((size_t)c.n * c.welem);
    return c.spec;
}

void ensure_pcg_buffers(Ctx& c) {
    if (c.r) return;
    const size_t bytes = (size_t)c.n * c.elem;
    c.r = dmalloc(bytes);
    c.p[0] = dmalloc(bytes);
    c.p[1] = dmalloc(bytes);
    c.q = dmalloc(bytes);
    c.dinv = dmalloc(bytes);
}

// Waits for the context's stream and reports a kernel whose bounded wait ran out.
void sync(Ctx& c) {
    PB_CUDA_TRY(cudaMemcpyAsync(c.h_err, c.d_err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    PB_CUDA_TRY(cudaStreamSynchronize(c.stream));
    c.prof.harvest();
    if (*c.h_err) {
        *c.h_err = 0;
        cudaMemsetAsync(c.d_err, 0, sizeof(int), c.stream);
        cudaStreamSynchronize(c.stream);
        throw Error{PB_ETIMEOUT, "a kernel's bounded wait for its TMA copies ran out"};
    }
}

template <class F>
int guarded(Ctx* c, F&& f) {
    try {
        f();
        if (c) c->err.clear();
        return PB_OK;
    } catch (const Error& e) {
        if (c) c->err = e.msg; else g_setup_error = e.msg;
        return e.code;
    } catch (const std::bad_alloc&) {
        if (c) c->err = "host allocation failed"; else g_setup_error = "host allocation failed";
        return PB_ENOMEM;
    }
}

pb_advance_opts resolve(const pb_advance_opts* o) {
    pb_advance_opts r;
    pb_advance_opts_init(&r);
    if (o) r = *o;
    if (r.max_cycles <= 0) r.max_cycles = 100000;
    if (!(r.ptl_floor >= 0.0)) r.ptl_floor = 1.0;
    if (!(r.rtol > 0.0)) r.rtol = 1e-10;
    if (r.max_iter < 0) r.max_iter = 100000;
    if (r.check_every <= 0) r.check_every = 8;
    if (!(r.inner_rtol > 0.0) || !(r.inner_rtol < 1.0)) r.inner_rtol = 1e-6;
    if (r.scheme != PB_RKL2 && r.scheme != PB_RKG2) throw Error{PB_EINVAL, "unknown scheme"};
    if (r.ptl_mode != PB_PTL_FMAX && r.ptl_mode != PB_PTL_FULL) throw Error{PB_EINVAL, "unknown ptl_mode"};
    if (r.precond != PB_PC_JACOBI && r.precond != PB_PC_CHEBYSHEV) throw Error{PB_EINVAL, "unknown precond"};
    if (r.precond == PB_PC_CHEBYSHEV && r.pc_degree <= 1) r.pc_degree = 3;
    if (r.pc_degree > 32) throw Error{PB_EINVAL, "pc_degree above 32"};
    if (r.dt_cycles == nullptr) r.n_forced = 0;
    if (r.n_forced < 0) throw Error{PB_EINVAL, "n_forced < 0"};
    return r;
}

void stats_begin(pb_stats* st, const Ctx& c) {
    if (!st) return;
    st->cycles = 0;
    st->status_cycle = -1;
    st->total_stages = 0;
    st->total_iters = 0;
    st->dt_explicit = c.dt_e;
    st->last_dt_ptl = std::numeric_limits<double>::quiet_NaN();
    st->fmax = std::numeric_limits<double>::quiet_NaN();
    st->k_index = -1;
    st->final_rel_residual = std::numeric_limits<double>::quiet_NaN();
    st->guess_used = 0;
}

void stats_cycle(pb_stats* st, double dt_c, int work, double dtp, long long k, double dt_full) {
    if (!st) return;
    const int c = st->cycles;
    if (c < st->cycle_capacity) {
        if (st->dt_cycle) st->dt_cycle[c] = dt_c;
        if (st->work_cycle) st->work_cycle[c] = work;
        if (st->dt_ptl_cycle) st->dt_ptl_cycle[c] = dtp;
        if (st->k_cycle) st->k_cycle[c] = k;
        if (st->dt_full_cycle) st->dt_full_cycle[c] = dt_full;
    }
    st->cycles = c + 1;
}

void check_operator(int kind, const pb_operator* op) {
    if (!op) throw Error{PB_EINVAL, "null operator"};
    if (op->kind != kind) throw Error{PB_EINVAL, "operator kind differs from the context's"};
    if (kind == PB_TC_ANISO) {
        if (!op->T0 || !op->n || !op->B[0] || !op->B[1] || !op->B[2]) throw Error{PB_EINVAL, "conduction needs T0, n, B"};
        if (!(op->C > 0.0)) throw Error{PB_EINVAL, "C must be > 0"};
    } else {
        for (int a = 0; a < 3; ++a)
            if (!op->rho[a] || !op->nu[a]) throw Error{PB_EINVAL, "viscosity needs rho[3], nu[3]"};
    }
}

// (Re)computes the float64 records, diag(A) and dt_E, and stores them in the context precision.
void update_coefficients(Ctx& c, const pb_operator& op) {
    // set-up reads the float64 inputs and writes the float64 and stored records once
    const double in_words = c.kind == PB_TC_ANISO ? 5.0 : 2.0;
    {
        KScope ks(c.prof, c.stream, K_SETUP, (double)c.n * (8.0 * in_words + 8.0 * 5 + 2.0 * 4 * (c.prec == PB_FP64 ? 8 : 4)));
        if (c.kind == PB_TC_ANISO) setup_tc(c, op, c.coef64, &c.dt_e);
        else setup_visc(c, op, c.coef64, &c.dt_e);
        ops_of(c)->store_coefs(c, c.coef64, c.s64);
    }
    mixed_refresh(c);      // the float32 / double-float shadow of mixed-precision BE, if built
    sync(c);
    if (!(c.dt_e > 0.0) || std::isinf(c.dt_e)) throw Error{PB_ENONFINITE, "dt_E is not a positive finite number"};
}

bool env_on(const char* name) {
    const char* e = getenv(name);
    return e && e[0] == '1';
}

// The next cycle's length (Sec. 2): n = ceil(t_rem / max(dt_PTL, floor)) cycles remain and the
// next one has t_rem / n; a quotient within 1e-12 of an integer takes the smaller n (the same
// rule as the stage counts), so a dt that is a whole multiple of dt_E gives that many cycles.
double cycle_length(double t_rem, double dt_ptl, double floor_dt) {
    const double dtl = std::max(dt_ptl, floor_dt);
    const double q = t_rem / dtl * kStageTie;
    const double n = q <= 1.0 ? 1.0 : std::ceil(q);
    return t_rem / n;
}

// Runs the PTL pass on u (y0 = F(u) in c.y0) and returns the result (host).
// PTL pass: F = L u into c.y0 with Eq. 5 at argmax |F|, and with `full` Eq. 4 over every pair.
PtlResult run_ptl(Ctx& c, Ops* ops, const void* u, bool full = false) {
    ops->y0_pass(c, u, c.y0, true, nullptr, 0.0);
    ops->ptl_finalize(c, u, c.y0);
    if (full) ops->ptl_full(c, u, c.y0);
    sync(c);                 // the finalisers write the result straight into mapped host memory
    return *c.h_ptl;
}

// The stages of one cycle of length dt_c (y0 = F(in) in c.y0) from `in` into `out`, in increment
// form d_k = u_k - u_0 (see EpiStage): stages 1 and 2 fused (d1 = mut_1 dt y0 in buf[0]), d_k in
// buf[(k-1) % 3], the last stage writes u_0 + d_s into out.  in == out is allowed: the last stage
// reads u_0 at its own point only.  Enqueue only: no host reads, no allocation.
void enqueue_stages(Ctx& c, Ops* ops, const Sts& co, double dt_c, const void* in, void* out) {
    const double a1 = co.mut[1] * dt_c;
    const StageCoef k2{co.mu[2], co.nu[2], co.mut[2] * dt_c, (co.mut[2] + co.gt[2]) * dt_c};
    if (co.s == 2) ops->stage2(c, c.y0, nullptr, in, out, a1, k2);
    else ops->stage2(c, c.y0, c.buf[0], nullptr, c.buf[1], a1, k2);
    for (int k = 3; k <= co.s; ++k) {
        const bool last = k == co.s;
        ops->stage(c, c.buf[(k - 2) % 3], c.buf[(k - 3) % 3], last ? in : nullptr, c.y0,
                   last ? out : c.buf[(k - 1) % 3],
                   StageCoef{co.mu[k], co.nu[k], co.mut[k] * dt_c, (co.mut[k] + co.gt[k]) * dt_c});
    }
}

// The Chebyshev preconditioner of a cycle: interval [b/30, b] with b = 1.05 x the Gershgorin
// bound of D^-1 S, and the coefficients of the three-term recurrence (cheb.cuh).
ChebPlan cheb_plan(double bound, int m) {
    ChebPlan pl;
    pl.m = m;
    const double b = 1.05 * bound, a = b / 30.0;
    const double theta = 0.5 * (b + a), delta = 0.5 * (b - a), sigma = theta / delta;
    pl.inv_theta = 1.0 / theta;
    double rho_prev = 1.0 / sigma;
    for (int j = 1; j < m; ++j) {
        const double rho = 1.0 / (2.0 * sigma - rho_prev);
        pl.c1[j] = rho * rho_prev;
        pl.c2[j] = 2.0 * rho / delta;
        rho_prev = rho;
    }
    return pl;
}

// Decides the next cycle length (Sec. 2): returns false when the step is complete.
struct CycleState {
    double dt, t_rem;
    int c;
};

}  // namespace
}  // namespace pb

using namespace pb;

extern "C" {

void pb_advance_opts_init(pb_advance_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->scheme = PB_RKL2;
    o->use_ptl = 1;
    o->max_cycles = 100000;
    o->ptl_floor = 1.0;
    o->dt_cycles = nullptr;
    o->n_forced = 0;
    o->rtol = 1e-10;
    o->max_iter = 100000;
    o->fixed_iters = 0;
    o->check_every = 8;
    o->judge_guess = 1;
    o->mixed_precision = 0;
    o->inner_rtol = 1e-6;
    o->ptl_mode = PB_PTL_FMAX;
    o->precond = PB_PC_JACOBI;
    o->pc_degree = 3;
}

const char* pb_status_string(int s) {
    switch (s) {
        case PB_OK: return "ok";
        case PB_EINVAL: return "invalid argument";
        case PB_ENOMEM: return "out of memory";
        case PB_ECUDA: return "CUDA error";
        case PB_ENOCONVERGE: return "PCG did not converge";
        case PB_EMAXCYCLES: return "too many PTL cycles";
        case PB_ENONFINITE: return "non-finite value";
        case PB_ETIMEOUT: return "device wait timed out";
        case PB_ENOTSUP: return "not supported";
        default: return "unknown status";
    }
}

const char* pb_last_error(const pb_ctx* h) {
    return h ? h->c.err.c_str() : g_setup_error.c_str();
}

int parabolic_setup(const pb_grid* g, const pb_operator* op, int32_t precision, void* stream, pb_ctx** out) {
    return guarded(nullptr, [&] {
        if (!g || !op || !out) throw Error{PB_EINVAL, "null argument"};
        *out = nullptr;
        if (g->geometry != PB_SPHERICAL && g->geometry != PB_CARTESIAN_PERIODIC) throw Error{PB_EINVAL, "unknown geometry"};
        if (g->geometry == PB_CARTESIAN_PERIODIC) {
            if (g->n_r < 3 || g->n_theta < 3 || g->n_phi < 3) throw Error{PB_EINVAL, "periodic box needs n_r, n_theta, n_phi >= 3"};
        } else {
            if (g->n_r < 2 || g->n_theta < 2 || g->n_phi < 3) throw Error{PB_EINVAL, "need n_r >= 2, n_theta >= 2, n_phi >= 3"};
            if (!g->r_face || !g->t_face) throw Error{PB_EINVAL, "null face array"};
            if (!(g->r_face[0] > 0.0)) throw Error{PB_EINVAL, "r_face[0] must be > 0"};
            for (int i = 0; i < g->n_r; ++i)
                if (!(g->r_face[i + 1] > g->r_face[i])) throw Error{PB_EINVAL, "r_face must increase"};
            if (!(g->t_face[0] >= 0.0) || !(g->t_face[g->n_theta] <= M_PI + 1e-12)) throw Error{PB_EINVAL, "t_face outside [0, pi]"};
            for (int j = 0; j < g->n_theta; ++j)
                if (!(g->t_face[j + 1] > g->t_face[j])) throw Error{PB_EINVAL, "t_face must increase"};
        }
        if ((long long)g->n_r * g->n_theta * g->n_phi > (1LL << 40)) throw Error{PB_EINVAL, "grid too large"};
        if (precision != PB_FP64 && precision != PB_FP32 && precision != PB_BF16_STORE && precision != PB_FP64_STORE)
            throw Error{PB_EINVAL, "bad precision"};
        if (op->kind != PB_TC_ANISO && op->kind != PB_VISC_ISO) throw Error{PB_EINVAL, "unknown operator kind"};
        check_operator(op->kind, op);
        int dev = 0;
        PB_CUDA_TRY(cudaGetDevice(&dev));
        pb_ctx* h = new pb_ctx();
        Ctx& c = h->c;
        try {
            c.kind = op->kind;
            c.prec = precision;
            c.elem = (precision == PB_FP64 || precision == PB_FP64_STORE) ? 8 : precision == PB_FP32 ? 4 : 2;
            c.welem = (precision == PB_FP64 || precision == PB_FP64_STORE) ? 8 : 4;
            c.stream = static_cast<cudaStream_t>(stream);
            c.nr = g->n_r; c.nt = g->n_theta; c.np = g->n_phi;
            c.geometry = g->geometry;
            PB_CUDA_TRY(cudaDeviceGetAttribute(&c.sm_count, cudaDevAttrMultiProcessorCount, dev));
            build_grid(c);
            const size_t csz = precision == PB_FP64 ? 8 : precision == PB_BF16_STORE ? 2 : 4;
            c.coef = dmalloc((size_t)c.n * 4 * csz);
            c.coef_be = dmalloc((size_t)c.n * 4 * csz);
            c.coef64 = static_cast<Coef4<double>*>(dmalloc((size_t)c.n * sizeof(Coef4<double>)));
            c.adiag = dmalloc((size_t)c.n * csz);
            c.y0 = dmalloc((size_t)c.n * c.welem);
            for (int b = 0; b < 3; ++b) c.buf[b] = dmalloc((size_t)c.n * c.welem);
            if (c.welem != c.elem) c.work = dmalloc((size_t)c.n * c.welem);
            c.partial_cap = std::max(c.grid.nblocks, 3 * reduce_blocks(c)) + 32;
            c.partials = dmalloc((size_t)c.partial_cap * 32);
            c.counter = static_cast<unsigned int*>(dmalloc(sizeof(unsigned int)));
            // the PTL result lives in mapped pinned host memory: the finalising kernels write it
            // there, so reading it back needs no copy in the stream
            PB_CUDA_TRY(cudaHostAlloc(&c.h_ptl, sizeof(PtlResult), cudaHostAllocMapped));
            PB_CUDA_TRY(cudaHostGetDevicePointer(reinterpret_cast<void**>(&c.d_ptl), c.h_ptl, 0));
            c.d_pcg = static_cast<PcgScalars*>(dmalloc(sizeof(PcgScalars)));
            c.d_scalar = static_cast<double*>(dmalloc(sizeof(double)));
            c.d_flag = static_cast<int*>(dmalloc(sizeof(int)));
            c.d_err = static_cast<int*>(dmalloc(sizeof(int)));
            PB_CUDA_TRY(cudaMallocHost(&c.h_err, sizeof(int)));
            *c.h_err = 0;
            PB_CUDA_TRY(cudaMemsetAsync(c.d_err, 0, sizeof(int), c.stream));
            {
                // the TMA kernel fills out-of-range halo points with zeros, so only the shell uses it
                const char* e = getenv("PB_DISABLE_TMA");
                c.use_tma = !(e && e[0] == '1') && c.geometry == PB_SPHERICAL;
            }
            PB_CUDA_TRY(cudaEventCreateWithFlags(&c.ev_ptl, cudaEventDisableTiming));
            PB_CUDA_TRY(cudaMallocHost(&c.h_pcg, sizeof(PcgScalars)));
            PB_CUDA_TRY(cudaMallocHost(&c.h_scalar, sizeof(double)));
            PB_CUDA_TRY(cudaMemsetAsync(c.counter, 0, sizeof(unsigned int), c.stream));
            PB_CUDA_TRY(cudaMemsetAsync(c.d_flag, 0, sizeof(int), c.stream));
            c.s64 = static_cast<double*>(dmalloc((size_t)c.n * sizeof(double)));
            c.arow = static_cast<double*>(dmalloc((size_t)c.n * sizeof(double)));
            setup_geometry(c, *g);
            update_coefficients(c, *op);
        } catch (...) {
            free_ctx(c);
            delete h;
            throw;
        }
        *out = h;
    });
}

int parabolic_update(pb_ctx* h, const pb_operator* op) {
    if (!h) return PB_EINVAL;
    Ctx& c = h->c;
    return guarded(&c, [&] {
        check_operator(c.kind, op);
        update_coefficients(c, *op);
    });
}

int pb_profile_enable(pb_ctx* h, int32_t on) {
    if (!h) return PB_EINVAL;
    Ctx& c = h->c;
    return guarded(&c, [&] {
        sync(c);
        c.prof.reset();
        c.prof.on = on != 0;
    });
}

int pb_profile_read(pb_ctx* h, pb_kernel_stat* out, int32_t cap, int32_t* count) {
    if (!h) return PB_EINVAL;
    Ctx& c = h->c;
    return guarded(&c, [&] {
        sync(c);
        int n = 0;
        for (int k = 0; k < K_NCLASS; ++k) {
            if (c.prof.launches[k] == 0) continue;
            if (out && n < cap) {
                pb_kernel_stat& s = out[n];
                std::memset(&s, 0, sizeof(s));
                std::snprintf(s.name, sizeof(s.name), "%s.%s", c.kind == PB_TC_ANISO ? "tc" : "visc", kclass_name(k));
                s.launches = c.prof.launches[k];
                s.timed_launches = c.prof.timed[k];
                s.total_ms = c.prof.ms[k];
                s.bytes = c.prof.bytes[k];
            }
            ++n;
        }
        if (count) *count = n;
    });
}

int parabolic_destroy(pb_ctx* h) {
    if (!h) return PB_OK;
    cudaStreamSynchronize(h->c.stream);
    free_ctx(h->c);
    delete h;
    return PB_OK;
}

int parabolic_state_size(const pb_ctx* h, int64_t* n, int32_t* elem) {
    if (!h) return PB_EINVAL;
    if (n) *n = h->c.n;
    if (elem) *elem = h->c.elem;
    return PB_OK;
}

int parabolic_dt_explicit(const pb_ctx* h, double* dt_e) {
    if (!h || !dt_e) return PB_EINVAL;
    *dt_e = h->c.dt_e;
    return PB_OK;
}

int parabolic_apply(pb_ctx* h, const void* u, void* F) {
    if (!h) return PB_EINVAL;
    Ctx& c = h->c;
    return guarded(&c, [&] {
        if (!u || !F) throw Error{PB_EINVAL, "null state pointer"};
        if (u == F) throw Error{PB_EINVAL, "u and F must not alias"};
        Ops* ops = ops_of(c);
        const void* wu = ops->enter(c, u);
        if (wu == u) {
            ops->apply(c, u, F);
        } else {           // bfloat16 storage: F in float32, then into the caller's bfloat16 array
            ops->apply(c, wu, c.y0);
            ops->leave(c, c.y0, F);
        }
        sync(c);
    });
}

int ptl_compute(pb_ctx* h, const void* u, double* dt_ptl, int64_t* k, double* fmax) {
    if (!h) return PB_EINVAL;
    Ctx& c = h->c;
    return guarded(&c, [&] {
        if (!u) throw Error{PB_EINVAL, "null state pointer"};
        Ops* ops = ops_of(c);
        const PtlResult r = run_ptl(c, ops, ops->enter(c, u));
        if (r.nonfinite) throw Error{PB_ENONFINITE, "non-finite F in the PTL pass"};
        if (dt_ptl) *dt_ptl = r.dt_ptl;
        if (k) *k = r.k;
        if (fmax) *fmax = r.fmax;
    });
}

int ptl_full_compute(pb_ctx* h, const void* u, double* dt_full, int64_t* cell, int32_t* direction) {
    if (!h) return PB_EINVAL;
    Ctx& c = h->c;
    return guarded(&c, [&] {
        if (!u) throw Error{PB_EINVAL, "null state pointer"};
        Ops* ops = ops_of(c);
        const PtlResult r = run_ptl(c, ops, ops->enter(c, u), true);
        if (r.nonfinite) throw Error{PB_ENONFINITE, "non-finite F in the PTL pass"};
        if (dt_full) *dt_full = r.dt_full;
        if (cell) *cell = r.key_full >= 0 ? r.key_full / 3 : -1;
        if (direction) *direction = r.key_full >= 0 ? (int32_t)(r.key_full % 3) : -1;
    });
}

int rkl2_advance_async(pb_ctx* h, void* u, double dt, const pb_advance_opts* opts) {
    if (!h) return PB_EINVAL;
    Ctx& c = h->c;
    return guarded(&c, [&] {
        const pb_advance_opts o = resolve(opts);
        if (!u) throw Error{PB_EINVAL, "null state pointer"};
        if (!(dt >= 0.0) || std::isinf(dt)) throw Error{PB_EINVAL, "dt must be finite and >= 0"};
        const bool forced = o.n_forced > 0;
        if (!forced && o.use_ptl)
            throw Error{PB_EINVAL, "the PTL needs a host round trip per cycle: use rkl2_advance, or a forced schedule"};
        Ops* ops = ops_of(c);
        const int n = forced ? o.n_forced : 1;
        for (int cycle = 0; cycle < n; ++cycle) {
            const double dt_c = forced ? o.dt_cycles[cycle] : dt;
            if (!(dt_c >= 0.0) || std::isinf(dt_c)) throw Error{PB_EINVAL, "cycle length must be finite and >= 0"};
        }
        void* wu = ops->enter(c, u);     // the caller's array, or the float32 working copy
        Sts co;
        for (int cycle = 0; cycle < n; ++cycle) {
            const double dt_c = forced ? o.dt_cycles[cycle] : dt;
            if (dt_c == 0.0) continue;
            make_sts(o.scheme, dt_c / c.dt_e, co);
            ops->apply(c, wu, c.y0);
            enqueue_stages(c, ops, co, dt_c, wu, wu);
        }
        if (wu != u) ops->leave(c, wu, u);
    });
}

int rkl2_advance(pb_ctx* h, void* u, double dt, const pb_advance_opts* opts, pb_stats* st) {
    if (!h) return PB_EINVAL;
    Ctx& c = h->c;
    stats_begin(st, c);
    int cycle = 0;
    void* cur = u;                  // holds the state of the last completed cycle
    const int rc = guarded(&c, [&] {
        const pb_advance_opts o = resolve(opts);
        if (!u) throw Error{PB_EINVAL, "null state pointer"};
        if (!(dt >= 0.0) || std::isinf(dt)) throw Error{PB_EINVAL, "dt must be finite and >= 0"};
        Ops* ops = ops_of(c);
        // the working state: u itself, or the float32 copy of a bfloat16-storage context's state
        void* const wu = ops->enter(c, u);
        cur = wu;
        const bool forced = o.n_forced > 0;
        const bool want_full = o.ptl_mode == PB_PTL_FULL || (st && st->dt_full_cycle);
        const double floor_dt = o.ptl_floor * c.dt_e;
        double t_rem = dt;
        Sts co;
        auto stages = [&](double dt_c, const void* in, void* out) { enqueue_stages(c, ops, co, dt_c, in, out); };
        auto take = [&](const PtlResult& r, double& dtp, double& dfull, long long& kk) {
            if (r.nonfinite) throw Error{PB_ENONFINITE, "non-finite F in the PTL pass"};
            dtp = o.ptl_mode == PB_PTL_FULL ? r.dt_full : r.dt_ptl;
            dfull = r.dt_full;
            kk = r.k;
            if (st) { st->last_dt_ptl = dtp; st->fmax = r.fmax; st->k_index = r.k; }
        };
        bool have_r = false;        // a PTL result of `cur` is at hand (y0 = F(cur) in c.y0)
        PtlResult pend{};
        for (cycle = 0;; ++cycle) {
            double dt_c, dtp = std::numeric_limits<double>::quiet_NaN(), dfull = dtp;
            long long kk = -1;
            bool y0_done = false, floored = false;
            if (forced) {
                if (cycle >= o.n_forced) break;
                dt_c = o.dt_cycles[cycle];
                if (!(dt_c >= 0.0) || std::isinf(dt_c)) throw Error{PB_EINVAL, "forced cycle length must be finite and >= 0"};
            } else {
                if (!(t_rem > 1e-12 * dt)) break;
                if (cycle >= o.max_cycles) throw Error{PB_EMAXCYCLES, "PTL cycle count above max_cycles"};
                if (o.use_ptl) {
                    const PtlResult r = have_r ? pend : run_ptl(c, ops, cur, want_full);
                    have_r = false;
                    take(r, dtp, dfull, kk);
                    dt_c = cycle_length(t_rem, dtp, floor_dt);
                    floored = !(dtp > floor_dt);
                    y0_done = true;
                } else {
                    dt_c = t_rem;
                }
            }
            make_sts(o.scheme, dt_c / c.dt_e, co);
            if (!y0_done) ops->apply(c, cur, c.y0);
            stages(dt_c, cur, cur);
            if (st) st->total_stages += co.s;
            stats_cycle(st, dt_c, co.s, dtp, kk, dfull);
            t_rem -= dt_c;
            // At the floor the next cycle most likely has the same length (t_rem / n, then
            // (t_rem - t_rem/n) / (n - 1)): its PTL pass and, speculatively, its stages are queued
            // into the other buffer before the host reads that PTL result, so the GPU does not
            // wait for the host.  The speculation is kept when the decided length matches.
            while (floored && t_rem > 1e-12 * dt && cycle + 1 < o.max_cycles) {
                ops->y0_pass(c, cur, c.y0, true, nullptr, 0.0);
                ops->ptl_finalize(c, cur, c.y0);
                if (want_full) ops->ptl_full(c, cur, c.y0);
                PB_CUDA_TRY(cudaEventRecord(c.ev_ptl, c.stream));
                void* nxt = cur == wu ? ensure_spec(c) : wu;
                stages(dt_c, cur, nxt);
                PB_CUDA_TRY(cudaEventSynchronize(c.ev_ptl));
                const PtlResult r = *c.h_ptl;
                double dtp2, dfull2;
                long long kk2;
                take(r, dtp2, dfull2, kk2);
                const double dt_c2 = cycle_length(t_rem, dtp2, floor_dt);
                if (!(std::fabs(dt_c2 - dt_c) <= 1e-12 * dt_c)) {   // not the speculated cycle
                    pend = r;
                    have_r = true;
                    break;
                }
                ++cycle;
                cur = nxt;
                if (st) st->total_stages += co.s;
                stats_cycle(st, dt_c, co.s, dtp2, kk2, dfull2);
                t_rem -= dt_c;
                floored = !(dtp2 > floor_dt);
            }
        }
        if (cur != u) {
            ops->leave(c, cur, u);
            cur = u;
        }
        sync(c);
    });
    if (rc != PB_OK && cur != u) {
        // the last completed cycle lives in the speculation buffer or the working copy: hand it back
        try {
            ops_of(c)->leave(c, cur, u);
        } catch (const Error&) {
        }
        cudaStreamSynchronize(c.stream);
    }
    if (rc != PB_OK && st) st->status_cycle = cycle;
    return rc;
}

int rkl2_advance_relag(pb_ctx* h, void* u, double dt, const pb_advance_opts* opts, const pb_operator* op,
                       pb_stats* st) {
    if (!h) return PB_EINVAL;
    Ctx& c = h->c;
    stats_begin(st, c);
    int cycle = 0;
    void* wu = nullptr;
    const int rc = guarded(&c, [&] {
        const pb_advance_opts o = resolve(opts);
        if (!u) throw Error{PB_EINVAL, "null state pointer"};
        if (!(dt >= 0.0) || std::isinf(dt)) throw Error{PB_EINVAL, "dt must be finite and >= 0"};
        if (c.kind != PB_TC_ANISO) throw Error{PB_EINVAL, "the per-cycle re-lag is for conduction contexts"};
        if (!op || op->kind != PB_TC_ANISO || !op->n || !op->B[0] || !op->B[1] || !op->B[2] || !(op->C > 0.0))
            throw Error{PB_EINVAL, "the re-lag needs the operator's n, B and C"};
        if (o.ptl_mode != PB_PTL_FMAX) throw Error{PB_EINVAL, "the re-lag cycles under Eq. 5"};
        Ops* ops = ops_of(c);
        wu = ops->enter(c, u);
        const bool forced = o.n_forced > 0;
        double t_rem = dt;
        Sts co;
        for (cycle = 0;; ++cycle) {
            if (forced) {
                if (cycle >= o.n_forced) break;
            } else {
                if (!(t_rem > 1e-12 * dt)) break;
                if (cycle >= o.max_cycles) throw Error{PB_EMAXCYCLES, "PTL cycle count above max_cycles"};
            }
            // the operator of this cycle: kappa = max(T, 0)^{5/2} from the current state, the
            // records and dt_E from it, frozen for the cycle
            ops->to_f64(c, wu, c.s64);
            pb_operator lag = *op;
            lag.T0 = c.s64;
            setup_tc(c, lag, c.coef64, &c.dt_e, true);
            ops->store_coefs(c, c.coef64, c.s64);
            mixed_refresh(c);
            sync(c);
            if (!(c.dt_e > 0.0) || std::isinf(c.dt_e)) throw Error{PB_ENONFINITE, "dt_E is not a positive finite number"};
            if (st) st->dt_explicit = c.dt_e;
            double dt_c, dtp = std::numeric_limits<double>::quiet_NaN();
            long long kk = -1;
            if (forced) {
                dt_c = o.dt_cycles[cycle];
                if (!(dt_c >= 0.0) || std::isinf(dt_c)) throw Error{PB_EINVAL, "forced cycle length must be finite and >= 0"};
                ops->apply(c, wu, c.y0);
            } else if (o.use_ptl) {
                const PtlResult r = run_ptl(c, ops, wu);
                if (r.nonfinite) throw Error{PB_ENONFINITE, "non-finite F in the PTL pass"};
                dtp = r.dt_ptl;
                kk = r.k;
                if (st) { st->last_dt_ptl = dtp; st->fmax = r.fmax; st->k_index = r.k; }
                dt_c = cycle_length(t_rem, dtp, o.ptl_floor * c.dt_e);
            } else {
                dt_c = t_rem;
                ops->apply(c, wu, c.y0);
            }
            make_sts(o.scheme, dt_c / c.dt_e, co);
            enqueue_stages(c, ops, co, dt_c, wu, wu);
            if (st) st->total_stages += co.s;
            stats_cycle(st, dt_c, co.s, dtp, kk, std::numeric_limits<double>::quiet_NaN());
            t_rem -= dt_c;
        }
        if (wu != u) ops->leave(c, wu, u);
        sync(c);
    });
    if (rc != PB_OK && wu && wu != u) {
        try {
            ops_of(c)->leave(c, wu, u);
        } catch (const Error&) {
        }
        cudaStreamSynchronize(c.stream);
    }
    if (rc != PB_OK && st) st->status_cycle = cycle;
    return rc;
}

int be_pcg_advance(pb_ctx* h, void* u, double dt, const pb_advance_opts* opts, const void* x0, pb_stats* st) {
    if (!h) return PB_EINVAL;
    Ctx& c = h->c;
    stats_begin(st, c);
    int cycle = 0;
    const int rc = guarded(&c, [&] {
        const pb_advance_opts o = resolve(opts);
        if (!u) throw Error{PB_EINVAL, "null state pointer"};
        if (!(dt >= 0.0) || std::isinf(dt)) throw Error{PB_EINVAL, "dt must be finite and >= 0"};
        Ops* ops = ops_of(c);
        if (!ops->supports_pcg()) throw Error{PB_ENOTSUP, "BE + PCG needs PB_FP64 or PB_FP32 contexts"};
        const bool cheb = o.precond == PB_PC_CHEBYSHEV;
        ensure_pcg_buffers(c);
        const bool forced = o.n_forced > 0;
        const bool want_full = o.ptl_mode == PB_PTL_FULL || (st && st->dt_full_cycle);
        const size_t bytes = (size_t)c.n * c.elem;
        double t_rem = dt;
        for (cycle = 0;; ++cycle) {
            double dt_c, dtp = std::numeric_limits<double>::quiet_NaN(), dfull = dtp;
            long long kk = -1;
            if (forced) {
                if (cycle >= o.n_forced) break;
                dt_c = o.dt_cycles[cycle];
                if (!(dt_c >= 0.0) || std::isinf(dt_c)) throw Error{PB_EINVAL, "forced cycle length must be finite and >= 0"};
            } else {
                if (!(t_rem > 1e-12 * dt)) break;
                if (cycle >= o.max_cycles) throw Error{PB_EMAXCYCLES, "PTL cycle count above max_cycles"};
                if (o.use_ptl) {
                    PtlResult r;
                    if (o.mixed_precision && c.prec == PB_FP64) {
                        // mixed precision: the decision on a float32 view of the state
                        mixed_ptl(c, u, want_full);
                        sync(c);
                        r = *c.h_ptl;
                    } else {
                        r = run_ptl(c, ops, u, want_full);
                    }
                    if (r.nonfinite) throw Error{PB_ENONFINITE, "non-finite F in the PTL pass"};
                    dtp = r.dt_ptl;
                    dfull = r.dt_full;
                    kk = r.k;
                    if (o.ptl_mode == PB_PTL_FULL) dtp = r.dt_full;
                    if (st) { st->last_dt_ptl = dtp; st->fmax = r.fmax; st->k_index = r.k; }
                    dt_c = cycle_length(t_rem, dtp, o.ptl_floor * c.dt_e);
                } else {
                    dt_c = t_rem;
                }
            }
            // u^n is kept in buf[0]: it is the right-hand side and the state restored on failure
            PB_CUDA_TRY(cudaMemcpyAsync(c.buf[0], u, bytes, cudaMemcpyDeviceToDevice, c.stream));
            PcgScalars& hs = *c.h_pcg;
            std::memset(&hs, 0, sizeof(hs));
            hs.tol2 = o.rtol * o.rtol;
            hs.max_iter = o.max_iter;
            hs.fixed = o.fixed_iters > 0 ? o.fixed_iters : 0;
            hs.dt = dt_c;
            const PcgScalars hs0 = hs;
            // mixed precision on conduction: the residuals that drive the refinements in
            // double-float arithmetic on the float32 pipes (about 48 bits), and a stop accepted only
            // once the float64 residual confirms it (PB_MIXED_FP64_RESIDUAL=1: float64 throughout)
            const bool df_residual = o.mixed_precision && c.prec == PB_FP64 && o.fixed_iters <= 0 &&
                                     c.kind == PB_TC_ANISO && !env_on("PB_MIXED_FP64_RESIDUAL");
            // iterative refinement (mixed precision): its outer residuals need no D^-1
            const bool refine = o.mixed_precision && c.prec == PB_FP64 && o.fixed_iters <= 0;
            bool exact = true;      // the residual at hand is the float64 one
            auto init = [&](bool want_exact = false) {
                *c.h_pcg = hs0;
                PB_CUDA_TRY(cudaMemcpyAsync(c.d_pcg, c.h_pcg, sizeof(PcgScalars), cudaMemcpyHostToDevice, c.stream));
                exact = want_exact || !df_residual;
                if (!exact) mixed_residual(c, u, c.buf[0], dt_c);
                else if (refine) ops->pcg_residual(c, u, c.buf[0], dt_c);
                else ops->pcg_init(c, u, c.buf[0], dt_c);
                PB_CUDA_TRY(cudaMemcpyAsync(c.h_pcg, c.d_pcg, sizeof(PcgScalars), cudaMemcpyDeviceToHost, c.stream));
                sync(c);
                return c.h_pcg->rr;
            };
            if (cycle == 0 && x0) {
                // the previous-step state is the fallback and the judge of a given guess
                const double rr_prev = o.judge_guess ? init() : 0.0;
                PB_CUDA_TRY(cudaMemcpyAsync(u, x0, bytes, cudaMemcpyDeviceToDevice, c.stream));
                const double rr_x0 = init();
                if (o.judge_guess && !(rr_x0 < rr_prev)) {
                    PB_CUDA_TRY(cudaMemcpyAsync(u, c.buf[0], bytes, cudaMemcpyDeviceToDevice, c.stream));
                    init();
                } else if (st) {
                    st->guess_used = 1;
                }
            } else {
                init();
            }
            ChebPlan plan;
            if (cheb) {
                plan = cheb_plan(ops->cheb_bound(c, dt_c), o.pc_degree);
                if (!refine) ops->pcg_precond(c, plan, dt_c);      // z_0 = P r_0 and <r_0, z_0>
            }
            if (refine) {
                // iterative refinement: float64 residual (the set-up pass above) and float32
                // corrections until r.r <= rtol^2 b.b
                long long inner = 0;
                int refine = 0;
                for (;;) {
                    const PcgScalars now = *c.h_pcg;
                    if (now.done == 2) break;
                    if (now.rr <= now.tol2 * now.bb) {
                        if (!exact) {       // confirm the stop on the float64 residual
                            init(true);
                            continue;
                        }
                        c.h_pcg->done = 1;
                        break;
                    }
                    if (refine >= 64 || inner >= o.max_iter) {
                        c.h_pcg->done = 3;
                        break;
                    }
                    // the last refinement solves only as far as the outer test still needs, with a
                    // factor 4 of margin for the float32 rounding of the correction
                    double tau = o.inner_rtol;
                    const double need = 0.25 * std::sqrt(now.tol2 * now.bb / now.rr);
                    const bool last = need > tau;
                    if (last) tau = std::min(need, 0.5);
                    int status = 0;
                    inner += mixed_inner(c, u, dt_c, tau, o.max_iter - inner, o.check_every, &status,
                                         cheb ? &plan : nullptr);
                    ++refine;
                    if (status == 2) {
                        c.h_pcg->done = 2;
                        break;
                    }
                    // after a correction meant to meet the outer test, the float64 residual decides
                    // at once (it would confirm the double-float one anyway)
                    init(last && status == 0);
                }
                c.h_pcg->iter = inner;
            } else {
                int parity = 0;
                for (;;) {
                    PB_CUDA_TRY(cudaMemcpyAsync(c.h_pcg, c.d_pcg, sizeof(PcgScalars), cudaMemcpyDeviceToHost, c.stream));
                    sync(c);
                    if (c.h_pcg->done) break;
                    for (int m = 0; m < o.check_every; ++m) {
                        if (cheb) ops->pcg_iter_poly(c, u, parity, dt_c, plan);
                        else ops->pcg_iter(c, u, parity, dt_c);
                        parity ^= 1;
                    }
                }
            }
            const PcgScalars r = *c.h_pcg;
            if (st) {
                st->total_iters += r.iter;
                st->final_rel_residual = r.bb > 0 ? std::sqrt(r.rr / r.bb) : 0.0;
            }
            if (r.done != 1) {
                PB_CUDA_TRY(cudaMemcpyAsync(u, c.buf[0], bytes, cudaMemcpyDeviceToDevice, c.stream));
                sync(c);
                if (r.done == 2) throw Error{PB_ENONFINITE, "PCG breakdown or non-finite scalar"};
                throw Error{PB_ENOCONVERGE, "PCG reached max_iter without meeting rtol"};
            }
            stats_cycle(st, dt_c, (int)r.iter, dtp, kk, dfull);
            t_rem -= dt_c;
        }
        sync(c);
    });
    if (rc != PB_OK && st) st->status_cycle = cycle;
    return rc;
}

}  // extern "C"
