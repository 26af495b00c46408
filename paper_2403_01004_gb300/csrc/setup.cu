// Set-up of the frozen operator coefficients (lagged kappa, Sec. 2) in float64 on the device:
// geometry, the packed per-point records, diag(A) and the Gershgorin bound that gives dt_E.
#include <cmath>
#include <vector>

#include "launch.h"
#include "reduce.cuh"

namespace pb {

namespace {

// kappa = T0^{5/2}; with clamp, max(T0, 0)^{5/2} (the lagged diffusivity of a state that may
// undershoot zero; kap may alias T0)
__global__ void kappa_kernel(long long n, const double* T0, double* kap, bool clamp) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const double T = clamp ? fmax(T0[t], 0.0) : T0[t];
        kap[t] = T * T * sqrt(T);          // T0^{5/2}
    }
}

struct TCArgs {
    int nr, nt, np;
    double dphi, C;
    const double* rf;
    const double* tf;
    const double* kap;
    const double* n;
    const double* B0;
    const double* B1;
    const double* B2;
    Coef4<double>* rec;
};

// phi planes per thread in the record kernels: a thread owns one (r, theta) column and a chunk of
// planes, so the metric factors (independent of phi; cosines, sines, divisions in float64) are
// formed once per chunk, not once per point
constexpr int kPlaneChunk = 32;

// Record of point [i,j,k]: ahat of corner (i+1/2, j+1/2, k+1/2) and w = C/(n V) of cell (i,j,k).
//   ahat = sqrt(W kappa_c) (h_r b_r, h_t b_t, h_p b_p) / 4,  kappa_c = mean of the 8 cells,
//   h_r = 1/(rc[i+1]-rc[i]), h_t = 1/(rf[i+1] (tc[j+1]-tc[j])), h_p = 1/(rf[i+1] sin tf[j+1] dphi),
//   W = rf[i+1]^2 (rc[i+1]-rc[i]) sin tf[j+1] (tc[j+1]-tc[j]) dphi, b = B/|B| at the corner.
__global__ void tc_coef_kernel(TCArgs a) {
    const long long pl = (long long)a.nr * a.nt;
    const int nchunk = (a.np + kPlaneChunk - 1) / kPlaneChunk;
    const long long total = pl * nchunk;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < total; w += (long long)gridDim.x * blockDim.x) {
        const long long col = w % pl;
        const int q = (int)(w / pl);
        const int i = (int)(col % a.nr);
        const int j = (int)(col / a.nr);
        const double V = (a.rf[i + 1] * a.rf[i + 1] * a.rf[i + 1] - a.rf[i] * a.rf[i] * a.rf[i]) / 3.0
                       * (cos(a.tf[j]) - cos(a.tf[j + 1])) * a.dphi;
        const bool corner = i < a.nr - 1 && j < a.nt - 1;
        double hr = 0.0, ht = 0.0, hp = 0.0, W = 0.0;
        if (corner) {
            const double rci = 0.5 * (a.rf[i] + a.rf[i + 1]), rcp = 0.5 * (a.rf[i + 1] + a.rf[i + 2]);
            const double tci = 0.5 * (a.tf[j] + a.tf[j + 1]), tcp = 0.5 * (a.tf[j + 1] + a.tf[j + 2]);
            const double drc = rcp - rci, dtc = tcp - tci;
            const double rfc = a.rf[i + 1], stf = sin(a.tf[j + 1]);
            hr = 1.0 / drc;
            ht = 1.0 / (rfc * dtc);
            hp = 1.0 / (rfc * stf * a.dphi);
            W = rfc * rfc * drc * (stf * dtc) * a.dphi;
        }
        const long long r0 = (long long)j * a.nr + i, r1 = (long long)(j + 1) * a.nr + i;
        const int k_end = min(a.np, (q + 1) * kPlaneChunk);
        for (int k = q * kPlaneChunk; k < k_end; ++k) {
            const long long t = (long long)k * pl + col;
            Coef4<double> r{0.0, 0.0, 0.0, a.C / (a.n[t] * V)};
            if (corner) {
                const int k1 = (k + 1) % a.np;
                const long long b0 = (long long)k * pl, b1 = (long long)k1 * pl;
                const double kc = (a.kap[b0 + r0] + a.kap[b0 + r0 + 1] + a.kap[b0 + r1] + a.kap[b0 + r1 + 1]
                                 + a.kap[b1 + r0] + a.kap[b1 + r0 + 1] + a.kap[b1 + r1] + a.kap[b1 + r1 + 1]) / 8.0;
                const double br = a.B0[t], bt = a.B1[t], bp = a.B2[t];
                const double bm = sqrt(br * br + bt * bt + bp * bp);
                const double root = sqrt(W * kc);
                r.a = root * hr * (br / bm) / 4.0;
                r.b = root * ht * (bt / bm) / 4.0;
                r.c = root * hp * (bp / bm) / 4.0;
            }
            a.rec[t] = r;
        }
    }
}

// Periodic box of unit cells (h = 1, W = V = 1), every corner present: record of point [i,j,k]
// is ahat = sqrt(kappa_c) b / 4 of corner (i+1/2, j+1/2, k+1/2), kappa_c the mean of its 8 cells
// (all indices wrap), and w = C / n.
__global__ void tc_coef_box_kernel(TCArgs a) {
    const long long n = (long long)a.nr * a.nt * a.np;
    const long long pl = (long long)a.nr * a.nt;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % a.nr);
        const long long q = t / a.nr;
        const int j = (int)(q % a.nt);
        const int k = (int)(q / a.nt);
        const int i1 = (i + 1) % a.nr, j1 = (j + 1) % a.nt, k1 = (k + 1) % a.np;
        const long long b0 = (long long)k * pl, b1 = (long long)k1 * pl;
        const long long r0 = (long long)j * a.nr, r1 = (long long)j1 * a.nr;
        const double kc = (a.kap[b0 + r0 + i] + a.kap[b0 + r0 + i1] + a.kap[b0 + r1 + i] + a.kap[b0 + r1 + i1]
                         + a.kap[b1 + r0 + i] + a.kap[b1 + r0 + i1] + a.kap[b1 + r1 + i] + a.kap[b1 + r1 + i1]) / 8.0;
        const double br = a.B0[t], bt = a.B1[t], bp = a.B2[t];
        const double bm = sqrt(br * br + bt * bt + bp * bp);
        const double root = sqrt(kc);
        a.rec[t] = Coef4<double>{root * (br / bm) / 4.0, root * (bt / bm) / 4.0, root * (bp / bm) / 4.0, a.C / a.n[t]};
    }
}

// Row of A at a cell from its 8 corners: A = -sum_c g_c g_c^T, g_c(p) = sigma(p) . ahat_c.
// Writes diag(A) and the block maximum of w sum_j |A_ij| (the Gershgorin bound of L).
__global__ void __launch_bounds__(256) tc_rows_kernel(int nr, int nt, int np, int periodic, const Coef4<double>* rec,
                                                      double* adiag, double* rowsum, double* part) {
    const long long n = (long long)nr * nt * np;
    const long long pl = (long long)nr * nt;
    double gmax = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % nr);
        const long long q = t / nr;
        const int j = (int)(q % nt);
        const int k = (int)(q / nt);
        double acc[27];
#pragma unroll
        for (int o = 0; o < 27; ++o) acc[o] = 0.0;
#pragma unroll
        for (int p = 0; p < 8; ++p) {
            const int pi = p & 1, pj = (p >> 1) & 1, pk = p >> 2;
            int ci = i - pi, cj = j - pj;
            const int ck = (k - pk + np) % np;
            if (ci < 0 || cj < 0) {
                if (!periodic) continue;
                ci = (ci + nr) % nr;
                cj = (cj + nt) % nt;
            }
            const Coef4<double> c = rec[(long long)ck * pl + (long long)cj * nr + ci];
            // g(q) = sigma(q) . ahat for the corner's 8 cells, from the 4 (r, theta) sign sums
            const double e[4] = {-c.a - c.b, c.a - c.b, -c.a + c.b, c.a + c.b};
            double g[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) g[q] = e[q & 3] + (q >= 4 ? c.c : -c.c);
            const double gp = g[p];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int qi = q & 1, qj = (q >> 1) & 1, qk = q >> 2;
                const int o = (qi - pi + 1) + 3 * (qj - pj + 1) + 9 * (qk - pk + 1);
                acc[o] -= gp * g[q];
            }
        }
        double s = 0.0;
#pragma unroll
        for (int o = 0; o < 27; ++o) s += fabs(acc[o]);
        adiag[t] = acc[13];
        rowsum[t] = s;
        gmax = fmax(gmax, rec[t].w * s);
    }
    gmax = warp_max(gmax);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = gmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = red[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
        part[blockIdx.x] = m;
    }
}

__global__ void max_finalize_kernel(const double* part, int n, double* out) {
    double m = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) m = fmax(m, part[b]);
    m = warp_max(m);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = red[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) x = fmax(x, red[w]);
        *out = 2.0 / x;
    }
}

struct ViscArgs {
    int nr, nt, np;          // this component's point counts
    double dphi;
    const double* pr;        // point radii [nr]
    const double* er;        // control-volume radial bounds [nr+1]
    const double* pt;        // point colatitudes [nt]
    const double* et;        // control-volume colatitude bounds [nt+1]
    const double* rho;
    const double* nu;
    Coef4<double>* rec;
};

// Record of point [i,j,k]: c_f = A_f nu_f rho_f / d_f on its +r, +theta, +phi faces (means of the
// two points for nu and rho; zero past the last r / theta point) and w = 1/(rho V).  One thread
// per (r, theta) column and chunk of phi planes, as for conduction.
__global__ void visc_coef_kernel(ViscArgs a) {
    const long long pl = (long long)a.nr * a.nt;
    const int nchunk = (a.np + kPlaneChunk - 1) / kPlaneChunk;
    const long long total = pl * nchunk;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < total; w += (long long)gridDim.x * blockDim.x) {
        const long long col = w % pl;
        const int q = (int)(w / pl);
        const int i = (int)(col % a.nr);
        const int j = (int)(col / a.nr);
        const double dcos = cos(a.et[j]) - cos(a.et[j + 1]);
        const double dr2 = (a.er[i + 1] * a.er[i + 1] - a.er[i] * a.er[i]) / 2.0;
        const double V = (a.er[i + 1] * a.er[i + 1] * a.er[i + 1] - a.er[i] * a.er[i] * a.er[i]) / 3.0 * dcos * a.dphi;
        double gr = 0.0, gt = 0.0;   // A_f / d_f of the +r and +theta faces
        if (i < a.nr - 1) {
            const double A = a.er[i + 1] * a.er[i + 1] * dcos * a.dphi;
            const double d = a.pr[i + 1] - a.pr[i];
            gr = A / d;
        }
        if (j < a.nt - 1) {
            const double A = dr2 * sin(a.et[j + 1]) * a.dphi;
            const double d = a.pr[i] * (a.pt[j + 1] - a.pt[j]);
            gt = A / d;
        }
        const double gp = (dr2 * (a.et[j + 1] - a.et[j])) / (a.pr[i] * sin(a.pt[j]) * a.dphi);
        const int k_end = min(a.np, (q + 1) * kPlaneChunk);
        for (int k = q * kPlaneChunk; k < k_end; ++k) {
            const long long t = (long long)k * pl + col;
            const double nu0 = a.nu[t], rho0 = a.rho[t];
            Coef4<double> r{0.0, 0.0, 0.0, 1.0 / (rho0 * V)};
            if (i < a.nr - 1) r.a = gr * ((0.5 * (nu0 + a.nu[t + 1])) * (0.5 * (rho0 + a.rho[t + 1])));
            if (j < a.nt - 1) r.b = gt * ((0.5 * (nu0 + a.nu[t + a.nr])) * (0.5 * (rho0 + a.rho[t + a.nr])));
            const long long tk = (long long)((k + 1) % a.np) * pl + col;
            r.c = gp * ((0.5 * (nu0 + a.nu[tk])) * (0.5 * (rho0 + a.rho[tk])));
            a.rec[t] = r;
        }
    }
}

// Periodic box of unit cells: every component on the full grid, c_f = nu_f rho_f on the +r,
// +theta, +phi faces (means of the two points, indices wrapping; A_f = d_f = 1), w = 1/rho.
__global__ void visc_coef_box_kernel(ViscArgs a) {
    const long long n = (long long)a.nr * a.nt * a.np;
    const long long pl = (long long)a.nr * a.nt;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % a.nr);
        const long long q = t / a.nr;
        const int j = (int)(q % a.nt);
        const int k = (int)(q / a.nt);
        const long long base = t - i - (long long)j * a.nr;     // start of plane k
        const long long tr = base + (long long)j * a.nr + (i + 1) % a.nr;
        const long long tt = base + (long long)((j + 1) % a.nt) * a.nr + i;
        const long long tp = (long long)((k + 1) % a.np) * pl + (t - (long long)k * pl);
        const double nu0 = a.nu[t], rho0 = a.rho[t];
        auto face = [&](long long o) { return (0.5 * (nu0 + a.nu[o])) * (0.5 * (rho0 + a.rho[o])); };
        a.rec[t] = Coef4<double>{face(tr), face(tt), face(tp), 1.0 / rho0};
    }
}

// diag(A) = -sum of the six face coefficients; Gershgorin bound of L = 2 w sum_f c_f.
__global__ void __launch_bounds__(256) visc_rows_kernel(int nr, int nt, int np, int periodic, const Coef4<double>* rec,
                                                        double* adiag, double* rowsum, double* part) {
    const long long n = (long long)nr * nt * np;
    const long long pl = (long long)nr * nt;
    double gmax = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % nr);
        const long long q = t / nr;
        const int j = (int)(q % nt);
        const int k = (int)(q / nt);
        const Coef4<double> c = rec[t];
        double s = c.a + c.b + c.c;
        if (i > 0) s += rec[t - 1].a;
        else if (periodic) s += rec[t + nr - 1].a;
        if (j > 0) s += rec[t - nr].b;
        else if (periodic) s += rec[t + (long long)(nt - 1) * nr].b;
        s += rec[(long long)((k + np - 1) % np) * pl + (t - (long long)k * pl)].c;
        adiag[t] = -s;
        rowsum[t] = 2.0 * s;
        gmax = fmax(gmax, 2.0 * c.w * s);
    }
    gmax = warp_max(gmax);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = gmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = red[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
        part[blockIdx.x] = m;
    }
}

template <typename T>
T* dev_copy(const std::vector<T>& h, cudaStream_t s) {
    T* d = nullptr;
    PB_CUDA_TRY(cudaMalloc(&d, h.size() * sizeof(T)));
    PB_CUDA_TRY(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return d;
}

int setup_blocks(const Ctx& c, long long n) {
    long long b = (n + 255) / 256;
    long long cap = (long long)c.sm_count * 8;
    return (int)std::max(1LL, std::min(b, cap));
}

}  // namespace

int reduce_blocks(const Ctx& c) { return setup_blocks(c, c.n); }

// Copies the face arrays (conduction) or the per-component point / bound arrays (viscosity) to
// the device once per context.
void setup_geometry(Ctx& c, const pb_grid& g) {
    if (c.geometry == PB_CARTESIAN_PERIODIC) return;     // unit cells: no metric arrays
    const int nr = g.n_r, nt = g.n_theta;
    std::vector<double> rf(g.r_face, g.r_face + nr + 1), tf(g.t_face, g.t_face + nt + 1);
    if (c.kind == PB_TC_ANISO) {
        c.geo[0] = dev_copy(rf, c.stream);
        c.geo[1] = dev_copy(tf, c.stream);
        return;
    }
    std::vector<double> rc(nr), tc(nt);
    for (int i = 0; i < nr; ++i) rc[i] = 0.5 * (rf[i] + rf[i + 1]);
    for (int j = 0; j < nt; ++j) tc[j] = 0.5 * (tf[j] + tf[j + 1]);
    for (int comp = 0; comp < 3; ++comp) {
        std::vector<double> pr, er, pt, et;
        if (comp == 0) { pr.assign(rf.begin() + 1, rf.begin() + nr); er = rc; }
        else { pr = rc; er = rf; }
        if (comp == 1) { pt.assign(tf.begin() + 1, tf.begin() + nt); et = tc; }
        else { pt = tc; et = tf; }
        c.geo[4 * comp + 0] = dev_copy(pr, c.stream);
        c.geo[4 * comp + 1] = dev_copy(er, c.stream);
        c.geo[4 * comp + 2] = dev_copy(pt, c.stream);
        c.geo[4 * comp + 3] = dev_copy(et, c.stream);
    }
}

// bfloat16-storage contexts: the float64 records rounded to the values the kernels will read, so
// that dt_E (the Gershgorin bound) and diag(A) belong to the operator actually applied.  A
// bfloat16 record may lie 2^-9 above its float64 value, and at the PTL floor a cycle runs at
// exactly the forward-Euler limit (RKL2 s = 2 has |R| = 1 there): a bound taken from the unrounded
// operator lets the highest modes grow by about 2^-8 per cycle.
__global__ void round_records_bf16_kernel(long long n, Coef4<double>* rec) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        Coef4<double> r = rec[t];
        r.a = (double)__bfloat162float(__double2bfloat16(r.a));
        r.b = (double)__bfloat162float(__double2bfloat16(r.b));
        r.c = (double)__bfloat162float(__double2bfloat16(r.c));
        r.w = (double)__bfloat162float(__double2bfloat16(r.w));
        rec[t] = r;
    }
}

static void round_records(Ctx& c, Coef4<double>* rec, long long n) {
    if (c.prec != PB_BF16_STORE) return;
    round_records_bf16_kernel<<<setup_blocks(c, n), 256, 0, c.stream>>>(n, rec);
}

void setup_tc(Ctx& c, const pb_operator& op, Coef4<double>* rec, double* dt_e, bool clamp) {
    const long long n = c.n;
    double* kap = c.s64;
    const int blocks = setup_blocks(c, n);
    kappa_kernel<<<blocks, 256, 0, c.stream>>>(n, op.T0, kap, clamp);
    TCArgs a{c.nr, c.nt, c.np, 2.0 * M_PI / c.np, op.C, c.geo[0], c.geo[1], kap, op.n, op.B[0], op.B[1], op.B[2], rec};
    const bool box = c.geometry == PB_CARTESIAN_PERIODIC;
    if (box) tc_coef_box_kernel<<<blocks, 256, 0, c.stream>>>(a);
    else tc_coef_kernel<<<blocks, 256, 0, c.stream>>>(a);
    round_records(c, rec, n);
    double* part = static_cast<double*>(c.partials);
    double* adiag = c.s64;   // kappa is no longer needed
    tc_rows_kernel<<<blocks, 256, 0, c.stream>>>(c.nr, c.nt, c.np, box ? 1 : 0, rec, adiag, c.arow, part);
    max_finalize_kernel<<<1, 256, 0, c.stream>>>(part, blocks, c.d_scalar);
    PB_CUDA_TRY(cudaGetLastError());
    PB_CUDA_TRY(cudaMemcpyAsync(c.h_scalar, c.d_scalar, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    PB_CUDA_TRY(cudaStreamSynchronize(c.stream));
    *dt_e = *c.h_scalar;
}

void setup_visc(Ctx& c, const pb_operator& op, Coef4<double>* rec, double* dt_e) {
    double* part = static_cast<double*>(c.partials);
    double* adiag = c.s64;
    int total_blocks = 0;
    for (int comp = 0; comp < 3; ++comp) {
        const CompGrid& cg = c.grid.c[comp];
        const long long n = (long long)cg.nr * cg.nt * cg.np;
        ViscArgs a{cg.nr, cg.nt, cg.np, 2.0 * M_PI / c.np, c.geo[4 * comp], c.geo[4 * comp + 1], c.geo[4 * comp + 2],
                   c.geo[4 * comp + 3], op.rho[comp], op.nu[comp], rec + cg.offset};
        const int blocks = setup_blocks(c, n);
        if (cg.periodic) visc_coef_box_kernel<<<blocks, 256, 0, c.stream>>>(a);
        else visc_coef_kernel<<<blocks, 256, 0, c.stream>>>(a);
    }
    round_records(c, rec, c.n);
    for (int comp = 0; comp < 3; ++comp) {
        const CompGrid& cg = c.grid.c[comp];
        const long long n = (long long)cg.nr * cg.nt * cg.np;
        const int blocks = setup_blocks(c, n);
        visc_rows_kernel<<<blocks, 256, 0, c.stream>>>(cg.nr, cg.nt, cg.np, cg.periodic, rec + cg.offset,
                                                       adiag + cg.offset, c.arow + cg.offset, part + total_blocks);
        total_blocks += blocks;
    }
    max_finalize_kernel<<<1, 256, 0, c.stream>>>(part, total_blocks, c.d_scalar);
    PB_CUDA_TRY(cudaGetLastError());
    PB_CUDA_TRY(cudaMemcpyAsync(c.h_scalar, c.d_scalar, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    PB_CUDA_TRY(cudaStreamSynchronize(c.stream));
    *dt_e = *c.h_scalar;
}

}  // namespace pb
