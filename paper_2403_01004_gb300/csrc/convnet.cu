// Learned initial guess for the Backward Euler PCG solve: a small 3-D convolutional network
// (four 3 x 3 x 3 layers, 16 channels, ReLU between them) that maps per-point features of the
// state to the BE increment x - u^n, with bfloat16 weights and activations and float32
// accumulation, plus its training (forward, backward, mean-squared-error loss, Adam) on
// samples produced by the library's own BE solves.  The paper has no network: this is the warm
// start the PCG of Sec. 3.1 is given; PCG still converges to the same tolerance from it.
//
// Tensors are channels-last: [sample][d][h][w][16] with w (r) fastest.  Every layer runs with
// 16 input and 16 output channels (layer 1 uses 6 of its inputs, layer 4 one of its outputs;
// the unused weights are held at zero).  Convolution is cross-correlation with zero padding;
// the d (phi) axis may wrap.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "epilogues.cuh"
#include "launch.h"
#include "umma.cuh"

namespace pb {

constexpr int NC = 16;          // channels
constexpr int NL = 4;           // layers
constexpr int NW = 27 * NC * NC;
constexpr int NPAR = NL * (NW + NC);
constexpr int NFEAT = 6;        // feature channels in use
constexpr int TD = 4, TH = 8, TW = 8;   // conv output tile (256 points)

struct Model {
    float* master = nullptr;    // float32 parameters: per layer W[27][ci][co] then b[co]
    float* m = nullptr;         // Adam moments
    float* v = nullptr;
    float* grad = nullptr;
    __nv_bfloat16* wfwd = nullptr;   // bfloat16 W[layer][27][ci][co]
    __nv_bfloat16* wbwd = nullptr;   // bfloat16 flipped / transposed: Wt[layer][off][co][ci] = W[26-off][ci][co]
    long long step = 0;
    // activation workspace (sized on demand)
    __nv_bfloat16* act[NL + 1] = {};   // act[0] input features, act[l] post-activation of layer l
    __nv_bfloat16* pre[NL] = {};       // pre-activation (for the ReLU masks)
    float* out = nullptr;              // layer 4 output, float32 [points]
    __nv_bfloat16* g0 = nullptr;       // gradient buffers
    __nv_bfloat16* g1 = nullptr;
    long long cap = 0;
    float* batch_target = nullptr;
    float* batch_mask = nullptr;
    double* loss_acc = nullptr;
    double* h_loss = nullptr;
    int* d_err = nullptr;              // set by a conv kernel whose bounded wait ran out
    std::string err;
};

namespace {

__device__ __forceinline__ long long pidx(int s, int d, int h, int w, int D, int H, int W) {
    return (((long long)s * D + d) * H + h) * W + w;
}

// One conv layer: out[p][co] = b[co] + sum_off sum_ci Wt[off][ci][co] in[p + off][ci].
// MODE 0: writes pre-activation (bf16, if pre != null) and relu (bf16) to act_out;
// MODE 1: writes float32 out (last layer, no activation);
// MODE 2: input-gradient pass (no bias), the result times the ReLU mask of `mask_pre`
//         written to act_out (bf16).
template <int MODE>
__global__ void __launch_bounds__(256)
conv_kernel(const __nv_bfloat16* __restrict__ in, int S, int D, int H, int W, int wrap_d,
            const __nv_bfloat16* __restrict__ wt, const float* __restrict__ bias,
            __nv_bfloat16* pre_out, __nv_bfloat16* act_out, float* fout, const __nv_bfloat16* __restrict__ mask_pre) {
    extern __shared__ __align__(16) unsigned char smem[];
    float* ws = reinterpret_cast<float*>(smem);                                  // [27][16][16]
    __nv_bfloat16* xs = reinterpret_cast<__nv_bfloat16*>(smem + NW * sizeof(float));   // [TD+2][TH+2][TW+2][16]
    const int tid = threadIdx.x;
    const int tw = tid % TW, th = (tid / TW) % TH, td = tid / (TW * TH);
    const int nbw = (W + TW - 1) / TW, nbh = (H + TH - 1) / TH, nbd = (D + TD - 1) / TD;
    int b = blockIdx.x;
    const int bw = b % nbw; b /= nbw;
    const int bh = b % nbh; b /= nbh;
    const int bd = b % nbd;
    const int s = b / nbd;
    const int w0 = bw * TW, h0 = bh * TH, d0 = bd * TD;
    for (int q = tid; q < NW; q += 256) ws[q] = __bfloat162float(wt[q]);
    constexpr int HW = TW + 2, HH = TH + 2, HD = TD + 2;
    for (int q = tid; q < HD * HH * HW; q += 256) {
        const int xw = q % HW, xh = (q / HW) % HH, xd = q / (HW * HH);
        int gd = d0 - 1 + xd;
        const int gh = h0 - 1 + xh, gw = w0 - 1 + xw;
        if (wrap_d) gd = (gd + D) % D;
        uint4* dst = reinterpret_cast<uint4*>(xs + (long long)q * NC);
        if (gd >= 0 && gd < D && gh >= 0 && gh < H && gw >= 0 && gw < W) {
            const uint4* src = reinterpret_cast<const uint4*>(in + pidx(s, gd, gh, gw, D, H, W) * NC);
            dst[0] = src[0];
            dst[1] = src[1];
        } else {
            dst[0] = make_uint4(0, 0, 0, 0);
            dst[1] = make_uint4(0, 0, 0, 0);
        }
    }
    __syncthreads();
    const int d = d0 + td, h = h0 + th, w = w0 + tw;
    if (d >= D || h >= H || w >= W) return;
    float acc[NC];
#pragma unroll
    for (int co = 0; co < NC; ++co) acc[co] = (MODE == 2) ? 0.f : bias[co];
    for (int off = 0; off < 27; ++off) {
        const int a = off / 9, bb = (off / 3) % 3, c = off % 3;
        const __nv_bfloat16* xp = xs + (((td + a) * HH + (th + bb)) * HW + (tw + c)) * NC;
        float xv[NC];
#pragma unroll
        for (int ci = 0; ci < NC; ci += 2) {
            const __nv_bfloat162 v2 = *reinterpret_cast<const __nv_bfloat162*>(xp + ci);
            xv[ci] = __low2float(v2);
            xv[ci + 1] = __high2float(v2);
        }
        const float4* wp = reinterpret_cast<const float4*>(ws + off * NC * NC);
#pragma unroll
        for (int ci = 0; ci < NC; ++ci) {
#pragma unroll
            for (int q4 = 0; q4 < NC / 4; ++q4) {
                const float4 wv = wp[ci * (NC / 4) + q4];
                acc[4 * q4 + 0] += xv[ci] * wv.x;
                acc[4 * q4 + 1] += xv[ci] * wv.y;
                acc[4 * q4 + 2] += xv[ci] * wv.z;
                acc[4 * q4 + 3] += xv[ci] * wv.w;
            }
        }
    }
    const long long p = pidx(s, d, h, w, D, H, W);
    if (MODE == 1) {
        fout[p] = acc[0];
        return;
    }
    __align__(16) __nv_bfloat16 ob[NC];
    if (MODE == 0) {
        __align__(16) __nv_bfloat16 pb_[NC];
#pragma unroll
        for (int co = 0; co < NC; ++co) {
            pb_[co] = __float2bfloat16_rn(acc[co]);
            ob[co] = __float2bfloat16_rn(fmaxf(acc[co], 0.f));
        }
        if (pre_out) {
            uint4* dst = reinterpret_cast<uint4*>(pre_out + p * NC);
            dst[0] = *reinterpret_cast<uint4*>(&pb_[0]);
            dst[1] = *reinterpret_cast<uint4*>(&pb_[8]);
        }
    } else {
        const __nv_bfloat16* mp = mask_pre + p * NC;
#pragma unroll
        for (int co = 0; co < NC; ++co) ob[co] = __float2bfloat16_rn(__bfloat162float(mp[co]) > 0.f ? acc[co] : 0.f);
    }
    uint4* dst = reinterpret_cast<uint4*>(act_out + p * NC);
    dst[0] = *reinterpret_cast<uint4*>(&ob[0]);
    dst[1] = *reinterpret_cast<uint4*>(&ob[8]);
}

// The same layer on the tensor cores (tcgen05): per output tile of 2 (d) x 16 (h) x 8 (w) points,
// each d slice is one M = 128, N = 16 accumulator in TMEM, summed over the 27 offsets by 27
// MMAs of K = 16 (the input channels).  Row m of a slice is the point (h0 + m / 8, w0 + m % 8).
// The input halo (4 x 18 x 10 points) sits in shared memory split by channel halves: plane c
// holds channels 8c..8c+7 of every point, 16 bytes a point, w fastest.  For offset (a, b, c) the
// A operand then starts at halo point (slice + a, b, c): its core matrices are the 8 consecutive
// w points of one h row (rows 16 bytes apart), the next h row is 10 points (160 bytes) on, and
// the second half of K is the other plane.  The weights of offset o are B = W[o] (N = co rows,
// K = ci), stored the same way: 512 bytes per offset.  One thread issues the MMAs; the four
// warps read the accumulators back (warp w owns TMEM lanes 32w..32w+31) and apply MODE's
// epilogue.  CTAs walk the tiles grid-stride, allocating 32 TMEM columns once.
constexpr int CT_D = 2, CT_H = 16, CT_W = 8;
constexpr int CH_D = CT_D + 2, CH_H = CT_H + 2, CH_W = CT_W + 2;
constexpr int CH_PTS = CH_D * CH_H * CH_W;
constexpr int CA_PLANE = CH_PTS * 16;            // one channel-half plane of the halo (bytes)
constexpr int CB_OFF = 2 * CA_PLANE;              // the weights follow the two planes
constexpr int CONV_TC_SMEM = CB_OFF + 27 * 512;
constexpr int CONV_TC_THREADS = 128;
constexpr uint32_t kConvIdesc = umma::idesc_bf16_f32(128, 16);

// 16-byte global -> shared copy; with valid == false nothing is read and 16 zero bytes land
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}

template <int MODE>
__global__ void __launch_bounds__(CONV_TC_THREADS, 6)
conv_tc_kernel(const __nv_bfloat16* __restrict__ in, int S, int D, int H, int W, int wrap_d,
               const __nv_bfloat16* __restrict__ wt, const float* __restrict__ bias, __nv_bfloat16* pre_out,
               __nv_bfloat16* act_out, float* fout, const __nv_bfloat16* __restrict__ mask_pre, int* err) {
    extern __shared__ __align__(16) unsigned char smem[];     // descriptors need 16-byte alignment
    __shared__ uint32_t tbase;
    __shared__ __align__(8) uint64_t bar;
    __shared__ float bias_s[NC];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* a_s = smem;
    unsigned char* b_s = smem + CB_OFF;
    if (MODE != 2 && tid < NC) bias_s[tid] = bias[tid];
    for (int q = tid; q < NW; q += CONV_TC_THREADS) {
        const int o = q / (NC * NC), ci = (q / NC) % NC, co = q % NC;
        *reinterpret_cast<__nv_bfloat16*>(b_s + o * 512 + (ci / 8) * 256 + (co / 8) * 128 + (co % 8) * 16 + (ci % 8) * 2) =
            wt[q];
    }
    __syncwarp();
    if (warp == 0) umma::tmem_alloc(&tbase, 32);
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tb = tbase;
    const int nbw = (W + CT_W - 1) / CT_W, nbh = (H + CT_H - 1) / CT_H, nbd = (D + CT_D - 1) / CT_D;
    const long long ntiles = (long long)S * nbd * nbh * nbw;
    unsigned phase = 0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        long long b = t;
        const int bw = (int)(b % nbw); b /= nbw;
        const int bh = (int)(b % nbh); b /= nbh;
        const int bd = (int)(b % nbd);
        const int s = (int)(b / nbd);
        const int w0 = bw * CT_W, h0 = bh * CT_H, d0 = bd * CT_D;
        // the halo by cp.async (all of a thread's copies in flight at once); points outside the
        // grid are zero-filled (source size 0)
        for (int q = tid; q < CH_PTS; q += CONV_TC_THREADS) {
            const int xw = q % CH_W, xh = (q / CH_W) % CH_H, xd = q / (CH_W * CH_H);
            int gd = d0 - 1 + xd;
            const int gh = h0 - 1 + xh, gw = w0 - 1 + xw;
            if (wrap_d) gd = (gd + D) % D;
            const bool inside = gd >= 0 && gd < D && gh >= 0 && gh < H && gw >= 0 && gw < W;
            const __nv_bfloat16* src = inside ? in + pidx(s, gd, gh, gw, D, H, W) * NC : in;
            cp_async16(a_s + q * 16, src, inside);
            cp_async16(a_s + CA_PLANE + q * 16, src + 8, inside);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        umma::fence_async_smem();
        umma::fence_before_sync();
        __syncthreads();
        umma::fence_after_sync();
        __shared__ int mma_ok;
        if (tid == 0) {
            // descriptors of offset 0; the start-address field counts 16-byte units, so moving the
            // operand by a multiple of 16 bytes is an add on the descriptor (shared memory stays
            // below 256 KB, so the 14-bit field cannot carry)
            const uint64_t da0 = umma::smem_desc(smem_u32(a_s), CA_PLANE, CH_W * 16);
            const uint64_t db0 = umma::smem_desc(smem_u32(b_s), 256, 128);
            // the slices' accumulations interleaved: consecutive MMAs write different
            // accumulators, so each does not wait for the one before it
#pragma unroll
            for (int o = 0; o < 27; ++o)
#pragma unroll
                for (int sl = 0; sl < CT_D; ++sl) {
                    const int od = o / 9, oh = (o / 3) % 3, ow = o % 3;
                    umma::mma_bf16(tb + (uint32_t)(sl * 16), da0 + (uint64_t)(((sl + od) * CH_H + oh) * CH_W + ow),
                                   db0 + (uint64_t)(o * 32), kConvIdesc, o > 0);
                }
            umma::commit(&bar);
            // one thread waits (bounded) for the MMAs; the others wait at the barrier
            mma_ok = mbar_wait(&bar, phase) ? 1 : 0;
        }
        __syncthreads();
        const int ok = mma_ok;
        phase ^= 1u;
        if (!ok) {
            // give the tensor core one more bounded interval before TMEM is released
            if (tid == 0) {
                atomicExch(err, 1);
                mbar_wait(&bar, phase ^ 1u);
            }
            __syncthreads();
            break;
        }
        umma::fence_after_sync();
        // both slices are read before any lane branches (the loads are warp-collective)
        float accs[CT_D][NC];
#pragma unroll
        for (int sl = 0; sl < CT_D; ++sl)
            umma::ld_32x32b_x16(tb + ((uint32_t)(32 * warp) << 16) + (uint32_t)(sl * 16), accs[sl]);
        for (int sl = 0; sl < CT_D; ++sl) {
            const float* acc = accs[sl];
            const int m = 32 * warp + lane;
            const int d = d0 + sl, h = h0 + m / CT_W, w = w0 + m % CT_W;
            if (d >= D || h >= H || w >= W) continue;
            const long long p = pidx(s, d, h, w, D, H, W);
            if (MODE == 1) {
                fout[p] = acc[0] + bias_s[0];
                continue;
            }
            __align__(16) __nv_bfloat16 ob[NC];
            if (MODE == 0) {
                __align__(16) __nv_bfloat16 pb_[NC];
#pragma unroll
                for (int co = 0; co < NC; ++co) {
                    const float z = acc[co] + bias_s[co];
                    pb_[co] = __float2bfloat16_rn(z);
                    ob[co] = __float2bfloat16_rn(fmaxf(z, 0.f));
                }
                if (pre_out) {
                    uint4* dst = reinterpret_cast<uint4*>(pre_out + p * NC);
                    dst[0] = *reinterpret_cast<uint4*>(&pb_[0]);
                    dst[1] = *reinterpret_cast<uint4*>(&pb_[8]);
                }
            } else {
                const __nv_bfloat16* mp = mask_pre + p * NC;
#pragma unroll
                for (int co = 0; co < NC; ++co) ob[co] = __float2bfloat16_rn(__bfloat162float(mp[co]) > 0.f ? acc[co] : 0.f);
            }
            uint4* dst = reinterpret_cast<uint4*>(act_out + p * NC);
            dst[0] = *reinterpret_cast<uint4*>(&ob[0]);
            dst[1] = *reinterpret_cast<uint4*>(&ob[8]);
        }
        // the halo planes and the accumulators are reused by the next tile
        umma::fence_before_sync();
        __syncthreads();
        umma::fence_after_sync();
    }
    if (warp == 0) umma::tmem_dealloc(tb, 32);
}

// dW[off][ci][co] += sum_p in[p + off][ci] g[p][co], db[co] += sum_p g[p][co] over one tile.
__global__ void __launch_bounds__(256)
wgrad_kernel(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ g, int S, int D, int H, int W,
             float* dW, float* db) {
    __shared__ __align__(16) __nv_bfloat16 xs[(TD + 2) * (TH + 2) * (TW + 2) * NC];
    __shared__ __align__(16) __nv_bfloat16 gs[TD * TH * TW * NC];
    const int tid = threadIdx.x;
    const int nbw = (W + TW - 1) / TW, nbh = (H + TH - 1) / TH, nbd = (D + TD - 1) / TD;
    int b = blockIdx.x;
    const int bw = b % nbw; b /= nbw;
    const int bh = b % nbh; b /= nbh;
    const int bd = b % nbd;
    const int s = b / nbd;
    const int w0 = bw * TW, h0 = bh * TH, d0 = bd * TD;
    constexpr int HW = TW + 2, HH = TH + 2, HD = TD + 2;
    for (int q = tid; q < HD * HH * HW; q += 256) {
        const int xw = q % HW, xh = (q / HW) % HH, xd = q / (HW * HH);
        const int gd = d0 - 1 + xd, gh = h0 - 1 + xh, gw = w0 - 1 + xw;
        uint4* dst = reinterpret_cast<uint4*>(xs + q * NC);
        if (gd >= 0 && gd < D && gh >= 0 && gh < H && gw >= 0 && gw < W) {
            const uint4* src = reinterpret_cast<const uint4*>(in + pidx(s, gd, gh, gw, D, H, W) * NC);
            dst[0] = src[0];
            dst[1] = src[1];
        } else {
            dst[0] = make_uint4(0, 0, 0, 0);
            dst[1] = make_uint4(0, 0, 0, 0);
        }
    }
    {
        const int tw = tid % TW, th = (tid / TW) % TH, td = tid / (TW * TH);
        const int d = d0 + td, h = h0 + th, w = w0 + tw;
        uint4* dst = reinterpret_cast<uint4*>(gs + tid * NC);
        if (d < D && h < H && w < W) {
            const uint4* src = reinterpret_cast<const uint4*>(g + pidx(s, d, h, w, D, H, W) * NC);
            dst[0] = src[0];
            dst[1] = src[1];
        } else {
            dst[0] = make_uint4(0, 0, 0, 0);
            dst[1] = make_uint4(0, 0, 0, 0);
        }
    }
    __syncthreads();
    const int ci = tid / NC, co = tid % NC;
    float acc[27];
#pragma unroll
    for (int o = 0; o < 27; ++o) acc[o] = 0.f;
    float bacc = 0.f;
    for (int p = 0; p < TD * TH * TW; ++p) {
        const int tw = p % TW, th = (p / TW) % TH, td = p / (TW * TH);
        const float gv = __bfloat162float(gs[p * NC + co]);
        bacc += gv;
#pragma unroll
        for (int o = 0; o < 27; ++o) {
            const int a = o / 9, bb = (o / 3) % 3, c = o % 3;
            acc[o] += __bfloat162float(xs[(((td + a) * HH + (th + bb)) * HW + (tw + c)) * NC + ci]) * gv;
        }
    }
#pragma unroll
    for (int o = 0; o < 27; ++o) atomicAdd(&dW[(o * NC + ci) * NC + co], acc[o]);
    if (ci == 0) atomicAdd(&db[co], bacc);
}

// loss = sum(mask (y - t)^2) / sum(mask); g = 2 mask (y - t) / sum(mask) into channel 0 of a
// 16-channel bf16 gradient tensor.
__global__ void loss_kernel(long long n, const float* y, const float* t, const float* mask, double msum,
                            __nv_bfloat16* g, double* acc) {
    double part = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const float r = (y[q] - t[q]) * mask[q];
        part += (double)r * r;
        __nv_bfloat16* gp = g + q * NC;
        gp[0] = __float2bfloat16_rn((float)(2.0 * r / msum));
        for (int c = 1; c < NC; ++c) gp[c] = __float2bfloat16_rn(0.f);
    }
    double v[1] = {part};
    block_sum<1>(v);
    if (threadIdx.x == 0) atomicAdd(acc, v[0]);
}

// Adam on the float32 parameters; refreshes the bf16 forward and flipped / transposed copies.
// Unused weights of the padded channels are held at zero.
__global__ void adam_kernel(float* w, float* m, float* v, const float* g, float lr, float b1, float b2, float eps,
                            float c1, float c2, __nv_bfloat16* wf, __nv_bfloat16* wb) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < NPAR; q += gridDim.x * blockDim.x) {
        const int layer = q / (NW + NC), r = q % (NW + NC);
        bool used = true;
        if (r < NW) {
            const int ci = (r / NC) % NC, co = r % NC;
            if (layer == 0 && ci >= NFEAT) used = false;
            if (layer == NL - 1 && co != 0) used = false;
        } else if (layer == NL - 1 && r - NW != 0) {
            used = false;
        }
        float x = w[q];
        if (used) {
            const float gq = g[q];
            const float mq = b1 * m[q] + (1.f - b1) * gq;
            const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
            m[q] = mq;
            v[q] = vq;
            x -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
        } else {
            x = 0.f;
        }
        w[q] = x;
        if (r < NW) {
            const int off = r / (NC * NC), ci = (r / NC) % NC, co = r % NC;
            wf[layer * NW + r] = __float2bfloat16_rn(x);
            wb[layer * NW + ((26 - off) * NC + co) * NC + ci] = __float2bfloat16_rn(x);
        }
    }
}

// crops[b] = src[sample[b]][d0 + z][h0 + y][w0 + x] for features (16 channels) and targets.
__global__ void crop_kernel(const __nv_bfloat16* feats, const float* targ, int D, int H, int W, const int* org, int nb,
                            int cd, int ch, int cw, __nv_bfloat16* out_f, float* out_t) {
    const long long per = (long long)cd * ch * cw;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < per * nb; q += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(q / per);
        long long r = q % per;
        const int x = (int)(r % cw); r /= cw;
        const int y = (int)(r % ch);
        const int z = (int)(r / ch);
        const int s = org[4 * b], d0 = org[4 * b + 1], h0 = org[4 * b + 2], w0 = org[4 * b + 3];
        const long long src = pidx(s, d0 + z, h0 + y, w0 + x, D, H, W);
        const uint4* a = reinterpret_cast<const uint4*>(feats + src * NC);
        uint4* o = reinterpret_cast<uint4*>(out_f + q * NC);
        o[0] = a[0];
        o[1] = a[1];
        out_t[q] = targ[src];
    }
}

// Feature channels per point of a conduction / viscosity state (see pb_guess_features):
// 0: e / S with e = dt F(u), S = rms(e);  1: log10(1 + sigma), sigma = dt w |A_ii|;
// 2: sigma / (1 + sigma);  3: (u - mean u) / S;  4: log10(w) / 10;  5: position along r in [0, 1].
template <class P>
__global__ void features_kernel(MarchGrid g, const typename P::S* u, const typename P::S* F,
                                const Coef4<typename P::C>* rec, const typename P::C* adiag, double dt, double S,
                                double umean, __nv_bfloat16* out, const typename P::S* x, float* target) {
    using A = typename P::A;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < (long long)g.c[g.ncomp - 1].offset +
                                                                                (long long)g.c[g.ncomp - 1].nr * g.c[g.ncomp - 1].nt * g.c[g.ncomp - 1].np;
         q += (long long)gridDim.x * blockDim.x) {
        int comp = 0;
        for (int c = 1; c < g.ncomp; ++c)
            if (q >= g.c[c].offset) comp = c;
        const int nr = g.c[comp].nr;
        const int i = (int)((q - g.c[comp].offset) % nr);
        const double w = (double)rec[q].w;
        const double e = dt * (double)cvt<A>(F[q]);
        const double sigma = dt * w * fabs((double)adiag[q]);
        float f[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) f[c] = 0.f;
        f[0] = (float)(e / S);
        f[1] = (float)log10(1.0 + sigma);
        f[2] = (float)(sigma / (1.0 + sigma));
        f[3] = (float)(((double)cvt<A>(u[q]) - umean) / S);
        f[4] = (float)(log10(w) / 10.0);
        f[5] = nr > 1 ? (float)i / (float)(nr - 1) : 0.f;
        __nv_bfloat16* o = out + q * NC;
#pragma unroll
        for (int c = 0; c < NC; ++c) o[c] = __float2bfloat16_rn(f[c]);
        if (target) target[q] = (float)(((double)cvt<A>(x[q]) - (double)cvt<A>(u[q])) / S);
    }
}

template <class P>
__global__ void moments_kernel(long long n, const typename P::S* u, const typename P::S* F, double dt, double* acc) {
    using A = typename P::A;
    double v[3] = {0.0, 0.0, 0.0};
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const double e = dt * (double)cvt<A>(F[q]);
        v[0] += e * e;
        v[1] += (double)cvt<A>(u[q]);
    }
    block_sum<3>(v);
    if (threadIdx.x == 0) {
        atomicAdd(acc, v[0]);
        atomicAdd(acc + 1, v[1]);
    }
}

// One pass of the binomial filter (1, 2, 1)/4 along one axis of [S][D][H][W] float fields (axis 0:
// W, r; 1: H, theta; 2: D, phi); the ends repeat their edge value (no flux through them), and phi
// wraps when wrap_d.
__global__ void smooth_axis_kernel(const float* __restrict__ in, float* __restrict__ out, int S_, int D, int H, int W,
                                   int axis, int wrap_d) {
    const long long n = (long long)S_ * D * H * W;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int w = (int)(q % W);
        const long long t = q / W;
        const int h = (int)(t % H);
        const int d = (int)((t / H) % D);
        long long lo, hi;
        if (axis == 0) {
            lo = w > 0 ? q - 1 : q;
            hi = w < W - 1 ? q + 1 : q;
        } else if (axis == 1) {
            lo = h > 0 ? q - W : q;
            hi = h < H - 1 ? q + W : q;
        } else {
            const long long pl = (long long)H * W;
            lo = d > 0 ? q - pl : (wrap_d ? q + (long long)(D - 1) * pl : q);
            hi = d < D - 1 ? q + pl : (wrap_d ? q - (long long)(D - 1) * pl : q);
        }
        out[q] = 0.25f * (in[lo] + 2.0f * in[q] + in[hi]);
    }
}

// `passes` passes of the filter along all three axes, in place in y (tmp: scratch of the same size)
void smooth_field(float* y, float* tmp, int S_, int D, int H, int W, int wrap_d, int passes, cudaStream_t s) {
    const long long n = (long long)S_ * D * H * W;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
    float* a = y;
    float* b = tmp;
    for (int p = 0; p < passes; ++p)
        for (int axis = 0; axis < 3; ++axis) {
            smooth_axis_kernel<<<blocks, 256, 0, s>>>(a, b, S_, D, H, W, axis, wrap_d);
            std::swap(a, b);
        }
    if (a != y) PB_CUDA_TRY(cudaMemcpyAsync(y, a, (size_t)n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    PB_CUDA_TRY(cudaGetLastError());
}

// Smoothing of the network's output before it becomes a guess: PCG's initial residual weights the
// guess's error by S = M + dt K, i.e. grid-scale error by up to dt / dt_E, and to rtol 1e-10 the
// iteration count grows with any rough error while a smooth, accurate increment shortens the
// solve; the learned part is therefore asked for the smooth part of the increment only.
constexpr int kGuessSmoothPasses = 4;

// x0 = u + S y
template <class P>
__global__ void guess_kernel(long long n, const typename P::S* u, const float* y, double S, typename P::S* x0) {
    using A = typename P::A;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        x0[q] = cvt<typename P::S>((A)((double)cvt<A>(u[q]) + S * (double)y[q]));
}

int conv_smem() { return NW * (int)sizeof(float) + (TD + 2) * (TH + 2) * (TW + 2) * NC * 2; }

int nblocks3(int S, int D, int H, int W) {
    return S * ((D + TD - 1) / TD) * ((H + TH - 1) / TH) * ((W + TW - 1) / TW);
}

void ensure_ws(Model& m, long long pts) {
    if (pts <= m.cap) return;
    for (auto*& p : m.act) if (p) { cudaFree(p); p = nullptr; }
    for (auto*& p : m.pre) if (p) { cudaFree(p); p = nullptr; }
    void* q[] = {m.out, m.g0, m.g1, m.batch_target, m.batch_mask};
    for (void* p : q) if (p) cudaFree(p);
    m.out = nullptr; m.g0 = m.g1 = nullptr; m.batch_target = m.batch_mask = nullptr;
    const size_t ab = (size_t)pts * NC * sizeof(__nv_bfloat16);
    for (auto*& p : m.act) PB_CUDA_TRY(cudaMalloc(&p, ab));
    for (auto*& p : m.pre) PB_CUDA_TRY(cudaMalloc(&p, ab));
    PB_CUDA_TRY(cudaMalloc(&m.out, (size_t)pts * sizeof(float)));
    PB_CUDA_TRY(cudaMalloc(&m.g0, ab));
    PB_CUDA_TRY(cudaMalloc(&m.g1, ab));
    PB_CUDA_TRY(cudaMalloc(&m.batch_target, (size_t)pts * sizeof(float)));
    PB_CUDA_TRY(cudaMalloc(&m.batch_mask, (size_t)pts * sizeof(float)));
    m.cap = pts;
}

void set_attr() {
    // once per process (a function-local static: thread-safe initialisation)
    static const cudaError_t e = [] {
        cudaError_t r = cudaFuncSetAttribute(conv_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, conv_smem());
        if (r == cudaSuccess) r = cudaFuncSetAttribute(conv_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, conv_smem());
        if (r == cudaSuccess) r = cudaFuncSetAttribute(conv_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, conv_smem());
        return r;
    }();
    PB_CUDA_TRY(e);
}

// The tensor-core layer is the default; PB_CONV_CUDA_CORES=1 selects the CUDA-core kernel (same
// layer, float32 FMAs), kept as the second implementation the tests compare it with.
bool conv_on_cuda_cores() {
    static const bool v = [] {
        const char* e = getenv("PB_CONV_CUDA_CORES");
        return e && e[0] == '1';
    }();
    return v;
}

int conv_tc_grid(long long ntiles) {
    static const int sms = [] {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            n = 1;
        }
        return std::max(1, n);
    }();
    return (int)std::min<long long>(ntiles, (long long)sms * 6);   // 6 CTAs per SM fit its shared memory
}

// One conv layer (see conv_kernel / conv_tc_kernel for MODE).
template <int MODE>
void conv(Model& m, const __nv_bfloat16* in, int S, int D, int H, int W, int wrap, const __nv_bfloat16* wt,
          const float* bias, __nv_bfloat16* pre, __nv_bfloat16* act, float* fout, const __nv_bfloat16* mask,
          cudaStream_t st) {
    if (conv_on_cuda_cores()) {
        set_attr();
        conv_kernel<MODE><<<nblocks3(S, D, H, W), 256, conv_smem(), st>>>(in, S, D, H, W, wrap, wt, bias, pre, act, fout,
                                                                          mask);
    } else {
        // the largest shared-memory carve-out, so that 6 CTAs (36.9 KB each) fit an SM
        static const cudaError_t carve = cudaFuncSetAttribute(conv_tc_kernel<MODE>,
                                                              cudaFuncAttributePreferredSharedMemoryCarveout,
                                                              (int)cudaSharedmemCarveoutMaxShared);
        PB_CUDA_TRY(carve);
        const long long ntiles = (long long)S * ((D + CT_D - 1) / CT_D) * ((H + CT_H - 1) / CT_H) * ((W + CT_W - 1) / CT_W);
        conv_tc_kernel<MODE><<<conv_tc_grid(ntiles), CONV_TC_THREADS, CONV_TC_SMEM, st>>>(
            in, S, D, H, W, wrap, wt, bias, pre, act, fout, mask, m.d_err);
    }
    PB_CUDA_TRY(cudaGetLastError());
}

// After a stream synchronisation: a conv kernel whose bounded wait for its MMAs ran out.
void check_conv(Model& m) {
    int e = 0;
    PB_CUDA_TRY(cudaMemcpy(&e, m.d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        PB_CUDA_TRY(cudaMemset(m.d_err, 0, sizeof(int)));
        throw Error{PB_ETIMEOUT, "a tensor-core conv layer timed out waiting for its MMAs"};
    }
}

// Forward over act[0] (already in place); keeps pre-activations for the backward pass.
void forward(Model& m, int S, int D, int H, int W, int wrap, cudaStream_t st) {
    for (int l = 0; l < NL; ++l) {
        const __nv_bfloat16* wl = m.wfwd + (size_t)l * NW;
        const float* bl = m.master + (size_t)l * (NW + NC) + NW;
        if (l < NL - 1)
            conv<0>(m, m.act[l], S, D, H, W, wrap, wl, bl, m.pre[l], m.act[l + 1], nullptr, nullptr, st);
        else
            conv<1>(m, m.act[l], S, D, H, W, wrap, wl, bl, nullptr, nullptr, m.out, nullptr, st);
    }
}

// Loss and gradients for the batch held in act[0] / batch_target / batch_mask; returns loss.
double backward(Model& m, int S, int D, int H, int W, double msum, cudaStream_t st) {
    const long long pts = (long long)S * D * H * W;
    const int nb = nblocks3(S, D, H, W);
    PB_CUDA_TRY(cudaMemsetAsync(m.loss_acc, 0, sizeof(double), st));
    PB_CUDA_TRY(cudaMemsetAsync(m.grad, 0, NPAR * sizeof(float), st));
    loss_kernel<<<std::max(1, (int)std::min<long long>((pts + 255) / 256, 2048)), 256, 0, st>>>(
        pts, m.out, m.batch_target, m.batch_mask, msum, m.g0, m.loss_acc);
    __nv_bfloat16* g = m.g0;
    __nv_bfloat16* gn = m.g1;
    for (int l = NL - 1; l >= 0; --l) {
        float* dW = m.grad + (size_t)l * (NW + NC);
        wgrad_kernel<<<nb, 256, 0, st>>>(m.act[l], g, S, D, H, W, dW, dW + NW);
        if (l > 0) {
            // gradient wrt act[l] (= relu(pre[l-1])), masked by pre[l-1] > 0
            conv<2>(m, g, S, D, H, W, 0, m.wbwd + (size_t)l * NW, nullptr, nullptr, gn, nullptr, m.pre[l - 1], st);
            std::swap(g, gn);
        }
    }
    PB_CUDA_TRY(cudaGetLastError());
    PB_CUDA_TRY(cudaMemcpyAsync(m.h_loss, m.loss_acc, sizeof(double), cudaMemcpyDeviceToHost, st));
    PB_CUDA_TRY(cudaStreamSynchronize(st));
    check_conv(m);
    return *m.h_loss / msum;
}

void adam(Model& m, float lr, cudaStream_t st) {
    m.step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)m.step), c2 = 1.f - powf(b2, (float)m.step);
    adam_kernel<<<(NPAR + 255) / 256, 256, 0, st>>>(m.master, m.m, m.v, m.grad, lr, b1, b2, 1e-8f, c1, c2, m.wfwd, m.wbwd);
    PB_CUDA_TRY(cudaGetLastError());
}

void upload(Model& m, const std::vector<float>& host, cudaStream_t st) {
    PB_CUDA_TRY(cudaMemcpyAsync(m.master, host.data(), NPAR * sizeof(float), cudaMemcpyHostToDevice, st));
    // refresh the bf16 copies (and zero the unused weights) with a zero-step Adam pass
    PB_CUDA_TRY(cudaMemsetAsync(m.grad, 0, NPAR * sizeof(float), st));
    adam_kernel<<<(NPAR + 255) / 256, 256, 0, st>>>(m.master, m.m, m.v, m.grad, 0.f, 0.9f, 0.999f, 1e-8f, 1.f, 1.f,
                                                   m.wfwd, m.wbwd);
    PB_CUDA_TRY(cudaGetLastError());
    PB_CUDA_TRY(cudaStreamSynchronize(st));
}

thread_local std::string g_model_error;

template <class F>
int mguard(Model* m, F&& f) {
    try {
        f();
        if (m) m->err.clear();
        return PB_OK;
    } catch (const Error& e) {
        if (m) m->err = e.msg; else g_model_error = e.msg;
        return e.code;
    } catch (const std::bad_alloc&) {
        return PB_ENOMEM;
    }
}

void free_model(Model* m) {
    void* p[] = {m->master, m->m, m->v, m->grad, m->wfwd, m->wbwd, m->out, m->g0, m->g1, m->batch_target,
                 m->batch_mask, m->loss_acc, m->d_err};
    for (void* q : p) if (q) cudaFree(q);
    for (auto* q : m->act) if (q) cudaFree(q);
    for (auto* q : m->pre) if (q) cudaFree(q);
    if (m->h_loss) cudaFreeHost(m->h_loss);
}

template <class P>
void features_t(Ctx& c, const void* u, double dt, void* feats, double* scale, const void* x = nullptr,
                float* target = nullptr) {
    using S = typename P::S;
    (c.prec == PB_FP64 ? ops_f64() : ops_f32())->apply(c, u, c.y0);
    double* acc = c.s64;       // float64 scratch of the context
    PB_CUDA_TRY(cudaMemsetAsync(acc, 0, 2 * sizeof(double), c.stream));
    const int blocks = reduce_blocks(c);
    moments_kernel<P><<<blocks, 256, 0, c.stream>>>(c.n, static_cast<const S*>(u), static_cast<const S*>(c.y0), dt, acc);
    double h[2];
    PB_CUDA_TRY(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, c.stream));
    PB_CUDA_TRY(cudaStreamSynchronize(c.stream));
    double scl = std::sqrt(h[0] / (double)c.n);
    if (!(scl > 0.0) || std::isinf(scl)) scl = 1.0;
    const double umean = h[1] / (double)c.n;
    features_kernel<P><<<blocks, 256, 0, c.stream>>>(c.grid, static_cast<const S*>(u), static_cast<const S*>(c.y0),
                                                     static_cast<const Coef4<typename P::C>*>(c.coef),
                                                     static_cast<const typename P::C*>(c.adiag), dt, scl, umean,
                                                     static_cast<__nv_bfloat16*>(feats), static_cast<const S*>(x), target);
    PB_CUDA_TRY(cudaGetLastError());
    if (scale) *scale = scl;
}

}  // namespace
}  // namespace pb

using namespace pb;

struct pb_model { Model m; };

extern "C" {

const char* pb_model_last_error(const pb_model* h) { return h ? h->m.err.c_str() : g_model_error.c_str(); }

int pb_model_create(uint64_t seed, pb_model** out) {
    return mguard(nullptr, [&] {
        if (!out) throw Error{PB_EINVAL, "null output"};
        *out = nullptr;
        pb_model* h = new pb_model();
        Model& m = h->m;
        try {
            PB_CUDA_TRY(cudaMalloc(&m.master, NPAR * sizeof(float)));
            PB_CUDA_TRY(cudaMalloc(&m.m, NPAR * sizeof(float)));
            PB_CUDA_TRY(cudaMalloc(&m.v, NPAR * sizeof(float)));
            PB_CUDA_TRY(cudaMalloc(&m.grad, NPAR * sizeof(float)));
            PB_CUDA_TRY(cudaMalloc(&m.wfwd, NL * NW * sizeof(__nv_bfloat16)));
            PB_CUDA_TRY(cudaMalloc(&m.wbwd, NL * NW * sizeof(__nv_bfloat16)));
            PB_CUDA_TRY(cudaMalloc(&m.loss_acc, sizeof(double)));
            PB_CUDA_TRY(cudaMalloc(&m.d_err, sizeof(int)));
            PB_CUDA_TRY(cudaMemset(m.d_err, 0, sizeof(int)));
            PB_CUDA_TRY(cudaMallocHost(&m.h_loss, sizeof(double)));
            PB_CUDA_TRY(cudaMemset(m.m, 0, NPAR * sizeof(float)));
            PB_CUDA_TRY(cudaMemset(m.v, 0, NPAR * sizeof(float)));
            // He-uniform initialisation over the channels in use; the last layer starts at zero
            // so that an untrained model predicts a zero increment (x0 = u)
            std::mt19937_64 rng(seed);
            std::vector<float> host(NPAR, 0.f);
            const int cin[NL] = {NFEAT, NC, NC, NC};
            for (int l = 0; l < NL - 1; ++l) {
                const double bound = std::sqrt(6.0 / (cin[l] * 27.0));
                std::uniform_real_distribution<double> U(-bound, bound);
                for (int r = 0; r < NW; ++r) host[(size_t)l * (NW + NC) + r] = (float)U(rng);
            }
            upload(m, host, nullptr);
        } catch (...) {
            free_model(&m);
            delete h;
            throw;
        }
        *out = h;
    });
}

int pb_model_destroy(pb_model* h) {
    if (!h) return PB_OK;
    cudaDeviceSynchronize();
    free_model(&h->m);
    delete h;
    return PB_OK;
}

int pb_model_num_params(void) { return NPAR; }

int pb_model_get_params(const pb_model* h, float* host, int64_t cap) {
    if (!h || !host || cap < NPAR) return PB_EINVAL;
    if (cudaMemcpy(host, h->m.master, NPAR * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return PB_ECUDA;
    return PB_OK;
}

int pb_model_set_params(pb_model* h, const float* host, int64_t n) {
    if (!h || !host || n != NPAR) return PB_EINVAL;
    return mguard(&h->m, [&] {
        std::vector<float> v(host, host + NPAR);
        upload(h->m, v, nullptr);
    });
}

int pb_model_save(const pb_model* h, const char* path) {
    if (!h || !path) return PB_EINVAL;
    std::vector<float> v(NPAR);
    if (cudaMemcpy(v.data(), h->m.master, NPAR * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return PB_ECUDA;
    FILE* f = std::fopen(path, "wb");
    if (!f) return PB_EINVAL;
    const char magic[8] = {'P', 'B', 'N', 'E', 'T', '0', '0', '1'};
    const int32_t hdr[4] = {NL, NC, NFEAT, NPAR};
    bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(int32_t), 4, f) == 4 &&
              std::fwrite(v.data(), sizeof(float), NPAR, f) == (size_t)NPAR;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? PB_OK : PB_EINVAL;
}

int pb_model_load(pb_model* h, const char* path) {
    if (!h || !path) return PB_EINVAL;
    FILE* f = std::fopen(path, "rb");
    if (!f) return PB_EINVAL;
    char magic[8];
    int32_t hdr[4];
    std::vector<float> v(NPAR);
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "PBNET001", 8) == 0 &&
              std::fread(hdr, sizeof(int32_t), 4, f) == 4 && hdr[0] == NL && hdr[1] == NC && hdr[2] == NFEAT &&
              hdr[3] == NPAR && std::fread(v.data(), sizeof(float), NPAR, f) == (size_t)NPAR;
    std::fclose(f);
    if (!ok) return PB_EINVAL;
    return pb_model_set_params(h, v.data(), NPAR);
}

int pb_guess_features(pb_ctx* h, const void* u, double dt, const void* x, void* feats, void* target, double* scale) {
    if (!h) return PB_EINVAL;
    Ctx& c = h->c;
    try {
        if (!u || !feats || !(dt > 0.0) || (x == nullptr) != (target == nullptr)) return PB_EINVAL;
        if (c.prec == PB_FP64) features_t<PolF64>(c, u, dt, feats, scale, x, static_cast<float*>(target));
        else if (c.prec == PB_FP32) features_t<PolF32>(c, u, dt, feats, scale, x, static_cast<float*>(target));
        else return PB_ENOTSUP;
        PB_CUDA_TRY(cudaStreamSynchronize(c.stream));
        return PB_OK;
    } catch (const Error& e) {
        c.err = e.msg;
        return e.code;
    }
}

int pb_model_forward(pb_model* h, const void* feats, int32_t S, int32_t D, int32_t H, int32_t W, int32_t wrap_d,
                     void* out, void* stream) {
    if (!h) return PB_EINVAL;
    Model& m = h->m;
    return mguard(&m, [&] {
        if (!feats || !out || S <= 0 || D <= 0 || H <= 0 || W <= 0) throw Error{PB_EINVAL, "bad forward arguments"};
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        const long long pts = (long long)S * D * H * W;
        ensure_ws(m, pts);
        PB_CUDA_TRY(cudaMemcpyAsync(m.act[0], feats, pts * NC * sizeof(__nv_bfloat16), cudaMemcpyDeviceToDevice, st));
        forward(m, S, D, H, W, wrap_d, st);
        PB_CUDA_TRY(cudaMemcpyAsync(out, m.out, pts * sizeof(float), cudaMemcpyDeviceToDevice, st));
        PB_CUDA_TRY(cudaStreamSynchronize(st));
        check_conv(m);
    });
}

int pb_model_grad(pb_model* h, const void* feats, const void* target, const void* mask, int32_t S, int32_t D, int32_t H,
                  int32_t W, double* loss, float* host_grad, void* stream) {
    if (!h) return PB_EINVAL;
    Model& m = h->m;
    return mguard(&m, [&] {
        if (!feats || !target || !mask || S <= 0) throw Error{PB_EINVAL, "bad gradient arguments"};
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        const long long pts = (long long)S * D * H * W;
        ensure_ws(m, pts);
        PB_CUDA_TRY(cudaMemcpyAsync(m.act[0], feats, pts * NC * sizeof(__nv_bfloat16), cudaMemcpyDeviceToDevice, st));
        PB_CUDA_TRY(cudaMemcpyAsync(m.batch_target, target, pts * sizeof(float), cudaMemcpyDeviceToDevice, st));
        PB_CUDA_TRY(cudaMemcpyAsync(m.batch_mask, mask, pts * sizeof(float), cudaMemcpyDeviceToDevice, st));
        std::vector<float> hm(pts);
        PB_CUDA_TRY(cudaMemcpyAsync(hm.data(), mask, pts * sizeof(float), cudaMemcpyDeviceToHost, st));
        PB_CUDA_TRY(cudaStreamSynchronize(st));
        double msum = 0.0;
        for (float x : hm) msum += x;
        if (!(msum > 0.0)) throw Error{PB_EINVAL, "empty mask"};
        forward(m, S, D, H, W, 0, st);
        const double L = backward(m, S, D, H, W, msum, st);
        if (loss) *loss = L;
        if (host_grad) PB_CUDA_TRY(cudaMemcpy(host_grad, m.grad, NPAR * sizeof(float), cudaMemcpyDeviceToHost));
    });
}

int pb_model_train(pb_model* h, const void* feats, const void* targets, int32_t nsamples, int32_t D, int32_t H,
                   int32_t W, const pb_train_opts* o, double* last_loss, void* stream) {
    if (!h || !o) return PB_EINVAL;
    Model& m = h->m;
    return mguard(&m, [&] {
        if (!feats || !targets || nsamples <= 0) throw Error{PB_EINVAL, "no training data"};
        const int cd = o->crop, bsz = o->batch, border = o->border;
        if (cd <= 2 * border || cd > D || cd > H || cd > W || bsz <= 0 || o->steps < 0)
            throw Error{PB_EINVAL, "crop must fit the samples and exceed twice the border"};
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        const long long pts = (long long)bsz * cd * cd * cd;
        ensure_ws(m, pts);
        // loss mask: the crop interior (the border sees the crop's zero padding)
        std::vector<float> hm((size_t)pts, 0.f);
        double msum = 0.0;
        for (long long q = 0; q < pts; ++q) {
            long long r = q % ((long long)cd * cd * cd);
            const int x = (int)(r % cd); r /= cd;
            const int y = (int)(r % cd);
            const int z = (int)(r / cd);
            const bool in = x >= border && x < cd - border && y >= border && y < cd - border && z >= border &&
                            z < cd - border;
            hm[q] = in ? 1.f : 0.f;
            msum += hm[q];
        }
        PB_CUDA_TRY(cudaMemcpyAsync(m.batch_mask, hm.data(), pts * sizeof(float), cudaMemcpyHostToDevice, st));
        int* d_org = nullptr;
        PB_CUDA_TRY(cudaMalloc(&d_org, (size_t)4 * bsz * sizeof(int)));
        std::mt19937_64 rng(o->seed);
        std::vector<int> org((size_t)4 * bsz);
        double L = 0.0;
        try {
            for (int it = 0; it < o->steps; ++it) {
                for (int b = 0; b < bsz; ++b) {
                    org[4 * b] = (int)(rng() % (uint64_t)nsamples);
                    org[4 * b + 1] = (int)(rng() % (uint64_t)(D - cd + 1));
                    org[4 * b + 2] = (int)(rng() % (uint64_t)(H - cd + 1));
                    org[4 * b + 3] = (int)(rng() % (uint64_t)(W - cd + 1));
                }
                PB_CUDA_TRY(cudaMemcpyAsync(d_org, org.data(), org.size() * sizeof(int), cudaMemcpyHostToDevice, st));
                crop_kernel<<<1024, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(feats), static_cast<const float*>(targets),
                                                  D, H, W, d_org, bsz, cd, cd, cd, m.act[0], m.batch_target);
                forward(m, bsz, cd, cd, cd, 0, st);
                L = backward(m, bsz, cd, cd, cd, msum, st);
                adam(m, (float)o->lr, st);
            }
            PB_CUDA_TRY(cudaStreamSynchronize(st));
        } catch (...) {
            cudaFree(d_org);
            throw;
        }
        cudaFree(d_org);
        if (last_loss) *last_loss = L;
    });
}

int pb_guess_smooth(const void* in, void* out, void* tmp, int32_t S_, int32_t D, int32_t H, int32_t W, int32_t wrap_d,
                    int32_t passes, void* stream) {
    if (!in || !out || !tmp || out == tmp || in == tmp || S_ <= 0 || D <= 0 || H <= 0 || W <= 0 || passes < 0)
        return PB_EINVAL;
    try {
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const size_t bytes = (size_t)S_ * D * H * W * sizeof(float);
        if (in != out) PB_CUDA_TRY(cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, s));
        smooth_field(static_cast<float*>(out), static_cast<float*>(tmp), S_, D, H, W, wrap_d, passes, s);
        PB_CUDA_TRY(cudaStreamSynchronize(s));
        return PB_OK;
    } catch (const Error& e) {
        return e.code;
    }
}

int pb_guess_smooth_passes(void) { return kGuessSmoothPasses; }

int learned_guess(pb_ctx* hc, pb_model* hm, const void* u, double dt, void* x0) {
    if (!hc || !hm) return PB_EINVAL;
    Ctx& c = hc->c;
    Model& m = hm->m;
    try {
        if (!u || !x0 || !(dt > 0.0)) return PB_EINVAL;
        if (c.kind != PB_TC_ANISO) throw Error{PB_ENOTSUP, "the learned guess is trained for conduction"};
        if (c.prec != PB_FP64 && c.prec != PB_FP32) throw Error{PB_ENOTSUP, "needs float64 or float32 states"};
        const long long pts = c.n;
        ensure_ws(m, pts);
        double S = 1.0;
        if (c.prec == PB_FP64) features_t<PolF64>(c, u, dt, m.act[0], &S);
        else features_t<PolF32>(c, u, dt, m.act[0], &S);
        forward(m, 1, c.np, c.nt, c.nr, 1, c.stream);
        smooth_field(m.out, m.batch_target, 1, c.np, c.nt, c.nr, 1, kGuessSmoothPasses, c.stream);
        const int blocks = reduce_blocks(c);
        if (c.prec == PB_FP64)
            guess_kernel<PolF64><<<blocks, 256, 0, c.stream>>>(pts, static_cast<const double*>(u), m.out, S, static_cast<double*>(x0));
        else
            guess_kernel<PolF32><<<blocks, 256, 0, c.stream>>>(pts, static_cast<const float*>(u), m.out, S, static_cast<float*>(x0));
        PB_CUDA_TRY(cudaGetLastError());
        PB_CUDA_TRY(cudaStreamSynchronize(c.stream));
        check_conv(m);
        return PB_OK;
    } catch (const Error& e) {
        c.err = e.msg;
        return e.code;
    }
}

}  // extern "C"
