// Learned warm start: a U-Net mapping a filtered-backprojection image to an
// initial point x^0 for the solves (not in the paper; the warm start changes only
// x^0, so the convergence of NCS is untouched).  Trained and run by this file's
// own kernels:
//   * 3x3 convolutions as implicit GEMMs on the tensor cores (mma.sync m16n8k16,
//     bfloat16 operands, FP32 accumulation): pixels x output channels tiles of
//     64 x 64 per block, K = 9 taps x input channels staged 16 at a time;
//   * the data gradient is the same kernel with flipped, transposed weights;
//   * the weight gradient is a split-K GEMM over pixels (output channels x input
//     channels per tap), partial sums reduced in a fixed order;
//   * 2x2 average pooling, nearest 2x upsampling, concatenation by channel
//     offsets (no copies), ReLU masks, MSE loss, Adam.
// Activations are NHWC bfloat16; gradients FP32 (rounded to bfloat16 where they
// enter a tensor-core GEMM); master weights FP32.
#include "../../include/ncs.h"
#include "ncs_internal.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <random>
#include <vector>

using namespace ncs;

namespace {

using bf16 = __nv_bfloat16;

constexpr int CM = 64;    // pixels per block
constexpr int CN = 64;    // output channels per block
constexpr int CK = 16;    // K per stage
constexpr int SP = 24;    // shared-memory row pitch (bf16): conflict-free fragment loads

__device__ __forceinline__ void mma_bf16(float* c, const unsigned* a, const unsigned* b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Fragments of a 64x16 (A, [m][k]) and 64x16 (B, [n][k]) stage for a warp's 32x32 tile.
__device__ __forceinline__ void warp_mma_stage(const bf16 (*As)[SP], const bf16 (*Bs)[SP], int wm, int wn, int lane,
                                               float (*acc)[4][4])
{
    const int g = lane >> 2, t4 = lane & 3;
    unsigned af[2][4], bfr[4][2];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
        const int r = wm * 32 + mi * 16;
        af[mi][0] = *reinterpret_cast<const unsigned*>(&As[r + g][2 * t4]);
        af[mi][1] = *reinterpret_cast<const unsigned*>(&As[r + g + 8][2 * t4]);
        af[mi][2] = *reinterpret_cast<const unsigned*>(&As[r + g][2 * t4 + 8]);
        af[mi][3] = *reinterpret_cast<const unsigned*>(&As[r + g + 8][2 * t4 + 8]);
    }
#pragma unroll
    for (int ni = 0; ni < 4; ++ni) {
        const int n = wn * 32 + ni * 8;
        bfr[ni][0] = *reinterpret_cast<const unsigned*>(&Bs[n + g][2 * t4]);
        bfr[ni][1] = *reinterpret_cast<const unsigned*>(&Bs[n + g][2 * t4 + 8]);
    }
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], af[mi], bfr[ni]);
}

// 8 consecutive bf16 of a channel slice, zero outside [0, limit).
__device__ __forceinline__ uint4 load8(const bf16* src, int c, int limit, bool vec)
{
    if (vec && c + 8 <= limit) return *reinterpret_cast<const uint4*>(src);
    union {
        uint4 v;
        bf16 h[8];
    } u;
#pragma unroll
    for (int k = 0; k < 8; ++k) u.h[k] = (c + k < limit) ? src[k] : __float2bfloat16_rn(0.0f);
    return u.v;
}

struct ConvArgs {
    const bf16* in;       // in[p * ldi + offi + ci], p = y * W + x
    int ldi, offi;
    const bf16* w;        // [Cout][9][Cin]
    const float* bias;    // [Cout] or null
    void* out;            // out[p * ldo + offo + co], bf16 or f32
    int ldo, offo, out_f32;
    int H, W, Cin, Cout;
    int relu;
};

// out = act(conv3x3(in, w) + bias), zero padding.
__global__ void __launch_bounds__(128) k_conv3x3(ConvArgs a)
{
    __shared__ __align__(16) bf16 As[CM][SP];
    __shared__ __align__(16) bf16 Bs[CN][SP];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;
    const int HW = a.H * a.W;
    const int p0 = blockIdx.x * CM, co0 = blockIdx.y * CN;
    const bool vin = ((a.ldi | a.offi | a.Cin) & 7) == 0;
    const bool vw = (a.Cin & 7) == 0;
    float acc[2][4][4];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[mi][ni][c] = 0.0f;
    const int m = tid >> 1, kh = (tid & 1) * 8;
    const int p = p0 + m;
    const int py = p / a.W, px = p - py * a.W;
    const int ksteps = (a.Cin + CK - 1) / CK;
    for (int kk = 0; kk < 9; ++kk) {
        const int y = py + kk / 3 - 1, x = px + kk % 3 - 1;
        const bool inside = p < HW && y >= 0 && y < a.H && x >= 0 && x < a.W;
        const bf16* srcA = a.in + (size_t)(y * a.W + x) * a.ldi + a.offi;
        const int co = co0 + m;
        const bf16* srcB = a.w + ((size_t)co * 9 + kk) * a.Cin;
        for (int ks = 0; ks < ksteps; ++ks) {
            const int c = ks * CK + kh;
            uint4 va = make_uint4(0, 0, 0, 0), vb = make_uint4(0, 0, 0, 0);
            if (inside) va = load8(srcA + c, c, a.Cin, vin);
            if (co < a.Cout) vb = load8(srcB + c, c, a.Cin, vw);
            *reinterpret_cast<uint4*>(&As[m][kh]) = va;
            *reinterpret_cast<uint4*>(&Bs[m][kh]) = vb;
            __syncthreads();
            warp_mma_stage(As, Bs, wm, wn, lane, acc);
            __syncthreads();
        }
    }
    const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int pp = p0 + wm * 32 + mi * 16 + g + (c >= 2 ? 8 : 0);
                const int cc = co0 + wn * 32 + ni * 8 + 2 * t4 + (c & 1);
                if (pp >= HW || cc >= a.Cout) continue;
                float v = acc[mi][ni][c] + (a.bias ? a.bias[cc] : 0.0f);
                if (a.relu) v = fmaxf(v, 0.0f);
                const size_t o = (size_t)pp * a.ldo + a.offo + cc;
                if (a.out_f32) static_cast<float*>(a.out)[o] = v;
                else static_cast<bf16*>(a.out)[o] = __float2bfloat16_rn(v);
            }
}

struct WgradArgs {
    const bf16* g;        // g[p * ldg + offg + co] (masked gradient of the conv output)
    int ldg, offg;
    const bf16* x;        // x[p * ldx + offx + ci] (conv input)
    int ldx, offx;
    float* part;          // [chunks][Cout][9][Cin]
    int H, W, Cin, Cout, chunk;
};

// part[chunk][co][kk][ci] = sum over the chunk's pixels p of g[p][co] x[p + off(kk)][ci]
__global__ void __launch_bounds__(128) k_wgrad(WgradArgs a)
{
    __shared__ __align__(16) bf16 As[CM][SP];   // [co][p]
    __shared__ __align__(16) bf16 Bs[CN][SP];   // [ci][p]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;
    const int co0 = blockIdx.x * CM, ci0 = blockIdx.y * CN;
    const int kk = blockIdx.z % 9, ch = blockIdx.z / 9;
    const int dy = kk / 3 - 1, dx = kk % 3 - 1;
    const int HW = a.H * a.W;
    const int pbeg = ch * a.chunk, pend = min(HW, pbeg + a.chunk);
    float acc[2][4][4];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[mi][ni][c] = 0.0f;
    const int k = tid >> 3, seg = (tid & 7) * 8;   // pixel k of the stage, channels seg..seg+7
    const bool vg = ((a.ldg | a.offg | a.Cout) & 7) == 0;
    const bool vx = ((a.ldx | a.offx | a.Cin) & 7) == 0;
    for (int ps = pbeg; ps < pend; ps += CK) {
        const int p = ps + k;
        union {
            uint4 v;
            bf16 h[8];
        } ug, ux;
        ug.v = make_uint4(0, 0, 0, 0);
        ux.v = make_uint4(0, 0, 0, 0);
        if (p < pend) {
            ug.v = load8(a.g + (size_t)p * a.ldg + a.offg + co0 + seg, co0 + seg, a.Cout, vg);
            const int py = p / a.W, px = p - py * a.W;
            const int y = py + dy, x = px + dx;
            if (y >= 0 && y < a.H && x >= 0 && x < a.W)
                ux.v = load8(a.x + (size_t)(y * a.W + x) * a.ldx + a.offx + ci0 + seg, ci0 + seg, a.Cin, vx);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            As[seg + j][k] = ug.h[j];
            Bs[seg + j][k] = ux.h[j];
        }
        __syncthreads();
        warp_mma_stage(As, Bs, wm, wn, lane, acc);
        __syncthreads();
    }
    const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int co = co0 + wm * 32 + mi * 16 + g + (c >= 2 ? 8 : 0);
                const int ci = ci0 + wn * 32 + ni * 8 + 2 * t4 + (c & 1);
                if (co >= a.Cout || ci >= a.Cin) continue;
                a.part[(((size_t)ch * a.Cout + co) * 9 + kk) * a.Cin + ci] = acc[mi][ni][c];
            }
}

// out[i] = sum over chunks (in order) of part[chunk][i]
__global__ void k_sum_chunks(const float* __restrict__ part, int chunks, size_t n, float* __restrict__ out)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int c = 0; c < chunks; ++c) s += part[(size_t)c * n + i];
        out[i] = s;
    }
}

// bias gradient partials: part[chunk][co] = sum over the chunk's pixels of g[p][co].
// With C < blockDim.x the block's threads form L = blockDim.x / C pixel lanes per
// channel (consecutive threads read consecutive channels of one pixel) and the lanes
// are summed in lane order; with C >= blockDim.x each thread sums whole channels.
__global__ void k_colsum(const bf16* __restrict__ g, int ldg, int offg, int HW, int C, int chunk, float* part)
{
    __shared__ float red[256];
    const int pbeg = blockIdx.x * chunk, pend = min(HW, pbeg + chunk);
    if (C >= (int)blockDim.x) {
        for (int co = threadIdx.x; co < C; co += blockDim.x) {
            float s = 0.0f;
            for (int p = pbeg; p < pend; ++p) s += __bfloat162float(g[(size_t)p * ldg + offg + co]);
            part[(size_t)blockIdx.x * C + co] = s;
        }
        return;
    }
    const int L = (int)blockDim.x / C;
    const int co = threadIdx.x % C, lp = threadIdx.x / C;
    float s = 0.0f;
    if (lp < L)
        for (int p = pbeg + lp; p < pend; p += L) s += __bfloat162float(g[(size_t)p * ldg + offg + co]);
    red[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < C) {
        float t = 0.0f;
        for (int q = 0; q < L; ++q) t += red[q * C + threadIdx.x];
        part[(size_t)blockIdx.x * C + threadIdx.x] = t;
    }
}

// gm = bf16(gin * (y > 0)) (relu) or bf16(gin)
__global__ void k_mask(const float* __restrict__ gin, const bf16* __restrict__ y, int ldy, int offy, int HW, int C,
                       int relu, bf16* __restrict__ gm)
{
    const size_t n = (size_t)HW * C;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t p = i / C, c = i - p * C;
        float v = gin[i];
        if (relu && !(__bfloat162float(y[p * ldy + offy + c]) > 0.0f)) v = 0.0f;
        gm[i] = __float2bfloat16_rn(v);
    }
}

// 2x2 average pooling: out[Y][X][c] = mean of in[2Y+dy][2X+dx][c]
__global__ void k_pool(const bf16* __restrict__ in, int ldi, int offi, int H, int W, int C, bf16* __restrict__ out)
{
    const int Ho = H / 2, Wo = W / 2;
    const size_t n = (size_t)Ho * Wo * C;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const size_t q = i / C;
        const int Y = (int)(q / Wo), X = (int)(q % Wo);
        float s = 0.0f;
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx)
                s += __bfloat162float(in[((size_t)(2 * Y + dy) * W + 2 * X + dx) * ldi + offi + c]);
        out[i] = __float2bfloat16_rn(0.25f * s);
    }
}

// gradient of the pooling: gin[y][x][c] (+)= 0.25 gout[y/2][x/2][c]
__global__ void k_pool_bwd(const float* __restrict__ gout, int H, int W, int C, float* __restrict__ gin, int ldg,
                           int offg, int accumulate)
{
    const size_t n = (size_t)H * W * C;
    const int Wo = W / 2;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const size_t q = i / C;
        const int y = (int)(q / W), x = (int)(q % W);
        const float v = 0.25f * gout[((size_t)(y / 2) * Wo + x / 2) * C + c];
        float* dst = gin + q * ldg + offg + c;
        *dst = accumulate ? *dst + v : v;
    }
}

// nearest 2x upsampling into a channel slice: out[y][x][offo + c] = in[y/2][x/2][c]
__global__ void k_up(const bf16* __restrict__ in, int Hi, int Wi, int C, bf16* __restrict__ out, int ldo, int offo)
{
    const int H = 2 * Hi, W = 2 * Wi;
    const size_t n = (size_t)H * W * C;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const size_t q = i / C;
        const int y = (int)(q / W), x = (int)(q % W);
        out[q * ldo + offo + c] = in[((size_t)(y / 2) * Wi + x / 2) * C + c];
    }
}

// gradient of the upsampling: gin[Y][X][c] = sum of gout[2Y+dy][2X+dx][offg + c]
__global__ void k_up_bwd(const float* __restrict__ gout, int ldg, int offg, int Hi, int Wi, int C, float* __restrict__ gin)
{
    const int W = 2 * Wi;
    const size_t n = (size_t)Hi * Wi * C;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const size_t q = i / C;
        const int Y = (int)(q / Wi), X = (int)(q % Wi);
        float s = 0.0f;
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) s += gout[((size_t)(2 * Y + dy) * W + 2 * X + dx) * ldg + offg + c];
        gin[i] = s;
    }
}

// add a channel slice: dst[p][c] += src[p * lds + offs + c]
__global__ void k_add_slice(const float* __restrict__ src, int lds, int offs, int HW, int C, float* __restrict__ dst)
{
    const size_t n = (size_t)HW * C;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t p = i / C, c = i - p * C;
        dst[i] += src[p * lds + offs + c];
    }
}

// float image -> bf16 one-channel tensor
__global__ void k_to_bf16(const float* __restrict__ x, size_t n, bf16* __restrict__ y)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

// head: y[p] = x[p] + sum_c h[p][c] w[c] + b (1x1 convolution to one channel, residual)
__global__ void k_head(const bf16* __restrict__ h, int C, const float* __restrict__ w, const float* __restrict__ b,
                       const float* __restrict__ x, int HW, float* __restrict__ y)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += gridDim.x * blockDim.x) {
        float s = b[0];
        for (int c = 0; c < C; ++c) s = fmaf(__bfloat162float(h[(size_t)p * C + c]), w[c], s);
        y[p] = x[p] + s;
    }
}

// MSE loss pieces: dy[p] = 2 (y[p] - t[p]) / HW; partial sums of (y - t)^2 per block (FP64)
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ t, int HW, float* __restrict__ dy,
                      double* __restrict__ part)
{
    __shared__ double red[256];
    double s = 0.0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += gridDim.x * blockDim.x) {
        const float d = y[p] - t[p];
        dy[p] = 2.0f * d / (float)HW;
        s += (double)d * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// head backward: gh[p][c] = dy[p] w[c]; partial sums of dy[p] h[p][c] and dy[p] per block
__global__ void k_head_bwd(const float* __restrict__ dy, const bf16* __restrict__ h, int C, const float* __restrict__ w,
                           int HW, float* __restrict__ gh, float* __restrict__ part /*[blocks][C+1]*/)
{
    extern __shared__ float sh[];   // [blockDim][C+1]
    float* mine = sh + threadIdx.x * (C + 1);
    for (int c = 0; c <= C; ++c) mine[c] = 0.0f;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += gridDim.x * blockDim.x) {
        const float d = dy[p];
        for (int c = 0; c < C; ++c) {
            gh[(size_t)p * C + c] = d * w[c];
            mine[c] = fmaf(d, __bfloat162float(h[(size_t)p * C + c]), mine[c]);
        }
        mine[C] += d;
    }
    __syncthreads();
    for (int c = threadIdx.x; c <= C; c += blockDim.x) {
        float s = 0.0f;
        for (int t = 0; t < (int)blockDim.x; ++t) s += sh[t * (C + 1) + c];
        part[(size_t)blockIdx.x * (C + 1) + c] = s;
    }
}

// Adam (Kingma & Ba 2015) on FP32 master weights; writes the bf16 copy.
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, size_t n, float lr, float b1, float b2, float eps, float c1,
                       float c2, bf16* __restrict__ wb)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        if (wb) wb[i] = __float2bfloat16_rn(wi);
    }
}

// bf16 copies of a conv's weights: wb[co][kk][ci] and the flipped, transposed wf[ci][8-kk][co]
__global__ void k_wcopies(const float* __restrict__ w, int Cout, int Cin, bf16* __restrict__ wb, bf16* __restrict__ wf)
{
    const size_t n = (size_t)Cout * 9 * Cin;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int ci = (int)(i % Cin);
        const int kk = (int)((i / Cin) % 9);
        const int co = (int)(i / ((size_t)9 * Cin));
        const bf16 v = __float2bfloat16_rn(w[i]);
        wb[i] = v;
        wf[((size_t)ci * 9 + (8 - kk)) * Cout + co] = v;
    }
}

int grid_of(size_t n)
{
    size_t g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

// ============================================================== network object

struct ncs_unet {
    struct Conv {
        int Cin, Cout, relu, level;
        size_t woff, boff;          // offsets in the flat parameter vector
        bf16 *wb = nullptr, *wf = nullptr;
    };
    struct Level {
        int c;                      // channels of this level
        int H, W;
        int ea, eb, da, db;         // conv indices (da, db = -1 at the bottom)
        bf16* in = nullptr;         // level input (level 0: the image, else pooled), cin channels
        int cin;
        bf16* a = nullptr;          // output of ea (c channels)
        bf16* cat = nullptr;        // [up(c_next) | skip(c)] (not at the bottom)
        bf16* bot = nullptr;        // output of eb at the bottom
        bf16* d1 = nullptr;         // output of da
        bf16* out = nullptr;        // output of db (or eb at the bottom): the level's result, c channels
        float *g_out = nullptr, *g_a = nullptr, *g_cat = nullptr, *g_in = nullptr, *g_d1 = nullptr, *g_skip = nullptr;
    };
    int dev = 0;
    int H = 0, W = 0, levels = 0, base = 0;
    std::vector<Conv> convs;
    std::vector<Level> L;
    size_t n_params = 0;
    size_t head_w = 0, head_b = 0;
    float *w = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;  // FP32 master, Adam moments, gradient
    bf16* xin = nullptr;            // input image as bf16
    float *y = nullptr, *dy = nullptr;
    float* part = nullptr;          // split-K partials
    size_t part_elems = 0;
    double* dpart = nullptr;
    double* h_pin = nullptr;
    bf16* gm = nullptr;             // masked bf16 gradient scratch
    float* gtmp = nullptr;          // FP32 gradient scratch
    long long step = 0;
    cudaStream_t st = nullptr;
};

namespace {

#define UCK(expr)                                                            \
    do {                                                                     \
        cudaError_t e_ = (expr);                                             \
        if (e_ != cudaSuccess) {                                             \
            fprintf(stderr, "ncs_unet: %s failed: %s\n", #expr, cudaGetErrorString(e_)); \
            return NCS_ERR_CUDA;                                             \
        }                                                                    \
    } while (0)

template <class T>
int ualloc(T** p, size_t n)
{
    if (cudaMalloc((void**)p, (n ? n : 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return NCS_ERR_NOMEM;
    }
    return NCS_OK;
}

#define UCKS(expr)                 \
    do {                           \
        int s_ = (expr);           \
        if (s_ < 0) return s_;     \
    } while (0)

int conv_fwd(ncs_unet* n, const ncs_unet::Conv& c, const bf16* in, int ldi, int offi, void* out, int ldo, int offo,
             int out_f32, int H, int W, const bf16* wts, int Cin, int Cout, const float* bias, int relu)
{
    ConvArgs a{};
    a.in = in; a.ldi = ldi; a.offi = offi;
    a.w = wts; a.bias = bias;
    a.out = out; a.ldo = ldo; a.offo = offo; a.out_f32 = out_f32;
    a.H = H; a.W = W; a.Cin = Cin; a.Cout = Cout; a.relu = relu;
    (void)c;
    dim3 grid((H * W + CM - 1) / CM, (Cout + CN - 1) / CN);
    k_conv3x3<<<grid, 128, 0, n->st>>>(a);
    UCK(cudaGetLastError());
    return NCS_OK;
}

// Backward of one conv: g_out (FP32, HW x Cout, dense) -> masked bf16 -> dW, db (into n->grad), g_in (optional)
int conv_bwd(ncs_unet* n, const ncs_unet::Conv& c, const float* g_out, const bf16* y, int ldy, int offy,
             const bf16* x, int ldx, int offx, int H, int W, float* g_in, int ld_gin, int off_gin)
{
    const int HW = H * W;
    k_mask<<<grid_of((size_t)HW * c.Cout), 256, 0, n->st>>>(g_out, y, ldy, offy, HW, c.Cout, c.relu, n->gm);
    UCK(cudaGetLastError());
    // weight gradient, split over pixel chunks
    const int chunk = 2048;
    const int chunks = (HW + chunk - 1) / chunk;
    const size_t nw = (size_t)c.Cout * 9 * c.Cin;
    if ((size_t)chunks * nw > n->part_elems) return NCS_ERR_UNSUPPORTED;
    WgradArgs a{};
    a.g = n->gm; a.ldg = c.Cout; a.offg = 0;
    a.x = x; a.ldx = ldx; a.offx = offx;
    a.part = n->part; a.H = H; a.W = W; a.Cin = c.Cin; a.Cout = c.Cout; a.chunk = chunk;
    dim3 grid((c.Cout + CM - 1) / CM, (c.Cin + CN - 1) / CN, 9 * chunks);
    k_wgrad<<<grid, 128, 0, n->st>>>(a);
    UCK(cudaGetLastError());
    k_sum_chunks<<<grid_of(nw), 256, 0, n->st>>>(n->part, chunks, nw, n->grad + c.woff);
    UCK(cudaGetLastError());
    k_colsum<<<chunks, 256, 0, n->st>>>(n->gm, c.Cout, 0, HW, c.Cout, chunk, n->part);
    UCK(cudaGetLastError());
    k_sum_chunks<<<grid_of(c.Cout), 256, 0, n->st>>>(n->part, chunks, c.Cout, n->grad + c.boff);
    UCK(cudaGetLastError());
    if (g_in) {
        // data gradient: the forward kernel with flipped, transposed weights
        ConvArgs d{};
        d.in = n->gm; d.ldi = c.Cout; d.offi = 0;
        d.w = c.wf; d.bias = nullptr;
        d.out = g_in; d.ldo = ld_gin; d.offo = off_gin; d.out_f32 = 1;
        d.H = H; d.W = W; d.Cin = c.Cout; d.Cout = c.Cin; d.relu = 0;
        dim3 g2((HW + CM - 1) / CM, (c.Cin + CN - 1) / CN);
        k_conv3x3<<<g2, 128, 0, n->st>>>(d);
        UCK(cudaGetLastError());
    }
    return NCS_OK;
}

int refresh_weights(ncs_unet* n)
{
    for (auto& c : n->convs) {
        k_wcopies<<<grid_of((size_t)c.Cout * 9 * c.Cin), 256, 0, n->st>>>(n->w + c.woff, c.Cout, c.Cin, c.wb, c.wf);
        UCK(cudaGetLastError());
    }
    return NCS_OK;
}

int forward(ncs_unet* n, const float* x)
{
    const int HW0 = n->H * n->W;
    k_to_bf16<<<grid_of(HW0), 256, 0, n->st>>>(x, HW0, n->xin);
    UCK(cudaGetLastError());
    const int NL = n->levels;
    // encoder
    for (int l = 0; l < NL; ++l) {
        auto& lv = n->L[l];
        const auto& ea = n->convs[lv.ea];
        const auto& eb = n->convs[lv.eb];
        UCKS(conv_fwd(n, ea, lv.in, lv.cin, 0, lv.a, lv.c, 0, 0, lv.H, lv.W, ea.wb, ea.Cin, ea.Cout, n->w + ea.boff, 1));
        if (l < NL - 1) {
            const int cn = n->L[l + 1].c;
            UCKS(conv_fwd(n, eb, lv.a, lv.c, 0, lv.cat, cn + lv.c, cn, 0, lv.H, lv.W, eb.wb, eb.Cin, eb.Cout,
                          n->w + eb.boff, 1));
            auto& nx = n->L[l + 1];
            k_pool<<<grid_of((size_t)nx.H * nx.W * lv.c), 256, 0, n->st>>>(lv.cat, cn + lv.c, cn, lv.H, lv.W, lv.c, nx.in);
            UCK(cudaGetLastError());
        } else {
            UCKS(conv_fwd(n, eb, lv.a, lv.c, 0, lv.out, lv.c, 0, 0, lv.H, lv.W, eb.wb, eb.Cin, eb.Cout, n->w + eb.boff, 1));
        }
    }
    // decoder
    for (int l = NL - 2; l >= 0; --l) {
        auto& lv = n->L[l];
        auto& nx = n->L[l + 1];
        const int cn = nx.c;
        k_up<<<grid_of((size_t)lv.H * lv.W * cn), 256, 0, n->st>>>(nx.out, nx.H, nx.W, cn, lv.cat, cn + lv.c, 0);
        UCK(cudaGetLastError());
        const auto& da = n->convs[lv.da];
        const auto& db = n->convs[lv.db];
        UCKS(conv_fwd(n, da, lv.cat, cn + lv.c, 0, lv.d1, lv.c, 0, 0, lv.H, lv.W, da.wb, da.Cin, da.Cout, n->w + da.boff, 1));
        UCKS(conv_fwd(n, db, lv.d1, lv.c, 0, lv.out, lv.c, 0, 0, lv.H, lv.W, db.wb, db.Cin, db.Cout, n->w + db.boff, 1));
    }
    auto& l0 = n->L[0];
    k_head<<<grid_of(HW0), 256, 0, n->st>>>(l0.out, l0.c, n->w + n->head_w, n->w + n->head_b, x, HW0, n->y);
    UCK(cudaGetLastError());
    return NCS_OK;
}

// loss and gradient of 1/HW ||y - t||^2 with respect to every parameter (into n->grad)
int backward(ncs_unet* n, const float* x, const float* t, double* loss)
{
    (void)x;
    const int HW0 = n->H * n->W;
    const int NL = n->levels;
    const int nb = 128;
    k_mse<<<nb, 256, 0, n->st>>>(n->y, t, HW0, n->dy, n->dpart);
    UCK(cudaGetLastError());
    UCK(launch_finalize(n->dpart, nb, 1.0 / HW0, nullptr, 0, 0.0, n->dpart + nb, n->st));
    auto& l0 = n->L[0];
    // head
    {
        // per-thread partials [threads][C + 1] within the default 48 KB of shared memory
        const int C = l0.c, blocks = 64;
        const int threads = std::max(32, std::min(128, (int)(48 * 1024 / ((C + 1) * sizeof(float))) / 32 * 32));
        const size_t smem = (size_t)threads * (C + 1) * sizeof(float);
        k_head_bwd<<<blocks, threads, smem, n->st>>>(n->dy, l0.out, C, n->w + n->head_w, HW0, l0.g_out, n->part);
        UCK(cudaGetLastError());
        // sum the block partials in order: w grads (C values) then b
        k_sum_chunks<<<grid_of(C + 1), 256, 0, n->st>>>(n->part, blocks, C + 1, n->gtmp);
        UCK(cudaGetLastError());
        UCK(cudaMemcpyAsync(n->grad + n->head_w, n->gtmp, C * sizeof(float), cudaMemcpyDeviceToDevice, n->st));
        UCK(cudaMemcpyAsync(n->grad + n->head_b, n->gtmp + C, sizeof(float), cudaMemcpyDeviceToDevice, n->st));
    }
    // decoder levels, top down in gradient order
    for (int l = 0; l <= NL - 2; ++l) {
        // processed after level l-1 provided g_out of level l (level 0: from the head)
    }
    // walk levels from 0 to the bottom: db, da, split the concat gradient
    for (int l = 0; l < NL - 1; ++l) {
        auto& lv = n->L[l];
        auto& nx = n->L[l + 1];
        const int cn = nx.c, ccat = cn + lv.c;
        const auto& db = n->convs[lv.db];
        const auto& da = n->convs[lv.da];
        UCKS(conv_bwd(n, db, lv.g_out, lv.out, lv.c, 0, lv.d1, lv.c, 0, lv.H, lv.W, lv.g_d1, lv.c, 0));
        UCKS(conv_bwd(n, da, lv.g_d1, lv.d1, lv.c, 0, lv.cat, ccat, 0, lv.H, lv.W, lv.g_cat, ccat, 0));
        // up part -> gradient of the next level's output
        k_up_bwd<<<grid_of((size_t)nx.H * nx.W * cn), 256, 0, n->st>>>(lv.g_cat, ccat, 0, nx.H, nx.W, cn, nx.g_out);
        UCK(cudaGetLastError());
    }
    // encoder, bottom up
    for (int l = NL - 1; l >= 0; --l) {
        auto& lv = n->L[l];
        const auto& eb = n->convs[lv.eb];
        const auto& ea = n->convs[lv.ea];
        float* g_eb_out;
        const bf16* eb_out;
        int ld_ebo, off_ebo;
        if (l == NL - 1) {
            g_eb_out = lv.g_out;
            eb_out = lv.out;
            ld_ebo = lv.c;
            off_ebo = 0;
        } else {
            // skip gradient: from the concat (its skip part) plus the pooling path
            auto& nx = n->L[l + 1];
            const int cn = nx.c, ccat = cn + lv.c;
            k_pool_bwd<<<grid_of((size_t)lv.H * lv.W * lv.c), 256, 0, n->st>>>(nx.g_in, lv.H, lv.W, lv.c, lv.g_skip,
                                                                               lv.c, 0, 0);
            UCK(cudaGetLastError());
            k_add_slice<<<grid_of((size_t)lv.H * lv.W * lv.c), 256, 0, n->st>>>(lv.g_cat, ccat, cn, lv.H * lv.W, lv.c,
                                                                               lv.g_skip);
            UCK(cudaGetLastError());
            g_eb_out = lv.g_skip;
            eb_out = lv.cat;
            ld_ebo = ccat;
            off_ebo = cn;
        }
        UCKS(conv_bwd(n, eb, g_eb_out, eb_out, ld_ebo, off_ebo, lv.a, lv.c, 0, lv.H, lv.W, lv.g_a, lv.c, 0));
        UCKS(conv_bwd(n, ea, lv.g_a, lv.a, lv.c, 0, lv.in, lv.cin, 0, lv.H, lv.W, l > 0 ? lv.g_in : nullptr, lv.cin, 0));
    }
    if (loss) {
        UCK(cudaMemcpyAsync(n->h_pin, n->dpart + nb, sizeof(double), cudaMemcpyDeviceToHost, n->st));
        UCK(cudaStreamSynchronize(n->st));
        *loss = n->h_pin[0];
    }
    return NCS_OK;
}

void free_unet(ncs_unet* n)
{
    for (auto& c : n->convs) { cudaFree(c.wb); cudaFree(c.wf); }
    for (auto& lv : n->L) {
        if (lv.in != n->xin) cudaFree(lv.in);
        cudaFree(lv.a); cudaFree(lv.cat); cudaFree(lv.d1); cudaFree(lv.out);
        cudaFree(lv.g_out); cudaFree(lv.g_a); cudaFree(lv.g_cat); cudaFree(lv.g_in); cudaFree(lv.g_d1);
        cudaFree(lv.g_skip);
    }
    cudaFree(n->w); cudaFree(n->m); cudaFree(n->v); cudaFree(n->grad); cudaFree(n->xin);
    cudaFree(n->y); cudaFree(n->dy); cudaFree(n->part); cudaFree(n->dpart); cudaFree(n->gm); cudaFree(n->gtmp);
    if (n->h_pin) cudaFreeHost(n->h_pin);
    if (n->st) cudaStreamDestroy(n->st);
}

int build_unet(ncs_unet* n, uint64_t seed)
{
    UCK(cudaGetDevice(&n->dev));
    UCK(cudaStreamCreateWithFlags(&n->st, cudaStreamNonBlocking));
    const int NL = n->levels;
    n->L.resize(NL);
    size_t off = 0;
    auto add_conv = [&](int cin, int cout, int level) {
        ncs_unet::Conv c;
        c.Cin = cin; c.Cout = cout; c.relu = 1; c.level = level;
        c.woff = off; off += (size_t)cout * 9 * cin;
        c.boff = off; off += cout;
        n->convs.push_back(c);
        return (int)n->convs.size() - 1;
    };
    for (int l = 0; l < NL; ++l) {
        auto& lv = n->L[l];
        lv.c = n->base << l;
        lv.H = n->H >> l;
        lv.W = n->W >> l;
        lv.cin = l == 0 ? 1 : n->L[l - 1].c;
        lv.ea = add_conv(lv.cin, lv.c, l);
        lv.eb = add_conv(lv.c, lv.c, l);
        lv.da = lv.db = -1;
    }
    for (int l = NL - 2; l >= 0; --l) {
        auto& lv = n->L[l];
        lv.da = add_conv(n->L[l + 1].c + lv.c, lv.c, l);
        lv.db = add_conv(lv.c, lv.c, l);
    }
    n->head_w = off; off += n->L[0].c;
    n->head_b = off; off += 1;
    n->n_params = off;
    UCKS(ualloc(&n->w, off)); UCKS(ualloc(&n->m, off)); UCKS(ualloc(&n->v, off)); UCKS(ualloc(&n->grad, off));
    UCK(cudaMemsetAsync(n->m, 0, off * sizeof(float), n->st));
    UCK(cudaMemsetAsync(n->v, 0, off * sizeof(float), n->st));
    UCK(cudaMemsetAsync(n->grad, 0, off * sizeof(float), n->st));
    // He initialisation (normal, std sqrt(2 / fan_in)); biases 0; head small
    std::vector<float> hw(off, 0.0f);
    std::mt19937_64 rng(seed);
    for (auto& c : n->convs) {
        std::normal_distribution<float> nd(0.0f, std::sqrt(2.0f / (9.0f * c.Cin)));
        for (size_t i = 0; i < (size_t)c.Cout * 9 * c.Cin; ++i) hw[c.woff + i] = nd(rng);
    }
    {
        std::normal_distribution<float> nd(0.0f, 1e-3f);
        for (int c = 0; c < n->L[0].c; ++c) hw[n->head_w + c] = nd(rng);
    }
    UCK(cudaMemcpyAsync(n->w, hw.data(), off * sizeof(float), cudaMemcpyHostToDevice, n->st));
    size_t max_part = 0, max_act = 0;
    for (auto& c : n->convs) {
        const size_t nw = (size_t)c.Cout * 9 * c.Cin;
        UCKS(ualloc(&c.wb, nw));
        UCKS(ualloc(&c.wf, nw));
        const size_t HW = (size_t)(n->H >> c.level) * (n->W >> c.level);
        max_part = std::max(max_part, ((HW + 2047) / 2048) * nw);
    }
    for (int l = 0; l < NL; ++l) {
        auto& lv = n->L[l];
        const size_t HW = (size_t)lv.H * lv.W;
        if (l == 0) {
            UCKS(ualloc(&n->xin, HW));
            lv.in = n->xin;
        } else {
            UCKS(ualloc(&lv.in, HW * lv.cin));
            UCKS(ualloc(&lv.g_in, HW * lv.cin));
        }
        UCKS(ualloc(&lv.a, HW * lv.c));
        UCKS(ualloc(&lv.g_a, HW * lv.c));
        UCKS(ualloc(&lv.g_out, HW * lv.c));
        if (l < NL - 1) {
            const int ccat = n->L[l + 1].c + lv.c;
            UCKS(ualloc(&lv.cat, HW * ccat));
            UCKS(ualloc(&lv.g_cat, HW * ccat));
            UCKS(ualloc(&lv.d1, HW * lv.c));
            UCKS(ualloc(&lv.g_d1, HW * lv.c));
            UCKS(ualloc(&lv.g_skip, HW * lv.c));
            max_act = std::max(max_act, HW * ccat);
        }
        UCKS(ualloc(&lv.out, HW * lv.c));
        max_act = std::max(max_act, HW * lv.c);
    }
    n->part_elems = std::max(max_part, (size_t)64 * (n->L[0].c + 1));
    UCKS(ualloc(&n->part, n->part_elems));
    UCKS(ualloc(&n->gm, max_act));
    UCKS(ualloc(&n->gtmp, std::max((size_t)n->L[0].c + 1, (size_t)16)));
    UCKS(ualloc(&n->y, (size_t)n->H * n->W));
    UCKS(ualloc(&n->dy, (size_t)n->H * n->W));
    UCKS(ualloc(&n->dpart, 256));
    if (cudaMallocHost((void**)&n->h_pin, 4 * sizeof(double)) != cudaSuccess) { cudaGetLastError(); return NCS_ERR_NOMEM; }
    UCKS(refresh_weights(n));
    UCK(cudaStreamSynchronize(n->st));
    return NCS_OK;
}

}  // namespace

extern "C" {

int ncs_unet_create(int H, int W, int levels, int base_channels, uint64_t seed, ncs_unet** out)
{
    if (!out) return NCS_ERR_BADARG;
    *out = nullptr;
    if (levels < 1 || levels > 6 || base_channels < 1 || base_channels > 256 || H < 1 || W < 1) return NCS_ERR_BADARG;
    if (H % (1 << (levels - 1)) != 0 || W % (1 << (levels - 1)) != 0) return NCS_ERR_UNSUPPORTED;
    ncs_unet* n = new (std::nothrow) ncs_unet();
    if (!n) return NCS_ERR_NOMEM;
    n->H = H; n->W = W; n->levels = levels; n->base = base_channels;
    int rc = build_unet(n, seed);
    if (rc != NCS_OK) { free_unet(n); delete n; return rc; }
    *out = n;
    return NCS_OK;
}

void ncs_unet_destroy(ncs_unet* n)
{
    if (!n) return;
    cudaSetDevice(n->dev);
    if (n->st) cudaStreamSynchronize(n->st);
    free_unet(n);
    delete n;
}

size_t ncs_unet_num_params(const ncs_unet* n) { return n ? n->n_params : 0; }

int ncs_unet_params(ncs_unet* n, float* host, int set)
{
    if (!n || !host) return NCS_ERR_BADARG;
    UCK(cudaSetDevice(n->dev));
    if (set) {
        UCK(cudaMemcpyAsync(n->w, host, n->n_params * sizeof(float), cudaMemcpyHostToDevice, n->st));
        UCKS(refresh_weights(n));
    } else {
        UCK(cudaMemcpyAsync(host, n->w, n->n_params * sizeof(float), cudaMemcpyDeviceToHost, n->st));
    }
    UCK(cudaStreamSynchronize(n->st));
    return NCS_OK;
}

int ncs_unet_forward(ncs_unet* n, const float* x, float* y)
{
    if (!n || !x || !y) return NCS_ERR_BADARG;
    UCK(cudaSetDevice(n->dev));
    UCKS(forward(n, x));
    UCK(cudaMemcpyAsync(y, n->y, (size_t)n->H * n->W * sizeof(float), cudaMemcpyDeviceToDevice, n->st));
    UCK(cudaStreamSynchronize(n->st));
    return NCS_OK;
}

int ncs_unet_gradient(ncs_unet* n, const float* x, const float* target, double* loss, float* grad_host)
{
    if (!n || !x || !target) return NCS_ERR_BADARG;
    UCK(cudaSetDevice(n->dev));
    UCKS(forward(n, x));
    UCKS(backward(n, x, target, loss));
    if (grad_host) {
        UCK(cudaMemcpyAsync(grad_host, n->grad, n->n_params * sizeof(float), cudaMemcpyDeviceToHost, n->st));
        UCK(cudaStreamSynchronize(n->st));
    }
    return NCS_OK;
}

int ncs_unet_train_step(ncs_unet* n, const float* x, const float* target, float lr, double* loss)
{
    if (!n || !x || !target || !(lr > 0.0f)) return NCS_ERR_BADARG;
    UCK(cudaSetDevice(n->dev));
    UCKS(forward(n, x));
    UCKS(backward(n, x, target, loss));
    n->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, (float)n->step), c2 = 1.0f - std::pow(b2, (float)n->step);
    k_adam<<<grid_of(n->n_params), 256, 0, n->st>>>(n->w, n->m, n->v, n->grad, n->n_params, lr, b1, b2, 1e-8f, c1, c2,
                                                   nullptr);
    UCK(cudaGetLastError());
    UCKS(refresh_weights(n));
    if (!loss) UCK(cudaStreamSynchronize(n->st));
    return NCS_OK;
}

}  // extern "C"
