// Joseph projector pair for sm_103a.
//
// K (forward, ray-driven): one thread per (angle, bin, row segment); the ray
// is stepped over the rows of x (row-branch angles) or of x^T (column-branch
// angles), so a warp of 32 consecutive bins always reads one contiguous row
// segment.  Partial sums of the segments are combined in shared memory in a
// fixed order, then a fused epilogue applies prox_{alpha g*} to the data dual
// (Sec. 4.1: divide by 1 + alpha; Sec. 4.2: the closed-form S(u; c)), or
// reduces the data term of the objective in FP64.
//
// K^T (gather, pixel-driven, no atomics): every pixel loops over the angles,
// finds the <= 2 rays that reach it and evaluates exactly the FP32 weight
// expression the forward kernel uses, so the two kernels hold the same matrix.
// The epilogue adds (beta/alpha) D^T v and kappa s (A^T of Sec. 4) and, for
// PDHG (eq. (PDHG)), applies the primal update.
#include "ncs_internal.cuh"

namespace ncs {

namespace {

constexpr int FWD_TB = 64;    // bins per block
constexpr int FWD_SEG = 4;    // row segments per ray

// Integer index k0 and interpolation weight w of the crossing f = H + L, where
// H = A_hi t + B_hi q + C_hi is exact and L = B_lo q + (A_lo t + C_lo) is small.
// The one expression both kernels use, so they hold the same FP32 matrix.
__device__ __forceinline__ float split_weight(float H, float L, float& k0)
{
    const float Hi = floorf(H);
    const float fr = (H - Hi) + L;
    const float fl = floorf(fr);
    k0 = Hi + fl;
    return fr - fl;
}

// Closed-form prox of alpha times the conjugate of l(.; b) (Sec. 4.2):
// S(z; c) = 1 + (z - 1 - sqrt((z-1)^2 + 4c)) / 2, evaluated without
// cancellation when z > 1.
__device__ __forceinline__ float kl_conj_prox(float z, float c)
{
    float d = z - 1.0f;
    float root = sqrtf(fmaf(d, d, 4.0f * c));
    return d > 0.0f ? 1.0f - 2.0f * c / (d + root) : 1.0f + 0.5f * (d - root);
}

template <int MODE>
__global__ void __launch_bounds__(FWD_TB * FWD_SEG)
k_fwd(FwdArgs g)
{
    __shared__ float red[FWD_SEG][FWD_TB];
    __shared__ double dred[FWD_TB];
    const int a = blockIdx.y;
    const AngleParam p = g.ap[a];
    const float* __restrict__ im = p.row ? g.img : g.imgT;
    const int N = g.N;
    const int t = blockIdx.x * FWD_TB + threadIdx.x;
    float acc = 0.0f;
    if (t < g.n_det) {
        const float ft = (float)t;
        const float Hr = fmaf(p.Ahi, ft, p.Chi);    // exact
        const float Lr = fmaf(p.Alo, ft, p.Clo);
        const float B = p.Bhi + p.Blo;
        // Rows where the ray can touch the image: f in [-1, N).  Found in FP32
        // with a 2-row margin; the per-step bounds checks stay, so the range
        // only skips steps whose contribution is zero.
        const float f0 = Hr + Lr;
        int jlo = 0, jhi = N;
        if (fabsf(B) > 1e-6f) {
            float j1 = (-1.0f - f0) / B, j2 = ((float)N - f0) / B;
            float lo = fminf(j1, j2), hi = fmaxf(j1, j2);
            lo = fmaxf(lo, -4.0f);
            hi = fminf(hi, (float)N + 4.0f);
            jlo = max(0, (int)floorf(lo) - 2);
            jhi = min(N, (int)ceilf(hi) + 2);
        } else if (!(f0 > -3.0f && f0 < (float)N + 2.0f)) {
            jhi = 0;
        }
        const int len = max(0, jhi - jlo);
        const int chunk = (len + FWD_SEG - 1) / FWD_SEG;
        const int js = jlo + threadIdx.y * chunk;
        const int je = min(jhi, js + chunk);
        for (int j = js; j < je; ++j) {
            const float jf = (float)j;
            float k0f;
            const float w = split_weight(fmaf(p.Bhi, jf, Hr), fmaf(p.Blo, jf, Lr), k0f);
            const int i0 = (int)k0f;
            const float* __restrict__ row = im + (size_t)j * N;
            const float x0 = (i0 >= 0 && i0 < N) ? __ldg(row + i0) : 0.0f;
            const float x1 = (i0 >= -1 && i0 + 1 < N) ? __ldg(row + i0 + 1) : 0.0f;
            acc = fmaf(1.0f - w, x0, acc);
            acc = fmaf(w, x1, acc);
        }
    }
    red[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    double term = 0.0;
    if (threadIdx.y == 0 && t < g.n_det) {
        float tot = red[0][threadIdx.x];
#pragma unroll
        for (int q = 1; q < FWD_SEG; ++q) tot += red[q][threadIdx.x];
        const float y = p.W * tot;
        const size_t idx = (size_t)a * g.n_det + t;
        if (MODE == FWD_PLAIN) {
            g.y[idx] = y;
        } else if (MODE == FWD_PROX_L2) {
            const float z = fmaf(g.alpha, y - g.b[idx], g.y[idx]);
            g.y[idx] = z * g.inv1pa;
        } else if (MODE == FWD_PROX_KL) {
            const float bgv = g.bg ? g.bg[idx] : 0.0f;
            const float z = fmaf(g.alpha, y + bgv, g.y[idx]);
            g.y[idx] = kl_conj_prox(z, g.alpha * g.b[idx]);
        } else if (MODE == FWD_RESID_L2) {
            const double d = (double)y - (double)g.b[idx];
            term = d * d;
        } else {  // FWD_RESID_KL
            const double mu = (double)y + (g.bg ? (double)g.bg[idx] : 0.0);
            const double bb = (double)g.b[idx];
            term = mu - bb;
            if (bb > 0.0) term += bb * log(bb / mu);
        }
    }
    if (MODE == FWD_RESID_L2 || MODE == FWD_RESID_KL) {
        if (threadIdx.y == 0) dred[threadIdx.x] = term;
        __syncthreads();
        if (threadIdx.y == 0 && threadIdx.x < 32) {
            double s = dred[threadIdx.x] + dred[threadIdx.x + 32];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (threadIdx.x == 0) g.partials[blockIdx.y * gridDim.x + blockIdx.x] = s;
        }
    }
}

constexpr int GB_X = 32, GB_Y = 8;     // gather block: 32 x 8 pixels
constexpr int GCHUNK = 256;            // angles staged in shared memory at a time

template <int MODE>
__global__ void __launch_bounds__(GB_X * GB_Y)
k_gather(GatherArgs g)
{
    __shared__ AngleParam sap[GCHUNK];
    const int N = g.N;
    const int i = blockIdx.x * GB_X + threadIdx.x;
    const int j = blockIdx.y * GB_Y + threadIdx.y;
    const bool inb = (i < N) && (j < N);
    const int tid = threadIdx.y * GB_X + threadIdx.x;
    const float fi_ = (float)i, fj_ = (float)j;
    float acc = 0.0f;
    for (int a0 = 0; a0 < g.n_ang; a0 += GCHUNK) {
        const int na = min(GCHUNK, g.n_ang - a0);
        __syncthreads();
        for (int q = tid; q < na; q += GB_X * GB_Y) sap[q] = g.ap[a0 + q];
        __syncthreads();
        if (!inb) continue;
        for (int aa = 0; aa < na; ++aa) {
            const AngleParam p = sap[aa];
            // own: the index interpolated along; other: the stepping index
            const float own = p.row ? fi_ : fj_;
            const float other = p.row ? fj_ : fi_;
            const float Hq = fmaf(p.Bhi, other, p.Chi);                 // exact
            const float base = Hq + fmaf(p.Blo, other, p.Clo);             // ~ B q + C
            const int tc = (int)rintf((own - base) * p.invA);
            const float* __restrict__ ua = g.u + (size_t)(a0 + aa) * g.n_det;
            float acc_a = 0.0f;
#pragma unroll
            for (int q = -1; q <= 1; ++q) {
                const int t = tc + q;
                if (t >= 0 && t < g.n_det) {
                    const float tf = (float)t;
                    float k0f;
                    const float w = split_weight(fmaf(p.Ahi, tf, Hq), fmaf(p.Blo, other, fmaf(p.Alo, tf, p.Clo)), k0f);
                    const float wt = (k0f == own) ? (1.0f - w) : ((k0f + 1.0f == own) ? w : 0.0f);
                    if (wt != 0.0f) acc_a = fmaf(wt, __ldg(ua + t), acc_a);
                }
            }
            acc = fmaf(p.W, acc_a, acc);
        }
    }
    if (!inb) return;
    const size_t pix = (size_t)j * N + i;
    float r = acc;
    if (g.v) {
        const float* vh = g.v;
        const float* vv = g.v + (size_t)N * N;
        float dt = 0.0f;
        if (i < N - 1) dt += vh[pix];
        if (i >= 1) dt -= vh[pix - 1];
        if (j < N - 1) dt += vv[pix];
        if (j >= 1) dt -= vv[pix - N];
        r = fmaf(g.dscale, dt, r);
    }
    if (g.s) r = fmaf(g.kappa, g.s[pix], r);
    if (MODE == GATHER_R) {
        g.r[pix] = r;
    } else {
        const float x = g.x[pix];
        const float x1 = fmaf(-g.inv_gamma, r, x);
        g.x[pix] = x1;
        g.xbar[pix] = 2.0f * x1 - x;
    }
}

}  // namespace

int fwd_num_blocks(int n_det, int n_ang)
{
    return ((n_det + FWD_TB - 1) / FWD_TB) * n_ang;
}

cudaError_t launch_fwd(int mode, const FwdArgs& a, cudaStream_t st)
{
    dim3 grid((a.n_det + FWD_TB - 1) / FWD_TB, a.n_ang), block(FWD_TB, FWD_SEG);
    switch (mode) {
        case FWD_PLAIN: k_fwd<FWD_PLAIN><<<grid, block, 0, st>>>(a); break;
        case FWD_PROX_L2: k_fwd<FWD_PROX_L2><<<grid, block, 0, st>>>(a); break;
        case FWD_PROX_KL: k_fwd<FWD_PROX_KL><<<grid, block, 0, st>>>(a); break;
        case FWD_RESID_L2: k_fwd<FWD_RESID_L2><<<grid, block, 0, st>>>(a); break;
        case FWD_RESID_KL: k_fwd<FWD_RESID_KL><<<grid, block, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_gather(int mode, const GatherArgs& a, cudaStream_t st)
{
    dim3 grid((a.N + GB_X - 1) / GB_X, (a.N + GB_Y - 1) / GB_Y), block(GB_X, GB_Y);
    if (mode == GATHER_R) k_gather<GATHER_R><<<grid, block, 0, st>>>(a);
    else if (mode == GATHER_PDHG) k_gather<GATHER_PDHG><<<grid, block, 0, st>>>(a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace ncs
