// Finite differences, TV dual prox, transposes and FP64 reductions for sm_103a.
//
// k_td works on 32 x 32 image tiles staged in shared memory with a one-pixel
// halo (right column, bottom row), so D (Sec. 2: (D_n x)_i = x_i - x_{i+1}) is
// formed from shared memory and the transposed image x^T (read by the
// column-branch rays of the projector) is written with coalesced stores.
//   TD_PROX : v+ = Pi(v + beta D xbar)  (box [-lam alpha/beta, lam alpha/beta]
//             of Sec. 4.1, or the per-pixel l2 ball for isotropic TV) and
//             s+ = min(0, s + alpha kappa xbar) (Sec. 4.2 nonnegativity row)
//   TD_APPLY: v = c D x, s = kappa x (the D and I rows of A)
//   TD_OBJ  : TV(x) partial sums in FP64 (optionally at max(x, 0))
// Every mode also writes the pair images of x and x^T that the forward
// projector reads (see PAIR_PAD), from the same shared-memory tile.
#include "ncs_internal.cuh"

namespace ncs {

namespace {

constexpr int TT = 32;      // tile side
constexpr int TR = 8;       // block rows

template <int MODE, bool IBF, bool PBF>
__global__ void __launch_bounds__(TT * TR)
k_td(TdArgs g)
{
    __shared__ float tile[TT + 1][TT + 1];
    __shared__ double red[TT * TR];
    const int N = g.N;
    const int i0 = blockIdx.x * TT, j0 = blockIdx.y * TT;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int r = ty; r <= TT; r += TR) {
        for (int c = tx; c <= TT; c += TT) {
            const int gj = j0 + r, gi = i0 + c;
            float val = (gj < N && gi < N) ? g.x[(size_t)gj * N + gi] : 0.0f;
            if (MODE == TD_OBJ && g.clamp) val = fmaxf(val, 0.0f);
            tile[r][c] = val;
        }
    }
    __syncthreads();
    double tv = 0.0;
    const size_t NN = (size_t)N * N;
#pragma unroll
    for (int q = 0; q < TT / TR; ++q) {
        const int r = ty + q * TR, c = tx;
        const int gj = j0 + r, gi = i0 + c;
        if (gj >= N || gi >= N) continue;
        const size_t pix = (size_t)gj * N + gi;
        const float xv = tile[r][c];
        const bool hx = gi < N - 1, hy = gj < N - 1;
        const float dh = hx ? xv - tile[r][c + 1] : 0.0f;
        const float dv = hy ? xv - tile[r + 1][c] : 0.0f;
        if (MODE == TD_PROX) {
            float zh = hx ? fmaf(g.beta, dh, St<IBF>::get(g.v, pix)) : 0.0f;
            float zv = hy ? fmaf(g.beta, dv, St<IBF>::get(g.v, NN + pix)) : 0.0f;
            if (g.iso) {
                const float n2 = fmaf(zh, zh, zv * zv);
                if (n2 > g.rad * g.rad) {
                    const float f = g.rad * rsqrtf(n2);
                    zh *= f;
                    zv *= f;
                }
            } else {
                zh = fminf(fmaxf(zh, -g.rad), g.rad);
                zv = fminf(fmaxf(zv, -g.rad), g.rad);
            }
            const unsigned long long it = IBF ? *g.iter : 0ull;
            St<IBF>::put_sr(g.v, pix, zh, IBF ? rand16(it, pix, 2u) : 0u);
            St<IBF>::put_sr(g.v, NN + pix, zv, IBF ? rand16(it, pix, 3u) : 0u);
            if (g.s)
                St<IBF>::put_sr(g.s, pix, fminf(fmaf(g.ak, xv, St<IBF>::get(g.s, pix)), 0.0f),
                                IBF ? rand16(it, pix, 4u) : 0u);
        } else if (MODE == TD_APPLY) {
            if (g.v) {
                St<IBF>::put(g.v, pix, g.beta * dh);
                St<IBF>::put(g.v, NN + pix, g.beta * dv);
            }
            if (g.s) St<IBF>::put(g.s, pix, g.ak * xv);
        } else if (MODE == TD_OBJ) {
            const double a = dh, b = dv;
            tv += g.iso ? sqrt(a * a + b * b) : fabs(a) + fabs(b);
        }
    }
    // pair images: x2 row j entry i = (x[j][i], x[j][i+1]); xT2 row i entry j = (x[j][i], x[j+1][i])
    const int P = pair_pitch(N);
    if (g.x2) {
#pragma unroll
        for (int q = 0; q < TT / TR; ++q) {
            const int r = ty + q * TR, c = tx;
            const int gj = j0 + r, gi = i0 + c;
            if (gj < N && gi < N) {
                const size_t rowp = (size_t)gj * P + PAIR_PAD;
                St<PBF>::put2(g.x2, rowp + gi, tile[r][c], tile[r][c + 1]);
                if (gi == 0) St<PBF>::put2(g.x2, rowp - 1, 0.0f, tile[r][0]);
            }
        }
    }
    if (g.xT2) {
#pragma unroll
        for (int q = 0; q < TT / TR; ++q) {
            const int oi = i0 + ty + q * TR, oj = j0 + tx;
            if (oi < N && oj < N) {
                const size_t rowp = (size_t)oi * P + PAIR_PAD;
                St<PBF>::put2(g.xT2, rowp + oj, tile[tx][ty + q * TR], tile[tx + 1][ty + q * TR]);
                if (oj == 0) St<PBF>::put2(g.xT2, rowp - 1, 0.0f, tile[0][ty + q * TR]);
            }
        }
    }
    if (MODE == TD_OBJ) {
        const int tid = ty * TT + tx;
        red[tid] = tv;
        __syncthreads();
        for (int s = TT * TR / 2; s > 0; s >>= 1) {
            if (tid < s) red[tid] += red[tid + s];
            __syncthreads();
        }
        if (tid == 0) g.partials[blockIdx.y * gridDim.x + blockIdx.x] = red[0];
    }
}

constexpr int RB = 256;     // reduction block

__global__ void k_dot_partials(const float* __restrict__ a, const float* __restrict__ b, size_t n,
                               double* __restrict__ partials)
{
    __shared__ double red[RB];
    double s = 0.0;
    for (size_t k = (size_t)blockIdx.x * RB + threadIdx.x; k < n; k += (size_t)gridDim.x * RB)
        s += (double)a[k] * (double)b[k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = RB / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__device__ double block_sum_fixed(const double* p, int n, double* red)
{
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += RB) s += p[k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = RB / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    double out = red[0];
    __syncthreads();
    return out;
}

__global__ void k_finalize(const double* p0, int n0, double c0, const double* p1, int n1, double c1, double* out)
{
    __shared__ double red[RB];
    double s0 = block_sum_fixed(p0, n0, red);
    double s1 = p1 ? block_sum_fixed(p1, n1, red) : 0.0;
    if (threadIdx.x == 0) out[0] = c0 * s0 + c1 * s1;
}

__global__ void k_scale_by_rsqrt(const float* __restrict__ x, float* __restrict__ y, size_t n,
                                 const double* __restrict__ nrm2)
{
    const float f = (float)(1.0 / sqrt(nrm2[0]));
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        y[k] = x[k] * f;
}

__global__ void k_scale(float* a, size_t n, float alpha)
{
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        a[k] *= alpha;
}

// ADMM comparator (Appendix, "Derivation from ADMM", with A = [K; f D], f = beta/alpha):
// z+ = prox_{(1/alpha) g}(A x - b - lambda) and the right-hand side y = z+ + b + lambda
// of the x-update.  Data block: z = (K x - b - l) / (1 + 1/alpha); TV block (fdx = f D x in
// the 2 N^2 layout): z = soft threshold of fdx - l at t = lambda / beta (the per-pixel
// block soft threshold for isotropic TV).
__global__ void k_admm_zu(const float* __restrict__ kx, const float* __restrict__ b, const float* __restrict__ lu,
                          float* __restrict__ zu, float* __restrict__ yu, size_t m, float inv1pia)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x) {
        const float l = lu[i], bb = b[i];
        const float z = (kx[i] - bb - l) * inv1pia;
        zu[i] = z;
        yu[i] = z + bb + l;
    }
}

__global__ void k_admm_zv(const float* __restrict__ fdx, const float* __restrict__ lv, float* __restrict__ zv,
                          float* __restrict__ yv, int N, float t, int iso)
{
    const size_t NN = (size_t)N * N;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < NN; i += (size_t)gridDim.x * blockDim.x) {
        const float lh = lv[i], lvv = lv[NN + i];
        const float wh = fdx[i] - lh, wv = fdx[NN + i] - lvv;
        float zh, zvv;
        if (iso) {
            const float nrm = sqrtf(fmaf(wh, wh, wv * wv));
            const float f = nrm > t ? 1.0f - t / nrm : 0.0f;
            zh = wh * f;
            zvv = wv * f;
        } else {
            zh = copysignf(fmaxf(fabsf(wh) - t, 0.0f), wh);
            zvv = copysignf(fmaxf(fabsf(wv) - t, 0.0f), wv);
        }
        zv[i] = zh;
        zv[NN + i] = zvv;
        yv[i] = zh + lh;
        yv[NN + i] = zvv + lvv;
    }
}

// lambda+ = lambda + z+ - A x+ + b, both blocks (A x+ = (kx, fdx) of the new x).
__global__ void k_admm_lambda(float* __restrict__ lu, const float* __restrict__ zu, const float* __restrict__ kx,
                              const float* __restrict__ b, size_t m, float* __restrict__ lv,
                              const float* __restrict__ zv, const float* __restrict__ fdx, size_t nv)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) lu[i] += zu[i] - kx[i] + b[i];
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) lv[i] += zv[i] - fdx[i];
}

// p = s + c p (conjugate-gradient direction update)
__global__ void k_xpby(const float* __restrict__ s, float c, float* __restrict__ p, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        p[i] = fmaf(c, p[i], s[i]);
}

__global__ void k_axpy(float alpha, const float* __restrict__ x, float* __restrict__ y, size_t n)
{
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        y[k] = fmaf(alpha, x[k], y[k]);
}

// SplitMix64 (Steele, Lea, Flood 2014): state seed + (k+1) * golden gamma, two
// xor-shift-multiply rounds; the top 53 bits give a uniform in [0, 1).
__global__ void k_splitmix(float* x, size_t n, uint64_t seed)
{
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + (uint64_t)(k + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z = z ^ (z >> 31);
        const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
        x[k] = (float)(2.0 * u - 1.0);
    }
}

// Ram-Lak filtering of one sinogram row per block (Kak & Slaney's discrete ramp
// kernel for bin pitch tau: h(0) = 1/(4 tau^2), h(n) = 0 for even n != 0,
// h(n) = -1/(n^2 pi^2 tau^2) for odd n), q = tau (h * b), as a direct sum.
__global__ void k_ramp(const float* __restrict__ b, float* __restrict__ q, int n_det, float inv_tau)
{
    extern __shared__ float sm[];
    float* row = sm;                 // n_det values
    float* c = sm + n_det;           // c[k] = 1 / (2k+1)^2
    const float* br = b + (size_t)blockIdx.x * n_det;
    for (int i = threadIdx.x; i < n_det; i += blockDim.x) {
        row[i] = br[i];
        const float n = (float)(2 * i + 1);
        c[i] = 1.0f / (n * n);
    }
    __syncthreads();
    constexpr float kInvPi2 = 0.10132118364233777f;   // 1 / pi^2
    for (int t = threadIdx.x; t < n_det; t += blockDim.x) {
        float acc = 0.0f;
        for (int k = 0; 2 * k + 1 <= t || t + 2 * k + 1 < n_det; ++k) {
            const int n = 2 * k + 1;
            float pair = 0.0f;
            if (t - n >= 0) pair += row[t - n];
            if (t + n < n_det) pair += row[t + n];
            acc = fmaf(c[k], pair, acc);
        }
        q[(size_t)blockIdx.x * n_det + t] = inv_tau * fmaf(-kInvPi2, acc, 0.25f * row[t]);
    }
}

int grid_for(size_t n)
{
    size_t g = (n + 255) / 256;
    if (g > 1216) g = 1216;     // 8 x 152 SMs
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

int td_num_blocks(int N)
{
    const int b = (N + TT - 1) / TT;
    return b * b;
}

template <bool IBF, bool PBF>
void td_dispatch(int mode, const TdArgs& a, dim3 grid, dim3 block, cudaStream_t st)
{
    switch (mode) {
        case TD_PROX: k_td<TD_PROX, IBF, PBF><<<grid, block, 0, st>>>(a); break;
        case TD_APPLY: k_td<TD_APPLY, IBF, PBF><<<grid, block, 0, st>>>(a); break;
        case TD_OBJ: k_td<TD_OBJ, IBF, PBF><<<grid, block, 0, st>>>(a); break;
        default: k_td<TD_TRANSPOSE, IBF, PBF><<<grid, block, 0, st>>>(a); break;
    }
}

cudaError_t launch_td(int mode, const TdArgs& a, cudaStream_t st)
{
    if (mode < TD_PROX || mode > TD_TRANSPOSE) return cudaErrorInvalidValue;
    const int b = (a.N + TT - 1) / TT;
    dim3 grid(b, b), block(TT, TR);
    if (a.img_bf && a.pair_bf) td_dispatch<true, true>(mode, a, grid, block, st);
    else if (a.img_bf) td_dispatch<true, false>(mode, a, grid, block, st);
    else if (a.pair_bf) td_dispatch<false, true>(mode, a, grid, block, st);
    else td_dispatch<false, false>(mode, a, grid, block, st);
    return cudaGetLastError();
}

cudaError_t launch_dot_partials(const float* a, const float* b, size_t n, double* partials, int nblk,
                                cudaStream_t st)
{
    k_dot_partials<<<nblk, RB, 0, st>>>(a, b, n, partials);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const double* p0, int n0, double c0, const double* p1, int n1, double c1,
                            double* out, cudaStream_t st)
{
    k_finalize<<<1, RB, 0, st>>>(p0, n0, c0, p1, n1, c1, out);
    return cudaGetLastError();
}

cudaError_t launch_scale_by_rsqrt(const float* x, float* y, size_t n, const double* nrm2, cudaStream_t st)
{
    k_scale_by_rsqrt<<<grid_for(n), 256, 0, st>>>(x, y, n, nrm2);
    return cudaGetLastError();
}

cudaError_t launch_scale(float* a, size_t n, float alpha, cudaStream_t st)
{
    k_scale<<<grid_for(n), 256, 0, st>>>(a, n, alpha);
    return cudaGetLastError();
}

cudaError_t launch_admm_z(const float* kx, const float* b, const float* lu, float* zu, float* yu, size_t m,
                          float inv1pia, const float* fdx, const float* lv, float* zv, float* yv, int N, float t,
                          int iso, cudaStream_t st)
{
    k_admm_zu<<<grid_for(m), 256, 0, st>>>(kx, b, lu, zu, yu, m, inv1pia);
    k_admm_zv<<<grid_for((size_t)N * N), 256, 0, st>>>(fdx, lv, zv, yv, N, t, iso);
    return cudaGetLastError();
}

cudaError_t launch_admm_lambda(float* lu, const float* zu, const float* kx, const float* b, size_t m, float* lv,
                               const float* zv, const float* fdx, size_t nv, cudaStream_t st)
{
    k_admm_lambda<<<grid_for(m > nv ? m : nv), 256, 0, st>>>(lu, zu, kx, b, m, lv, zv, fdx, nv);
    return cudaGetLastError();
}

cudaError_t launch_xpby(const float* s, float c, float* p, size_t n, cudaStream_t st)
{
    k_xpby<<<grid_for(n), 256, 0, st>>>(s, c, p, n);
    return cudaGetLastError();
}

cudaError_t launch_axpy(float a, const float* x, float* y, size_t n, cudaStream_t st)
{
    k_axpy<<<grid_for(n), 256, 0, st>>>(a, x, y, n);
    return cudaGetLastError();
}

cudaError_t launch_ramp(const float* b, float* q, int n_ang, int n_det, float tau, cudaStream_t st)
{
    const size_t smem = (size_t)2 * n_det * sizeof(float);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_ramp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_ramp<<<n_ang, 256, smem, st>>>(b, q, n_det, 1.0f / tau);
    return cudaGetLastError();
}

cudaError_t launch_splitmix(float* x, size_t n, uint64_t seed, cudaStream_t st)
{
    k_splitmix<<<grid_for(n), 256, 0, st>>>(x, n, seed);
    return cudaGetLastError();
}

}  // namespace ncs
