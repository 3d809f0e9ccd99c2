// Cone-beam Joseph projector pair for sm_103a (Sec. 4, "fan beam and cone beam geometry": the
// 3-D divergent-beam transform on a circular orbit), as plan-free operators.
//
// Geometry (include/ncs.h, ncs_cone_geometry): the source circles in the plane w = 0 like the
// fan beam's; detector row r holds the rays of slope sigma_r (rise in w per unit of in-plane
// distance from the source), so the in-plane trace of ray (a, r, t) is the fan ray (a, t).
// Volume x[k][j][i] (Nz slices of N x N), voxel centre (i - (N-1)/2, (N-1)/2 - j, k - (Nz-1)/2).
//
// K (k_cone_fwd): one thread per (view, row, channel, line segment).  The ray is stepped over
// the in-plane lines of its trace; the in-plane crossing and weight come from the fan beam's
// split coefficients (split_weight, as in joseph.cu), the slice coordinate
// g = sigma (Bz q + Cz) + (Nz-1)/2 (Bz q + Cz is the in-plane distance from the source to the
// crossing on line q) from a per-ray 32.32 fixed-point pair evaluated exactly in 64-bit
// integers (fix_weight), and the four taps are interpolated bilinearly in (position, slice)
// with bounds-checked loads; the sum is scaled by |W| sqrt(1 + sigma^2).
//
// K^T (k_cone_gather, no atomics): one thread per 2 x 2 in-plane pixel quad of one slice.
// Per view it scans the channels whose in-plane trace can reach the quad (the fan-beam quad
// window) and, for each, the rows whose slope can put a slice weight on slice k over the
// quad's lines (from the in-plane distance of the quad, widened by 2.5 pixels and 1% of a
// slice), and evaluates exactly the forward kernel's in-plane weight and fixed-point slice
// coordinate.
// Views, channels and rows are summed in increasing order, so the result is deterministic.
#include "../../include/ncs.h"
#include "ncs_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <vector>

using namespace ncs;

struct ncs_cone {
    int dev = 0;
    int N = 0, Nz = 0, na = 0, nr = 0, nd = 0;
    cudaStream_t st = nullptr;
    FanRay* d_rays = nullptr;
    float* d_rayw = nullptr;
    FanView* d_views = nullptr;
    longlong2* d_zfix = nullptr; // per ray (view, row, channel): the slice coordinate, 32.32 fixed point
    float* d_rowf = nullptr;     // per row: sqrt(1 + sigma_r^2)
    float inv_pitch = 0.f, t_off = 0.f, inv_rp = 0.f, r_off = 0.f;
    double row_offset = 0.0;
};

namespace {

struct ConeArgs {
    const FanRay* rays;
    const float* rayw;
    const FanView* views;
    const longlong2* zfix;       // slice coordinate of ray (a, r, t) on line q: (Zi q + Ci) / 2^32 (see below)
    const float* rowf;           // path-length factor sqrt(1 + sigma_r^2) per row
    int N, Nz, na, nr, nd;
    float inv_pitch, t_off;      // channel coordinate of a fan angle: gamma * inv_pitch + t_off
    float inv_rp, r_off;         // row coordinate of a slope: sigma * inv_rp + r_off
    const float* x;
    const float* y;
    float* out;
    // K^T epilogue: out += dscale D^T v, v = three N*N*Nz blocks (x, y, z differences), when set
    const float* v;
    float dscale;
    // K epilogues, by the kernel's mode: FWD_PLAIN out = K x; FWD_PROX_L2 the data prox of the
    // dual held in out, u = (u + alpha (K x - b)) / (1 + alpha), with the running K x in kx
    // updated to (K x + kx)/2 and the FP64 partials of its data term (if partials); FWD_RESID_L2
    // the partials of (K x - b)^2
    const float* b;
    float alpha, inv1pa;
    float* kx;
    double* partials;
};

// The integer index and weight of a crossing f = H + L (the same expression as the
// parallel- and fan-beam kernels of joseph.cu).
// The floors are taken on the FP32 pipe: for |v| < 2^22, v + 1.5 * 2^23 rounded toward -infinity
// is floor(v) + 1.5 * 2^23 exactly (floats in [2^23, 2^24) are spaced 1 apart).
__device__ __forceinline__ float cone_split_weight(float H, float L, float& k0)
{
    const float Hi = __fadd_rd(H, 12582912.0f) - 12582912.0f;
    const float fr = (H - Hi) + L;
    const float fl = __fadd_rd(fr, 12582912.0f) - 12582912.0f;
    k0 = Hi + fl;
    return fr - fl;
}

__device__ __forceinline__ float vox(const float* x, int N, int Nz, int k, int j, int i)
{
    return (k >= 0 && k < Nz && j >= 0 && j < N && i >= 0 && i < N) ? __ldg(x + ((size_t)k * N + j) * N + i) : 0.0f;
}

// Path length per step of a ray with in-plane weight ws in a row with factor rowf =
// sqrt(1 + sigma^2) (the same expression in both kernels).
__device__ __forceinline__ float cone_path(float ws, float rowf)
{
    return fabsf(ws) * rowf;
}

constexpr int CF_TB = 64;      // channels per forward block
constexpr int CF_SEG = 4;      // line segments per ray

template <int MODE>
__global__ void __launch_bounds__(CF_TB * CF_SEG) k_cone_fwd(ConeArgs g)
{
    __shared__ float red[CF_SEG][CF_TB];
    __shared__ double dred[CF_TB];
    const int t = blockIdx.x * CF_TB + threadIdx.x, r = blockIdx.y, a = blockIdx.z;
    const int N = g.N, Nz = g.Nz;
    float acc = 0.0f, W3 = 0.0f;
    if (t < g.nd) {
        const size_t rt = (size_t)a * g.nd + t;
        const float4 q = __ldg(g.rays + rt);
        const float ws = __ldg(g.rayw + rt);
        const longlong2 zf = g.zfix[((size_t)a * g.nr + r) * g.nd + t];
        const bool row = !(ws < 0.0f);
        const int chunk = (N + CF_SEG - 1) / CF_SEG;
        const int ls = threadIdx.y * chunk, le = min(N, ls + chunk);
        for (int l = ls; l < le; ++l) {
            const float lf = (float)l;
            float k0f;
            const float w = cone_split_weight(fmaf(q.x, lf, q.z), fmaf(q.y, lf, q.w), k0f);
            if (!(k0f >= -1.0f && k0f < (float)N)) continue;        // both in-plane taps outside
            const int p0 = (int)k0f;
            int k0;
            const float wz = fix_weight(zf.x * (long long)l + zf.y, k0);
            if (!(k0 >= -1 && k0 < Nz)) continue;                    // both slice taps outside
            float v00, v01, v10, v11;                                // (slice k0 / k0+1, position p0 / p0+1)
            if (row) {
                v00 = vox(g.x, N, Nz, k0, l, p0);
                v01 = vox(g.x, N, Nz, k0, l, p0 + 1);
                v10 = vox(g.x, N, Nz, k0 + 1, l, p0);
                v11 = vox(g.x, N, Nz, k0 + 1, l, p0 + 1);
            } else {
                v00 = vox(g.x, N, Nz, k0, p0, l);
                v01 = vox(g.x, N, Nz, k0, p0 + 1, l);
                v10 = vox(g.x, N, Nz, k0 + 1, p0, l);
                v11 = vox(g.x, N, Nz, k0 + 1, p0 + 1, l);
            }
            const float a0 = fmaf(w, v01, (1.0f - w) * v00);
            const float a1 = fmaf(w, v11, (1.0f - w) * v10);
            acc += fmaf(wz, a1, (1.0f - wz) * a0);
        }
        W3 = cone_path(ws, __ldg(g.rowf + r));
    }
    red[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    double term = 0.0;
    if (threadIdx.y == 0 && t < g.nd) {
        float tot = red[0][threadIdx.x];
#pragma unroll
        for (int s = 1; s < CF_SEG; ++s) tot += red[s][threadIdx.x];
        const float yv = W3 * tot;
        const size_t idx = ((size_t)a * g.nr + r) * g.nd + t;
        if (MODE == FWD_PLAIN) {
            g.out[idx] = yv;
        } else if (MODE == FWD_PROX_L2) {
            const float bv = __ldg(g.b + idx);
            g.out[idx] = fmaf(g.alpha, yv - bv, g.out[idx]) * g.inv1pa;
            if (g.kx) {
                // x+ = (xbar + x) / 2, so K x+ = (K xbar + K x) / 2 without another projection
                const float kxp = 0.5f * (yv + g.kx[idx]);
                g.kx[idx] = kxp;
                const double d = (double)kxp - (double)bv;
                term = d * d;
            }
        } else {
            const double d = (double)yv - (double)__ldg(g.b + idx);
            term = d * d;
        }
    }
    if (MODE == FWD_RESID_L2 || (MODE == FWD_PROX_L2 && g.partials)) {
        if (threadIdx.y == 0) dred[threadIdx.x] = term;
        __syncthreads();
        if (threadIdx.y == 0 && threadIdx.x < 32) {
            double s2 = dred[threadIdx.x] + dred[threadIdx.x + 32];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s2 += __shfl_down_sync(0xffffffffu, s2, o);
            if (threadIdx.x == 0) g.partials[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = s2;
        }
    }
}

// (D^T v) at voxel (k, j, i) for the three difference blocks of v (forward differences of
// Sec. 2 along x, y and z, each block N*N*Nz with zeros at the last index of its axis).
__device__ __forceinline__ float cone_dt(const float* v, int N, int Nz, int k, int j, int i)
{
    const size_t n = (size_t)N * N * Nz;
    const size_t e = ((size_t)k * N + j) * N + i;
    float d = 0.0f;
    if (i < N - 1) d += __ldg(v + e);
    if (i >= 1) d -= __ldg(v + e - 1);
    if (j < N - 1) d += __ldg(v + n + e);
    if (j >= 1) d -= __ldg(v + n + e - N);
    if (k < Nz - 1) d += __ldg(v + 2 * n + e);
    if (k >= 1) d -= __ldg(v + 2 * n + e - (size_t)N * N);
    return d;
}

constexpr int CQX = 16;    // gather block: 16 x 8 threads, each a 2 x 2 pixel quad of one slice
constexpr int CQY = 8;

// Weights that a crossing (index k0f, fraction w) of a line puts on positions p and p + 1.
__device__ __forceinline__ void cone_quad_weights(int p, float k0f, float w, float& c0, float& c1)
{
    const int d = p - (int)k0f;
    c0 = d == 0 ? 1.0f - w : (d == 1 ? w : 0.0f);
    c1 = d == -1 ? 1.0f - w : (d == 0 ? w : 0.0f);
}

// Weight that the fixed-point slice coordinate G puts on slice k (fix_weight: the forward
// kernel's slice index and weight).
__device__ __forceinline__ float slice_weight(long long G, int k)
{
    int kz;
    const float wz = fix_weight(G, kz);
    return kz == k ? 1.0f - wz : (kz == k - 1 ? wz : 0.0f);
}

__global__ void __launch_bounds__(CQX * CQY) k_cone_gather(ConeArgs g)
{
    const int N = g.N, Nz = g.Nz, nd = g.nd, nr = g.nr;
    const int i = blockIdx.x * (2 * CQX) + 2 * (int)(threadIdx.x % CQX);
    const int j = blockIdx.y * (2 * CQY) + 2 * (int)(threadIdx.x / CQX);
    const int k = blockIdx.z;
    if (i >= N || j >= N) return;           // N is even: a quad is inside or outside
    const float cN = 0.5f * (float)(N - 1);
    const float qu = ((float)i + 0.5f) - cN, qv = cN - ((float)j + 0.5f);
    const float fi = (float)i, fj = (float)j;
    const float wv = (float)k - 0.5f * (float)(Nz - 1);
    float a00 = 0.0f, a01 = 0.0f, a10 = 0.0f, a11 = 0.0f;
    for (int a = 0; a < g.na; ++a) {
        const float4 sv = __ldg(g.views + a);
        const float du = qu - sv.x, dv = qv - sv.y;
        const float tc = fmaf(atan2f(fmaf(sv.z, dv, -sv.w * du), fmaf(sv.z, du, sv.w * dv)), g.inv_pitch, g.t_off);
        const float dist = sqrtf(fmaf(du, du, dv * dv));
        const float x = fminf(1.0f, 1.7092f / dist);
        const float half = fmaf(fmaf(x, x * x, x), g.inv_pitch, 0.02f);
        const int t0 = max(0, (int)ceilf(tc - half));
        const int t1 = min(nd - 1, (int)floorf(tc + half));
        // slopes that reach slice k at an in-plane distance h in [dist - 2.5, dist + 2.5]
        const float hlo = fmaxf(dist - 2.5f, 0.5f), hhi = dist + 2.5f;
        const float slo = fminf((wv - 1.01f) / hlo, (wv - 1.01f) / hhi);
        const float shi = fmaxf((wv + 1.01f) / hlo, (wv + 1.01f) / hhi);
        const int r0 = max(0, (int)ceilf(fmaf(slo, g.inv_rp, g.r_off) - 0.01f));
        const int r1 = min(nr - 1, (int)floorf(fmaf(shi, g.inv_rp, g.r_off) + 0.01f));
        if (r0 > r1) continue;
        for (int t = t0; t <= t1; ++t) {
            const size_t rt = (size_t)a * nd + t;
            const float4 q = __ldg(g.rays + rt);
            const float ws = __ldg(g.rayw + rt);
            const bool row = !(ws < 0.0f);
            const float l0 = row ? fj : fi, l1 = l0 + 1.0f;
            const int p0 = row ? i : j;
            float kA, kB, cA0, cA1, cB0, cB1;
            const float wA = cone_split_weight(fmaf(q.x, l0, q.z), fmaf(q.y, l0, q.w), kA);
            const float wB = cone_split_weight(fmaf(q.x, l1, q.z), fmaf(q.y, l1, q.w), kB);
            cone_quad_weights(p0, kA, wA, cA0, cA1);
            cone_quad_weights(p0, kB, wB, cB0, cB1);
            if (cA0 == 0.0f && cA1 == 0.0f && cB0 == 0.0f && cB1 == 0.0f) continue;
            const long long lA = (long long)(row ? j : i);
            for (int r = r0; r <= r1; ++r) {
                const longlong2 zf = __ldg(g.zfix + ((size_t)a * nr + r) * nd + t);
                const long long GA = zf.x * lA + zf.y;
                const float zA = slice_weight(GA, k);
                const float zB = slice_weight(GA + zf.x, k);
                if (zA == 0.0f && zB == 0.0f) continue;
                const float Wu = cone_path(ws, __ldg(g.rowf + r)) * __ldg(g.y + ((size_t)a * nr + r) * nd + t);
                // row branch: line A is row j, B row j + 1; column branch: A is column i, B column i + 1
                const float c00 = zA * cA0, c11 = zB * cB1;
                const float c01 = row ? zA * cA1 : zB * cB0;
                const float c10 = row ? zB * cB0 : zA * cA1;
                a00 = c00 != 0.0f ? fmaf(c00, Wu, a00) : a00;
                a01 = c01 != 0.0f ? fmaf(c01, Wu, a01) : a01;
                a10 = c10 != 0.0f ? fmaf(c10, Wu, a10) : a10;
                a11 = c11 != 0.0f ? fmaf(c11, Wu, a11) : a11;
            }
        }
    }
    if (g.v) {
        // A^T of Sec. 4.1 in 3-D: add dscale D^T v at the four voxels
        a00 = fmaf(g.dscale, cone_dt(g.v, N, Nz, k, j, i), a00);
        a01 = fmaf(g.dscale, cone_dt(g.v, N, Nz, k, j, i + 1), a01);
        a10 = fmaf(g.dscale, cone_dt(g.v, N, Nz, k, j + 1, i), a10);
        a11 = fmaf(g.dscale, cone_dt(g.v, N, Nz, k, j + 1, i + 1), a11);
    }
    float* o = g.out + ((size_t)k * N + j) * N + i;
    o[0] = a00;
    o[1] = a01;
    o[N] = a10;
    o[N + 1] = a11;
}

// ---------------------------------------------------------------- 3-D differences and TV prox

enum { TD3_PROX = 0, TD3_APPLY = 1, TD3_OBJ = 2 };
constexpr int T3B = 256;

// One pass over the volume, one voxel per thread: the forward differences (Sec. 2) along x, y
// and z (zero at the last index of each axis), then
//   TD3_PROX : v <- Pi(v + beta D xbar), the box [-rad, rad] per component (anisotropic TV) or
//              the ball of radius rad per voxel over the three components (isotropic);
//   TD3_APPLY: v = beta D x (the D rows of A with beta = beta/alpha);
//   TD3_OBJ  : FP64 partial sums of TV(x), one per block.
template <int MODE>
__global__ void __launch_bounds__(T3B) k_cone_td(const float* __restrict__ x, float* __restrict__ v, int N, int Nz,
                                                 float beta, float rad, int iso, double* __restrict__ partials)
{
    __shared__ double red[T3B];
    const size_t n = (size_t)N * N * Nz, NN = (size_t)N * N;
    double tv = 0.0;
    for (size_t e = (size_t)blockIdx.x * T3B + threadIdx.x; e < n; e += (size_t)gridDim.x * T3B) {
        const int i = (int)(e % N);
        const size_t rest = e / N;
        const int j = (int)(rest % N), k = (int)(rest / N);
        const float xv = __ldg(x + e);
        const bool hx = i < N - 1, hy = j < N - 1, hz = k < Nz - 1;
        const float dx = hx ? xv - __ldg(x + e + 1) : 0.0f;
        const float dy = hy ? xv - __ldg(x + e + N) : 0.0f;
        const float dz = hz ? xv - __ldg(x + e + NN) : 0.0f;
        if (MODE == TD3_PROX) {
            float zx = hx ? fmaf(beta, dx, v[e]) : 0.0f;
            float zy = hy ? fmaf(beta, dy, v[n + e]) : 0.0f;
            float zz = hz ? fmaf(beta, dz, v[2 * n + e]) : 0.0f;
            if (iso) {
                const float n2 = fmaf(zx, zx, fmaf(zy, zy, zz * zz));
                if (n2 > rad * rad) {
                    const float f = rad * rsqrtf(n2);
                    zx *= f;
                    zy *= f;
                    zz *= f;
                }
            } else {
                zx = fminf(fmaxf(zx, -rad), rad);
                zy = fminf(fmaxf(zy, -rad), rad);
                zz = fminf(fmaxf(zz, -rad), rad);
            }
            v[e] = zx;
            v[n + e] = zy;
            v[2 * n + e] = zz;
        } else if (MODE == TD3_APPLY) {
            v[e] = beta * dx;
            v[n + e] = beta * dy;
            v[2 * n + e] = beta * dz;
        } else {
            const double a = dx, b = dy, c = dz;
            tv += iso ? sqrt(a * a + b * b + c * c) : fabs(a) + fabs(b) + fabs(c);
        }
    }
    if (MODE == TD3_OBJ) {
        red[threadIdx.x] = tv;
        __syncthreads();
        for (int w = T3B / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
    }
}

// Eq. (H-fan) in least-squares form, one probe's terms: num += Re(W conj(V)), den += |V|^2 over
// the stacked half spectra of the probe v (V) and of w = K^T K v (W).
__global__ void k_cone_ratio(const float2* __restrict__ W, const float2* __restrict__ V, double* __restrict__ num,
                             double* __restrict__ den, size_t count)
{
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
        const float2 w = W[e], v = V[e];
        num[e] += (double)w.x * v.x + (double)w.y * v.y;
        den[e] += (double)v.x * v.x + (double)v.y * v.y;
    }
}

ConeArgs args_of(const ncs_cone* c)
{
    ConeArgs a{};
    a.rays = c->d_rays;
    a.rayw = c->d_rayw;
    a.views = c->d_views;
    a.zfix = c->d_zfix;
    a.rowf = c->d_rowf;
    a.N = c->N;
    a.Nz = c->Nz;
    a.na = c->na;
    a.nr = c->nr;
    a.nd = c->nd;
    a.inv_pitch = c->inv_pitch;
    a.t_off = c->t_off;
    a.inv_rp = c->inv_rp;
    a.r_off = c->r_off;
    return a;
}

void free_cone(ncs_cone* c)
{
    cudaFree(c->d_rays);
    cudaFree(c->d_rayw);
    cudaFree(c->d_views);
    cudaFree(c->d_zfix);
    cudaFree(c->d_rowf);
}

template <class T>
int cone_alloc(T** p, size_t n)
{
    if (cudaMalloc((void**)p, (n ? n : 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return NCS_ERR_NOMEM;
    }
    return NCS_OK;
}

}  // namespace

extern "C" {

int ncs_cone_create(const ncs_cone_geometry* geom, int N, int Nz, void* cuda_stream, ncs_cone** out)
{
    if (!out) return NCS_ERR_BADARG;
    *out = nullptr;
    if (!geom || N < 8 || N % 2 != 0 || N > 4096 || Nz < 1 || Nz > 4096 || geom->n_views < 1 || geom->n_rows < 1 ||
        geom->n_det < 1)
        return NCS_ERR_BADARG;
    if (!(geom->pitch > 0.0) || !std::isfinite(geom->pitch) || !std::isfinite(geom->offset) ||
        !(geom->row_pitch > 0.0) || !std::isfinite(geom->row_pitch) || !std::isfinite(geom->row_offset) ||
        !std::isfinite(geom->src_dist) || !(geom->src_dist >= 0.5 * (N - 1) * std::sqrt(2.0) + 3.0))
        return NCS_ERR_BADARG;
    const int na = geom->n_views, nr = geom->n_rows, nd = geom->n_det;
    std::vector<double> sig(nr);
    for (int r = 0; r < nr; ++r) {
        sig[r] = (r - 0.5 * (nr - 1)) * geom->row_pitch + geom->row_offset;
        if (!(std::fabs(sig[r]) < 1.0 / std::sqrt(2.0))) return NCS_ERR_BADARG;
    }
    if (geom->views)
        for (int a = 0; a < na; ++a)
            if (!std::isfinite(geom->views[a])) return NCS_ERR_BADARG;
    std::vector<FanRay> rays;
    std::vector<float> rayw;
    std::vector<FanView> views;
    std::vector<double> geo;
    if (!fan_ray_tables(N, na, nd, geom->src_dist, geom->pitch, geom->offset, geom->views, rays, rayw, views, &geo))
        return NCS_ERR_UNSUPPORTED;
    // in-plane distance from the source to the crossing on line q: Bz q + Cz (FP64)
    const double cN = 0.5 * (N - 1), R = geom->src_dist;
    const size_t m = (size_t)na * nd;
    std::vector<double2> zc(m);
    std::vector<longlong2> zfix((size_t)na * nr * nd);
    std::vector<float> rowf(nr);
    for (int r = 0; r < nr; ++r) rowf[r] = (float)std::sqrt(1.0 + sig[r] * sig[r]);
    for (int a = 0; a < na; ++a) {
        const double be = geom->views ? geom->views[a] : 2.0 * M_PI * a / na;
        const double Su = -R * std::sin(be), Sv = R * std::cos(be);
        for (int t = 0; t < nd; ++t) {
            const size_t r = (size_t)a * nd + t;
            const double c = geo[3 * r], sn = geo[3 * r + 1], s = geo[3 * r + 2];
            double Bz = 0.0, Cz = 0.0;
            if (rayw[r] > 0.0f) {          // stepped over rows: v = cN - q, u = (s - v sn) / c
                Bz = 1.0 / c;
                Cz = ((s - cN * sn) / c - Su) * sn - (cN - Sv) * c;
            } else if (rayw[r] < 0.0f) {   // over columns: u = q - cN, v = (s - u c) / sn
                Bz = 1.0 / sn;
                Cz = -(cN + Su) * sn - ((s + cN * c) / sn - Sv) * c;
            }
            zc[r] = make_double2(Bz, Cz);
        }
    }
    // slice coordinate of ray (a, row, t) on line q: g = sigma (Bz q + Cz) + (Nz-1)/2, as
    // (Zi q + Ci) / 2^32 with Zi, Ci the integers nearest to sigma Bz 2^32 and (sigma Cz +
    // (Nz-1)/2) 2^32; both kernels evaluate it exactly in 64-bit integers (fix_weight)
    const double cZ = 0.5 * (Nz - 1), two32 = 4294967296.0;
    for (int a = 0; a < na; ++a)
        for (int rr = 0; rr < nr; ++rr)
            for (int t = 0; t < nd; ++t) {
                const double2 z = zc[(size_t)a * nd + t];
                longlong2& f = zfix[((size_t)a * nr + rr) * nd + t];
                f.x = std::llround(sig[rr] * z.x * two32);
                f.y = std::llround((sig[rr] * z.y + cZ) * two32);
            }
    ncs_cone* c = new (std::nothrow) ncs_cone();
    if (!c) return NCS_ERR_NOMEM;
    c->N = N;
    c->Nz = Nz;
    c->na = na;
    c->nr = nr;
    c->nd = nd;
    c->st = (cudaStream_t)cuda_stream;
    c->inv_pitch = (float)(1.0 / geom->pitch);
    c->t_off = (float)(0.5 * (nd - 1) - geom->offset / geom->pitch);
    c->inv_rp = (float)(1.0 / geom->row_pitch);
    c->r_off = (float)(0.5 * (nr - 1) - geom->row_offset / geom->row_pitch);
    int rc = cudaGetDevice(&c->dev) == cudaSuccess ? NCS_OK : NCS_ERR_CUDA;
    if (rc == NCS_OK) rc = cone_alloc(&c->d_rays, m);
    if (rc == NCS_OK) rc = cone_alloc(&c->d_rayw, m);
    if (rc == NCS_OK) rc = cone_alloc(&c->d_views, (size_t)na);
    if (rc == NCS_OK) rc = cone_alloc(&c->d_zfix, zfix.size());
    if (rc == NCS_OK) rc = cone_alloc(&c->d_rowf, (size_t)nr);
    if (rc == NCS_OK &&
        (cudaMemcpy(c->d_rays, rays.data(), m * sizeof(FanRay), cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(c->d_rayw, rayw.data(), m * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(c->d_views, views.data(), na * sizeof(FanView), cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(c->d_zfix, zfix.data(), zfix.size() * sizeof(longlong2), cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(c->d_rowf, rowf.data(), nr * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess))
        rc = NCS_ERR_CUDA;
    if (rc != NCS_OK) {
        cudaGetLastError();
        free_cone(c);
        delete c;
        return rc;
    }
    *out = c;
    return NCS_OK;
}

void ncs_cone_destroy(ncs_cone* c)
{
    if (!c) return;
    cudaSetDevice(c->dev);
    if (c->st) cudaStreamSynchronize(c->st);
    else cudaDeviceSynchronize();
    free_cone(c);
    delete c;
}

int ncs_cone_apply_K(ncs_cone* c, const float* x, float* y)
{
    if (!c || !x || !y) return NCS_ERR_BADARG;
    if (cudaSetDevice(c->dev) != cudaSuccess) return NCS_ERR_CUDA;
    ConeArgs a = args_of(c);
    a.x = x;
    a.out = y;
    dim3 grid((c->nd + CF_TB - 1) / CF_TB, c->nr, c->na), block(CF_TB, CF_SEG);
    if (c->nr > 65535 || c->na > 65535) return NCS_ERR_UNSUPPORTED;
    k_cone_fwd<FWD_PLAIN><<<grid, block, 0, c->st>>>(a);
    if (cudaGetLastError() != cudaSuccess) return NCS_ERR_CUDA;
    return NCS_OK;
}

int ncs_cone_apply_KT(ncs_cone* c, const float* y, float* x)
{
    if (!c || !x || !y) return NCS_ERR_BADARG;
    if (cudaSetDevice(c->dev) != cudaSuccess) return NCS_ERR_CUDA;
    ConeArgs a = args_of(c);
    a.y = y;
    a.out = x;
    dim3 grid((c->N + 2 * CQX - 1) / (2 * CQX), (c->N + 2 * CQY - 1) / (2 * CQY), c->Nz), block(CQX * CQY);
    if (c->Nz > 65535) return NCS_ERR_UNSUPPORTED;
    k_cone_gather<<<grid, block, 0, c->st>>>(a);
    if (cudaGetLastError() != cudaSuccess) return NCS_ERR_CUDA;
    return NCS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- the 3-D NCS plan
//
// NCS for min 1/2 ||K x - b||^2 + lam TV(x) on the cone beam, A = [K; (beta/alpha) D] with the
// 3-D forward differences (eq. (NCS), the updates of Sec. 4.1 in 3-D):
//   r = K^T u + (beta/alpha) D^T v         (k_cone_gather with its D^T epilogue)
//   x+ = x - M^{-1} r, xbar = 2 x+ - x       (3-D FFT solve: per-slice row and column passes, the
//                                            direct transform along z, the update in the last pass)
//   u+ = (u + alpha (K xbar - b))/(1 + alpha) (k_cone_fwd's data-prox epilogue)
//   v+ = Pi(v + beta D xbar)                (k_cone_td)
// with M = gamma I + alpha C on the periodic N x N x Nz grid: eq. (H-fan) in least-squares form
// over SplitMix64 probe volumes for K^T K (DC entry ||K 1||^2 / ||1||^2) and the 3-D Laplacian
// spectrum for D^T D, rescaled so that rho(M^{-1} alpha A^T A) = 1/(1 + margin) (A3).

struct ncs_cone_plan {
    ncs_cone* op = nullptr;
    int N = 0, Nz = 0, na = 0, nr = 0, nd = 0;
    size_t n = 0, m = 0, plane = 0;
    double lam = 0, alpha = 0, beta = 0, gamma = 0, rho = std::numeric_limits<double>::quiet_NaN(), h_dc = 0;
    bool iso = false;
    ncs_options opt{};
    cudaStream_t st = nullptr;
    bool own_stream = false;
    RadixPlan rp{};
    float2 *d_tw = nullptr, *d_twz = nullptr, *d_spec = nullptr, *d_spec2 = nullptr;
    std::vector<double> mu;                     // Nz x N x N, [l][p][q]
    float *d_invmu = nullptr, *d_mu = nullptr;  // 1/(N^2 Nz mu), mu/(N^2 Nz): [l][k][p], k <= N/2
    float *d_xbar = nullptr, *d_r = nullptr, *d_tmp = nullptr, *d_y = nullptr, *d_vt = nullptr;
    float *d_u = nullptr, *d_v = nullptr, *d_kx = nullptr;   // solver state
    double *d_part0 = nullptr, *d_part1 = nullptr, *d_scal = nullptr, *h_pin = nullptr;
    int n_part0 = 0, n_part1 = 0;
    cudaGraphExec_t gexec = nullptr;
    const void* gkey[2] = {nullptr, nullptr};
    int gT = 0;
    long long n_kern = 0;    // kernels enqueued on the stream (a captured graph counts once, at capture)
};

namespace {

#define CONE_CK(expr)                                                \
    do {                                                             \
        cudaError_t e_ = (expr);                                     \
        if (e_ != cudaSuccess) {                                     \
            fprintf(stderr, "ncs: %s failed: %s (%s:%d)\n", #expr,   \
                    cudaGetErrorString(e_), __FILE__, __LINE__);     \
            return NCS_ERR_CUDA;                                     \
        }                                                            \
    } while (0)

#define CONE_CKS(expr)                    \
    do {                                  \
        int s_ = (expr);                  \
        if (s_ < 0) return s_;            \
    } while (0)

bool cone_radices(int L, RadixPlan* rp)
{
    rp->n = 0;
    while (L % 8 == 0 && rp->n < 12) { rp->r[rp->n++] = 8; L /= 8; }
    while (L % 4 == 0 && rp->n < 12) { rp->r[rp->n++] = 4; L /= 4; }
    while (L % 3 == 0 && rp->n < 12) { rp->r[rp->n++] = 3; L /= 3; }
    while (L % 2 == 0 && rp->n < 12) { rp->r[rp->n++] = 2; L /= 2; }
    return L == 1;
}

int td_blocks(size_t n) { return (int)std::min<size_t>((n + T3B - 1) / T3B, 2048); }
int fwd_blocks(const ncs_cone_plan* p) { return ((p->nd + CF_TB - 1) / CF_TB) * p->nr * p->na; }

// r = K^T u (+ dscale D^T v)
int cenq_gather(ncs_cone_plan* p, const float* u, const float* v, float dscale, float* out)
{
    ConeArgs a = args_of(p->op);
    a.y = u;
    a.out = out;
    a.v = v;
    a.dscale = dscale;
    dim3 grid((p->N + 2 * CQX - 1) / (2 * CQX), (p->N + 2 * CQY - 1) / (2 * CQY), p->Nz), block(CQX * CQY);
    k_cone_gather<<<grid, block, 0, p->st>>>(a);
    CONE_CK(cudaGetLastError());
    p->n_kern += 1;
    return NCS_OK;
}

int cenq_fwd(ncs_cone_plan* p, int mode, const float* x, float* out, const float* b, float* kx, double* partials)
{
    ConeArgs a = args_of(p->op);
    a.x = x;
    a.out = out;
    a.b = b;
    a.alpha = (float)p->alpha;
    a.inv1pa = (float)(1.0 / (1.0 + p->alpha));
    a.kx = kx;
    a.partials = partials;
    dim3 grid((p->nd + CF_TB - 1) / CF_TB, p->nr, p->na), block(CF_TB, CF_SEG);
    if (mode == FWD_PLAIN) k_cone_fwd<FWD_PLAIN><<<grid, block, 0, p->st>>>(a);
    else if (mode == FWD_PROX_L2) k_cone_fwd<FWD_PROX_L2><<<grid, block, 0, p->st>>>(a);
    else k_cone_fwd<FWD_RESID_L2><<<grid, block, 0, p->st>>>(a);
    CONE_CK(cudaGetLastError());
    p->n_kern += 1;
    return NCS_OK;
}

int cenq_td(ncs_cone_plan* p, int mode, const float* x, float* v, float beta, double* partials)
{
    const float rad = (float)(p->lam * p->alpha / p->beta);
    const int nb = td_blocks(p->n);
    if (mode == TD3_PROX) k_cone_td<TD3_PROX><<<nb, T3B, 0, p->st>>>(x, v, p->N, p->Nz, beta, rad, p->iso, nullptr);
    else if (mode == TD3_APPLY) k_cone_td<TD3_APPLY><<<nb, T3B, 0, p->st>>>(x, v, p->N, p->Nz, beta, rad, p->iso, nullptr);
    else k_cone_td<TD3_OBJ><<<nb, T3B, 0, p->st>>>(x, v, p->N, p->Nz, beta, rad, p->iso, partials);
    CONE_CK(cudaGetLastError());
    p->n_kern += 1;
    return NCS_OK;
}

// The 3-D circulant pass on r: mode 0 x <- x - delta, xbar <- 2 x+ - x; mode 1 out <- delta,
// delta = F^{-1} diag(table * N^2 Nz) F r.
int cenq_solve(ncs_cone_plan* p, const float* r, const float* table, int mode, float* x, float* xbar, float* out)
{
    CONE_CK(launch_rows_fwd_stack(r, p->d_spec, p->d_tw, p->rp, p->N, p->Nz, p->st));
    CONE_CK(launch_cols_fft_stack(p->d_spec, p->d_tw, p->rp, p->N, p->Nz, 0, p->st));
    CONE_CK(launch_z_dft(p->d_spec, table, p->d_twz, p->Nz, p->plane, 1, p->st));
    CONE_CK(launch_cols_fft_stack(p->d_spec, p->d_tw, p->rp, p->N, p->Nz, 1, p->st));
    CONE_CK(launch_rows_inv_stack(p->d_spec, p->d_tw, p->rp, p->N, p->Nz, mode, x, xbar, out, p->st));
    p->n_kern += 5;
    return NCS_OK;
}

// the forward 3-D transform of r into spec (stacked half spectra)
int cenq_fft3(ncs_cone_plan* p, const float* r, float2* spec)
{
    CONE_CK(launch_rows_fwd_stack(r, spec, p->d_tw, p->rp, p->N, p->Nz, p->st));
    CONE_CK(launch_cols_fft_stack(spec, p->d_tw, p->rp, p->N, p->Nz, 0, p->st));
    CONE_CK(launch_z_dft(spec, nullptr, p->d_twz, p->Nz, p->plane, 0, p->st));
    return NCS_OK;
}

int cenq_dot(ncs_cone_plan* p, const float* a, const float* b, size_t n, int slot)
{
    CONE_CK(launch_dot_partials(a, b, n, p->d_part0, p->n_part0, p->st));
    CONE_CK(launch_finalize(p->d_part0, p->n_part0, 1.0, nullptr, 0, 0.0, p->d_scal + slot, p->st));
    return NCS_OK;
}

int cread(ncs_cone_plan* p, int count)
{
    CONE_CK(cudaMemcpyAsync(p->h_pin, p->d_scal, count * sizeof(double), cudaMemcpyDeviceToHost, p->st));
    CONE_CK(cudaStreamSynchronize(p->st));
    return NCS_OK;
}

// w = A^T A x = K^T K x + (beta/alpha)^2 D^T D x
int cenq_AtA(ncs_cone_plan* p, const float* x, float* w)
{
    const float f = (float)(p->beta / p->alpha);
    CONE_CKS(cenq_fwd(p, FWD_PLAIN, x, p->d_y, nullptr, nullptr, nullptr));
    CONE_CKS(cenq_td(p, TD3_APPLY, x, p->d_vt, f, nullptr));
    return cenq_gather(p, p->d_y, p->d_vt, f, w);
}

int cupload_mu(ncs_cone_plan* p)
{
    const int N = p->N, Nz = p->Nz, H = N / 2;
    const double s = 1.0 / ((double)N * N * Nz);
    std::vector<float> inv((size_t)Nz * p->plane), fwd((size_t)Nz * p->plane);
    for (int l = 0; l < Nz; ++l)
        for (int k = 0; k <= H; ++k)
            for (int q = 0; q < N; ++q) {
                const double mv = p->mu[((size_t)l * N + q) * N + k];
                const size_t e = (size_t)l * p->plane + (size_t)k * N + q;
                inv[e] = (float)(s / mv);
                fwd[e] = (float)(s * mv);
            }
    CONE_CK(cudaMemcpyAsync(p->d_invmu, inv.data(), inv.size() * sizeof(float), cudaMemcpyHostToDevice, p->st));
    CONE_CK(cudaMemcpyAsync(p->d_mu, fwd.data(), fwd.size() * sizeof(float), cudaMemcpyHostToDevice, p->st));
    CONE_CK(cudaStreamSynchronize(p->st));
    return NCS_OK;
}

// rho = lambda_max(M^{-1} alpha A^T A) by power iteration (Rayleigh quotients in the M inner
// product, FP64 reductions), as for the 2-D plans
int cpower_rho(ncs_cone_plan* p, double* out)
{
    float* x = p->d_tmp;
    float* w = p->d_r;
    float* y = p->d_xbar;
    const size_t n = p->n;
    CONE_CK(launch_splitmix(x, n, p->opt.power_seed, p->st));
    CONE_CKS(cenq_dot(p, x, x, n, 0));
    CONE_CK(launch_scale_by_rsqrt(x, x, n, p->d_scal + 0, p->st));
    CONE_CKS(cenq_solve(p, x, p->d_mu, 1, nullptr, nullptr, y));
    CONE_CKS(cenq_dot(p, x, y, n, 3));
    CONE_CKS(cread(p, 4));
    double xMx = p->h_pin[3], rho = 0.0, rho_old = 0.0;
    for (int it = 1; it <= p->opt.power_max_iter; ++it) {
        CONE_CKS(cenq_AtA(p, x, w));
        CONE_CK(launch_scale(w, n, (float)p->alpha, p->st));
        CONE_CKS(cenq_dot(p, x, w, n, 0));
        CONE_CKS(cenq_solve(p, w, p->d_invmu, 1, nullptr, nullptr, y));
        CONE_CKS(cenq_dot(p, y, w, n, 1));
        CONE_CKS(cenq_dot(p, y, y, n, 2));
        CONE_CK(launch_scale_by_rsqrt(y, x, n, p->d_scal + 2, p->st));
        CONE_CKS(cread(p, 3));
        rho = p->h_pin[0] / xMx;
        xMx = p->h_pin[1] / p->h_pin[2];
        if (!std::isfinite(rho)) return NCS_ERR_DIVERGED;
        if (it > 1 && std::fabs(rho - rho_old) <= p->opt.power_tol * std::fabs(rho)) break;
        rho_old = rho;
    }
    *out = rho;
    return NCS_OK;
}

// Eq. (H-fan) over P probe volumes: h on the stacked half spectra ([l][k][p]) into *h
int cprobe_h(ncs_cone_plan* p, int P, std::vector<double>* h)
{
    const size_t cnt = (size_t)p->Nz * p->plane;
    double *num = nullptr, *den = nullptr;
    if (cudaMalloc(&num, cnt * sizeof(double)) != cudaSuccess || cudaMalloc(&den, cnt * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(num);
        return NCS_ERR_NOMEM;
    }
    int rc = NCS_OK;
    if (cudaMemsetAsync(num, 0, cnt * sizeof(double), p->st) != cudaSuccess ||
        cudaMemsetAsync(den, 0, cnt * sizeof(double), p->st) != cudaSuccess)
        rc = NCS_ERR_CUDA;
    for (int q = 0; q < P && rc == NCS_OK; ++q) {
        float* v = p->d_tmp;
        float* w = p->d_r;
        if (launch_splitmix(v, p->n, p->opt.power_seed + 1 + (uint64_t)q, p->st) != cudaSuccess) rc = NCS_ERR_CUDA;
        if (rc == NCS_OK) rc = cenq_fwd(p, FWD_PLAIN, v, p->d_y, nullptr, nullptr, nullptr);
        if (rc == NCS_OK) rc = cenq_gather(p, p->d_y, nullptr, 0.f, w);
        if (rc == NCS_OK) rc = cenq_fft3(p, w, p->d_spec);
        if (rc == NCS_OK) rc = cenq_fft3(p, v, p->d_spec2);
        if (rc == NCS_OK) {
            k_cone_ratio<<<(unsigned)std::min<size_t>((cnt + 255) / 256, 4096), 256, 0, p->st>>>(p->d_spec, p->d_spec2,
                                                                                              num, den, cnt);
            if (cudaGetLastError() != cudaSuccess) rc = NCS_ERR_CUDA;
        }
    }
    if (rc == NCS_OK) {
        std::vector<double> d(cnt);
        h->assign(cnt, 0.0);
        if (cudaMemcpyAsync(h->data(), num, cnt * sizeof(double), cudaMemcpyDeviceToHost, p->st) != cudaSuccess ||
            cudaMemcpyAsync(d.data(), den, cnt * sizeof(double), cudaMemcpyDeviceToHost, p->st) != cudaSuccess ||
            cudaStreamSynchronize(p->st) != cudaSuccess)
            rc = NCS_ERR_CUDA;
        for (size_t e = 0; e < cnt; ++e) (*h)[e] = d[e] > 0.0 ? (*h)[e] / d[e] : 0.0;
    }
    cudaGetLastError();
    cudaFree(num);
    cudaFree(den);
    return rc;
}

template <class T>
int calloc_dev(T** ptr, size_t count)
{
    if (cudaMalloc((void**)ptr, (count ? count : 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return NCS_ERR_NOMEM;
    }
    return NCS_OK;
}

void free_cone_plan(ncs_cone_plan* p)
{
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    cudaFree(p->d_tw); cudaFree(p->d_twz); cudaFree(p->d_spec); cudaFree(p->d_spec2);
    cudaFree(p->d_invmu); cudaFree(p->d_mu); cudaFree(p->d_xbar); cudaFree(p->d_r); cudaFree(p->d_tmp);
    cudaFree(p->d_y); cudaFree(p->d_vt); cudaFree(p->d_u); cudaFree(p->d_v); cudaFree(p->d_kx);
    cudaFree(p->d_part0); cudaFree(p->d_part1); cudaFree(p->d_scal);
    if (p->h_pin) cudaFreeHost(p->h_pin);
    if (p->op) ncs_cone_destroy(p->op);
    if (p->own_stream && p->st) cudaStreamDestroy(p->st);
}

int build_cone_plan(ncs_cone_plan* p, const ncs_cone_geometry* geom)
{
    const int N = p->N, Nz = p->Nz, H = N / 2;
    if (p->opt.cuda_stream) {
        p->st = (cudaStream_t)p->opt.cuda_stream;
    } else {
        CONE_CK(cudaStreamCreateWithFlags(&p->st, cudaStreamNonBlocking));
        p->own_stream = true;
    }
    CONE_CKS(ncs_cone_create(geom, N, Nz, p->st, &p->op));
    p->na = geom->n_views;
    p->nr = geom->n_rows;
    p->nd = geom->n_det;
    p->n = (size_t)N * N * Nz;
    p->m = (size_t)p->na * p->nr * p->nd;
    p->plane = (size_t)(H + 1) * N;
    CONE_CK(fft_prepare(N));
    std::vector<float2> tw(N), twz(Nz);
    for (int q = 0; q < N; ++q) {
        const double ang = -2.0 * M_PI * (double)q / (double)N;
        tw[q] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    for (int q = 0; q < Nz; ++q) {
        const double ang = -2.0 * M_PI * (double)q / (double)Nz;
        twz[q] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    CONE_CKS(calloc_dev(&p->d_tw, (size_t)N));
    CONE_CKS(calloc_dev(&p->d_twz, (size_t)Nz));
    CONE_CK(cudaMemcpyAsync(p->d_tw, tw.data(), N * sizeof(float2), cudaMemcpyHostToDevice, p->st));
    CONE_CK(cudaMemcpyAsync(p->d_twz, twz.data(), Nz * sizeof(float2), cudaMemcpyHostToDevice, p->st));
    const size_t spec = (size_t)Nz * p->plane;
    CONE_CKS(calloc_dev(&p->d_spec, spec));
    CONE_CKS(calloc_dev(&p->d_spec2, spec));
    CONE_CKS(calloc_dev(&p->d_invmu, spec));
    CONE_CKS(calloc_dev(&p->d_mu, spec));
    CONE_CKS(calloc_dev(&p->d_xbar, p->n));
    CONE_CKS(calloc_dev(&p->d_r, p->n));
    CONE_CKS(calloc_dev(&p->d_tmp, p->n));
    CONE_CKS(calloc_dev(&p->d_y, p->m));
    CONE_CKS(calloc_dev(&p->d_vt, 3 * p->n));
    p->n_part0 = std::max(td_blocks(p->n), 1024);
    p->n_part1 = fwd_blocks(p);
    CONE_CKS(calloc_dev(&p->d_part0, (size_t)p->n_part0));
    CONE_CKS(calloc_dev(&p->d_part1, (size_t)p->n_part1));
    CONE_CKS(calloc_dev(&p->d_scal, (size_t)16));
    if (cudaMallocHost((void**)&p->h_pin, 16 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return NCS_ERR_NOMEM;
    }
    // DC entry: ||K 1||^2 / ||1||^2 unless given
    if (std::isnan(p->h_dc)) {
        std::vector<float> ones(p->n, 1.0f);
        CONE_CK(cudaMemcpyAsync(p->d_tmp, ones.data(), p->n * sizeof(float), cudaMemcpyHostToDevice, p->st));
        CONE_CKS(cenq_fwd(p, FWD_PLAIN, p->d_tmp, p->d_y, nullptr, nullptr, nullptr));
        CONE_CKS(cenq_dot(p, p->d_y, p->d_y, p->m, 0));
        CONE_CKS(cread(p, 1));
        p->h_dc = p->h_pin[0] / (double)p->n;
    }
    // eq. (H-fan) for K^T K, the periodic 3-D Laplacian for D^T D
    std::vector<double> hh;
    CONE_CKS(cprobe_h(p, p->opt.h_probes > 0 ? p->opt.h_probes : 128, &hh));
    p->mu.assign(p->n, 0.0);
    const double b2a = p->beta * p->beta / p->alpha;
    for (int l = 0; l < Nz; ++l) {
        const double sl = std::sin(M_PI * l / Nz);
        for (int pp = 0; pp < N; ++pp) {
            const double sp = std::sin(M_PI * pp / N);
            for (int q = 0; q < N; ++q) {
                const double sq = std::sin(M_PI * q / N);
                double hr;
                if (l == 0 && pp == 0 && q == 0) {
                    hr = p->h_dc;
                } else if (q <= H) {
                    hr = hh[(size_t)l * p->plane + (size_t)q * N + pp];
                } else {
                    // a real operator's estimate is even: h(l, p, q) = h(-l, -p, -q)
                    const int l2 = (Nz - l) % Nz, p2 = (N - pp) % N;
                    hr = hh[(size_t)l2 * p->plane + (size_t)(N - q) * N + p2];
                }
                const double hd = 4.0 * (sl * sl + sp * sp + sq * sq);
                p->mu[((size_t)l * N + pp) * N + q] = p->gamma + p->alpha * std::max(0.0, hr) + b2a * hd;
            }
        }
    }
    for (double v : p->mu)
        if (!(v > 0.0)) return NCS_ERR_BADARG;
    CONE_CKS(cupload_mu(p));
    if (p->opt.a3_margin >= 0.0) {
        CONE_CKS(cpower_rho(p, &p->rho));
        const double f = p->rho * (1.0 + p->opt.a3_margin);
        for (double& v : p->mu) v *= f;
        CONE_CKS(cupload_mu(p));
    }
    return NCS_OK;
}

// one NCS iteration on (x, u, v); with kx, the running K x and (if partials) the data term
int cenq_iter(ncs_cone_plan* p, float* x, float* u, float* v, const float* b, float* kx, double* partials)
{
    CONE_CKS(cenq_gather(p, u, v, (float)(p->beta / p->alpha), p->d_r));
    CONE_CKS(cenq_solve(p, p->d_r, p->d_invmu, 0, x, p->d_xbar, nullptr));
    CONE_CKS(cenq_fwd(p, FWD_PROX_L2, p->d_xbar, u, b, kx, partials));
    return cenq_td(p, TD3_PROX, p->d_xbar, v, (float)p->beta, nullptr);
}

// the FP64 objective 1/2 ||K x - b||^2 + lam TV(x) into d_scal[slot]; with the data partials
// already in d_part1 (the last iteration's running K x+) unless resid
int cenq_objective(ncs_cone_plan* p, const float* x, const float* b, bool resid, int slot)
{
    if (resid) CONE_CKS(cenq_fwd(p, FWD_RESID_L2, x, p->d_y, b, nullptr, p->d_part1));
    CONE_CKS(cenq_td(p, TD3_OBJ, x, nullptr, 0.f, p->d_part0));
    CONE_CK(launch_finalize(p->d_part1, p->n_part1, 0.5, p->d_part0, td_blocks(p->n), p->lam, p->d_scal + slot,
                            p->st));
    p->n_kern += 1;
    return NCS_OK;
}

int cenq_block(ncs_cone_plan* p, const float* b, float* x, int n_it)
{
    for (int k = 0; k < n_it; ++k)
        CONE_CKS(cenq_iter(p, x, p->d_u, p->d_v, b, p->d_kx, k == n_it - 1 ? p->d_part1 : nullptr));
    CONE_CKS(cenq_objective(p, x, b, false, 0));
    CONE_CK(cudaMemcpyAsync(p->h_pin, p->d_scal, sizeof(double), cudaMemcpyDeviceToHost, p->st));
    return NCS_OK;
}

}  // namespace

extern "C" {

int ncs_cone_plan_create(const ncs_cone_geometry* geom, int N, int Nz, double lambda, double alpha,
                         const ncs_options* opt, ncs_cone_plan** out)
{
    if (!out) return NCS_ERR_BADARG;
    *out = nullptr;
    if (!geom || !(lambda >= 0.0) || !(alpha > 0.0) || N < 8 || N % 2 != 0 || N > 4096 || Nz < 2) return NCS_ERR_BADARG;
    ncs_options o;
    if (opt) o = *opt;
    else ncs_options_default(&o);
    if (o.data != NCS_DATA_L2 || o.nonneg || o.prec != NCS_FP32 || o.warm_dual || o.autotune || o.pdhg_only)
        return NCS_ERR_UNSUPPORTED;
    if (o.power_max_iter < 1 || !(o.power_tol >= 0.0) || o.h_probes < 0) return NCS_ERR_BADARG;
    RadixPlan rp;
    if (Nz > 64 || !cone_radices(N, &rp)) return NCS_ERR_UNSUPPORTED;
    ncs_cone_plan* p = new (std::nothrow) ncs_cone_plan();
    if (!p) return NCS_ERR_NOMEM;
    p->N = N;
    p->Nz = Nz;
    p->lam = lambda;
    p->alpha = alpha;
    p->beta = std::isnan(o.beta) ? alpha : o.beta;
    p->gamma = o.gamma;
    p->h_dc = o.h_dc;
    p->iso = o.tv == NCS_TV_ISO;
    p->opt = o;
    p->rp = rp;
    if (!(p->beta > 0.0) || !(p->gamma >= 0.0)) {
        delete p;
        return NCS_ERR_BADARG;
    }
    int rc = build_cone_plan(p, geom);
    if (rc != NCS_OK) {
        if (p->st) cudaStreamSynchronize(p->st);
        free_cone_plan(p);
        delete p;
        return rc;
    }
    *out = p;
    return NCS_OK;
}

void ncs_cone_plan_destroy(ncs_cone_plan* p)
{
    if (!p) return;
    if (p->st) cudaStreamSynchronize(p->st);
    free_cone_plan(p);
    delete p;
}

int ncs_cone_step(ncs_cone_plan* p, float* x, float* u, float* v, const float* b, int n_iter)
{
    if (!p || !x || !u || !v || !b || n_iter < 1) return NCS_ERR_BADARG;
    for (int k = 0; k < n_iter; ++k) CONE_CKS(cenq_iter(p, x, u, v, b, nullptr, nullptr));
    return NCS_OK;
}

int ncs_cone_objective(ncs_cone_plan* p, const float* x, const float* b, double* f)
{
    if (!p || !x || !b || !f) return NCS_ERR_BADARG;
    CONE_CKS(cenq_objective(p, x, b, true, 1));
    CONE_CK(cudaMemcpyAsync(p->h_pin + 1, p->d_scal + 1, sizeof(double), cudaMemcpyDeviceToHost, p->st));
    CONE_CK(cudaStreamSynchronize(p->st));
    *f = p->h_pin[1];
    return NCS_OK;
}

int ncs_cone_kernels(const ncs_cone_plan* p, long long* n)
{
    if (!p || !n) return NCS_ERR_BADARG;
    *n = p->n_kern;
    return NCS_OK;
}

int ncs_cone_apply_Minv(ncs_cone_plan* p, const float* r, float* out)
{
    if (!p || !r || !out) return NCS_ERR_BADARG;
    return cenq_solve(p, r, p->d_invmu, 1, nullptr, nullptr, out);
}

int ncs_cone_get_mu(ncs_cone_plan* p, double* mu_host)
{
    if (!p || !mu_host) return NCS_ERR_BADARG;
    memcpy(mu_host, p->mu.data(), p->mu.size() * sizeof(double));
    return NCS_OK;
}

int ncs_cone_power_bound(ncs_cone_plan* p, double* rho)
{
    if (!p || !rho) return NCS_ERR_BADARG;
    *rho = p->rho;
    return NCS_OK;
}

int ncs_cone_solve(ncs_cone_plan* p, const float* b, float* x, double tol, int max_iter, double f_star, ncs_report* rep)
{
    if (!p || !b || !x || max_iter < 1 || !(tol >= 0.0)) return NCS_ERR_BADARG;
    if (!p->d_u) {
        CONE_CKS(calloc_dev(&p->d_u, p->m));
        CONE_CKS(calloc_dev(&p->d_v, 3 * p->n));
        CONE_CKS(calloc_dev(&p->d_kx, p->m));
    }
    CONE_CK(cudaMemsetAsync(p->d_u, 0, p->m * sizeof(float), p->st));
    CONE_CK(cudaMemsetAsync(p->d_v, 0, 3 * p->n * sizeof(float), p->st));
    CONE_CKS(cenq_fwd(p, FWD_PLAIN, x, p->d_kx, nullptr, nullptr, nullptr));     // running K x from x^0
    const int T = p->opt.check_every > 0 ? p->opt.check_every : 10;
    if (!(p->gexec && p->gkey[0] == b && p->gkey[1] == x && p->gT == T)) {
        if (p->gexec) { cudaGraphExecDestroy(p->gexec); p->gexec = nullptr; }
        cudaGraph_t graph;
        CONE_CK(cudaStreamBeginCapture(p->st, cudaStreamCaptureModeThreadLocal));
        const int rc = cenq_block(p, b, x, T);
        cudaError_t e = cudaStreamEndCapture(p->st, &graph);
        if (rc != NCS_OK) { if (e == cudaSuccess) cudaGraphDestroy(graph); return rc; }
        CONE_CK(e);
        e = cudaGraphInstantiate(&p->gexec, graph, 0);
        cudaGraphDestroy(graph);
        CONE_CK(e);
        p->gkey[0] = b;
        p->gkey[1] = x;
        p->gT = T;
    }
    cudaEvent_t e0, e1;
    CONE_CK(cudaEventCreate(&e0));
    CONE_CK(cudaEventCreate(&e1));
    CONE_CK(cudaEventRecord(e0, p->st));
    int it = 0, status = NCS_NOT_CONVERGED;
    const double nan = std::numeric_limits<double>::quiet_NaN();
    double f = nan, f_prev = nan, gap = nan;
    while (it < max_iter) {
        const int n_it = std::min(T, max_iter - it);
        if (n_it == T) CONE_CK(cudaGraphLaunch(p->gexec, p->st));
        else CONE_CKS(cenq_block(p, b, x, n_it));
        CONE_CK(cudaStreamSynchronize(p->st));
        it += n_it;
        f = p->h_pin[0];
        if (!std::isfinite(f)) { status = NCS_ERR_DIVERGED; break; }
        if (std::isfinite(f_star)) gap = (f - f_star) / std::fabs(f_star);
        else gap = std::isfinite(f_prev) ? std::fabs(f - f_prev) / std::fabs(f) : nan;
        if (std::isfinite(gap) && gap <= tol) { status = NCS_OK; break; }
        f_prev = f;
    }
    CONE_CK(cudaEventRecord(e1, p->st));
    CONE_CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rep) {
        rep->iters = it;
        rep->status = status;
        rep->time_ms = ms;
        rep->f = f;
        rep->gap = gap;
        rep->rho = p->rho;
    }
    return status;
}

}  // extern "C"
