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
// split coefficients (split_weight, as in joseph.cu), the slice coordinate from
// g = sigma (Bz q + Cz) + (Nz-1)/2 evaluated in FP64 (Bz q + Cz is the in-plane distance from
// the source to the crossing on line q), and the four taps are interpolated bilinearly in
// (position, slice) with bounds-checked loads; the sum is scaled by |W| sqrt(1 + sigma^2).
//
// K^T (k_cone_gather, no atomics): one thread per 2 x 2 in-plane pixel quad of one slice.
// Per view it scans the channels whose in-plane trace can reach the quad (the fan-beam quad
// window) and, for each, the rows whose slope can put a slice weight on slice k over the
// quad's lines (from the in-plane distance of the quad, widened by 2.5 pixels and 1% of a
// slice), and evaluates exactly the forward kernel's in-plane weight and FP64 slice coordinate.
// Views, channels and rows are summed in increasing order, so the result is deterministic.
#include "../../include/ncs.h"
#include "ncs_internal.cuh"

#include <cmath>
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
    double2* d_zc = nullptr;     // per (view, channel): (Bz, Cz) of the in-plane distance Bz q + Cz
    double* d_sig = nullptr;     // per row: slope sigma_r
    float inv_pitch = 0.f, t_off = 0.f, inv_rp = 0.f, r_off = 0.f;
    double row_offset = 0.0;
};

namespace {

struct ConeArgs {
    const FanRay* rays;
    const float* rayw;
    const FanView* views;
    const double2* zc;
    const double* sig;
    int N, Nz, na, nr, nd;
    float inv_pitch, t_off;      // channel coordinate of a fan angle: gamma * inv_pitch + t_off
    float inv_rp, r_off;         // row coordinate of a slope: sigma * inv_rp + r_off
    const float* x;
    const float* y;
    float* out;
};

// The integer index and weight of a crossing f = H + L (the same expression as the
// parallel- and fan-beam kernels of joseph.cu).
__device__ __forceinline__ float cone_split_weight(float H, float L, float& k0)
{
    const float Hi = floorf(H);
    const float fr = (H - Hi) + L;
    const float fl = floorf(fr);
    k0 = Hi + fl;
    return fr - fl;
}

__device__ __forceinline__ float vox(const float* x, int N, int Nz, int k, int j, int i)
{
    return (k >= 0 && k < Nz && j >= 0 && j < N && i >= 0 && i < N) ? __ldg(x + ((size_t)k * N + j) * N + i) : 0.0f;
}

// Path length per step of a ray with in-plane weight ws and slope sig (the same expression in
// both kernels).
__device__ __forceinline__ float cone_path(float ws, double sig)
{
    return fabsf(ws) * sqrtf(1.0f + (float)(sig * sig));
}

constexpr int CF_TB = 64;      // channels per forward block
constexpr int CF_SEG = 4;      // line segments per ray

__global__ void __launch_bounds__(CF_TB * CF_SEG) k_cone_fwd(ConeArgs g)
{
    __shared__ float red[CF_SEG][CF_TB];
    const int t = blockIdx.x * CF_TB + threadIdx.x, r = blockIdx.y, a = blockIdx.z;
    const int N = g.N, Nz = g.Nz;
    float acc = 0.0f, W3 = 0.0f;
    if (t < g.nd) {
        const size_t rt = (size_t)a * g.nd + t;
        const float4 q = __ldg(g.rays + rt);
        const float ws = __ldg(g.rayw + rt);
        const double2 zc = g.zc[rt];
        const double sig = g.sig[r];
        const bool row = !(ws < 0.0f);
        const double cZ = 0.5 * (double)(Nz - 1);
        const int chunk = (N + CF_SEG - 1) / CF_SEG;
        const int ls = threadIdx.y * chunk, le = min(N, ls + chunk);
        for (int l = ls; l < le; ++l) {
            const float lf = (float)l;
            float k0f;
            const float w = cone_split_weight(fmaf(q.x, lf, q.z), fmaf(q.y, lf, q.w), k0f);
            if (!(k0f >= -1.0f && k0f < (float)N)) continue;        // both in-plane taps outside
            const int p0 = (int)k0f;
            const double gz = fma(sig, fma(zc.x, (double)l, zc.y), cZ);
            const double kz = floor(gz);
            if (!(kz >= -1.0 && kz < (double)Nz)) continue;         // both slice taps outside
            const int k0 = (int)kz;
            const float wz = (float)(gz - kz);
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
        W3 = cone_path(ws, sig);
    }
    red[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.y == 0 && t < g.nd) {
        float tot = red[0][threadIdx.x];
#pragma unroll
        for (int s = 1; s < CF_SEG; ++s) tot += red[s][threadIdx.x];
        g.out[((size_t)a * g.nr + r) * g.nd + t] = W3 * tot;
    }
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

// Weight that slice coordinate g puts on slice k.
__device__ __forceinline__ float slice_weight(double g, int k)
{
    const double kz = floor(g);
    const float wz = (float)(g - kz);
    return kz == (double)k ? 1.0f - wz : (kz == (double)(k - 1) ? wz : 0.0f);
}

__global__ void __launch_bounds__(CQX * CQY) k_cone_gather(ConeArgs g)
{
    const int N = g.N, Nz = g.Nz, nd = g.nd, nr = g.nr;
    const int i = blockIdx.x * (2 * CQX) + 2 * (int)(threadIdx.x % CQX);
    const int j = blockIdx.y * (2 * CQY) + 2 * (int)(threadIdx.x / CQX);
    const int k = blockIdx.z;
    if (i >= N || j >= N) return;           // N is even: a quad is inside or outside
    const float cN = 0.5f * (float)(N - 1);
    const double cZ = 0.5 * (double)(Nz - 1);
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
            const double2 zc = g.zc[rt];
            const double hA = fma(zc.x, (double)l0, zc.y), hB = fma(zc.x, (double)l1, zc.y);
            for (int r = r0; r <= r1; ++r) {
                const double sig = g.sig[r];
                const float zA = slice_weight(fma(sig, hA, cZ), k);
                const float zB = slice_weight(fma(sig, hB, cZ), k);
                if (zA == 0.0f && zB == 0.0f) continue;
                const float Wu = cone_path(ws, sig) * __ldg(g.y + ((size_t)a * nr + r) * nd + t);
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
    float* o = g.out + ((size_t)k * N + j) * N + i;
    o[0] = a00;
    o[1] = a01;
    o[N] = a10;
    o[N + 1] = a11;
}

ConeArgs args_of(const ncs_cone* c)
{
    ConeArgs a{};
    a.rays = c->d_rays;
    a.rayw = c->d_rayw;
    a.views = c->d_views;
    a.zc = c->d_zc;
    a.sig = c->d_sig;
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
    cudaFree(c->d_zc);
    cudaFree(c->d_sig);
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
    if (rc == NCS_OK) rc = cone_alloc(&c->d_zc, m);
    if (rc == NCS_OK) rc = cone_alloc(&c->d_sig, (size_t)nr);
    if (rc == NCS_OK &&
        (cudaMemcpy(c->d_rays, rays.data(), m * sizeof(FanRay), cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(c->d_rayw, rayw.data(), m * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(c->d_views, views.data(), na * sizeof(FanView), cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(c->d_zc, zc.data(), m * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(c->d_sig, sig.data(), nr * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess))
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
    k_cone_fwd<<<grid, block, 0, c->st>>>(a);
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
