// Joseph projector pair for sm_103a.
//
// K (forward, ray-driven): one thread per (angle, bin, row segment); the ray
// is stepped over the rows of x (row-branch angles) or of x^T (column-branch
// angles), so a warp of 32 consecutive bins always reads one contiguous row
// segment; both taps of a step come from one 8-byte load of the pair image.  Partial sums of the segments are combined in shared memory in a
// fixed order, then a fused epilogue applies prox_{alpha g*} to the data dual
// (Sec. 4.1: divide by 1 + alpha; Sec. 4.2: the closed-form S(u; c)), or
// reduces the data term of the objective in FP64.  With L2 data the prox epilogue can
// also carry the running K x of a solve and the FP64 data term at K x+.
//
// K^T (gather, no atomics on data): a block owns a 32 x 32 pixel tile and a
// slice of the angles.  Each warp takes whole angles and walks the (ray, line)
// pairs that cross the tile, evaluating exactly the FP32 crossing and weight
// expression of the forward kernel (so the two kernels hold the same matrix),
// and accumulates into its own shared-memory tile.  The warp tiles are summed
// in a fixed order; when the angles are split over several blocks, the last
// block of a tile (an arrival counter) sums the slices in slice order.  The
// epilogue adds (beta/alpha) D^T v and kappa s (A^T of Sec. 4) and, for PDHG
// (eq. (PDHG)), applies the primal update.
//
// Fan beam (Sec. 4, fan beam geometry): the forward kernel reads per-ray
// coefficients instead of per-angle ones (same stepping, taps and epilogues), and
// K^T is a pixel-driven gather (k_gather_fan) that evaluates the same weights.
#include "ncs_internal.cuh"

#include <algorithm>
#include <climits>

namespace ncs {

namespace {

constexpr int FWD_TB = 64;    // bins per block
constexpr int FWD_SEG = 4;    // row segments per ray

// floor(v) for |v| < 2^22 on the FP32 pipe (no conversion instructions): v + 1.5 * 2^23
// rounded toward -infinity is the integer floor(v) + 1.5 * 2^23, since floats in [2^23, 2^24)
// are spaced 1 apart; subtracting 1.5 * 2^23 again is exact.  bits gets the sum's bit
// pattern, which exceeds FLOOR_MAG_BITS by floor(v).
constexpr float FLOOR_MAG = 12582912.0f;       // 1.5 * 2^23
constexpr int FLOOR_MAG_BITS = 0x4B400000;      // its bit pattern
__device__ __forceinline__ float floor_fp32(float v, int& bits)
{
    const float m = __fadd_rd(v, FLOOR_MAG);
    bits = __float_as_int(m);
    return m - FLOOR_MAG;
}

// Integer index k0 and interpolation weight w of the crossing f = H + L, where
// H = A_hi t + B_hi q + C_hi is exact and L = A_lo t + (B_lo q + C_lo) is small:
// k0 = floor(H) + floor(frac(H) + L), w = (frac(H) + L) - that second floor.
// The one expression every projector kernel uses, so they hold the same FP32 matrix.
__device__ __forceinline__ float split_weight(float H, float L, int& k0)
{
    int bh, bf;
    const float Hi = floor_fp32(H, bh);
    const float fr = (H - Hi) + L;
    const float fl = floor_fp32(fr, bf);
    k0 = (bh - FLOOR_MAG_BITS) + (bf - FLOOR_MAG_BITS);
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

// Lines [jlo, jhi) of the stepping axis where a ray f = f0 + B q can touch the image:
// f in [-1, N), found in FP32 with a 2-line margin (|B| <= 1, so f stays in (-4, N + 3) on
// every line of the range and the pair image's zero border absorbs the steps outside the
// image).  Every line outside the range has f outside [-1, N), where both taps are zero.
__device__ __forceinline__ void fwd_lines(float f0, float B, int N, int& jlo, int& jhi)
{
    jlo = 0;
    jhi = N;
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
}

// The mode's epilogue for sinogram entry idx with y = (K x)[idx]: the prox of the data dual
// (Sec. 4.1: divide by 1 + alpha; Sec. 4.2: the closed-form S(u; c)), the running K x, or a
// data-term summand.  Returns the FP64 summand (0 where the mode has none).
template <int MODE, bool SBF>
__device__ __forceinline__ double fwd_finish(const FwdArgs& g, size_t idx, float y)
{
    double term = 0.0;
    if (MODE == FWD_PLAIN) {
        St<false>::put(g.y, idx, y);
    } else if (MODE == FWD_PROX_L2) {
        const float bv = St<false>::ld(g.b, idx);
        const float z = fmaf(g.alpha, y - bv, St<SBF>::get(g.y, idx));
        St<SBF>::put_sr(g.y, idx, z * g.inv1pa, SBF ? rand16(*g.iter, idx, 1u) : 0u);
        if (g.kx) {
            // x+ = (xbar + x) / 2, so K x+ = (K xbar + K x) / 2 without another projection
            const float kxp = 0.5f * (y + g.kx[idx]);
            g.kx[idx] = kxp;
            const double d = (double)kxp - (double)bv;
            term = d * d;
        }
    } else if (MODE == FWD_PROX_KL) {
        const float bgv = g.bg ? St<false>::ld(g.bg, idx) : 0.0f;
        const float z = fmaf(g.alpha, y + bgv, St<SBF>::get(g.y, idx));
        St<SBF>::put_sr(g.y, idx, kl_conj_prox(z, g.alpha * St<false>::ld(g.b, idx)),
                        SBF ? rand16(*g.iter, idx, 1u) : 0u);
    } else if (MODE == FWD_RESID_L2) {
        const double d = (double)y - (double)St<false>::ld(g.b, idx);
        term = d * d;
    } else {  // FWD_RESID_KL
        const double mu = (double)y + (g.bg ? (double)St<false>::ld(g.bg, idx) : 0.0);
        const double bb = (double)St<false>::ld(g.b, idx);
        term = mu - bb;
        if (bb > 0.0) term += bb * log(bb / mu);
    }
    return term;
}

// The end of a forward launch in a (FWD_TB x FWD_SEG) block for ray (a, t): the FWD_SEG
// partial sums in red are added in a fixed order and scaled by the path length Wr, and the
// mode's epilogue runs; the RESID modes (and PROX_L2 with a running K x) leave one FP64
// partial sum per block.  Called by every thread of the block.
template <int MODE, bool SBF>
__device__ __forceinline__ void fwd_epilogue(const FwdArgs& g, int a, int t, float Wr, float (*red)[FWD_TB],
                                             double* dred)
{
    __syncthreads();
    double term = 0.0;
    if (threadIdx.y == 0 && t < g.n_det) {
        float tot = red[0][threadIdx.x];
#pragma unroll
        for (int q = 1; q < FWD_SEG; ++q) tot += red[q][threadIdx.x];
        term = fwd_finish<MODE, SBF>(g, (size_t)a * g.n_det + t, Wr * tot);
    }
    if (MODE == FWD_RESID_L2 || MODE == FWD_RESID_KL || (MODE == FWD_PROX_L2 && g.partials)) {
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

// FAN: the ray's coefficients come from the per-ray table (fan beam) instead of the
// block's angle; with no per-bin term the crossing is H = Bhi q + Chi, L = Blo q + Clo.
template <int MODE, bool PBF, bool SBF, bool FAN>
__global__ void __launch_bounds__(FWD_TB * FWD_SEG)
k_fwd(FwdArgs g)
{
    __shared__ float red[FWD_SEG][FWD_TB];
    __shared__ double dred[FWD_TB];
    const int a = blockIdx.y;
    const int t = blockIdx.x * FWD_TB + threadIdx.x;
    // FAN: the ray's split coefficients (see FanRay); parallel beam: the angle's 32.32 ones
    float Bhi = 0.f, Blo = 0.f, Chi = 0.f, Clo = 0.f, Wr, B, f0 = 0.f;
    long long Fi = 0, Bi = 0;
    int row;
    const float ft = (float)t;
    if (FAN) {
        const size_t r = (size_t)a * g.n_det + min(t, g.n_det - 1);
        const float4 q = __ldg(g.rays + r);
        const float ws = __ldg(g.rayw + r);
        Bhi = q.x;
        Blo = q.y;
        Chi = q.z;
        Clo = q.w;
        Wr = fabsf(ws);
        row = ws < 0.0f ? 0 : 1;
        B = Bhi + Blo;
        f0 = Chi + Clo;
    } else {
        const AngleParam p = g.ap[a];
        Wr = p.W;
        row = p.row;
        B = p.Bf;
        f0 = fmaf(p.Af, ft, p.Cf);
        Fi = p.Ai * (long long)t + p.Ci;       // crossing of line 0, 32.32
        Bi = p.Bi;
    }
    const void* im2 = row ? g.img2 : g.imgT2;
    const int pitch = pair_pitch(g.N);
    const int N = g.N;
    float acc = 0.0f;
    if (t < g.n_det) {
        // rows where the ray can touch the image
        int jlo, jhi;
        fwd_lines(f0, B, N, jlo, jhi);
        const int len = max(0, jhi - jlo);
        const int chunk = (len + FWD_SEG - 1) / FWD_SEG;
        const int js = jlo + threadIdx.y * chunk;
        const int je = min(jhi, js + chunk);
        if (FAN) {
            for (int j = js; j < je; ++j) {
                const float jf = (float)j;
                int i0;
                const float w = split_weight(fmaf(Bhi, jf, Chi), fmaf(Blo, jf, Clo), i0);
                const float2 xv = St<PBF>::ld2(im2, (size_t)j * pitch + PAIR_PAD + i0);
                acc = fmaf(1.0f - w, xv.x, acc);
                acc = fmaf(w, xv.y, acc);
            }
        } else {
            long long F = Fi + Bi * (long long)js;
            const size_t rs = (size_t)pitch * 2 * St<PBF>::bytes;      // bytes per pair-image row
            const char* rowp = static_cast<const char*>(im2) + ((size_t)js * pitch + PAIR_PAD) * 2 * St<PBF>::bytes;
            int j = js;
            // four rows at a time: their loads are independent, so all four are issued before
            // the first is used (the taps are summed in row order, as in the loop below)
            for (; j + 4 <= je; j += 4) {
                int k0, k1, k2, k3;
                const float w0 = fix_weight(F, k0);
                const float w1 = fix_weight(F + Bi, k1);
                const float w2 = fix_weight(F + 2 * Bi, k2);
                const float w3 = fix_weight(F + 3 * Bi, k3);
                const float2 x0 = St<PBF>::ld2(rowp, k0);
                const float2 x1 = St<PBF>::ld2(rowp + rs, k1);
                const float2 x2 = St<PBF>::ld2(rowp + 2 * rs, k2);
                const float2 x3 = St<PBF>::ld2(rowp + 3 * rs, k3);
                acc = fmaf(1.0f - w0, x0.x, acc);
                acc = fmaf(w0, x0.y, acc);
                acc = fmaf(1.0f - w1, x1.x, acc);
                acc = fmaf(w1, x1.y, acc);
                acc = fmaf(1.0f - w2, x2.x, acc);
                acc = fmaf(w2, x2.y, acc);
                acc = fmaf(1.0f - w3, x3.x, acc);
                acc = fmaf(w3, x3.y, acc);
                F += 4 * Bi;
                rowp += 4 * rs;
            }
            for (; j < je; ++j) {
                int i0;
                const float w = fix_weight(F, i0);
                const float2 xv = St<PBF>::ld2(rowp, i0);
                acc = fmaf(1.0f - w, xv.x, acc);
                acc = fmaf(w, xv.y, acc);
                F += Bi;
                rowp += rs;
            }
        }
    }
    red[threadIdx.y][threadIdx.x] = acc;
    fwd_epilogue<MODE, SBF>(g, a, t, Wr, red, dred);
}

// Strip form of the parallel-beam K.  A block holds image rows [r0, r0 + R) of x (row-branch
// angles) or of x^T (column-branch angles) in shared memory, x[j][i] at column i + PAIR_PAD
// of a row of SPC floats (N + 2 PAIR_PAD of them used, zeros beyond the image), and runs a
// slice of that branch's angles through it: one warp per 32 consecutive bins of one angle,
// lane = ray.  The strip is read from L2 once per block instead of once per angle.  The warp
// walks the lines of the strip that any of its rays touches (a host table of exact 32.32
// ranges, wrange), all lanes on the same line, so the two tap loads of a step hit one row of
// shared memory; a line outside a lane's own range contributes an exact zero (its crossing
// lies outside [-1, N), and the tap index is clamped to the zero border).  The sum over the
// strip goes to plane s of spart; k_fwd_sum adds the planes in strip order and runs the
// epilogue.  Rows are stepped with the same 32.32 crossing and fix_weight as k_fwd and the
// gather, so all three hold one matrix.  SPC is a compile-time row pitch (fwd_strip_pitch),
// so the four rows of an unrolled step sit at constant offsets from one another.
constexpr int FS_WARPS = 32;                 // warps per strip block (one block per SM)
constexpr int FSUM_T = 256;                  // threads per block of the strip sum, 4 rays each
constexpr int FS_SMEM = 220 * 1024;          // strip bytes per block
constexpr int FWD_MAX_STRIPS = 16;
constexpr int FS_PITCHES[] = {72, 136, 264, 392, 520, 656, 776, 872};   // strip row pitches (floats)

template <bool PBF, int SPC>
__global__ void __launch_bounds__(FS_WARPS * 32, 1)
k_fwd_strip(FwdArgs g)
{
    extern __shared__ float strip[];
    const int N = g.N, SP = pair_pitch(N);
    const int r0 = blockIdx.y * g.strip_rows;
    const int nr = min(g.strip_rows, N - r0);
    const bool colb = blockIdx.z != 0;
    const void* im2 = colb ? g.imgT2 : g.img2;
    // pair entry c of a row holds (x[c - PAIR_PAD], x[c + 1 - PAIR_PAD]): the even entries fill
    // the strip's row two floats at a time
    const int half = (SP + 1) >> 1;
    for (int e = threadIdx.x; e < nr * half; e += FS_WARPS * 32) {
        const int i = e / half;
        const int c = 2 * (e - i * half);
        const float2 v = St<PBF>::ld2(im2, (ptrdiff_t)(r0 + i) * SP + c);
        strip[i * SPC + c] = v.x;
        if (c + 1 < SP) strip[i * SPC + c + 1] = v.y;
    }
    __syncthreads();
    const int nb = colb ? g.n_ang - g.n_row : g.n_row;
    const int* list = g.order + (colb ? g.n_row : 0);
    const int per = (nb + gridDim.x - 1) / gridDim.x;
    const int lo = blockIdx.x * per;
    const int cnt = max(0, min(nb, lo + per) - lo);
    const int chunks = (g.n_det + 31) >> 5;
    const int lane = threadIdx.x & 31;
    float* out = g.spart + (size_t)blockIdx.y * fwd_strip_plane(g.n_ang, g.n_det);
    const unsigned last = (unsigned)(SP - 2);      // the last tap pair inside a strip row
    // items (angle ai of the slice, 32-bin chunk c) in order, FS_WARPS apart: (ai, c) advanced
    // without a division
    int ai = (threadIdx.x >> 5) / chunks, c = (threadIdx.x >> 5) - ai * chunks;
    for (; ai < cnt; c += FS_WARPS) {
        while (c >= chunks) {
            c -= chunks;
            ++ai;
        }
        if (ai >= cnt) break;
        const int a = __ldg(list + lo + ai);
        const int t = c * 32 + lane;
        const short2 wr = __ldg(g.wrange + (size_t)a * chunks + c);
        const int wa = max((int)wr.x, r0);
        const int wb = min((int)wr.y, r0 + nr);
        float acc = 0.0f;
        if (wa < wb) {
            const AngleParam& p = g.ap[a];
            const long long Bi = p.Bi;
            // crossing of line wa, 32.32, biased by PAIR_PAD so that its integer part is the
            // strip column of the first tap
            long long F = p.Ai * (long long)t + p.Ci + Bi * (long long)wa + ((long long)PAIR_PAD << 32);
            int ro = (wa - r0) * SPC;                       // strip offset of line j
            int j = wa;
            for (; j + 4 <= wb; j += 4) {
                int k0, k1, k2, k3;
                const float w0 = fix_weight(F, k0);
                const float w1 = fix_weight(F + Bi, k1);
                const float w2 = fix_weight(F + 2 * Bi, k2);
                const float w3 = fix_weight(F + 3 * Bi, k3);
                const float* q0 = strip + ro + min((unsigned)k0, last);
                const float* q1 = strip + ro + min((unsigned)k1, last);
                const float* q2 = strip + ro + min((unsigned)k2, last);
                const float* q3 = strip + ro + min((unsigned)k3, last);
                acc = fmaf(1.0f - w0, q0[0], acc);
                acc = fmaf(w0, q0[1], acc);
                acc = fmaf(1.0f - w1, q1[SPC], acc);
                acc = fmaf(w1, q1[SPC + 1], acc);
                acc = fmaf(1.0f - w2, q2[2 * SPC], acc);
                acc = fmaf(w2, q2[2 * SPC + 1], acc);
                acc = fmaf(1.0f - w3, q3[3 * SPC], acc);
                acc = fmaf(w3, q3[3 * SPC + 1], acc);
                F += 4 * Bi;
                ro += 4 * SPC;
            }
            for (; j < wb; ++j) {
                int k0;
                const float w = fix_weight(F, k0);
                const float* q = strip + ro + min((unsigned)k0, last);
                acc = fmaf(1.0f - w, q[0], acc);
                acc = fmaf(w, q[1], acc);
                F += Bi;
                ro += SPC;
            }
        }
        if (t < g.n_det) out[(size_t)a * g.n_det + t] = acc;
    }
}

// Sum of the strip planes of k_fwd_strip in strip order, then the epilogue of k_fwd: a thread
// takes four consecutive sinogram entries (one 16-byte load per plane; planes are padded to a
// multiple of four entries), and a block leaves one FP64 partial sum in the modes that have one.
template <int MODE, bool SBF>
__global__ void __launch_bounds__(FSUM_T)
k_fwd_sum(FwdArgs g)
{
    __shared__ double dred[FSUM_T / 32];
    const unsigned m = (unsigned)g.n_ang * (unsigned)g.n_det;
    const size_t plane = fwd_strip_plane(g.n_ang, g.n_det);
    const unsigned i0 = (blockIdx.x * FSUM_T + threadIdx.x) * 4u;
    double term = 0.0;
    if (i0 < m) {
        const float4* src = reinterpret_cast<const float4*>(g.spart + i0);
        const size_t pl4 = plane / 4;
        float4 tot = src[0];
#pragma unroll
        for (int q = 1; q < FWD_MAX_STRIPS; ++q) {
            if (q < g.n_strip) {
                const float4 v = src[q * pl4];
                tot.x += v.x;
                tot.y += v.y;
                tot.z += v.z;
                tot.w += v.w;
            }
        }
        const float tv[4] = {tot.x, tot.y, tot.z, tot.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const unsigned i = i0 + e;
            if (i < m) term += fwd_finish<MODE, SBF>(g, i, g.ap[i / (unsigned)g.n_det].W * tv[e]);
        }
    }
    if (MODE == FWD_RESID_L2 || MODE == FWD_RESID_KL || (MODE == FWD_PROX_L2 && g.partials)) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) term += __shfl_down_sync(0xffffffffu, term, o);
        if ((threadIdx.x & 31) == 0) dred[threadIdx.x >> 5] = term;
        __syncthreads();
        if (threadIdx.x == 0) {
            double sum = dred[0];
#pragma unroll
            for (int w = 1; w < FSUM_T / 32; ++w) sum += dred[w];
            g.partials[blockIdx.x] = sum;
        }
    }
}

constexpr int GT = 32;             // gather tile side (pixels)
constexpr int GW = 8;              // warps per gather block
constexpr int GP = GT + 1;         // pitch of a warp tile
constexpr int GU = 96;             // staged W u per warp: the rays one angle's walks visit (<= 2 GT + 2)

// Gather epilogue for pixel (j, i) with K^T u summed in r: adds dscale D^T v and kappa s
// (A^T of Sec. 4), then stores r (GATHER_R) or applies the PDHG primal update.
template <int MODE, bool IBF>
__device__ __forceinline__ void gather_epilogue(const GatherArgs& g, int j, int i, float r)
{
    const int N = g.N;
    const size_t pix = (size_t)j * N + i;
    if (g.v) {
        const size_t NN = (size_t)N * N;
        float dt = 0.0f;
        if (i < N - 1) dt += St<IBF>::get(g.v, pix);
        if (i >= 1) dt -= St<IBF>::get(g.v, pix - 1);
        if (j < N - 1) dt += St<IBF>::get(g.v, NN + pix);
        if (j >= 1) dt -= St<IBF>::get(g.v, NN + pix - N);
        r = fmaf(g.dscale, dt, r);
    }
    if (g.s) r = fmaf(g.kappa, St<IBF>::get(g.s, pix), r);
    if (MODE == GATHER_R) {
        g.r[pix] = r;
    } else {
        const float x = g.x[pix];
        const float x1 = fmaf(-g.inv_gamma, r, x);
        g.x[pix] = x1;
        g.xbar[pix] = 2.0f * x1 - x;
    }
}

// K^T for the parallel beam (no atomics on data).  A block owns a 32 x 32 pixel tile and a slice
// z of the angles: entries z, z + P, z + 2P, ... of the list of row-branch angles and of the list
// of column-branch angles (so that every slice holds angles of both branches); warps 0-3 take
// the slice's row-branch angles, warps 4-7 its column-branch ones, round robin.  For one angle, lane l owns line l of the tile (row l, or
// column l) and walks the tile's 32 positions along it in order, holding the 32 sums of its
// line in registers across all its angles.  Rays are visited in order of their crossing with
// the line, F = Ai t + Bi q + Ci in 32.32 fixed point (the forward kernel's exact expression,
// so the two kernels hold the same matrix): the crossing at k0 with weight w puts (1 - w) W u_t
// on position k0 and w W u_t on k0 + 1, and since rays cross a line at distinct k0 (|A| >= 1),
// position k receives at most the w-part of the ray at k - 1 and the (1 - w)-part of the ray at
// k; the walk advances to the next ray after taking a w-part.  W u of the warp's rays is staged
// in shared memory per angle (zero beyond the detector).  At the end the warps write their lines
// to shared tiles, summed per pixel in a fixed order; with several slices the last block of a
// tile (an arrival counter) sums the slices in slice order.
template <int MODE, bool SBF, bool IBF>
__global__ void __launch_bounds__(GT * GW)
k_gather(GatherArgs g)
{
    __shared__ float tiles[GW][GT * GP];      // warp tiles: pixel (r, c) at r GP + c
    __shared__ float su[GW][GU];
    __shared__ int s_last;
    const int N = g.N;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int i0 = blockIdx.x * GT, j0 = blockIdx.y * GT;
    float* U = su[wid];
    if (g.iter && tid == 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) *g.iter += 1ull;
    const bool rowwarp = wid < GW / 2;
    const int wsub = rowwarp ? wid : wid - GW / 2;
    const int q = (rowwarp ? j0 : i0) + lane;       // this lane's line: a row, or a column
    const int o0 = rowwarp ? i0 : j0;               // the tile's first position along it
    const bool live = q < N;
    float acc[GT];
#pragma unroll
    for (int k = 0; k < GT; ++k) acc[k] = 0.0f;
    const int P = gridDim.z, part = blockIdx.z;
    // this warp's angles: entries part + P (wsub + 4 m) of its branch's list
    const int n_row = min(max(g.n_row, 0), g.n_ang);
    const int nb = rowwarp ? n_row : g.n_ang - n_row;
    const int* ord = g.order + (rowwarp ? 0 : n_row);
    for (int r = part + P * wsub; r < nb; r += P * (GW / 2)) {
        const int a = __ldg(ord + r);
        const AngleParam& pa = g.ap[a];
        const long long Ai = __ldg(&pa.Ai), Bi = __ldg(&pa.Bi), Ci = __ldg(&pa.Ci);
        const float Bf = __ldg(&pa.Bf), Cf = __ldg(&pa.Cf), W = __ldg(&pa.W), invA = __ldg(&pa.invA);
        // walk order: increasing crossing, so t goes up when Ai > 0 and down when Ai < 0
        const bool upw = Ai > 0;
        const int dir = upw ? 1 : -1;
        const long long step = upw ? Ai : -Ai;
        // crossing of ray t relative to the tile's first position: G = Ai t + Bi q + Ci - o0 2^32
        const long long Gq = Bi * (long long)q + Ci - ((long long)o0 << 32);
        // the first ray in walk order whose crossing is >= -1 (it gives position 0 its w-part):
        // the FP32 estimate of where the crossing is -1 is within 0.05 rays, so the rounded
        // estimate is that ray or the one before it
        const float c = fmaf(Bf, (float)q, Cf) - (float)o0;
        const float tr = (-1.0f - c) * invA;
        int t0 = upw ? __float2int_rd(tr + 0.05f) : __float2int_ru(tr - 0.05f);
        long long G = Ai * (long long)t0 + Gq;
        if ((int)(G >> 32) < -1) {
            t0 += dir;
            G += step;
        }
        // the lane visits at most GT + 1 rays from t0; stage W u for the warp's rays
        int tlo = upw ? t0 : t0 - GT, thi = upw ? t0 + GT : t0;
        if (!live) {
            tlo = 0x3FFFFFFF;
            thi = -0x3FFFFFFF;
        }
        const int Tmin = __reduce_min_sync(0xffffffffu, tlo);
        const int Tmax = __reduce_max_sync(0xffffffffu, thi);
        const int nU = min(Tmax - Tmin + 1, GU);     // <= 2 GT + 2: the bound never binds
        const void* ua = static_cast<const char*>(g.u) + (size_t)a * g.n_det * St<SBF>::bytes;
        for (int e = lane; e < nU; e += 32) {
            const int t = Tmin + e;
            U[e] = (t >= 0 && t < g.n_det) ? W * St<SBF>::ld(ua, t) : 0.0f;
        }
        __syncwarp();
        if (live) {
            int ui = t0 - Tmin;
            int k0;
            float w = fix_weight(G, k0);
            float wu = U[ui];
            float vr = fmaf(-w, wu, wu), vl = w * wu;
            // branch-free: only the step to the next ray is conditional; the weight and W u of
            // the current ray are recomputed at every position.  One compare per position: the
            // test "the current ray crosses at k" of position k is "at (k + 1) - 1" for position
            // k + 1, and its 0/1 factor m serves both adds by a multiply-add
            bool adv = k0 == -1;
            float m = adv ? 1.0f : 0.0f;
#pragma unroll
            for (int k = 0; k < GT; ++k) {
                acc[k] = fmaf(m, vl, acc[k]);
                if (adv) {
                    G += step;
                    ui += dir;
                }
                w = fix_weight(G, k0);
                wu = U[ui];
                vr = fmaf(-w, wu, wu);
                vl = w * wu;
                adv = k0 == k;
                m = adv ? 1.0f : 0.0f;
                acc[k] = fmaf(m, vr, acc[k]);
            }
        }
        __syncwarp();
    }
    // each warp's lines into its tile (row lanes along rows, column lanes along columns)
    float* T = tiles[wid];
#pragma unroll
    for (int k = 0; k < GT; ++k) {
        if (rowwarp) T[lane * GP + k] = acc[k];
        else T[k * GP + lane] = acc[k];
    }
    __syncthreads();
    // sum the warp tiles in a fixed order; thread -> pixels (q*8 + wid, lane)
    float tot[GT / GW];
#pragma unroll
    for (int qq = 0; qq < GT / GW; ++qq) {
        const int rr = qq * GW + wid;
        float sum = 0.0f;
#pragma unroll
        for (int w = 0; w < GW; ++w) sum += tiles[w][rr * GP + lane];
        tot[qq] = sum;
    }
    if (P > 1) {
        // angle slices of this tile: the last block to arrive sums them in slice order
        const size_t NN = (size_t)N * N;
#pragma unroll
        for (int qq = 0; qq < GT / GW; ++qq) {
            const int j = j0 + qq * GW + wid, i = i0 + lane;
            if (j < N && i < N) g.part[(size_t)part * NN + (size_t)j * N + i] = tot[qq];
        }
        __threadfence();
        __syncthreads();
        const int tile = blockIdx.y * gridDim.x + blockIdx.x;
        if (tid == 0) s_last = (atomicAdd(&g.counters[tile], 1) == P - 1);
        __syncthreads();
        if (!s_last) return;
        __threadfence();
#pragma unroll
        for (int qq = 0; qq < GT / GW; ++qq) {
            const int j = j0 + qq * GW + wid, i = i0 + lane;
            float sum = 0.0f;
            if (j < N && i < N)
                for (int pp = 0; pp < P; ++pp) sum += __ldcg(g.part + (size_t)pp * NN + (size_t)j * N + i);
            tot[qq] = sum;
        }
        if (tid == 0) g.counters[tile] = 0;
    }
#pragma unroll
    for (int qq = 0; qq < GT / GW; ++qq) {
        const int j = j0 + qq * GW + wid, i = i0 + lane;
        if (j >= N || i >= N) continue;
        gather_epilogue<MODE, IBF>(g, j, i, tot[qq]);
    }
}

constexpr int FQX = 16;    // fan-beam gather block: 16 x 8 threads, each owning a 2 x 2 pixel quad,
constexpr int FQY = 8;     // so a block covers 32 columns x 16 rows

// Weights that one crossing (integer part k0, fraction w) of a line puts on the two
// positions p and p + 1 of that line: 1 - w where k0 is the position, w where k0 is one less.
__device__ __forceinline__ void quad_weights(int p, int k0, float w, float& c0, float& c1)
{
    const int d = p - k0;
    c0 = d == 0 ? 1.0f - w : (d == 1 ? w : 0.0f);
    c1 = d == -1 ? 1.0f - w : (d == 0 ? w : 0.0f);
}

// K^T for the fan beam (pixel-driven, no atomics).  Rays of one view are not parallel, and
// adjacent rays can cross a line less than a pixel apart, so the tile walk above does not
// carry over.  Instead each thread owns a 2 x 2 pixel quad (N is even, so a quad is inside
// the image or outside it) and, per view a, finds the channels whose ray can reach it: a ray
// that puts a nonzero Joseph weight on a pixel passes within one pixel of its centre (|f - k|
// < 1 along the interpolation axis, and the perpendicular distance is that times |cos| or
// |sin| <= 1), hence within 1 + sqrt(2)/2 of the quad's centre Q, so its fan angle differs
// from Q's fan angle, atan2(cross, dot) of (Q - S_a) against the central direction, by less
// than asin((1 + sqrt(2)/2) / |Q - S_a|) <= x + x^3.  That window, widened for FP32 rounding,
// is scanned; each candidate ray's weights on the quad's two lines (rows j, j + 1 for a ray
// stepped over rows, columns i, i + 1 otherwise) come from the forward kernel's split_weight
// on the ray's own coefficients, so the pair holds the same FP32 matrix.  Each pixel sums
// its views in order and their channels in increasing order (deterministic).  With view slices
// (gridDim.z > 1) the last block of a tile sums the slices in slice order.
template <int MODE, bool SBF, bool IBF>
__global__ void __launch_bounds__(FQX * FQY)
k_gather_fan(GatherArgs g)
{
    __shared__ int s_last;
    const int N = g.N, nd = g.n_det;
    const int i = blockIdx.x * (2 * FQX) + 2 * (int)(threadIdx.x % FQX);
    const int j = blockIdx.y * (2 * FQY) + 2 * (int)(threadIdx.x / FQX);
    const bool inside = i < N && j < N;
    if (g.iter && threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) *g.iter += 1ull;
    const int P = gridDim.z, part = blockIdx.z;
    const int a_beg = (int)(((long long)g.n_ang * part) / P);
    const int a_end = (int)(((long long)g.n_ang * (part + 1)) / P);
    float a00 = 0.0f, a01 = 0.0f, a10 = 0.0f, a11 = 0.0f;     // pixel (j + r, i + c) in a{r}{c}
    if (inside) {
        const float cN = 0.5f * (float)(N - 1);
        const float qu = ((float)i + 0.5f) - cN, qv = cN - ((float)j + 0.5f);   // quad centre (exact)
        const float fi = (float)i, fj = (float)j;
        for (int a = a_beg; a < a_end; ++a) {
            const float4 sv = __ldg(g.views + a);
            const float du = qu - sv.x, dv = qv - sv.y;
            const float cr = fmaf(sv.z, dv, -sv.w * du);          // |Q - S| sin(gamma_Q)
            const float dt = fmaf(sv.z, du, sv.w * dv);           // |Q - S| cos(gamma_Q)
            const float tc = fmaf(atan2f(cr, dt), g.inv_pitch, g.t_off);
            // x = (1 + sqrt(2)/2) / |Q - S| with a relative margin of 2e-3
            const float x = fminf(1.0f, 1.7092f * rsqrtf(fmaf(du, du, dv * dv)));
            const float half = fmaf(fmaf(x, x * x, x), g.inv_pitch, 0.02f);
            const int t0 = max(0, (int)ceilf(tc - half));
            const int t1 = min(nd - 1, (int)floorf(tc + half));
            const size_t base = (size_t)a * nd;
            const void* ua = static_cast<const char*>(g.u) + base * St<SBF>::bytes;
            for (int t = t0; t <= t1; ++t) {
                const float4 q = __ldg(g.rays + base + t);
                const float ws = __ldg(g.rayw + base + t);
                const bool row = !(ws < 0.0f);
                const float Wu = fabsf(ws) * St<SBF>::ld(ua, t);
                const float l0 = row ? fj : fi;             // the quad's first line for this ray
                const float l1 = l0 + 1.0f;
                const int p0 = row ? i : j;                 // its first position along the line
                int kA, kB;
                float cA0, cA1, cB0, cB1;
                const float wA = split_weight(fmaf(q.x, l0, q.z), fmaf(q.y, l0, q.w), kA);
                const float wB = split_weight(fmaf(q.x, l1, q.z), fmaf(q.y, l1, q.w), kB);
                quad_weights(p0, kA, wA, cA0, cA1);
                quad_weights(p0, kB, wB, cB0, cB1);
                // row branch: line A is row j, line B row j + 1; column branch: A is column i, B column i + 1
                const float c01 = row ? cA1 : cB0;
                const float c10 = row ? cB0 : cA1;
                a00 = cA0 != 0.0f ? fmaf(cA0, Wu, a00) : a00;
                a01 = c01 != 0.0f ? fmaf(c01, Wu, a01) : a01;
                a10 = c10 != 0.0f ? fmaf(c10, Wu, a10) : a10;
                a11 = cB1 != 0.0f ? fmaf(cB1, Wu, a11) : a11;
            }
        }
    }
    if (P > 1) {
        const size_t NN = (size_t)N * N;
        float* pp0 = g.part + (size_t)part * NN + (size_t)j * N + i;
        if (inside) {
            *reinterpret_cast<float2*>(pp0) = make_float2(a00, a01);
            *reinterpret_cast<float2*>(pp0 + N) = make_float2(a10, a11);
        }
        __threadfence();
        __syncthreads();
        const int tile = blockIdx.y * gridDim.x + blockIdx.x;
        if (threadIdx.x == 0) s_last = (atomicAdd(&g.counters[tile], 1) == P - 1);
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        a00 = a01 = a10 = a11 = 0.0f;
        if (inside)
            for (int k = 0; k < P; ++k) {
                const float* src = g.part + (size_t)k * NN + (size_t)j * N + i;
                const float2 r0 = __ldcg(reinterpret_cast<const float2*>(src));
                const float2 r1 = __ldcg(reinterpret_cast<const float2*>(src + N));
                a00 += r0.x;
                a01 += r0.y;
                a10 += r1.x;
                a11 += r1.y;
            }
        if (threadIdx.x == 0) g.counters[tile] = 0;
    }
    if (inside) {
        gather_epilogue<MODE, IBF>(g, j, i, a00);
        gather_epilogue<MODE, IBF>(g, j, i + 1, a01);
        gather_epilogue<MODE, IBF>(g, j + 1, i, a10);
        gather_epilogue<MODE, IBF>(g, j + 1, i + 1, a11);
    }
}

constexpr int LT = 32;     // line-walk fan gather: 32 x 32 pixel tile per block
constexpr int LW = 4;      // warps per block, each with a private shared tile
constexpr int LCAP = 32;   // rays staged per warp at a time

// K^T for the fan beam, ray-driven (no atomics).  A block owns a 32 x 32 tile and a slice of
// the views; warps take whole views round robin.  Lane l owns line l of the tile: row j0 + l
// for rays stepped over rows, column i0 + l for rays stepped over columns, so whatever ray a
// lane works on it writes only its own row (or column) of the warp's tile, and rays closer
// than a pixel (adjacent fan rays can be) never collide.  The rays that can put a weight on
// the tile cross the tile widened by one pixel, so their channels lie between the fan angles
// of its four corners (atan2 of each corner seen from the source, widened for FP32
// rounding).  They are staged, up to 64 at a time, in the warp's shared arrays by coalesced
// loads (coefficients and W u), rays stepped over rows from the front in channel order and
// rays stepped over columns from the back; each lane then walks the row list and, after a
// warp barrier, the column list, starting at a lane-dependent offset (11 l mod n) so that
// simultaneous shared-memory writes spread over the banks.  The crossing and weight come
// from the forward's split_weight on the ray's coefficients and the lane's line.  Per pixel
// the order of the sums is fixed (views by warp and slice, rays by lane), so the result is
// deterministic.  Warp tiles are summed in a fixed order and view slices by the last block
// of a tile, as in k_gather.
template <int MODE, bool SBF, bool IBF>
__global__ void __launch_bounds__(LT * LW)
k_gather_fan_lines(GatherArgs g)
{
    // the sums of rays stepped over rows (pitch LT + 2) and over columns (pitch LT) go to separate
    // tiles: all lanes walk the same staged ray (broadcast reads), and a ray of slope B in
    // (-1, 1) puts lane l's tap in bank (2 + B) l + c of the row tile and in bank l of the
    // column tile, so the read-modify-writes conflict at most two ways
    __shared__ float tr[LW][LT][LT + 2];
    __shared__ float tc[LW][LT][LT];
    __shared__ float stage[LW][5][LCAP];      // Bhi, Blo, Chi, Clo, |W| u of the staged rays
    __shared__ int s_last;
    const int N = g.N, nd = g.n_det;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int i0 = blockIdx.x * LT, j0 = blockIdx.y * LT;
    float (*AR)[LT + 2] = tr[wid];
    float (*AC)[LT] = tc[wid];
    float (*S)[LCAP] = stage[wid];
    if (g.iter && tid == 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) *g.iter += 1ull;
    for (int rr = 0; rr < LT; ++rr) {
        AR[rr][lane] = 0.0f;
        AC[rr][lane] = 0.0f;
    }
    __syncwarp();
    const int P = gridDim.z, part = blockIdx.z;
    const int a_beg = (int)(((long long)g.n_ang * part) / P);
    const int a_end = (int)(((long long)g.n_ang * (part + 1)) / P);
    const float cN = 0.5f * (float)(N - 1);
    // corner (lane & 3) of the tile widened by one pixel: columns i0 - 1 / i0 + 32, rows j0 - 1 / j0 + 32
    const float cu = ((lane & 1) ? (float)(i0 + LT) : (float)(i0 - 1)) - cN;
    const float cv = cN - ((lane & 2) ? (float)(j0 + LT) : (float)(j0 - 1));
    const float lrow = (float)(j0 + lane), lcol = (float)(i0 + lane);
    const unsigned below = (1u << lane) - 1u;
    for (int a = a_beg + wid; a < a_end; a += LW) {
        const float4 sv = __ldg(g.views + a);
        const float du = cu - sv.x, dv = cv - sv.y;
        const float tcor = fmaf(atan2f(fmaf(sv.z, dv, -sv.w * du), fmaf(sv.z, du, sv.w * dv)), g.inv_pitch, g.t_off);
        float tmin = fminf(tcor, __shfl_xor_sync(0xffffffffu, tcor, 1));
        float tmax = fmaxf(tcor, __shfl_xor_sync(0xffffffffu, tcor, 1));
        tmin = fminf(tmin, __shfl_xor_sync(0xffffffffu, tmin, 2));
        tmax = fmaxf(tmax, __shfl_xor_sync(0xffffffffu, tmax, 2));
        const int t0 = max(0, (int)ceilf(tmin - 0.02f));
        const int t1 = min(nd - 1, (int)floorf(tmax + 0.02f));
        const size_t base = (size_t)a * nd;
        const void* ua = static_cast<const char*>(g.u) + base * St<SBF>::bytes;
        for (int c0 = t0; c0 <= t1; c0 += LCAP) {                  // warp-uniform
            const int c1 = min(t1, c0 + LCAP - 1);
            int nR = 0, nC = 0;
            for (int tb = c0; tb <= c1; tb += 32) {
                const int t = tb + lane;
                const bool valid = t <= c1;
                float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
                float ws = 0.0f, uu = 0.0f;
                if (valid) {
                    q = __ldg(g.rays + base + t);
                    ws = __ldg(g.rayw + base + t);
                    uu = St<SBF>::ld(ua, t);
                }
                const bool isrow = valid && !(ws < 0.0f);
                const bool iscol = valid && ws < 0.0f;
                const unsigned mr = __ballot_sync(0xffffffffu, isrow);
                const unsigned mc = __ballot_sync(0xffffffffu, iscol);
                if (valid) {
                    const int slot = isrow ? nR + __popc(mr & below) : LCAP - 1 - (nC + __popc(mc & below));
                    S[0][slot] = q.x;
                    S[1][slot] = q.y;
                    S[2][slot] = q.z;
                    S[3][slot] = q.w;
                    S[4][slot] = fabsf(ws) * uu;
                }
                nR += __popc(mr);
                nC += __popc(mc);
            }
            __syncwarp();
            for (int pass = 0; pass < 2; ++pass) {
                const int n = pass == 0 ? nR : nC;
                if (pass == 1) __syncwarp();
                if (n == 0) continue;                                // warp-uniform
                const bool rowpass = pass == 0;
                const int s0 = rowpass ? 0 : LCAP - nC;
                const float lf = rowpass ? lrow : lcol;
                const int o0 = rowpass ? i0 : j0;
                for (int k = 0; k < n; ++k) {
                    const int e = s0 + k;                            // the same ray in every lane
                    int k0;
                    const float w = split_weight(fmaf(S[0][e], lf, S[2][e]), fmaf(S[1][e], lf, S[3][e]), k0);
                    const float Wu = S[4][e];
                    const int kk = k0 - o0;
                    if ((unsigned)kk < (unsigned)LT) {
                        float& d = rowpass ? AR[lane][kk] : AC[kk][lane];
                        d = fmaf(1.0f - w, Wu, d);
                    }
                    if ((unsigned)(kk + 1) < (unsigned)LT) {
                        float& d = rowpass ? AR[lane][kk + 1] : AC[kk + 1][lane];
                        d = fmaf(w, Wu, d);
                    }
                }
            }
            __syncwarp();
        }
    }
    __syncthreads();
    // sum the warp tiles in a fixed order (row tiles, then column tiles); thread -> pixels
    // (q*LW + wid, lane)
    float tot[LT / LW];
#pragma unroll
    for (int q = 0; q < LT / LW; ++q) {
        const int rr = q * LW + wid;
        float sum = 0.0f;
#pragma unroll
        for (int w = 0; w < LW; ++w) sum += tr[w][rr][lane];
#pragma unroll
        for (int w = 0; w < LW; ++w) sum += tc[w][rr][lane];
        tot[q] = sum;
    }
    if (P > 1) {
        const size_t NN = (size_t)N * N;
#pragma unroll
        for (int q = 0; q < LT / LW; ++q) {
            const int j = j0 + q * LW + wid, i = i0 + lane;
            if (j < N && i < N) g.part[(size_t)part * NN + (size_t)j * N + i] = tot[q];
        }
        __threadfence();
        __syncthreads();
        const int tile = blockIdx.y * gridDim.x + blockIdx.x;
        if (tid == 0) s_last = (atomicAdd(&g.counters[tile], 1) == P - 1);
        __syncthreads();
        if (!s_last) return;
        __threadfence();
#pragma unroll
        for (int q = 0; q < LT / LW; ++q) {
            const int j = j0 + q * LW + wid, i = i0 + lane;
            float sum = 0.0f;
            if (j < N && i < N)
                for (int pp = 0; pp < P; ++pp) sum += __ldcg(g.part + (size_t)pp * NN + (size_t)j * N + i);
            tot[q] = sum;
        }
        if (tid == 0) g.counters[tile] = 0;
    }
#pragma unroll
    for (int q = 0; q < LT / LW; ++q) {
        const int j = j0 + q * LW + wid, i = i0 + lane;
        if (j < N && i < N) gather_epilogue<MODE, IBF>(g, j, i, tot[q]);
    }
}

}  // namespace

int fwd_num_blocks(int n_det, int n_ang)
{
    return ((n_det + FWD_TB - 1) / FWD_TB) * n_ang;
}

template <bool PBF, bool SBF, bool FAN>
void fwd_dispatch(int mode, const FwdArgs& a, dim3 grid, dim3 block, cudaStream_t st)
{
    switch (mode) {
        case FWD_PLAIN: k_fwd<FWD_PLAIN, PBF, SBF, FAN><<<grid, block, 0, st>>>(a); break;
        case FWD_PROX_L2: k_fwd<FWD_PROX_L2, PBF, SBF, FAN><<<grid, block, 0, st>>>(a); break;
        case FWD_PROX_KL: k_fwd<FWD_PROX_KL, PBF, SBF, FAN><<<grid, block, 0, st>>>(a); break;
        case FWD_RESID_L2: k_fwd<FWD_RESID_L2, PBF, SBF, FAN><<<grid, block, 0, st>>>(a); break;
        default: k_fwd<FWD_RESID_KL, PBF, SBF, FAN><<<grid, block, 0, st>>>(a); break;
    }
}

template <bool FAN>
void fwd_dispatch_prec(int mode, const FwdArgs& a, dim3 grid, dim3 block, cudaStream_t st)
{
    if (a.pair_bf && a.sino_bf) fwd_dispatch<true, true, FAN>(mode, a, grid, block, st);
    else if (a.pair_bf) fwd_dispatch<true, false, FAN>(mode, a, grid, block, st);
    else if (a.sino_bf) fwd_dispatch<false, true, FAN>(mode, a, grid, block, st);
    else fwd_dispatch<false, false, FAN>(mode, a, grid, block, st);
}

// Row pitch (floats) of the strip kernel's shared-memory rows for an N x N image: the
// smallest of FS_PITCHES that holds N + 2 PAIR_PAD floats, or 0 if none does.
int fwd_strip_pitch(int N)
{
    for (int sp : FS_PITCHES)
        if (sp >= pair_pitch(N)) return sp;
    return 0;
}

// Strip shape of the parallel-beam K for an N x N image: the rows per strip that leave room
// for one block per SM (FS_SMEM bytes) and the number of strips; false when more than
// FWD_MAX_STRIPS would be needed (the row walk k_fwd serves such images).
bool fwd_strip_shape(int N, int* rows, int* strips)
{
    const int sp = fwd_strip_pitch(N);
    if (N < 1 || sp == 0) return false;
    const int rmax = FS_SMEM / (int)(sizeof(float) * sp);
    const int s = (N + rmax - 1) / rmax;
    if (s > FWD_MAX_STRIPS) return false;
    *strips = s;
    *rows = (N + s - 1) / s;
    return true;
}

template <bool PBF, int SPC>
cudaError_t fwd_strip_attr()
{
    return cudaFuncSetAttribute(k_fwd_strip<PBF, SPC>, cudaFuncAttributeMaxDynamicSharedMemorySize, FS_SMEM);
}

// Opt-in to FS_SMEM bytes of dynamic shared memory for the strip kernels (once, before the
// first launch and outside any stream capture).
cudaError_t fwd_prepare()
{
    const cudaError_t e[] = {fwd_strip_attr<false, 72>(), fwd_strip_attr<false, 136>(), fwd_strip_attr<false, 264>(),
                             fwd_strip_attr<false, 392>(), fwd_strip_attr<false, 520>(), fwd_strip_attr<false, 656>(),
                             fwd_strip_attr<false, 776>(), fwd_strip_attr<false, 872>(),
                             fwd_strip_attr<true, 72>(), fwd_strip_attr<true, 136>(), fwd_strip_attr<true, 264>(),
                             fwd_strip_attr<true, 392>(), fwd_strip_attr<true, 520>(), fwd_strip_attr<true, 656>(),
                             fwd_strip_attr<true, 776>(), fwd_strip_attr<true, 872>()};
    for (cudaError_t x : e)
        if (x != cudaSuccess) return x;
    return cudaSuccess;
}

template <bool PBF>
void fwd_strip_dispatch(int sp, const FwdArgs& a, dim3 grid, size_t smem, cudaStream_t st)
{
    switch (sp) {
        case 72: k_fwd_strip<PBF, 72><<<grid, FS_WARPS * 32, smem, st>>>(a); break;
        case 136: k_fwd_strip<PBF, 136><<<grid, FS_WARPS * 32, smem, st>>>(a); break;
        case 264: k_fwd_strip<PBF, 264><<<grid, FS_WARPS * 32, smem, st>>>(a); break;
        case 392: k_fwd_strip<PBF, 392><<<grid, FS_WARPS * 32, smem, st>>>(a); break;
        case 520: k_fwd_strip<PBF, 520><<<grid, FS_WARPS * 32, smem, st>>>(a); break;
        case 656: k_fwd_strip<PBF, 656><<<grid, FS_WARPS * 32, smem, st>>>(a); break;
        case 776: k_fwd_strip<PBF, 776><<<grid, FS_WARPS * 32, smem, st>>>(a); break;
        default: k_fwd_strip<PBF, 872><<<grid, FS_WARPS * 32, smem, st>>>(a); break;
    }
}

// Per (angle, 32-bin chunk) the lines [lo, hi) of the stepping axis on which some ray of the
// chunk touches the image (its 32.32 crossing F has F >> 32 in [-1, N - 1]): exact, in 64-bit
// integers.  F is linear in t and in the line q with the same slope Bi for every ray, so the
// lines form one interval.  Rays past n_det are left out; an empty chunk gets lo = hi = 0.
void fwd_warp_ranges(int N, int n_det, const std::vector<AngleParam>& ap, std::vector<short2>& out)
{
    const int chunks = (n_det + 31) / 32;
    out.assign(ap.size() * chunks, short2{0, 0});
    const long long lo_f = -(1LL << 32), hi_f = (long long)N << 32;
    for (size_t a = 0; a < ap.size(); ++a) {
        const AngleParam& p = ap[a];
        for (int c = 0; c < chunks; ++c) {
            const int t0 = 32 * c, t1 = std::min(n_det - 1, t0 + 31);
            const long long f0 = p.Ai * t0 + p.Ci, f1 = p.Ai * t1 + p.Ci;
            const long long fmin = std::min(f0, f1), fmax = std::max(f0, f1);
            int lo = -1, hi = -1;
            for (int q = 0; q < N; ++q) {
                const long long d = p.Bi * (long long)q;
                if (fmax + d >= lo_f && fmin + d < hi_f) {
                    if (lo < 0) lo = q;
                    hi = q + 1;
                }
            }
            if (lo >= 0) out[a * chunks + c] = short2{(short)lo, (short)hi};
        }
    }
}

// FP64 partial sums one RESID launch (or PROX_L2 launch with a running K x) leaves
int fwd_num_partials(const FwdArgs& a)
{
    if (a.spart && !a.rays) {
        const long long m = (long long)a.n_ang * a.n_det;
        return (int)((m + 4LL * FSUM_T - 1) / (4LL * FSUM_T));
    }
    return fwd_num_blocks(a.n_det, a.n_ang);
}

template <bool SBF>
void fwd_sum_dispatch(int mode, const FwdArgs& a, dim3 grid, dim3 block, cudaStream_t st)
{
    switch (mode) {
        case FWD_PLAIN: k_fwd_sum<FWD_PLAIN, SBF><<<grid, block, 0, st>>>(a); break;
        case FWD_PROX_L2: k_fwd_sum<FWD_PROX_L2, SBF><<<grid, block, 0, st>>>(a); break;
        case FWD_PROX_KL: k_fwd_sum<FWD_PROX_KL, SBF><<<grid, block, 0, st>>>(a); break;
        case FWD_RESID_L2: k_fwd_sum<FWD_RESID_L2, SBF><<<grid, block, 0, st>>>(a); break;
        default: k_fwd_sum<FWD_RESID_KL, SBF><<<grid, block, 0, st>>>(a); break;
    }
}

cudaError_t launch_fwd(int mode, const FwdArgs& a, cudaStream_t st)
{
    if (mode < FWD_PLAIN || mode > FWD_RESID_KL) return cudaErrorInvalidValue;
    if (mode == FWD_PLAIN && a.sino_bf) return cudaErrorInvalidValue;    // y is float
    if (a.rays && !a.rayw) return cudaErrorInvalidValue;
    dim3 grid((a.n_det + FWD_TB - 1) / FWD_TB, a.n_ang), block(FWD_TB, FWD_SEG);
    if (a.spart && !a.rays) {
        const int sp = fwd_strip_pitch(a.N);
        if (!a.order || !a.ap || !a.wrange || sp == 0 || a.n_row < 0 || a.n_row > a.n_ang || a.n_strip < 1 ||
            a.strip_rows < 1 || a.n_strip > FWD_MAX_STRIPS || (long long)a.n_strip * a.strip_rows < a.N ||
            (long long)(a.n_strip - 1) * a.strip_rows >= a.N ||
            (size_t)a.strip_rows * sp * sizeof(float) > (size_t)FS_SMEM || a.N > 32767)
            return cudaErrorInvalidValue;
        int dev = 0, sms = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        // one resident block per SM: n_strip x 2 branches x G angle slices fill them once
        const dim3 sgrid(std::max(1, sms / (2 * a.n_strip)), a.n_strip, 2);
        const size_t smem = (size_t)a.strip_rows * sp * sizeof(float);
        if (a.pair_bf) fwd_strip_dispatch<true>(sp, a, sgrid, smem, st);
        else fwd_strip_dispatch<false>(sp, a, sgrid, smem, st);
        const dim3 sum_grid((unsigned)fwd_num_partials(a)), sum_block(FSUM_T);
        if (a.sino_bf) fwd_sum_dispatch<true>(mode, a, sum_grid, sum_block, st);
        else fwd_sum_dispatch<false>(mode, a, sum_grid, sum_block, st);
        return cudaGetLastError();
    }
    if (a.rays) fwd_dispatch_prec<true>(mode, a, grid, block, st);
    else fwd_dispatch_prec<false>(mode, a, grid, block, st);
    return cudaGetLastError();
}

size_t gather_tiles(int N)
{
    const size_t b = (size_t)(N + GT - 1) / GT;
    return b * b;
}

int gather_parts(int N, int n_ang)
{
    // about 2048 blocks (several waves of 152 SMs x 6 blocks); at most 64 slices
    const long long tiles = (long long)gather_tiles(N);
    long long p = (2048 + tiles - 1) / tiles;
    if (p > 64) p = 64;
    if (p > n_ang) p = n_ang;
    if (p < 1) p = 1;
    return (int)p;
}

template <int MODE>
void gather_dispatch(const GatherArgs& a, dim3 grid, dim3 block, cudaStream_t st)
{
    if (a.sino_bf && a.img_bf) k_gather<MODE, true, true><<<grid, block, 0, st>>>(a);
    else if (a.sino_bf) k_gather<MODE, true, false><<<grid, block, 0, st>>>(a);
    else if (a.img_bf) k_gather<MODE, false, true><<<grid, block, 0, st>>>(a);
    else k_gather<MODE, false, false><<<grid, block, 0, st>>>(a);
}

template <int MODE>
void gather_fan_dispatch(const GatherArgs& a, dim3 grid, dim3 block, cudaStream_t st)
{
    if (a.sino_bf && a.img_bf) k_gather_fan<MODE, true, true><<<grid, block, 0, st>>>(a);
    else if (a.sino_bf) k_gather_fan<MODE, true, false><<<grid, block, 0, st>>>(a);
    else if (a.img_bf) k_gather_fan<MODE, false, true><<<grid, block, 0, st>>>(a);
    else k_gather_fan<MODE, false, false><<<grid, block, 0, st>>>(a);
}

template <int MODE>
void gather_fan_lines_dispatch(const GatherArgs& a, dim3 grid, dim3 block, cudaStream_t st)
{
    if (a.sino_bf && a.img_bf) k_gather_fan_lines<MODE, true, true><<<grid, block, 0, st>>>(a);
    else if (a.sino_bf) k_gather_fan_lines<MODE, true, false><<<grid, block, 0, st>>>(a);
    else if (a.img_bf) k_gather_fan_lines<MODE, false, true><<<grid, block, 0, st>>>(a);
    else k_gather_fan_lines<MODE, false, false><<<grid, block, 0, st>>>(a);
}

cudaError_t launch_gather(int mode, const GatherArgs& a, cudaStream_t st)
{
    if (mode != GATHER_R && mode != GATHER_PDHG) return cudaErrorInvalidValue;
    if (a.parts < 1 || (a.parts > 1 && (!a.part || !a.counters))) return cudaErrorInvalidValue;
    if (a.rays && a.fan_lines) {
        if (!a.rayw || !a.views || (a.n_ang > 0 && !a.u)) return cudaErrorInvalidValue;
        const int b = (a.N + LT - 1) / LT;
        dim3 grid(b, b, a.parts), block(LT * LW);
        if (mode == GATHER_R) gather_fan_lines_dispatch<GATHER_R>(a, grid, block, st);
        else gather_fan_lines_dispatch<GATHER_PDHG>(a, grid, block, st);
        return cudaGetLastError();
    }
    if (a.rays) {
        if (!a.rayw || !a.views || (a.n_ang > 0 && !a.u)) return cudaErrorInvalidValue;
        if (a.N % 2 != 0) return cudaErrorInvalidValue;
        dim3 grid((a.N + 2 * FQX - 1) / (2 * FQX), (a.N + 2 * FQY - 1) / (2 * FQY), a.parts), block(FQX * FQY);
        if (mode == GATHER_R) gather_fan_dispatch<GATHER_R>(a, grid, block, st);
        else gather_fan_dispatch<GATHER_PDHG>(a, grid, block, st);
        return cudaGetLastError();
    }
    if (a.n_ang > 0 && (!a.u || !a.ap || !a.order || a.n_row < 0 || a.n_row > a.n_ang)) return cudaErrorInvalidValue;
    const int b = (a.N + GT - 1) / GT;
    dim3 grid(b, b, a.parts), block(GT * GW);
    if (mode == GATHER_R) gather_dispatch<GATHER_R>(a, grid, block, st);
    else gather_dispatch<GATHER_PDHG>(a, grid, block, st);
    return cudaGetLastError();
}

size_t fan_gather_tiles(int N)
{
    return (size_t)((N + 2 * FQX - 1) / (2 * FQX)) * (size_t)((N + 2 * FQY - 1) / (2 * FQY));
}

int fan_lines_parts(int N, int n_views)
{
    // about 2048 blocks of 4 warps; at most 64 slices
    const long long tiles = (long long)gather_tiles(N);
    long long p = (2048 + tiles - 1) / tiles;
    if (p > 64) p = 64;
    if (p > n_views) p = n_views;
    if (p < 1) p = 1;
    return (int)p;
}

int fan_gather_parts(int N, int n_views)
{
    // about 152 x 8 blocks of 128 threads (2048 pixels each); at most 64 slices
    const long long tiles = (long long)fan_gather_tiles(N);
    long long p = (1216 + tiles - 1) / tiles;
    if (p > 64) p = 64;
    if (p > n_views) p = n_views;
    if (p < 1) p = 1;
    return (int)p;
}

}  // namespace ncs
