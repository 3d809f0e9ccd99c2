// Internal declarations shared by the CUDA translation units of the NCS library.
// Not part of the public C ABI (include/ncs.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#include <vector>

namespace ncs {

// Storage precision of the iteration state (FP32 arithmetic either way):
// St<false> stores float, St<true> stores bfloat16 rounded to nearest.
template <bool BF>
struct St;

// 16 random bits for element i of a store made at iteration ctr (SplitMix64
// finaliser of a counter; Steele, Lea, Flood 2014).
__device__ __forceinline__ unsigned rand16(unsigned long long ctr, size_t i, unsigned salt)
{
    unsigned long long z = ctr * 0x9E3779B97F4A7C15ull + (unsigned long long)i * 0xD1B54A32D192ED03ull + salt;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return (unsigned)(z >> 48);
}

template <>
struct St<false> {
    static constexpr size_t bytes = 4;
    __device__ static void put_sr(void* p, size_t i, float v, unsigned) { static_cast<float*>(p)[i] = v; }
    __device__ static float ld(const void* p, size_t i) { return __ldg(static_cast<const float*>(p) + i); }
    __device__ static float get(const void* p, size_t i) { return static_cast<const float*>(p)[i]; }
    __device__ static void put(void* p, size_t i, float v) { static_cast<float*>(p)[i] = v; }
    __device__ static float2 ld2(const void* p, ptrdiff_t i) { return __ldg(static_cast<const float2*>(p) + i); }
    __device__ static void put2(void* p, size_t i, float a, float b)
    {
        static_cast<float2*>(p)[i] = make_float2(a, b);
    }
};

template <>
struct St<true> {
    static constexpr size_t bytes = 2;
    // Stochastic rounding: add 16 random bits below the bfloat16 mantissa and
    // truncate, so the stored value is unbiased (small increments to an
    // accumulator survive in expectation).  Inf / NaN are stored unchanged.
    __device__ static void put_sr(void* p, size_t i, float v, unsigned r16)
    {
        unsigned bits = __float_as_uint(v);
        if ((bits & 0x7F800000u) != 0x7F800000u) bits += r16;
        static_cast<unsigned short*>(p)[i] = (unsigned short)(bits >> 16);
    }
    __device__ static float ld(const void* p, size_t i)
    {
        return __bfloat162float(__ldg(static_cast<const __nv_bfloat16*>(p) + i));
    }
    __device__ static float get(const void* p, size_t i)
    {
        return __bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]);
    }
    __device__ static void put(void* p, size_t i, float v)
    {
        static_cast<__nv_bfloat16*>(p)[i] = __float2bfloat16_rn(v);
    }
    __device__ static float2 ld2(const void* p, ptrdiff_t i)
    {
        return __bfloat1622float2(__ldg(static_cast<const __nv_bfloat162*>(p) + i));
    }
    __device__ static void put2(void* p, size_t i, float a, float b)
    {
        static_cast<__nv_bfloat162*>(p)[i] = __floats2bfloat162_rn(a, b);
    }
};

// Per-angle Joseph coefficients of the parallel beam, FP64 on the host, rounded once to
// 32.32 fixed point.  A ray (a, t) crosses stepping line q (an image row, or a row of x^T for
// column-branch angles) at the fractional index f = A t + B q + C along the interpolation
// axis.  With Ai, Bi, Ci the integers nearest to A 2^32, B 2^32, C 2^32, the kernels evaluate
// F = Ai t + Bi q + Ci exactly in 64-bit integers, in any order, directly or by steps of Ai or
// Bi: the crossing's integer part is k0 = F >> 32 and its interpolation weight is the top 23
// bits of the low word, w = (low >> 9) 2^-23, exact in FP32 together with 1 - w (fix_weight).
// So the forward projector and the gather hold the same FP32 matrix, and consecutive rays
// (|A| >= 1) always cross a line at distinct k0.  Af, Bf, Cf are FP32 copies of A, B, C for
// range estimates only; W = 1/|cos| or 1/|sin| is the path length per step; invA ~ 1/A.
struct AngleParam {
    long long Ai, Bi, Ci;
    float Af, Bf, Cf, W, invA;
    int row;       // 1: stepped over rows of x; 0: over rows of x^T
};

// Index k0 and weight w of a 32.32 fixed-point crossing F (see AngleParam): k0 = floor(F / 2^32)
// and w = the fraction truncated to 23 bits, built as the float 1.m minus 1 (exact).
__host__ __device__ inline float fix_weight(long long F, int& k0)
{
    k0 = (int)(F >> 32);
#ifdef __CUDA_ARCH__
    // (low >> 9) + 0x3F800000 as one multiply-high-add (low * 2^23 / 2^32 is low >> 9; the sum
    // has no carries into the exponent), which runs on the FMA pipe instead of a shift and an or
    unsigned bits;
    asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(bits) : "r"((unsigned)(unsigned long long)F), "r"(0x800000u),
        "r"(0x3F800000u));
    return __uint_as_float(bits) - 1.0f;
#else
    const unsigned bits = 0x3F800000u | ((unsigned)(unsigned long long)F >> 9);
    float f;
    memcpy(&f, &bits, sizeof f);
    return f - 1.0f;
#endif
}

// Fan-beam rays (Sec. 4, fan beam geometry), one entry per ray r = a * n_det + t, FP64 on
// the host and rounded once.  Ray r crosses stepping line q (a row of x, or a row of x^T)
// at f = B q + C; B and C are split into a multiple of 2^-10 and a remainder, so that
// H = Bhi q + Chi is exact in FP32 (|H| < 2^14) and L = Blo q + Clo small, and every fan-beam
// kernel evaluates the crossing with the same split_weight.  FanRay = (Bhi, Blo, Chi, Clo);
// the path length W goes in a separate float array, +W for a ray stepped over rows of x,
// -W for one stepped over rows of x^T.  A ray that passes no pixel has B = 0, C = -8, W = 0.
// FanView = (Su, Sv, du, dv): the source position of the view and the unit direction of
// its central ray (towards the rotation centre), used by the gather to find the channels
// that reach a pixel.
using FanRay = float4;
using FanView = float4;

// Images read by the forward projector are stored as "pair images": entry i of
// row j holds (x[j][i], x[j][i+1]) as one float2, so one aligned 8-byte load
// serves both interpolation taps, and each row carries PAIR_PAD zero entries on
// either side (row pitch N + 2 PAIR_PAD), so the projector's steps need no
// bounds checks.  Entry i sits at offset i + PAIR_PAD, i in [-PAIR_PAD, N + PAIR_PAD).
constexpr int PAIR_PAD = 4;
inline __host__ __device__ int pair_pitch(int N) { return N + 2 * PAIR_PAD; }

// Entries of one strip plane of the strip-form K's scratch: n_ang * n_det rounded up to a
// multiple of 4, so that every plane starts on a 16-byte boundary.
inline __host__ __device__ size_t fwd_strip_plane(int n_ang, int n_det)
{
    return ((size_t)n_ang * (size_t)n_det + 3) & ~(size_t)3;
}

// Forward-projection epilogues.
enum FwdMode {
    FWD_PLAIN = 0,     // y = K x
    FWD_PROX_L2 = 1,   // u+ = (u + alpha (K x - b)) / (1 + alpha)
    FWD_PROX_KL = 2,   // u+ = S(u + alpha (K x + bg); alpha b)
    FWD_RESID_L2 = 3,  // partial sums of (K x - b)^2 (FP64)
    FWD_RESID_KL = 4,  // partial sums of mu - b + b log(b/mu), mu = K x + bg (FP64)
};

struct FwdArgs {
    const void* img2;    // pair image of x (row-branch angles)
    const void* imgT2;   // pair image of x^T (column-branch angles)
    const AngleParam* ap;
    int N, n_ang, n_det;
    void* y;             // PLAIN: output (float); PROX: dual u, updated in place
    const float* b;      // data (float32 in every precision)
    const float* bg;     // KL background or nullptr (float32)
    int pair_bf;         // pair images stored as bfloat16
    int sino_bf;         // the dual u (y in PROX modes) stored as bfloat16 (stochastic rounding)
    const unsigned long long* iter;  // device iteration counter (random bits of the rounding)
    float alpha, inv1pa;
    double* partials;    // RESID: one partial per block (gridDim.x * gridDim.y); PROX_L2 with kx:
                         // the same partials of the data term at the running K x+
    float* kx;           // PROX_L2 or nullptr: running K x, updated to (K xbar + K x) / 2 = K x+
    const FanRay* rays;  // fan beam: per-ray table (ap unused), or nullptr for the parallel beam
    const float* rayw;   // fan beam: signed path length per ray
    // parallel beam, strip form (k_fwd_strip): spart non-null selects it
    const int* order;    // angle indices, the n_row row-branch ones first (angle_order)
    int n_row;
    float* spart;        // scratch: n_strip planes of fwd_strip_plane(n_ang, n_det) partial sums
    const short2* wrange;  // per (angle, 32-bin chunk): lines touched by the chunk's rays (fwd_warp_ranges)
    int n_strip, strip_rows;  // strips of strip_rows image rows (fwd_strip_shape)
};

// Gather epilogues.
enum GatherMode {
    GATHER_R = 0,        // r = K^T u + dscale D^T v + kappa s
    GATHER_PDHG = 1,     // x+ = x - inv_gamma * r ; xbar = 2 x+ - x
};

struct GatherArgs {
    const void* u;       // sinogram (float, or bfloat16 if sino_bf)
    const AngleParam* ap;
    const int* order;    // parallel beam: angle indices, the n_row row-branch ones first (angle_order)
    int n_row;
    int N, n_ang, n_det;
    int parts;           // angle slices per tile (gridDim.z)
    float* part;         // scratch: parts * N * N partial sums (parts > 1)
    int* counters;       // scratch: one arrival counter per 32 x 32 tile, zero between launches
    const void* v;       // 2*N*N or nullptr (float, or bfloat16 if img_bf)
    float dscale;
    const void* s;       // N*N or nullptr (float, or bfloat16 if img_bf)
    float kappa;
    int sino_bf, img_bf;
    float* r;            // GATHER_R output
    float* x;            // GATHER_PDHG: primal, updated in place
    float* xbar;         // GATHER_PDHG: extrapolated primal
    float inv_gamma;
    unsigned long long* iter;  // if set, block (0,0,0) advances this device iteration counter
    const FanRay* rays;  // fan beam: per-ray table (ap unused), or nullptr for the parallel beam
    const float* rayw;   // fan beam: signed path length per ray
    const FanView* views;// fan beam: per-view source and central direction
    float inv_pitch;     // fan beam: 1 / (fan angle between adjacent channels)
    float t_off;         // fan beam: channel coordinate of fan angle 0, (n_det-1)/2 - offset / pitch
    int fan_lines;       // fan beam: 1 = ray-driven tile walk (k_gather_fan_lines), 0 = pixel quads (k_gather_fan)
};

// Transpose / finite-difference pass.
enum TdMode {
    TD_PROX = 0,         // v+ = Pi(v + beta D xbar), s+ = min(0, s + alpha kappa xbar), pair images
    TD_APPLY = 1,        // v = dscale D x, s = kappa x (if s), pair images
    TD_OBJ = 2,          // pair images of x (clamped at 0 if clamp), TV partial sums (FP64)
    TD_TRANSPOSE = 3,    // pair images only
};

struct TdArgs {
    const float* x;
    void* x2;            // pair image of x (or nullptr)
    void* xT2;           // pair image of x^T (or nullptr)
    void* v;             // 2*N*N
    void* s;             // N*N or nullptr
    int img_bf;          // v, s stored as bfloat16 (stochastic rounding)
    int pair_bf;         // pair images stored as bfloat16 (round to nearest)
    const unsigned long long* iter;  // device iteration counter (random bits of the rounding)
    int N;
    float beta;          // TD_PROX: beta; TD_APPLY: dscale
    float rad;           // TV ball / box radius lambda alpha / beta
    float ak;            // alpha * kappa (TD_PROX) or kappa (TD_APPLY)
    int iso;             // 1: isotropic TV
    int clamp;           // TD_OBJ: evaluate at max(x, 0)
    double* partials;
};

struct RadixPlan {
    int n;               // number of stages
    int r[12];           // radices (2, 3, 4 or 8)
};

// Host: the parallel-beam angle table (see AngleParam) for N x N images and n_det bins at
// spacing ds (>= 1) with centre offset, angles a pi / na or the given ones.  Returns false when
// an angle is not finite or the crossings leave the range of the 32.32 fixed point.
bool angle_table(int N, int na, int nd, double ds, double offset, const double* angles,
                 std::vector<AngleParam>& ap);

// Host: the angle indices with the row-branch angles first, each group in increasing order;
// *n_row gets the number of row-branch angles.
inline void angle_order(const std::vector<AngleParam>& ap, std::vector<int>& order, int* n_row)
{
    order.clear();
    for (int a = 0; a < (int)ap.size(); ++a)
        if (ap[a].row) order.push_back(a);
    *n_row = (int)order.size();
    for (int a = 0; a < (int)ap.size(); ++a)
        if (!ap[a].row) order.push_back(a);
}

// Host: the fan-beam ray tables of N x N images for n_views x n_det rays (see FanRay): FP64,
// rounded once.  geo (optional) receives (cos, sin, s) of every ray in FP64.  Returns false
// when a ray's coefficients leave the range in which H = Bhi q + Chi is exact.
bool fan_ray_tables(int N, int na, int nd, double R, double pitch, double offset, const double* views,
                    std::vector<FanRay>& rays, std::vector<float>& rayw, std::vector<FanView>& vws,
                    std::vector<double>* geo);

// ---- launchers (all asynchronous on `st`) ----
cudaError_t launch_fwd(int mode, const FwdArgs& a, cudaStream_t st);
int fwd_num_blocks(int n_det, int n_ang);
bool fwd_strip_shape(int N, int* rows, int* strips);
void fwd_warp_ranges(int N, int n_det, const std::vector<AngleParam>& ap, std::vector<short2>& out);
int fwd_num_partials(const FwdArgs& a);
cudaError_t fwd_prepare();
cudaError_t launch_gather(int mode, const GatherArgs& a, cudaStream_t st);
int gather_parts(int N, int n_ang);          // angle slices the gather uses for this size
size_t gather_tiles(int N);                  // 32 x 32 tiles of an N x N image
int fan_gather_parts(int N, int n_views);    // view slices of the fan-beam gather (pixel quads)
int fan_lines_parts(int N, int n_views);     // view slices of the fan-beam gather (ray-driven tiles)
size_t fan_gather_tiles(int N);              // blocks (arrival counters) of the fan-beam gather
cudaError_t launch_td(int mode, const TdArgs& a, cudaStream_t st);
int td_num_blocks(int N);

// once per plan (per device), before any launch below or graph capture: opt the FFT kernels in
// to more than 48 KB of dynamic shared memory when N needs it
cudaError_t fft_prepare(int N);
cudaError_t launch_rows_fwd(const float* r, float2* S, const float2* tw, const RadixPlan& rp, int N,
                            cudaStream_t st);
cudaError_t launch_cols_ratio(const float2* Sw, float2* Sv, double* num, double* den, const float2* tw,
                              const RadixPlan& rp, int N, cudaStream_t st);   // eq. (H-fan) probe terms
cudaError_t launch_cols_solve(float2* S, const float* invmu, const float2* tw, const RadixPlan& rp, int N,
                              cudaStream_t st);
// mode 0: x <- x - delta, xbar <- x_old - 2 delta ; mode 1: out <- delta
cudaError_t launch_rows_inv(const float2* S, const float2* tw, const RadixPlan& rp, int N, int mode,
                            float* x, float* xbar, float* out, cudaStream_t st);

// Stacks of nz N x N slices (the 3-D circulant solve): the row pass and the row inverse per
// slice (spectra (N/2 + 1) x N apart), column transforms forward or inverse per slice, and
// the direct transform along z of the stacked half spectra, plane = (N/2 + 1) N entries per
// slice apart (mode 0 forward; 1 forward, times table, inverse; 2 inverse; Nz <= 64).
cudaError_t launch_rows_fwd_stack(const float* r, float2* S, const float2* tw, const RadixPlan& rp, int N, int nz,
                                  cudaStream_t st);
cudaError_t launch_cols_fft_stack(float2* S, const float2* tw, const RadixPlan& rp, int N, int nz, int inverse,
                                  cudaStream_t st);
cudaError_t launch_z_dft(float2* S, const float* table, const float2* twz, int Nz, size_t plane, int mode,
                         cudaStream_t st);
cudaError_t launch_rows_inv_stack(const float2* S, const float2* tw, const RadixPlan& rp, int N, int nz, int mode,
                                  float* x, float* xbar, float* out, cudaStream_t st);

// FP64 reductions.  Partial sums go to `partials` (one per block), finalize
// sums them in a fixed order, so results are deterministic.
cudaError_t launch_dot_partials(const float* a, const float* b, size_t n, double* partials, int nblk,
                                cudaStream_t st);
// out[0] = c0 * sum(p0[0..n0)) + c1 * sum(p1[0..n1))   (p1 may be null)
cudaError_t launch_finalize(const double* p0, int n0, double c0, const double* p1, int n1, double c1,
                            double* out, cudaStream_t st);
// y = x * rsqrt(*nrm2)  (nrm2 on the device)
cudaError_t launch_scale_by_rsqrt(const float* x, float* y, size_t n, const double* nrm2, cudaStream_t st);
// a = alpha * a
cudaError_t launch_scale(float* a, size_t n, float alpha, cudaStream_t st);
// Ram-Lak filtered sinogram q = tau (h * b), one row per angle
cudaError_t launch_ramp(const float* b, float* q, int n_ang, int n_det, float tau, cudaStream_t st);
// SplitMix64 uniforms in [-1, 1)
cudaError_t launch_splitmix(float* x, size_t n, uint64_t seed, cudaStream_t st);
// y = a*x + y ; y = x
cudaError_t launch_axpy(float a, const float* x, float* y, size_t n, cudaStream_t st);
// ADMM comparator: z-update with the x-update's right-hand side, lambda-update, p = s + c p
cudaError_t launch_admm_z(const float* kx, const float* b, const float* lu, float* zu, float* yu, size_t m,
                          float inv1pia, const float* fdx, const float* lv, float* zv, float* yv, int N, float t,
                          int iso, cudaStream_t st);
cudaError_t launch_admm_lambda(float* lu, const float* zu, const float* kx, const float* b, size_t m, float* lv,
                               const float* zv, const float* fdx, size_t nv, cudaStream_t st);
cudaError_t launch_xpby(const float* s, float c, float* p, size_t n, cudaStream_t st);

}  // namespace ncs
