// Real 2-D FFT solve with the circulant M (Sec. 2: C^+ = F^{-1} diag(h)^+ F) on
// sm_103a, written as three passes over an N x N image:
//
//   rows_fwd   : each block transforms a pair of image rows at once, packed as
//                the real and imaginary parts of one complex sequence, and
//                unpacks the two half spectra (k = 0..N/2); the result is
//                stored transposed, S[k][p], so the column pass reads rows.
//   cols_solve : each block loads one spectrum column S[k][.], transforms it,
//                multiplies by 1/(N^2 mu), transforms back, and stores it.
//   rows_inv   : each block rebuilds the full spectra of two rows from their
//                Hermitian halves, inverts them as one complex sequence and
//                applies the primal update x+ = x - delta, xbar = 2x+ - x (NCS,
//                eq. (NCS)) or writes delta.
//
// Every 1-D transform is a Stockham autosort FFT in shared memory (ping-pong
// buffers, radices 8/4/3/2 in registers, twiddles from a table computed in FP64
// on the host).  The inverse is taken as conj(FFT(conj(.))); the 1/N^2 of the
// inverse is folded into the 1/mu table.
#include "ncs_internal.cuh"

namespace ncs {

namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 conj2(float2 a) { return make_float2(a.x, -a.y); }
// multiply by -i
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }

constexpr float kS2 = 0.70710678118654752440f;   // sqrt(2)/2
constexpr float kS3 = 0.86602540378443864676f;   // sqrt(3)/2

// Forward DFTs of length R in registers, X_k = sum_q v_q exp(-2 pi i q k / R).
__device__ __forceinline__ void dft2(float2* v)
{
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

__device__ __forceinline__ void dft4(float2& v0, float2& v1, float2& v2, float2& v3)
{
    float2 t0 = cadd(v0, v2), t1 = csub(v0, v2);
    float2 t2 = cadd(v1, v3), t3 = mul_mi(csub(v1, v3));
    v0 = cadd(t0, t2);
    v2 = csub(t0, t2);
    v1 = cadd(t1, t3);
    v3 = csub(t1, t3);
}

__device__ __forceinline__ void dft3(float2* v)
{
    float2 s = cadd(v[1], v[2]), d = csub(v[1], v[2]);
    float2 m = make_float2(fmaf(-0.5f, s.x, v[0].x), fmaf(-0.5f, s.y, v[0].y));
    float2 e = mul_mi(make_float2(kS3 * d.x, kS3 * d.y));   // -i sqrt(3)/2 d
    v[0] = cadd(v[0], s);
    v[1] = cadd(m, e);
    v[2] = csub(m, e);
}

__device__ __forceinline__ void dft8(float2* v)
{
    // even / odd radix-4 halves, then W8^k twiddles
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4(e0, e1, e2, e3);
    dft4(o0, o1, o2, o3);
    // W8^1 = s2 (1 - i), W8^2 = -i, W8^3 = s2 (-1 - i)
    float2 w1 = make_float2(kS2 * (o1.x + o1.y), kS2 * (o1.y - o1.x));
    float2 w2 = mul_mi(o2);
    float2 w3 = make_float2(kS2 * (o3.y - o3.x), -kS2 * (o3.x + o3.y));
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, w1);
    v[5] = csub(e1, w1);
    v[2] = cadd(e2, w2);
    v[6] = csub(e2, w2);
    v[3] = cadd(e3, w3);
    v[7] = csub(e3, w3);
}

template <int R>
__device__ __forceinline__ void dftR(float2* v)
{
    if (R == 2) dft2(v);
    else if (R == 3) dft3(v);
    else if (R == 4) dft4(v[0], v[1], v[2], v[3]);
    else dft8(v);
}

// One Stockham stage: src -> dst, Ns = product of the radices already applied.
template <int R>
__device__ __forceinline__ void stockham_stage(const float2* __restrict__ src, float2* __restrict__ dst,
                                               int L, int Ns, const float2* __restrict__ tw, int tid, int nthr)
{
    const int nb = L / R;
    const int tws = L / (Ns * R);   // twiddle stride in the length-L table
    for (int jj = tid; jj < nb; jj += nthr) {
        const int k = jj % Ns;
        float2 v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = src[jj + q * nb];
#pragma unroll
        for (int q = 1; q < R; ++q) v[q] = cmul(v[q], __ldg(tw + q * k * tws));
        dftR<R>(v);
        const int base = (jj / Ns) * Ns * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) dst[base + q * Ns] = v[q];
    }
}

// Forward FFT of length L held in a (ping-pong with b); returns the buffer
// holding the result.  All threads of the group [0, nthr) take part; the
// caller's block must call this with every thread (it syncs the block).
__device__ float2* fft_smem(float2* a, float2* b, int L, const RadixPlan& rp, const float2* tw,
                            int tid, int nthr)
{
    int Ns = 1;
    for (int s = 0; s < rp.n; ++s) {
        const int R = rp.r[s];
        if (R == 8) stockham_stage<8>(a, b, L, Ns, tw, tid, nthr);
        else if (R == 4) stockham_stage<4>(a, b, L, Ns, tw, tid, nthr);
        else if (R == 3) stockham_stage<3>(a, b, L, Ns, tw, tid, nthr);
        else stockham_stage<2>(a, b, L, Ns, tw, tid, nthr);
        __syncthreads();
        float2* t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

__global__ void k_rows_fwd(const float* __restrict__ r, float2* __restrict__ S, const float2* __restrict__ tw,
                           RadixPlan rp, int N)
{
    extern __shared__ float2 sm[];
    float2* a = sm;
    float2* b = sm + N;
    const int j = 2 * blockIdx.x;
    const int tid = threadIdx.x, nthr = blockDim.x;
    // slice blockIdx.y of a stack of N x N images (3-D solves); one slice in 2-D
    r += (size_t)blockIdx.y * N * N;
    S += (size_t)blockIdx.y * (N / 2 + 1) * N;
    const float* r0 = r + (size_t)j * N;
    const float* r1 = r0 + N;
    for (int i = tid; i < N; i += nthr) a[i] = make_float2(r0[i], r1[i]);
    __syncthreads();
    float2* Z = fft_smem(a, b, N, rp, tw, tid, nthr);
    // unpack: X_j[k] = (Z[k] + conj Z[N-k]) / 2, X_{j+1}[k] = (Z[k] - conj Z[N-k]) / (2i)
    for (int k = tid; k <= N / 2; k += nthr) {
        const float2 zk = Z[k];
        const float2 zn = conj2(Z[k == 0 ? 0 : N - k]);
        const float2 s = cadd(zk, zn), d = csub(zk, zn);
        const float4 out = make_float4(0.5f * s.x, 0.5f * s.y, 0.5f * d.y, -0.5f * d.x);
        *reinterpret_cast<float4*>(S + (size_t)k * N + j) = out;
    }
}

__global__ void k_cols_solve(float2* __restrict__ S, const float* __restrict__ invmu,
                             const float2* __restrict__ tw, RadixPlan rp, int N)
{
    extern __shared__ float2 sm[];
    float2* a = sm;
    float2* b = sm + N;
    const int k = blockIdx.x;
    const int tid = threadIdx.x, nthr = blockDim.x;
    float2* col = S + (size_t)k * N;
    const float* im = invmu + (size_t)k * N;
    for (int p = tid; p < N; p += nthr) a[p] = col[p];
    __syncthreads();
    float2* X = fft_smem(a, b, N, rp, tw, tid, nthr);
    float2* Y = (X == a) ? b : a;
    // multiply by 1/(N^2 mu) and conjugate for the inverse transform
    for (int p = tid; p < N; p += nthr) {
        const float s = im[p];
        const float2 v = X[p];
        Y[p] = make_float2(v.x * s, -v.y * s);
    }
    __syncthreads();
    float2* Z = fft_smem(Y, X, N, rp, tw, tid, nthr);
    for (int p = tid; p < N; p += nthr) col[p] = conj2(Z[p]);
}

// Eq. (H-fan), least-squares form: one probe's terms of the circulant-eigenvalue
// estimate h_p = sum_v Re(W_p conj(V_p)) / sum_v |V_p|^2.  Column k of the
// row-transformed probe v (Sv) and of w = E^T E v (Sw) are transformed along the
// column and num[k][p] += Re(W_p conj(V_p)), den[k][p] += |V_p|^2.  The row pass is
// k_rows_fwd; Sv is overwritten.
__global__ void k_cols_ratio(const float2* __restrict__ Sw, float2* __restrict__ Sv, double* __restrict__ num,
                             double* __restrict__ den, const float2* __restrict__ tw, RadixPlan rp, int N)
{
    extern __shared__ float2 sm[];
    float2* a = sm;
    float2* b = sm + N;
    const int k = blockIdx.x;
    const int tid = threadIdx.x, nthr = blockDim.x;
    float2* colv = Sv + (size_t)k * N;
    for (int q = tid; q < N; q += nthr) a[q] = colv[q];
    __syncthreads();
    float2* V = fft_smem(a, b, N, rp, tw, tid, nthr);
    for (int q = tid; q < N; q += nthr) colv[q] = V[q];
    __syncthreads();
    const float2* colw = Sw + (size_t)k * N;
    for (int q = tid; q < N; q += nthr) a[q] = colw[q];
    __syncthreads();
    float2* W = fft_smem(a, b, N, rp, tw, tid, nthr);
    for (int q = tid; q < N; q += nthr) {
        const float2 v = colv[q], w = W[q];
        num[(size_t)k * N + q] += (double)w.x * v.x + (double)w.y * v.y;
        den[(size_t)k * N + q] += (double)v.x * v.x + (double)v.y * v.y;
    }
}

__global__ void k_rows_inv(const float2* __restrict__ S, const float2* __restrict__ tw, RadixPlan rp, int N,
                           int mode, float* __restrict__ x, float* __restrict__ xbar, float* __restrict__ out)
{
    extern __shared__ float2 sm[];
    float2* a = sm;
    float2* b = sm + N;
    const int j = 2 * blockIdx.x;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int H = N / 2;
    {   // slice blockIdx.y of a stack (3-D solves)
        const size_t z = blockIdx.y;
        S += z * (H + 1) * N;
        if (x) x += z * N * N;
        if (xbar) xbar += z * N * N;
        if (out) out += z * N * N;
    }
    // full spectra of rows j, j+1 from their halves; Z = X_j + i X_{j+1}, conjugated
    for (int k = tid; k < N; k += nthr) {
        const int kk = (k <= H) ? k : N - k;
        float4 q = *reinterpret_cast<const float4*>(S + (size_t)kk * N + j);
        float2 A = make_float2(q.x, q.y), B = make_float2(q.z, q.w);
        if (k == 0 || k == H) {
            A.y = 0.0f;
            B.y = 0.0f;
        } else if (k > H) {
            A = conj2(A);
            B = conj2(B);
        }
        const float2 z = make_float2(A.x - B.y, A.y + B.x);
        a[k] = conj2(z);
    }
    __syncthreads();
    float2* Z = fft_smem(a, b, N, rp, tw, tid, nthr);
    // conj(Z) = delta_j + i delta_{j+1}
    float* x0 = x ? x + (size_t)j * N : nullptr;
    for (int i = tid; i < N; i += nthr) {
        const float d0 = Z[i].x, d1 = -Z[i].y;
        if (mode == 0) {
            const float xa = x0[i], xb = x0[N + i];
            const float xa1 = xa - d0, xb1 = xb - d1;
            x0[i] = xa1;
            x0[N + i] = xb1;
            xbar[(size_t)j * N + i] = 2.0f * xa1 - xa;
            xbar[(size_t)j * N + N + i] = 2.0f * xb1 - xb;
        } else {
            out[(size_t)j * N + i] = d0;
            out[(size_t)j * N + N + i] = d1;
        }
    }
}

// One column transform of the half spectrum per block (slice blockIdx.y): forward, or the
// unnormalised inverse conj(FFT(conj(.))), in place.
__global__ void k_cols_fft(float2* __restrict__ S, const float2* __restrict__ tw, RadixPlan rp, int N, int inverse)
{
    extern __shared__ float2 sm[];
    float2* a = sm;
    float2* b = sm + N;
    const int k = blockIdx.x;
    const int tid = threadIdx.x, nthr = blockDim.x;
    float2* col = S + (size_t)blockIdx.y * (N / 2 + 1) * N + (size_t)k * N;
    for (int p = tid; p < N; p += nthr) a[p] = inverse ? conj2(col[p]) : col[p];
    __syncthreads();
    float2* X = fft_smem(a, b, N, rp, tw, tid, nthr);
    for (int p = tid; p < N; p += nthr) col[p] = inverse ? conj2(X[p]) : X[p];
}

constexpr int ZB = 32;    // z columns per block of k_z_dft

// The transform along z of a stack of Nz half spectra (entry (z, e) at S[z * plane + e]), one
// thread per e, as a direct DFT with twiddles twz[m] = exp(-2 pi i m / Nz) (FP64 on the
// host, rounded once).  mode 0: forward; 1: forward, times table[l * plane + e], unnormalised
// inverse (the 3-D circulant solve or apply); 2: unnormalised inverse.  In place.
__global__ void __launch_bounds__(ZB) k_z_dft(float2* __restrict__ S, const float* __restrict__ table,
                                              const float2* __restrict__ twz, int Nz, size_t plane, int mode)
{
    extern __shared__ float2 sm[];
    const size_t e = (size_t)blockIdx.x * ZB + threadIdx.x;
    if (e >= plane) return;                      // no block-wide synchronisation below
    float2* a = sm + threadIdx.x;                // a[z * ZB]: this thread's column
    float2* c = sm + (size_t)Nz * ZB + threadIdx.x;
    for (int z = 0; z < Nz; ++z) a[z * ZB] = S[z * plane + e];
    if (mode != 2) {
        for (int l = 0; l < Nz; ++l) {
            float2 acc = make_float2(0.0f, 0.0f);
            int m = 0;
            for (int z = 0; z < Nz; ++z) {
                const float2 w = __ldg(twz + m);
                const float2 v = a[z * ZB];
                acc.x = fmaf(v.x, w.x, fmaf(-v.y, w.y, acc.x));
                acc.y = fmaf(v.x, w.y, fmaf(v.y, w.x, acc.y));
                m += l;
                if (m >= Nz) m -= Nz;
            }
            if (mode == 1) {
                const float t = __ldg(table + l * plane + e);
                acc.x *= t;
                acc.y *= t;
            }
            c[l * ZB] = acc;
        }
        if (mode == 0) {
            for (int l = 0; l < Nz; ++l) S[l * plane + e] = c[l * ZB];
            return;
        }
        for (int l = 0; l < Nz; ++l) a[l * ZB] = c[l * ZB];
    }
    // inverse: y[z] = sum_l X[l] exp(+2 pi i l z / Nz)
    for (int z = 0; z < Nz; ++z) {
        float2 acc = make_float2(0.0f, 0.0f);
        int m = 0;
        for (int l = 0; l < Nz; ++l) {
            const float2 w = __ldg(twz + m);
            const float2 v = a[l * ZB];
            acc.x = fmaf(v.x, w.x, fmaf(v.y, w.y, acc.x));
            acc.y = fmaf(v.y, w.x, fmaf(-v.x, w.y, acc.y));
            m += z;
            if (m >= Nz) m -= Nz;
        }
        S[z * plane + e] = acc;
    }
}

int fft_threads(int N)
{
    int t = N / 8;
    if (t < 32) t = 32;
    if (t > 256) t = 256;
    return t;
}

}  // namespace

cudaError_t fft_prepare(int N)
{
    // each FFT block stages two length-N complex sequences: above 48 KB (N > 3072) the
    // kernels must opt in to the larger dynamic shared memory of the current device
    // (the attribute belongs to the kernel, not to a plan: it is set to what the largest side,
    // 4096, needs, so that a smaller plan made later does not lower it below an earlier one's)
    if (2 * N * (int)sizeof(float2) <= 48 * 1024) return cudaSuccess;
    const int smem = 2 * 4096 * (int)sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_rows_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cols_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cols_ratio, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rows_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cols_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

cudaError_t launch_rows_fwd_stack(const float* r, float2* S, const float2* tw, const RadixPlan& rp, int N, int nz,
                                  cudaStream_t st)
{
    k_rows_fwd<<<dim3(N / 2, nz), fft_threads(N), 2 * N * sizeof(float2), st>>>(r, S, tw, rp, N);
    return cudaGetLastError();
}

cudaError_t launch_cols_fft_stack(float2* S, const float2* tw, const RadixPlan& rp, int N, int nz, int inverse,
                                  cudaStream_t st)
{
    k_cols_fft<<<dim3(N / 2 + 1, nz), fft_threads(N), 2 * N * sizeof(float2), st>>>(S, tw, rp, N, inverse);
    return cudaGetLastError();
}

cudaError_t launch_z_dft(float2* S, const float* table, const float2* twz, int Nz, size_t plane, int mode,
                         cudaStream_t st)
{
    if (Nz < 1 || Nz > 64 || mode < 0 || mode > 2 || (mode == 1 && !table)) return cudaErrorInvalidValue;
    const unsigned blocks = (unsigned)((plane + ZB - 1) / ZB);
    k_z_dft<<<blocks, ZB, 2 * (size_t)Nz * ZB * sizeof(float2), st>>>(S, table, twz, Nz, plane, mode);
    return cudaGetLastError();
}

cudaError_t launch_rows_inv_stack(const float2* S, const float2* tw, const RadixPlan& rp, int N, int nz, int mode,
                                  float* x, float* xbar, float* out, cudaStream_t st)
{
    k_rows_inv<<<dim3(N / 2, nz), fft_threads(N), 2 * N * sizeof(float2), st>>>(S, tw, rp, N, mode, x, xbar, out);
    return cudaGetLastError();
}

cudaError_t launch_rows_fwd(const float* r, float2* S, const float2* tw, const RadixPlan& rp, int N,
                            cudaStream_t st)
{
    k_rows_fwd<<<N / 2, fft_threads(N), 2 * N * sizeof(float2), st>>>(r, S, tw, rp, N);
    return cudaGetLastError();
}

cudaError_t launch_cols_solve(float2* S, const float* invmu, const float2* tw, const RadixPlan& rp, int N,
                              cudaStream_t st)
{
    k_cols_solve<<<N / 2 + 1, fft_threads(N), 2 * N * sizeof(float2), st>>>(S, invmu, tw, rp, N);
    return cudaGetLastError();
}

cudaError_t launch_cols_ratio(const float2* Sw, float2* Sv, double* num, double* den, const float2* tw,
                              const RadixPlan& rp, int N, cudaStream_t st)
{
    k_cols_ratio<<<N / 2 + 1, fft_threads(N), 2 * N * sizeof(float2), st>>>(Sw, Sv, num, den, tw, rp, N);
    return cudaGetLastError();
}

cudaError_t launch_rows_inv(const float2* S, const float2* tw, const RadixPlan& rp, int N, int mode, float* x,
                            float* xbar, float* out, cudaStream_t st)
{
    k_rows_inv<<<N / 2, fft_threads(N), 2 * N * sizeof(float2), st>>>(S, tw, rp, N, mode, x, xbar, out);
    return cudaGetLastError();
}

}  // namespace ncs
