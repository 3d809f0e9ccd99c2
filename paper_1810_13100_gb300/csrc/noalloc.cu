// K^T without any device allocation: ncs_apply_KT_static (declared in include/ncs.h).
//
// Some callers cannot allocate device memory at the point where they need a
// backprojection: code running under a memory pool that owns the whole device,
// inside a framework whose allocator must not be bypassed, or in a process
// that has reserved all memory up front.  For them this entry point runs the
// same tiled gather kernel as ncs_apply_KT but takes its working memory (the
// per-angle coefficient table, the per-tile arrival counters and the partial
// sums of the angle slices) from one file-scope device array instead of a plan.
// It needs no plan and calls no allocating routine.
//
// Limits: image side N <= NCS_STATIC_MAX_N (512), n_angles <= NCS_STATIC_MAX_ANGLES
// (2048); larger sizes are rejected with NCS_ERR_UNSUPPORTED, and so is a det_spacing
// in (0, 1) (the gather needs rays at least a pixel apart) or a geometry outside the
// range of ncs_plan_create.  The array
// (about 4.1 MiB) lives on every GPU that loads the library until the process
// exits.  Every call shares it, so calls whose work overlaps on the GPU (two
// streams, or two host threads) race; serialise them.  The first call on a
// device looks up the array's device address (cudaGetSymbolAddress) with that
// device current.  Calls are not capturable into a CUDA graph (the angle table is
// copied from host memory the call owns); on a capturing stream they return
// NCS_ERR_UNSUPPORTED before touching the GPU.
#include "../../include/ncs.h"
#include "ncs_internal.cuh"

#include <mutex>
#include <vector>

using namespace ncs;

namespace {

constexpr int kTile = 32;
constexpr int kMaxTiles = (NCS_STATIC_MAX_N / kTile) * (NCS_STATIC_MAX_N / kTile);
constexpr int kMaxParts = 4;
constexpr size_t kParamBytes = sizeof(AngleParam) * NCS_STATIC_MAX_ANGLES;
constexpr size_t kOrderBytes = sizeof(int) * NCS_STATIC_MAX_ANGLES;
constexpr size_t kCounterBytes = sizeof(int) * kMaxTiles;
constexpr size_t kPartBytes = sizeof(float) * kMaxParts * NCS_STATIC_MAX_N * NCS_STATIC_MAX_N;
constexpr size_t kScratchBytes = kParamBytes + kOrderBytes + kCounterBytes + kPartBytes;
static_assert(kParamBytes % 256 == 0 && kOrderBytes % 256 == 0 && kCounterBytes % 256 == 0,
              "scratch regions stay 256-byte aligned");

// The working memory of ncs_apply_KT_static: [angle table | angle order | counters | partials].
static __device__ __align__(256) unsigned char g_kt_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {nullptr};

// Device address of g_kt_scratch for the current device (looked up once per device).
int scratch_address(unsigned char** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return NCS_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return NCS_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_kt_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return NCS_ERR_CUDA;
        }
        g_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_addr[dev];
    return NCS_OK;
}

}  // namespace

extern "C" int ncs_apply_KT_static(const ncs_geometry* geom, int N, const float* y, float* x, void* cuda_stream)
{
    if (!geom || !y || !x || geom->n_angles < 1 || geom->n_det < 1 || N < 8) return NCS_ERR_BADARG;
    if (N > NCS_STATIC_MAX_N || geom->n_angles > NCS_STATIC_MAX_ANGLES) return NCS_ERR_UNSUPPORTED;
    if (geom->det_spacing != 0.0 && !(geom->det_spacing >= 1.0)) return NCS_ERR_UNSUPPORTED;
    // per-angle Joseph coefficients, the same FP64 construction as a plan's
    std::vector<AngleParam> ap;
    const double ds = geom->det_spacing > 0.0 ? geom->det_spacing : 1.0;
    if (!angle_table(N, geom->n_angles, geom->n_det, ds, geom->det_offset, geom->angles, ap))
        return NCS_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the angle table is copied from host memory owned by this call: no graph capture
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return NCS_ERR_UNSUPPORTED;
    }
    if (cs != cudaStreamCaptureStatusNone) return NCS_ERR_UNSUPPORTED;
    unsigned char* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != NCS_OK) return rc;
    AngleParam* d_ap = reinterpret_cast<AngleParam*>(base);
    int* d_order = reinterpret_cast<int*>(base + kParamBytes);
    int* d_count = reinterpret_cast<int*>(base + kParamBytes + kOrderBytes);
    float* d_part = reinterpret_cast<float*>(base + kParamBytes + kOrderBytes + kCounterBytes);
    const int tiles = (int)gather_tiles(N);
    std::vector<int> order;
    int n_row = 0;
    angle_order(ap, order, &n_row);
    // the angle table and order, and arrival counters that must start at zero
    if (cudaMemcpyAsync(d_ap, ap.data(), ap.size() * sizeof(AngleParam), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(d_count, 0, (size_t)tiles * sizeof(int), st) != cudaSuccess) {
        cudaGetLastError();
        return NCS_ERR_CUDA;
    }
    GatherArgs g{};
    g.u = y;
    g.ap = d_ap;
    g.order = d_order;
    g.n_row = n_row;
    g.N = N;
    g.n_ang = geom->n_angles;
    g.n_det = geom->n_det;
    int parts = gather_parts(N, geom->n_angles);
    if (parts > kMaxParts) parts = kMaxParts;
    g.parts = parts;
    g.part = d_part;
    g.counters = d_count;
    g.r = x;
    if (launch_gather(GATHER_R, g, st) != cudaSuccess) {
        cudaGetLastError();
        return NCS_ERR_CUDA;
    }
    return NCS_OK;
}
