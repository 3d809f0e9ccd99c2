// Host runtime and C ABI of the NCS library (declarations in include/ncs.h).
//
// A plan owns: per-angle Joseph coefficients (FP64 on the host, rounded once),
// the Stockham twiddle table and radix schedule, the eigenvalue table of M
// (eqs. (circ_R), (circ_D)) after the (A3) rescale, the iteration workspace
// (xbar, xbar^T, r, half spectrum), the solver state used by ncs_solve /
// pdhg_solve, and cached CUDA graphs of check_every iterations.
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

namespace {

constexpr int kMaxPartials = 16384;

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    int kind = -1;
    const void* key[4] = {nullptr, nullptr, nullptr, nullptr};
    int T = 0;
};

}  // namespace

namespace ncs {

// Fan-beam rays (Sec. 4, fan beam geometry; equiangular detector): view a puts the source at
// S_a = R (-sin beta_a, cos beta_a); channel t is the ray leaving S_a at the fan angle
// gamma_t = (t - (n_det-1)/2) pitch + offset, counted counter-clockwise from the central ray
// (S_a towards the centre).  It is the line u cos(theta) + v sin(theta) = s with theta =
// beta_a + gamma_t and s = R sin(gamma_t) (every quantity in FP64, rounded once), stepped over
// rows when |cos theta| >= |sin theta| with the parallel beam's crossing, interpolation and
// path length.
// Parallel beam (Sec. 2, eq. (radon-def)): ray t of angle theta is u cos + v sin = s_t with
// s_t = (t - (n_det-1)/2) ds + offset.  Stepped over rows (|cos| >= |sin|; ties, decided
// exactly on the integer angle index for the default angles, step over rows) it crosses row j
// at column f = (s_t - v_j sin)/cos + (N-1)/2; stepped over columns it crosses column i at row
// f = (N-1)/2 - (s_t - u_i cos)/sin.  Both are f = A t + B q + C, rounded once to 32.32 fixed point.
bool angle_table(int N, int na, int nd, double ds, double offset, const double* angles, std::vector<AngleParam>& ap)
{
    const double cN = 0.5 * (N - 1);
    const double s0 = -0.5 * (nd - 1) * ds + offset;
    const double two32 = 4294967296.0;
    ap.resize(na);
    for (int a = 0; a < na; ++a) {
        double th, c, sn;
        int row;
        if (angles) {
            th = angles[a];
            if (!std::isfinite(th)) return false;
            c = std::cos(th);
            sn = std::sin(th);
            row = std::fabs(c) >= std::fabs(sn) ? 1 : 0;
        } else {
            th = a * M_PI / na;
            c = std::cos(th);
            sn = std::sin(th);
            row = (4 * a <= na || 4 * a >= 3 * na) ? 1 : 0;   // exact test; ties step over rows
        }
        double A, B, C, W, invA;
        if (row) {
            A = ds / c;
            B = sn / c;
            C = (s0 - cN * sn) / c + cN;
            W = 1.0 / std::fabs(c);
            invA = c / ds;
        } else {
            A = -ds / sn;
            B = c / sn;
            C = cN - (s0 + cN * c) / sn;
            W = 1.0 / std::fabs(sn);
            invA = -sn / ds;
        }
        // every crossing evaluated (rays a tile's width beyond the detector included) stays
        // well inside the 32.32 range
        if (!(std::fabs(A) * (nd + 64.0) + std::fabs(B) * (N + 64.0) + std::fabs(C) < 1073741824.0)) return false;
        AngleParam& q = ap[a];
        q.Ai = std::llround(A * two32);
        q.Bi = std::llround(B * two32);
        q.Ci = std::llround(C * two32);
        q.Af = (float)A;
        q.Bf = (float)B;
        q.Cf = (float)C;
        q.W = (float)W;
        q.invA = (float)invA;
        q.row = row;
    }
    return true;
}

bool fan_ray_tables(int N, int na, int nd, double R, double pitch, double offset, const double* views_in,
                    std::vector<FanRay>& rays, std::vector<float>& rayw, std::vector<FanView>& views,
                    std::vector<double>* geo)
{
    const double cN = 0.5 * (N - 1), cd = 0.5 * (nd - 1);
    const double reach = cN * std::sqrt(2.0) + 2.0;   // farther from the centre a ray touches no pixel
    const size_t m = (size_t)na * nd;
    auto split_hi = [](double X) { return std::nearbyint(X * 1024.0) / 1024.0; };
    rays.resize(m);
    rayw.resize(m);
    views.resize(na);
    if (geo) geo->resize(3 * m);
    for (int a = 0; a < na; ++a) {
        const double be = views_in ? views_in[a] : 2.0 * M_PI * a / na;
        const double sb = std::sin(be), cb = std::cos(be);
        views[a] = make_float4((float)(-R * sb), (float)(R * cb), (float)sb, (float)(-cb));
        for (int t = 0; t < nd; ++t) {
            const double gam = (t - cd) * pitch + offset;
            const double th = be + gam;
            const double c = std::cos(th), sn = std::sin(th), s = R * std::sin(gam);
            const int row = std::fabs(c) >= std::fabs(sn) ? 1 : 0;
            double B, C, W;
            if (std::fabs(s) > reach) {
                B = 0.0;
                C = -8.0;
                W = 0.0;
            } else if (row) {
                B = sn / c;
                C = (s - cN * sn) / c + cN;
                W = 1.0 / std::fabs(c);
            } else {
                B = c / sn;
                C = cN - (s + cN * c) / sn;
                W = 1.0 / std::fabs(sn);
            }
            if (std::fabs(split_hi(B)) * (N - 1) + std::fabs(split_hi(C)) >= 16384.0) return false;
            const size_t r = (size_t)a * nd + t;
            rays[r] = make_float4((float)split_hi(B), (float)(B - split_hi(B)), (float)split_hi(C),
                                  (float)(C - split_hi(C)));
            rayw[r] = row ? (float)W : -(float)W;
            if (geo) {
                (*geo)[3 * r] = c;
                (*geo)[3 * r + 1] = sn;
                (*geo)[3 * r + 2] = s;
            }
        }
    }
    return true;
}

}  // namespace ncs

struct ncs_plan {
    int dev = 0;
    int N = 0, na = 0, nd = 0;
    double lam = 0, alpha = 0, beta = 0, gamma = 0, kappa = 0, c_r = 0, h_dc = 0;
    bool kl = false, iso = false, nonneg = false;
    bool bf = false;                 // duals u, v, s stored as bfloat16 (NCS_BF16_STORE, NCS_BF16_DUALS)
    bool bf_img = false;             // projector images of xbar stored as bfloat16 (NCS_BF16_STORE)
    unsigned long long* d_iter = nullptr;  // device iteration counter (stochastic rounding of bfloat16 duals)
    float* d_q = nullptr;            // filtered sinogram of ncs_fbp (allocated on first use)
    double ds = 1.0;                 // detector pitch
    ncs_options opt{};
    cudaStream_t st = nullptr;
    bool own_stream = false;
    std::vector<AngleParam> h_ap;
    AngleParam* d_ap = nullptr;
    int* d_order = nullptr;          // angle indices, row-branch ones first (the gather's work split)
    int n_row = 0;
    // fan beam (ncs_plan_create_fan): per-ray coefficients, signed path lengths, views
    bool fan = false;
    std::vector<FanRay> h_rays;
    std::vector<float> h_rayw;
    FanRay* d_rays = nullptr;
    float* d_rayw = nullptr;
    FanView* d_views = nullptr;
    float inv_pitch = 0.f, t_off = 0.f;
    bool fan_lines = true;           // fan-beam K^T: ray-driven tiles (true) or pixel quads (false)
    float2* d_tw = nullptr;
    RadixPlan rp{};
    std::vector<double> mu;          // eigenvalues of M, N x N, [p][q]
    float* d_invmu = nullptr;        // 1/(N^2 mu), [q][p], q = 0..N/2
    float* d_mu = nullptr;           // mu/N^2 (power iteration start only)
    float *d_xbar = nullptr, *d_r = nullptr, *d_tmp = nullptr;
    // pair images (see PAIR_PAD) of xbar / xbar^T and of a scratch image / its transpose
    float2 *d_xb2 = nullptr, *d_xbT2 = nullptr, *d_tmp2 = nullptr, *d_tmpT2 = nullptr;
    float2* d_spec = nullptr;
    double *d_part0 = nullptr, *d_part1 = nullptr, *d_scal = nullptr, *h_pin = nullptr;
    float* d_kx = nullptr;        // running K x of a solve (L2 data)
    void* d_bfpair = nullptr;     // bfloat16 pair images of x and x^T for ncs_apply_K_bf16 (on first use)
    float* d_adm = nullptr;       // ADMM comparator workspace (allocated on first use)
    float *d_u = nullptr, *d_v = nullptr, *d_s = nullptr;   // solver state
    int gparts = 1;                  // angle slices of the gather
    float* d_gpart = nullptr;        // gather scratch: gparts * N * N partial sums
    float* d_spart = nullptr;        // strip form of K: n_strip planes of partial sums (nullptr: row walk)
    short2* d_wrange = nullptr;      // strip form of K: lines touched per (angle, 32-bin chunk)
    int n_strip = 0, strip_rows = 0;
    int* d_gcount = nullptr;         // gather scratch: arrival counter per 32 x 32 tile
    double rho = std::numeric_limits<double>::quiet_NaN();
    double lmax = std::numeric_limits<double>::quiet_NaN();
    float gamma_p = 0.0f;
    GraphCache graph;
    // per-kernel event timing (ncs_profile_enable / ncs_profile_read)
    unsigned prof = 0;            // bit k: kernel class k is timed
    bool capturing = false;
    struct Rec { int cls, n; cudaEvent_t a, b; };   // n: kernels launched between a and b
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> ev_pool;
    double nnz_K = -1.0;
};

struct ncs_batch {
    int dev = 0;
    std::vector<ncs_plan*> plans;
    cudaStream_t main = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    int lanes = 0;   // slices in flight at once (0 = all)
};

namespace {

#define CK(expr)                                                     \
    do {                                                             \
        cudaError_t e_ = (expr);                                     \
        if (e_ != cudaSuccess) {                                     \
            fprintf(stderr, "ncs: %s failed: %s (%s:%d)\n", #expr,   \
                    cudaGetErrorString(e_), __FILE__, __LINE__);     \
            return NCS_ERR_CUDA;                                     \
        }                                                            \
    } while (0)

#define CKS(expr)                         \
    do {                                  \
        int s_ = (expr);                  \
        if (s_ < 0) return s_;            \
    } while (0)

constexpr size_t kMaxProfRecords = 1u << 18;

cudaEvent_t prof_event(ncs_plan* p)
{
    if (!p->ev_pool.empty()) {
        cudaEvent_t e = p->ev_pool.back();
        p->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Brackets one kernel launch with CUDA events on the plan's stream while
// profiling is on (never inside graph capture).
struct ProfScope {
    ncs_plan* p;
    int cls, n;
    cudaEvent_t a = nullptr;
    ProfScope(ncs_plan* p_, int cls_, int n_ = 1) : p(p_), cls(cls_), n(n_)
    {
        if (((p->prof >> cls) & 1u) && !p->capturing && p->recs.size() < kMaxProfRecords) {
            a = prof_event(p);
            if (a) cudaEventRecord(a, p->st);
        }
    }
    ~ProfScope()
    {
        if (!a) return;
        cudaEvent_t b = prof_event(p);
        if (!b) { p->ev_pool.push_back(a); return; }
        cudaEventRecord(b, p->st);
        p->recs.push_back({cls, n, a, b});
    }
};

#define CKP(cls, expr)              \
    do {                            \
        ProfScope ps_(p, (cls));    \
        CK(expr);                   \
    } while (0)

// the same for a call that launches n kernels
#define CKPN(cls, n, expr)             \
    do {                               \
        ProfScope ps_(p, (cls), (n));  \
        CK(expr);                      \
    } while (0)

size_t NN(const ncs_plan* p) { return (size_t)p->N * p->N; }
size_t MM(const ncs_plan* p) { return (size_t)p->na * p->nd; }

bool factor_radices(int N, RadixPlan* rp)
{
    rp->n = 0;
    int n = N;
    while (n % 8 == 0 && n > 1) { rp->r[rp->n++] = 8; n /= 8; if (rp->n >= 12) return false; }
    while (n % 4 == 0 && n > 1) { rp->r[rp->n++] = 4; n /= 4; if (rp->n >= 12) return false; }
    while (n % 2 == 0 && n > 1) { rp->r[rp->n++] = 2; n /= 2; if (rp->n >= 12) return false; }
    while (n % 3 == 0 && n > 1) { rp->r[rp->n++] = 3; n /= 3; if (rp->n >= 12) return false; }
    return n == 1;
}

template <class T>
int dalloc(T** p, size_t count)
{
    if (count == 0) count = 1;
    if (cudaMalloc((void**)p, count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return NCS_ERR_NOMEM;
    }
    return NCS_OK;
}

// ---------------------------------------------------------------- enqueue helpers

size_t pair_elems(const ncs_plan* p) { return (size_t)p->N * pair_pitch(p->N); }

// allocate a pair image with its zero border
int alloc_pair(ncs_plan* p, float2** out)
{
    CKS(dalloc(out, pair_elems(p)));
    CK(cudaMemsetAsync(*out, 0, pair_elems(p) * sizeof(float2), p->st));
    return NCS_OK;
}

// pair images of x and x^T
int enq_pairs(ncs_plan* p, const float* x, float2* x2, float2* xT2)
{
    TdArgs a{};
    a.x = x;
    a.x2 = x2;
    a.xT2 = xT2;
    a.N = p->N;
    CKP(NCS_KERNEL_TD, launch_td(TD_TRANSPOSE, a, p->st));
    return NCS_OK;
}

// The projector tables and the strip scratch of a forward launch.
FwdArgs fwd_args(const ncs_plan* p)
{
    FwdArgs f{};
    f.ap = p->d_ap;
    f.rays = p->d_rays;
    f.rayw = p->d_rayw;
    f.N = p->N;
    f.n_ang = p->na;
    f.n_det = p->nd;
    f.order = p->d_order;
    f.n_row = p->n_row;
    f.spart = p->d_spart;
    f.wrange = p->d_wrange;
    f.n_strip = p->n_strip;
    f.strip_rows = p->strip_rows;
    return f;
}

// kernels one launch_fwd enqueues: the strip pass and the strip sum, or the row walk
int fwd_kernels(const FwdArgs& f) { return f.spart && !f.rays ? 2 : 1; }

int enq_K(ncs_plan* p, const float2* x2, const float2* xT2, float* y)
{
    FwdArgs f = fwd_args(p);
    f.img2 = x2;
    f.imgT2 = xT2;
    f.y = y;
    CKPN(NCS_KERNEL_FWD, fwd_kernels(f), launch_fwd(FWD_PLAIN, f, p->st));
    return NCS_OK;
}

int enq_gather(ncs_plan* p, int mode, const void* u, const void* v, float dscale, const void* s, float kappa,
               float* r, float* x, float* xbar, float inv_gamma, int n_ang, bool bf = false, bool advance = true)
{
    GatherArgs g{};
    g.u = u;
    g.ap = p->d_ap;
    g.order = p->d_order;
    g.n_row = n_ang > 0 ? p->n_row : 0;      // n_ang is p->na, or 0 for D^T / kappa s alone
    g.rays = p->d_rays;
    g.rayw = p->d_rayw;
    g.views = p->d_views;
    g.inv_pitch = p->inv_pitch;
    g.t_off = p->t_off;
    g.fan_lines = p->fan_lines ? 1 : 0;
    g.N = p->N;
    g.n_ang = n_ang;
    g.n_det = p->nd;
    g.parts = n_ang > 0 ? p->gparts : 1;
    g.part = p->d_gpart;
    g.counters = p->d_gcount;
    g.v = v;
    g.dscale = dscale;
    g.s = s;
    g.kappa = kappa;
    g.r = r;
    g.x = x;
    g.xbar = xbar;
    g.inv_gamma = inv_gamma;
    g.sino_bf = bf ? 1 : 0;
    g.img_bf = bf ? 1 : 0;
    g.iter = (bf && advance) ? p->d_iter : nullptr;
    CKP(NCS_KERNEL_GATHER, launch_gather(mode, g, p->st));
    return NCS_OK;
}

// out = M^{-1} r (mode 1) or x <- x - M^{-1} r, xbar = 2 x+ - x (mode 0)
int enq_solve(ncs_plan* p, const float* r, const float* table, int mode, float* x, float* xbar, float* out)
{
    CKP(NCS_KERNEL_ROWS_FWD, launch_rows_fwd(r, p->d_spec, p->d_tw, p->rp, p->N, p->st));
    CKP(NCS_KERNEL_COLS_SOLVE, launch_cols_solve(p->d_spec, table, p->d_tw, p->rp, p->N, p->st));
    CKP(NCS_KERNEL_ROWS_INV, launch_rows_inv(p->d_spec, p->d_tw, p->rp, p->N, mode, x, xbar, out, p->st));
    return NCS_OK;
}

// v+, s+ prox and the pair images of xbar and xbar^T
int enq_td_prox(ncs_plan* p, void* v, void* s)
{
    TdArgs a{};
    a.x = p->d_xbar;
    a.x2 = p->d_xb2;
    a.xT2 = p->d_xbT2;
    a.v = v;
    a.s = p->nonneg ? s : nullptr;
    a.N = p->N;
    a.beta = (float)p->beta;
    a.rad = (float)(p->lam * p->alpha / p->beta);
    a.ak = (float)(p->alpha * p->kappa);
    a.iso = p->iso ? 1 : 0;
    a.img_bf = p->bf ? 1 : 0;
    a.pair_bf = p->bf_img ? 1 : 0;
    a.iter = p->d_iter;
    CKP(NCS_KERNEL_TD, launch_td(TD_PROX, a, p->st));
    return NCS_OK;
}

int enq_fwd_prox(ncs_plan* p, void* u, const float* b, const float* bg, float* kx = nullptr,
                 double* partials = nullptr)
{
    FwdArgs f = fwd_args(p);
    f.img2 = p->d_xb2;
    f.imgT2 = p->d_xbT2;
    f.y = u;
    f.b = b;
    f.bg = bg;
    f.alpha = (float)p->alpha;
    f.inv1pa = (float)(1.0 / (1.0 + p->alpha));
    f.pair_bf = p->bf_img ? 1 : 0;
    f.sino_bf = p->bf ? 1 : 0;
    f.iter = p->d_iter;
    f.kx = p->kl ? nullptr : kx;
    f.partials = f.kx ? partials : nullptr;
    CKPN(NCS_KERNEL_FWD, fwd_kernels(f), launch_fwd(p->kl ? FWD_PROX_KL : FWD_PROX_L2, f, p->st));
    return NCS_OK;
}

// One NCS iteration (eq. (NCS), Sec. 4.1 / 4.2).  kx (solves with L2 data): the running
// K x, advanced to K x+; partials: where the data term at K x+ goes (check iterations).
int enq_ncs_iter(ncs_plan* p, float* x, void* u, void* v, void* s, const float* b, const float* bg,
                 float* kx = nullptr, double* partials = nullptr)
{
    const void* sv = p->nonneg ? s : nullptr;
    // r = K^T u + (beta/alpha) D^T v + kappa s
    CKS(enq_gather(p, GATHER_R, u, v, (float)(p->beta / p->alpha), sv, (float)p->kappa, p->d_r, nullptr,
                   nullptr, 0.f, p->na, p->bf));
    // x+ = x - M^+ r ; xbar = 2 x+ - x
    CKS(enq_solve(p, p->d_r, p->d_invmu, 0, x, p->d_xbar, nullptr));
    // v+ = Pi(v + beta D xbar), s+ = min(0, s + alpha kappa xbar), xbar^T
    CKS(enq_td_prox(p, v, s));
    // u+ = prox_{alpha g1*}(u + alpha (K xbar - b))
    CKS(enq_fwd_prox(p, u, b, bg, kx, partials));
    return NCS_OK;
}

// One PDHG iteration (eq. (PDHG)); kx, partials as for NCS (xbar = 2 x+ - x here too).
int enq_pdhg_iter(ncs_plan* p, float* x, void* u, void* v, void* s, const float* b, const float* bg,
                  float* kx = nullptr, double* partials = nullptr)
{
    const void* sv = p->nonneg ? s : nullptr;
    CKS(enq_gather(p, GATHER_PDHG, u, v, (float)(p->beta / p->alpha), sv, (float)p->kappa, nullptr, x,
                   p->d_xbar, 1.0f / p->gamma_p, p->na, p->bf));
    CKS(enq_td_prox(p, v, s));
    CKS(enq_fwd_prox(p, u, b, bg, kx, partials));
    return NCS_OK;
}

// FP64 objective at x into d_scal[slot] (x, its pair images, b and bg in FP32 in every precision).
int enq_objective(ncs_plan* p, const float* x, const float* b, const float* bg, int slot)
{
    TdArgs a{};
    a.x = x;
    a.x2 = p->d_tmp2;
    a.xT2 = p->d_tmpT2;
    a.clamp = p->kl ? 1 : 0;
    a.N = p->N;
    a.iso = p->iso ? 1 : 0;
    a.partials = p->d_part0;
    CKP(NCS_KERNEL_TD, launch_td(TD_OBJ, a, p->st));
    FwdArgs f = fwd_args(p);
    f.img2 = p->d_tmp2;
    f.imgT2 = p->d_tmpT2;
    f.b = b;
    f.bg = bg;
    f.partials = p->d_part1;
    CKPN(NCS_KERNEL_FWD_RESID, fwd_kernels(f), launch_fwd(p->kl ? FWD_RESID_KL : FWD_RESID_L2, f, p->st));
    CKP(NCS_KERNEL_REDUCE, launch_finalize(p->d_part1, fwd_num_partials(f), p->kl ? 1.0 : 0.5, p->d_part0,
                       td_num_blocks(p->N), p->lam, p->d_scal + slot, p->st));
    return NCS_OK;
}

int enq_dot(ncs_plan* p, const float* a, const float* b, size_t n, int slot)
{
    CK(launch_dot_partials(a, b, n, p->d_part0, 1024, p->st));
    CK(launch_finalize(p->d_part0, 1024, 1.0, nullptr, 0, 0.0, p->d_scal + slot, p->st));
    return NCS_OK;
}

int read_scalars(ncs_plan* p, int count)
{
    CK(cudaMemcpyAsync(p->h_pin, p->d_scal, count * sizeof(double), cudaMemcpyDeviceToHost, p->st));
    CK(cudaStreamSynchronize(p->st));
    return NCS_OK;
}

// w = A^T A x (yk, vb, sb: scratch buffers provided by the caller)
int enq_AtA(ncs_plan* p, const float* x, float* yk, float* vb, float* sb, float* w)
{
    TdArgs a{};
    a.x = x;
    a.x2 = p->d_tmp2;
    a.xT2 = p->d_tmpT2;
    a.v = vb;
    a.s = p->nonneg ? sb : nullptr;
    a.N = p->N;
    a.beta = (float)(p->beta / p->alpha);
    a.ak = (float)p->kappa;
    CK(launch_td(TD_APPLY, a, p->st));
    CKS(enq_K(p, p->d_tmp2, p->d_tmpT2, yk));
    CKS(enq_gather(p, GATHER_R, yk, vb, (float)(p->beta / p->alpha), p->nonneg ? sb : nullptr, (float)p->kappa,
                   w, nullptr, nullptr, 0.f, p->na));
    return NCS_OK;
}

struct PowerBufs {
    float *x = nullptr, *w = nullptr, *y = nullptr, *u = nullptr, *v = nullptr, *s = nullptr;
    ~PowerBufs()
    {
        cudaFree(x); cudaFree(w); cudaFree(y); cudaFree(u); cudaFree(v); cudaFree(s);
    }
};

int alloc_power(ncs_plan* p, PowerBufs& B)
{
    CKS(dalloc(&B.x, NN(p)));
    CKS(dalloc(&B.w, NN(p)));
    CKS(dalloc(&B.y, NN(p)));
    CKS(dalloc(&B.u, MM(p)));
    CKS(dalloc(&B.v, 2 * NN(p)));
    CKS(dalloc(&B.s, NN(p)));
    return NCS_OK;
}

// rho = lambda_max(M^{-1} alpha A^T A): x <- M^{-1} alpha A^T A x normalised; Rayleigh
// quotient <x, alpha A^T A x> / <x, M x> (M inner product).  <x, M x> of the
// next iterate comes for free: M (y/|y|) = w/|y|.
int power_rho(ncs_plan* p, double* rho_out)
{
    PowerBufs B;
    CKS(alloc_power(p, B));
    const size_t n = NN(p);
    CK(launch_splitmix(B.x, n, p->opt.power_seed, p->st));
    CKS(enq_dot(p, B.x, B.x, n, 0));
    CK(launch_scale_by_rsqrt(B.x, B.x, n, p->d_scal + 0, p->st));
    // <x0, M x0> with one application of M
    CKS(enq_solve(p, B.x, p->d_mu, 1, nullptr, nullptr, B.y));
    CKS(enq_dot(p, B.x, B.y, n, 3));
    CKS(read_scalars(p, 4));
    double xMx = p->h_pin[3];
    double rho = 0.0, rho_old = std::numeric_limits<double>::quiet_NaN();
    for (int it = 1; it <= p->opt.power_max_iter; ++it) {
        CKS(enq_AtA(p, B.x, B.u, B.v, B.s, B.w));
        CK(launch_scale(B.w, n, (float)p->alpha, p->st));
        CKS(enq_dot(p, B.x, B.w, n, 0));
        CKS(enq_solve(p, B.w, p->d_invmu, 1, nullptr, nullptr, B.y));
        CKS(enq_dot(p, B.y, B.w, n, 1));
        CKS(enq_dot(p, B.y, B.y, n, 2));
        CK(launch_scale_by_rsqrt(B.y, B.x, n, p->d_scal + 2, p->st));
        CKS(read_scalars(p, 3));
        rho = p->h_pin[0] / xMx;
        xMx = p->h_pin[1] / p->h_pin[2];
        if (!std::isfinite(rho)) return NCS_ERR_DIVERGED;
        if (it > 1 && std::fabs(rho - rho_old) <= p->opt.power_tol * std::fabs(rho)) break;
        rho_old = rho;
    }
    *rho_out = rho;
    return NCS_OK;
}

// lambda_max(A^T A) with the Rayleigh quotient <x, A^T A x>/<x, x>.
int power_lmax(ncs_plan* p, double* out)
{
    PowerBufs B;
    CKS(alloc_power(p, B));
    const size_t n = NN(p);
    CK(launch_splitmix(B.x, n, p->opt.power_seed, p->st));
    CKS(enq_dot(p, B.x, B.x, n, 0));
    CK(launch_scale_by_rsqrt(B.x, B.x, n, p->d_scal + 0, p->st));
    double lm = 0.0, lm_old = 0.0;
    for (int it = 1; it <= p->opt.power_max_iter; ++it) {
        CKS(enq_AtA(p, B.x, B.u, B.v, B.s, B.w));
        CKS(enq_dot(p, B.x, B.w, n, 0));
        CKS(enq_dot(p, B.x, B.x, n, 1));
        CKS(enq_dot(p, B.w, B.w, n, 2));
        CK(launch_scale_by_rsqrt(B.w, B.x, n, p->d_scal + 2, p->st));
        CKS(read_scalars(p, 3));
        lm = p->h_pin[0] / p->h_pin[1];
        if (!std::isfinite(lm)) return NCS_ERR_DIVERGED;
        if (it > 1 && std::fabs(lm - lm_old) <= p->opt.power_tol * std::fabs(lm)) break;
        lm_old = lm;
    }
    *out = lm;
    return NCS_OK;
}

int upload_mu(ncs_plan* p)
{
    const int N = p->N, H = N / 2;
    std::vector<float> inv((size_t)(H + 1) * N), fwd((size_t)(H + 1) * N);
    const double s = 1.0 / ((double)N * N);
    for (int q = 0; q <= H; ++q)
        for (int pp = 0; pp < N; ++pp) {
            const double m = p->mu[(size_t)pp * N + q];
            inv[(size_t)q * N + pp] = (float)(s / m);
            fwd[(size_t)q * N + pp] = (float)(s * m);
        }
    CK(cudaMemcpyAsync(p->d_invmu, inv.data(), inv.size() * sizeof(float), cudaMemcpyHostToDevice, p->st));
    CK(cudaMemcpyAsync(p->d_mu, fwd.data(), fwd.size() * sizeof(float), cudaMemcpyHostToDevice, p->st));
    CK(cudaStreamSynchronize(p->st));
    return NCS_OK;
}

int ensure_state(ncs_plan* p)
{
    if (!p->d_u) CKS(dalloc(&p->d_u, MM(p)));
    if (!p->d_v) CKS(dalloc(&p->d_v, 2 * NN(p)));
    if (!p->d_s) CKS(dalloc(&p->d_s, NN(p)));
    if (!p->kl && !p->d_kx) CKS(dalloc(&p->d_kx, MM(p)));
    return NCS_OK;
}

int ensure_gamma_p(ncs_plan* p)
{
    if (!std::isfinite(p->lmax)) CKS(power_lmax(p, &p->lmax));
    const double m = p->opt.a3_margin >= 0 ? p->opt.a3_margin : 0.0;
    p->gamma_p = (float)(p->alpha * p->lmax * (1.0 + m));
    return NCS_OK;
}

void free_plan(ncs_plan* p)
{
    for (auto& r : p->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : p->ev_pool) cudaEventDestroy(e);
    p->recs.clear();
    p->ev_pool.clear();
    if (p->graph.exec) cudaGraphExecDestroy(p->graph.exec);
    cudaFree(p->d_ap); cudaFree(p->d_order); cudaFree(p->d_rays); cudaFree(p->d_rayw); cudaFree(p->d_views); cudaFree(p->d_tw); cudaFree(p->d_invmu); cudaFree(p->d_mu);
    cudaFree(p->d_xbar); cudaFree(p->d_r); cudaFree(p->d_tmp);
    cudaFree(p->d_xb2); cudaFree(p->d_xbT2); cudaFree(p->d_tmp2); cudaFree(p->d_tmpT2);
    cudaFree(p->d_spec); cudaFree(p->d_part0); cudaFree(p->d_part1); cudaFree(p->d_scal);
    cudaFree(p->d_u); cudaFree(p->d_v); cudaFree(p->d_s); cudaFree(p->d_kx); cudaFree(p->d_adm); cudaFree(p->d_bfpair);
    cudaFree(p->d_gpart); cudaFree(p->d_gcount); cudaFree(p->d_iter); cudaFree(p->d_q); cudaFree(p->d_spart); cudaFree(p->d_wrange);
    if (p->h_pin) cudaFreeHost(p->h_pin);
    if (p->own_stream && p->st) cudaStreamDestroy(p->st);
}

int autotune_plan(ncs_plan* p);

// Eq. (H-fan) on the GPU, least-squares form: h = sum_v Re((F K^T K v) conj(F v)) /
// sum_v |F v|^2 over P probe images v, into *h in the [k][p] half-spectrum layout of the
// solve's tables (0 where every F v vanishes).
int probe_h(ncs_plan* p, int P, std::vector<double>* h)
{
    const int N = p->N, H = N / 2;
    const size_t n = NN(p), half = (size_t)(H + 1) * N;
    float* v = p->d_tmp;
    float* w = p->d_r;
    float* y = nullptr;
    float2* sv = nullptr;
    double *num = nullptr, *den = nullptr;
    int rc = dalloc(&y, MM(p));
    if (rc == NCS_OK) rc = dalloc(&sv, half);
    if (rc == NCS_OK) rc = dalloc(&num, half);
    if (rc == NCS_OK) rc = dalloc(&den, half);
    if (rc == NCS_OK && (cudaMemsetAsync(num, 0, half * sizeof(double), p->st) != cudaSuccess ||
                         cudaMemsetAsync(den, 0, half * sizeof(double), p->st) != cudaSuccess))
        rc = NCS_ERR_CUDA;
    for (int q = 0; q < P && rc == NCS_OK; ++q) {
        if (launch_splitmix(v, n, p->opt.power_seed + 1 + (uint64_t)q, p->st) != cudaSuccess) rc = NCS_ERR_CUDA;
        if (rc == NCS_OK) rc = enq_pairs(p, v, p->d_tmp2, p->d_tmpT2);
        if (rc == NCS_OK) rc = enq_K(p, p->d_tmp2, p->d_tmpT2, y);
        if (rc == NCS_OK)
            rc = enq_gather(p, GATHER_R, y, nullptr, 0.f, nullptr, 0.f, w, nullptr, nullptr, 0.f, p->na, false);
        if (rc == NCS_OK && (launch_rows_fwd(w, p->d_spec, p->d_tw, p->rp, N, p->st) != cudaSuccess ||
                             launch_rows_fwd(v, sv, p->d_tw, p->rp, N, p->st) != cudaSuccess ||
                             launch_cols_ratio(p->d_spec, sv, num, den, p->d_tw, p->rp, N, p->st) != cudaSuccess))
            rc = NCS_ERR_CUDA;
    }
    if (rc == NCS_OK) {
        std::vector<double> d(half);
        h->assign(half, 0.0);
        if (cudaMemcpyAsync(h->data(), num, half * sizeof(double), cudaMemcpyDeviceToHost, p->st) != cudaSuccess ||
            cudaMemcpyAsync(d.data(), den, half * sizeof(double), cudaMemcpyDeviceToHost, p->st) != cudaSuccess ||
            cudaStreamSynchronize(p->st) != cudaSuccess)
            rc = NCS_ERR_CUDA;
        for (size_t i = 0; i < half; ++i) (*h)[i] = d[i] > 0.0 ? (*h)[i] / d[i] : 0.0;
    }
    cudaGetLastError();
    cudaFree(y);
    cudaFree(sv);
    cudaFree(num);
    cudaFree(den);
    return rc;
}

int open_stream(ncs_plan* p)
{
    CK(cudaGetDevice(&p->dev));
    if (p->opt.cuda_stream) {
        p->st = (cudaStream_t)p->opt.cuda_stream;
    } else {
        CK(cudaStreamCreateWithFlags(&p->st, cudaStreamNonBlocking));
        p->own_stream = true;
    }
    return NCS_OK;
}


// Fan-beam rays (Sec. 4, fan beam geometry; equiangular detector): view a puts the source at
// S_a = R (-sin beta_a, cos beta_a); channel t is the ray leaving S_a at the fan angle
// gamma_t = (t - (n_det-1)/2) pitch + offset, counted counter-clockwise from the central ray
// (S_a towards the centre).  It is the line u cos(theta) + v sin(theta) = s with theta =
// beta_a + gamma_t and s = R sin(gamma_t) (every quantity in FP64, rounded once), stepped over
// rows when |cos theta| >= |sin theta| with the parallel beam's crossing, interpolation and
// path length.
int build_fan_tables(ncs_plan* p, const ncs_fan_geometry* fg)
{
    const int N = p->N, na = p->na, nd = p->nd;
    const double cd = 0.5 * (nd - 1);
    const size_t m = (size_t)na * nd;
    std::vector<FanView> views;
    if (!fan_ray_tables(N, na, nd, fg->src_dist, fg->pitch, fg->offset, fg->views, p->h_rays, p->h_rayw, views,
                        nullptr))
        return NCS_ERR_UNSUPPORTED;
    p->fan = true;
    p->inv_pitch = (float)(1.0 / fg->pitch);
    p->t_off = (float)(cd - fg->offset / fg->pitch);
    CKS(dalloc(&p->d_rays, m));
    CKS(dalloc(&p->d_rayw, m));
    CKS(dalloc(&p->d_views, (size_t)na));
    CK(cudaMemcpyAsync(p->d_rays, p->h_rays.data(), m * sizeof(FanRay), cudaMemcpyHostToDevice, p->st));
    CK(cudaMemcpyAsync(p->d_rayw, p->h_rayw.data(), m * sizeof(float), cudaMemcpyHostToDevice, p->st));
    CK(cudaMemcpyAsync(p->d_views, views.data(), na * sizeof(FanView), cudaMemcpyHostToDevice, p->st));
    CK(cudaStreamSynchronize(p->st));
    return NCS_OK;
}

int build_common(ncs_plan* p);

int build_plan(ncs_plan* p, const ncs_geometry* geom)
{
    const int N = p->N, na = p->na, nd = p->nd;
    CKS(open_stream(p));
    // per-angle Joseph coefficients in FP64, rounded once
    const double ds = (geom->det_spacing > 0.0) ? geom->det_spacing : 1.0;
    p->ds = ds;
    if (!angle_table(N, na, nd, ds, geom->det_offset, geom->angles, p->h_ap)) return NCS_ERR_UNSUPPORTED;
    CKS(dalloc(&p->d_ap, na));
    CK(cudaMemcpyAsync(p->d_ap, p->h_ap.data(), na * sizeof(AngleParam), cudaMemcpyHostToDevice, p->st));
    std::vector<int> order;
    angle_order(p->h_ap, order, &p->n_row);
    CKS(dalloc(&p->d_order, na));
    CK(cudaMemcpyAsync(p->d_order, order.data(), na * sizeof(int), cudaMemcpyHostToDevice, p->st));
    CK(cudaStreamSynchronize(p->st));
    return build_common(p);
}

// Everything after the projector tables: FFT twiddles, workspace, the DC entry and the
// eigenvalues of M, the (A3) power iteration and rescale, the optional autotuner.
int build_common(ncs_plan* p)
{
    const int N = p->N, na = p->na, nd = p->nd;
    CK(fft_prepare(N));
    // twiddles exp(-2 pi i m / N) in FP64, rounded once
    std::vector<float2> tw(N);
    for (int m = 0; m < N; ++m) {
        const double ang = -2.0 * M_PI * (double)m / (double)N;
        tw[m] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    CKS(dalloc(&p->d_tw, N));
    CK(cudaMemcpyAsync(p->d_tw, tw.data(), N * sizeof(float2), cudaMemcpyHostToDevice, p->st));
    const size_t n = NN(p), H = N / 2;
    CKS(dalloc(&p->d_invmu, (H + 1) * N));
    CKS(dalloc(&p->d_mu, (H + 1) * N));
    CKS(dalloc(&p->d_xbar, n));
    CKS(dalloc(&p->d_r, n));
    CKS(dalloc(&p->d_tmp, n));
    CKS(alloc_pair(p, &p->d_xb2));
    CKS(alloc_pair(p, &p->d_xbT2));
    CKS(alloc_pair(p, &p->d_tmp2));
    CKS(alloc_pair(p, &p->d_tmpT2));
    CKS(dalloc(&p->d_spec, (H + 1) * N));
    p->gparts = !p->fan ? gather_parts(N, na) : p->fan_lines ? fan_lines_parts(N, na) : fan_gather_parts(N, na);
    const size_t counters = p->fan ? fan_gather_tiles(N) : gather_tiles(N);   // fan: enough for either kernel
    const size_t slices = p->fan ? (size_t)std::max(fan_lines_parts(N, na), fan_gather_parts(N, na)) : p->gparts;
    CKS(dalloc(&p->d_gpart, slices > 1 ? slices * n : 1));
    CKS(dalloc(&p->d_gcount, counters));
    // K in strips (k_fwd_strip) unless the options ask for the row walk or the image is too large
    if (!p->fan && p->opt.fwd_kernel != 1) {
        if (fwd_strip_shape(N, &p->strip_rows, &p->n_strip)) {
            CK(fwd_prepare());
            CKS(dalloc(&p->d_spart, (size_t)p->n_strip * fwd_strip_plane(na, nd)));
            std::vector<short2> wr;
            fwd_warp_ranges(N, nd, p->h_ap, wr);
            CKS(dalloc(&p->d_wrange, wr.size()));
            CK(cudaMemcpyAsync(p->d_wrange, wr.data(), wr.size() * sizeof(short2), cudaMemcpyHostToDevice, p->st));
            CK(cudaStreamSynchronize(p->st));
        } else if (p->opt.fwd_kernel == 2) {
            return NCS_ERR_UNSUPPORTED;
        }
    }
    CKS(dalloc(&p->d_iter, 1));
    CK(cudaMemsetAsync(p->d_iter, 0, sizeof(unsigned long long), p->st));
    CK(cudaMemsetAsync(p->d_gcount, 0, counters * sizeof(int), p->st));
    CKS(dalloc(&p->d_part0, kMaxPartials));
    CKS(dalloc(&p->d_part1, (size_t)std::max(fwd_num_blocks(nd, na), (int)((size_t)na * nd / 1024 + 1))));
    CKS(dalloc(&p->d_scal, 16));
    if (cudaMallocHost((void**)&p->h_pin, 16 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return NCS_ERR_NOMEM;
    }
    if (td_num_blocks(N) > kMaxPartials) return NCS_ERR_UNSUPPORTED;
    if (p->opt.pdhg_only) {
        // PDHG needs no M: no eigenvalues, probes or (A3) power iteration
        if (p->opt.autotune) CKS(autotune_plan(p));
        return NCS_OK;
    }
    // DC of H_R: ||K 1||^2 / ||1||^2 unless given
    if (std::isnan(p->h_dc)) {
        float* ones = p->d_tmp;
        std::vector<float> h1(n, 1.0f);
        CK(cudaMemcpyAsync(ones, h1.data(), n * sizeof(float), cudaMemcpyHostToDevice, p->st));
        float* y = nullptr;
        CKS(dalloc(&y, MM(p)));
        int rc = enq_pairs(p, ones, p->d_tmp2, p->d_tmpT2);
        if (rc == NCS_OK) rc = enq_K(p, p->d_tmp2, p->d_tmpT2, y);
        if (rc == NCS_OK) rc = enq_dot(p, y, y, MM(p), 0);
        if (rc == NCS_OK) rc = read_scalars(p, 1);
        cudaFree(y);
        if (rc != NCS_OK) return rc;
        p->h_dc = p->h_pin[0] / (double)n;
    }
    if (std::isnan(p->c_r)) p->c_r = (double)na * N / M_PI;
    // eq. (H-fan): the projector part estimated from probe images, in the [k][p] half layout
    std::vector<double> hprobe;
    if (p->opt.h_probes > 0) CKS(probe_h(p, p->opt.h_probes, &hprobe));
    // eigenvalues of M = gamma I + alpha C, C ~ A^T A (eqs. (circ_R) or (H-fan), (circ_D))
    p->mu.assign(n, 0.0);
    const double b2a = p->beta * p->beta / p->alpha;
    const double kap = p->nonneg ? p->alpha * p->kappa * p->kappa : 0.0;
    for (int pp = 0; pp < N; ++pp) {
        const double jp = std::min(pp, N - pp);
        const double sp = std::sin(M_PI * pp / N);
        for (int q = 0; q < N; ++q) {
            const double kq = std::min(q, N - q);
            const double sq = std::sin(M_PI * q / N);
            double hr;
            if (pp == 0 && q == 0) hr = p->h_dc;
            else if (!hprobe.empty()) {
                // a real operator's estimate is even: h(p, q) = h(-p, -q) for the half above N/2
                const int qq = q <= N / 2 ? q : N - q, pr = q <= N / 2 ? pp : (N - pp) % N;
                hr = std::max(0.0, hprobe[(size_t)qq * N + pr]);
            } else hr = p->c_r / std::sqrt(jp * jp + kq * kq);
            const double hd = 4.0 * (sp * sp + sq * sq);
            p->mu[(size_t)pp * N + q] = p->gamma + p->alpha * hr + b2a * hd + kap;
        }
    }
    for (double m : p->mu)
        if (!(m > 0.0)) return NCS_ERR_BADARG;
    CKS(upload_mu(p));
    // (A3): rho = lambda_max(M^{-1} alpha A^T A); rescale M to rho = 1/(1+margin)
    CKS(power_rho(p, &p->rho));
    if (p->opt.a3_margin >= 0.0) {
        const double f = p->rho * (1.0 + p->opt.a3_margin);
        for (double& m : p->mu) m *= f;
        CKS(upload_mu(p));
    }
    if (p->opt.autotune) CKS(autotune_plan(p));
    return NCS_OK;
}

int check_plan(const ncs_plan* p) { return p ? NCS_OK : NCS_ERR_BADARG; }

// Entry points that need M: refused for a plan created with pdhg_only.
int check_plan_m(const ncs_plan* p)
{
    if (!p) return NCS_ERR_BADARG;
    return p->opt.pdhg_only ? NCS_ERR_UNSUPPORTED : NCS_OK;
}

// Time `reps` launches of fn on the plan's stream (ms per launch, CUDA events).
template <class F>
int time_launches(ncs_plan* p, int reps, F fn, float* ms)
{
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    int rc = NCS_OK;
    for (int k = 0; k < 2 && rc == NCS_OK; ++k) rc = fn();      // warm-up
    cudaEventRecord(a, p->st);
    for (int k = 0; k < reps && rc == NCS_OK; ++k) rc = fn();
    cudaEventRecord(b, p->st);
    cudaEventSynchronize(b);
    float t = 0.f;
    cudaEventElapsedTime(&t, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *ms = t / reps;
    return rc;
}

// Fan beam: time the two K^T kernels (pixel quads, ray-driven tiles), each with its default
// view slices, on the plan's sizes, and keep the faster.
int autotune_fan_gather(ncs_plan* p)
{
    float* y = nullptr;
    float* xo = nullptr;
    CKS(dalloc(&y, MM(p)));
    int rc = dalloc(&xo, NN(p));
    if (rc == NCS_OK && cudaMemsetAsync(y, 0, MM(p) * sizeof(float), p->st) != cudaSuccess) rc = NCS_ERR_CUDA;
    float ms[2] = {1e30f, 1e30f};
    for (int k = 0; k < 2 && rc == NCS_OK; ++k) {
        p->fan_lines = k == 1;
        p->gparts = p->fan_lines ? fan_lines_parts(p->N, p->na) : fan_gather_parts(p->N, p->na);
        rc = time_launches(p, 5, [&]() {
            return enq_gather(p, GATHER_R, y, nullptr, 0.f, nullptr, 0.f, xo, nullptr, nullptr, 0.f, p->na);
        }, &ms[k]);
    }
    p->fan_lines = ms[1] <= ms[0];
    p->gparts = p->fan_lines ? fan_lines_parts(p->N, p->na) : fan_gather_parts(p->N, p->na);
    cudaFree(y);
    cudaFree(xo);
    return rc;
}

// Autotuner: the gather's number of angle slices (half, same, double the default)
// and the order of the FFT radices (distinct permutations), each timed on the plan's
// own sizes with CUDA events; the fastest is kept.
int autotune_plan(ncs_plan* p)
{
    if (p->fan) CKS(autotune_fan_gather(p));
    const int base = p->gparts;
    int cand[3] = {std::max(1, base / 2), base, std::min(std::min(64, p->na), base * 2)};
    if (p->fan) cand[0] = cand[2] = base;      // the fan gather's view slices are set with its kernel
    const int cmax = std::max(cand[2], base);
    if (cmax > 1) {
        float* bigger = nullptr;
        CKS(dalloc(&bigger, (size_t)cmax * NN(p)));
        cudaFree(p->d_gpart);
        p->d_gpart = bigger;
    }
    float *y = nullptr, *xo = nullptr, *xo2 = nullptr;
    CKS(dalloc(&y, MM(p)));
    int rc = dalloc(&xo, NN(p));
    if (rc == NCS_OK) rc = dalloc(&xo2, NN(p));
    if (rc == NCS_OK && cudaMemsetAsync(y, 0, MM(p) * sizeof(float), p->st) != cudaSuccess) rc = NCS_ERR_CUDA;
    if (rc == NCS_OK && cudaMemsetAsync(xo, 0, NN(p) * sizeof(float), p->st) != cudaSuccess) rc = NCS_ERR_CUDA;
    float best = 1e30f;
    int best_parts = base;
    for (int c = 0; c < 3 && rc == NCS_OK; ++c) {
        if (c > 0 && cand[c] == cand[c - 1]) continue;
        p->gparts = cand[c];
        float ms = 0.f;
        rc = time_launches(p, 5, [&]() {
            return enq_gather(p, GATHER_R, y, nullptr, 0.f, nullptr, 0.f, xo, nullptr, nullptr, 0.f, p->na);
        }, &ms);
        if (ms < best) { best = ms; best_parts = cand[c]; }
    }
    p->gparts = best_parts;
    if (p->opt.pdhg_only) {            // no M: the FFT solve is never run
        cudaFree(y);
        cudaFree(xo);
        cudaFree(xo2);
        return rc;
    }
    // FFT radix orders
    RadixPlan rp0 = p->rp, best_rp = p->rp;
    std::vector<int> r(rp0.r, rp0.r + rp0.n);
    std::sort(r.begin(), r.end());
    best = 1e30f;
    int tried = 0;
    do {
        if (rc != NCS_OK || tried >= 8) break;
        for (int k = 0; k < rp0.n; ++k) p->rp.r[k] = r[k];
        float ms = 0.f;
        rc = time_launches(p, 5, [&]() { return enq_solve(p, xo, p->d_invmu, 1, nullptr, nullptr, xo2); }, &ms);
        if (ms < best) { best = ms; best_rp = p->rp; }
        ++tried;
    } while (std::next_permutation(r.begin(), r.end()));
    p->rp = best_rp;
    cudaFree(y);
    cudaFree(xo);
    cudaFree(xo2);
    return rc;
}

// The TV term of the objective at x, added to the data-term partials already in d_part1
// (left by the forward pass of the last iteration), into d_scal[slot].
int enq_objective_tv(ncs_plan* p, const float* x, int slot)
{
    TdArgs a{};
    a.x = x;
    a.x2 = p->d_tmp2;
    a.xT2 = p->d_tmpT2;
    a.clamp = 0;
    a.N = p->N;
    a.iso = p->iso ? 1 : 0;
    a.partials = p->d_part0;
    CKP(NCS_KERNEL_TD, launch_td(TD_OBJ, a, p->st));
    CKP(NCS_KERNEL_REDUCE, launch_finalize(p->d_part1, fwd_num_partials(fwd_args(p)), 0.5, p->d_part0,
                       td_num_blocks(p->N), p->lam, p->d_scal + slot, p->st));
    return NCS_OK;
}

// n_it iterations of NCS (kind 0) or PDHG (kind 1) on the plan's solver state, then
// the FP64 objective at x copied to the plan's pinned host slot.
int enq_solve_block(ncs_plan* p, int kind, const float* b, const float* bg, float* x, int n_it)
{
    // L2 data: the last iteration's forward pass leaves K x+ and the data term's partials
    // (Sec. 4.1 objective without another projection); the TV term is summed here
    float* kx = p->kl ? nullptr : p->d_kx;
    for (int k = 0; k < n_it; ++k) {
        double* part = (kx && k == n_it - 1) ? p->d_part1 : nullptr;
        if (kind == 0) CKS(enq_ncs_iter(p, x, p->d_u, p->d_v, p->d_s, b, bg, kx, part));
        else CKS(enq_pdhg_iter(p, x, p->d_u, p->d_v, p->d_s, b, bg, kx, part));
    }
    if (kx) CKS(enq_objective_tv(p, x, 0));
    else CKS(enq_objective(p, x, b, bg, 0));
    CK(cudaMemcpyAsync(p->h_pin, p->d_scal, sizeof(double), cudaMemcpyDeviceToHost, p->st));
    return NCS_OK;
}

// Solver state zeroed for a new solve (and gamma_P for PDHG).
int prepare_solve(ncs_plan* p, int kind, const float* b, const float* x)
{
    CKS(ensure_state(p));
    if (kind == 1) CKS(ensure_gamma_p(p));
    if (p->opt.warm_dual && !p->kl) {
        // dual start consistent with x^0: u^0 = K x^0 - b, the gradient of 1/2||.||^2 at K x^0 - b
        CKS(enq_pairs(p, x, p->d_tmp2, p->d_tmpT2));
        CKS(enq_K(p, p->d_tmp2, p->d_tmpT2, p->d_u));
        CK(launch_axpy(-1.0f, b, p->d_u, MM(p), p->st));
    } else {
        CK(cudaMemsetAsync(p->d_u, 0, MM(p) * sizeof(float), p->st));
    }
    CK(cudaMemsetAsync(p->d_v, 0, 2 * NN(p) * sizeof(float), p->st));
    CK(cudaMemsetAsync(p->d_s, 0, NN(p) * sizeof(float), p->st));
    if (!p->kl) {
        // running K x of the solve, starting at K x^0
        CKS(enq_pairs(p, x, p->d_tmp2, p->d_tmpT2));
        CKS(enq_K(p, p->d_tmp2, p->d_tmpT2, p->d_kx));
    }
    return NCS_OK;
}

// Gap measure of a solve: (f - f*)/|f*|, or the relative change of f when f* is NaN.
double solve_gap(double f, double f_prev, double f_star)
{
    if (std::isfinite(f_star)) return (f - f_star) / std::fabs(f_star);
    return std::isfinite(f_prev) ? std::fabs(f - f_prev) / std::fabs(f) : std::numeric_limits<double>::quiet_NaN();
}

int solve_common(ncs_plan* p, int kind, const float* b, const float* bg, float* x, double tol, int max_iter,
                 double f_star, ncs_report* rep)
{
    if (!b || !x || max_iter < 1 || !(tol >= 0.0)) return NCS_ERR_BADARG;
    if (!p->kl && bg) return NCS_ERR_BADARG;
    CK(cudaSetDevice(p->dev));
    CKS(prepare_solve(p, kind, b, x));
    const int T = p->opt.check_every > 0 ? p->opt.check_every : 10;
    auto enq_block = [&](int n_it) -> int { return enq_solve_block(p, kind, b, bg, x, n_it); };
    // CUDA graph of T iterations + objective, cached per (kind, pointers)
    GraphCache& G = p->graph;
    const void* key[4] = {b, bg, x, nullptr};
    bool hit = G.exec && G.kind == kind && G.T == T && !memcmp(G.key, key, sizeof(key));
    if (!hit) {
        if (G.exec) { cudaGraphExecDestroy(G.exec); G.exec = nullptr; }
        cudaGraph_t graph;
        CK(cudaStreamBeginCapture(p->st, cudaStreamCaptureModeThreadLocal));
        p->capturing = true;
        int rc = enq_block(T);
        p->capturing = false;
        cudaError_t e = cudaStreamEndCapture(p->st, &graph);
        if (rc != NCS_OK) { if (e == cudaSuccess) cudaGraphDestroy(graph); return rc; }
        CK(e);
        e = cudaGraphInstantiate(&G.exec, graph, 0);
        cudaGraphDestroy(graph);
        CK(e);
        G.kind = kind;
        G.T = T;
        memcpy(G.key, key, sizeof(key));
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, p->st));
    int it = 0, status = NCS_NOT_CONVERGED;
    double f = std::numeric_limits<double>::quiet_NaN(), f_prev = f, gap = f;
    while (it < max_iter) {
        const int n_it = std::min(T, max_iter - it);
        if (n_it == T) CK(cudaGraphLaunch(G.exec, p->st));
        else CKS(enq_block(n_it));
        CK(cudaStreamSynchronize(p->st));
        it += n_it;
        f = p->h_pin[0];
        if (!std::isfinite(f)) { status = NCS_ERR_DIVERGED; break; }
        gap = solve_gap(f, f_prev, f_star);
        if (std::isfinite(gap) && gap <= tol) { status = NCS_OK; break; }
        f_prev = f;
    }
    CK(cudaEventRecord(e1, p->st));
    CK(cudaEventSynchronize(e1));
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
        rep->rho = kind == 0 ? p->rho : (double)p->gamma_p;
    }
    return status;
}

// ADMM comparator (Appendix, "Derivation from ADMM"; Ramani and Fessler's scheme, Sec. 1.3)
// for L2 data: z+ = prox_{(1/alpha) g}(A x - b - lambda), x+ from n_cg steps of conjugate
// gradients on A^T A x = A^T (z+ + b + lambda) preconditioned by the plan's circulant M and
// started from x, lambda+ = lambda + z+ - A x+ + b.  One outer step costs n_cg + 2 passes
// of A^T A-like work; the objective is checked every check_every outer steps.
int admm_common(ncs_plan* p, const float* b, float* x, double tol, int max_outer, int n_cg, double f_star,
                ncs_report* rep)
{
    if (!b || !x || max_outer < 1 || n_cg < 1 || !(tol >= 0.0)) return NCS_ERR_BADARG;
    if (p->kl || p->bf || p->bf_img || p->nonneg) return NCS_ERR_UNSUPPORTED;
    CK(cudaSetDevice(p->dev));
    const size_t n = NN(p), m = MM(p), nv = 2 * n;
    // workspace: lu zu yu kx yk (m each) | lv zv yv fdx vb (2n each) | rhs r s q w pd sb (n each)
    const size_t words = 5 * m + 5 * nv + 7 * n;
    if (!p->d_adm) CKS(dalloc(&p->d_adm, words));
    float* lu = p->d_adm;
    float* zu = lu + m;
    float* yu = zu + m;
    float* kx = yu + m;
    float* yk = kx + m;
    float* lv = yk + m;
    float* zv = lv + nv;
    float* yv = zv + nv;
    float* fdx = yv + nv;
    float* vb = fdx + nv;
    float* rhs = vb + nv;
    float* r = rhs + n;
    float* sv = r + n;
    float* q = sv + n;
    float* w = q + n;
    float* pd = w + n;
    float* sb = pd + n;
    const float f = (float)(p->beta / p->alpha);
    const float inv1pia = (float)(1.0 / (1.0 + 1.0 / p->alpha));
    const float thr = (float)(p->lam / p->beta);
    auto apply_A = [&](const float* xin) -> int {
        // fdx = f D x (and the pair images), kx = K x
        TdArgs a{};
        a.x = xin;
        a.x2 = p->d_tmp2;
        a.xT2 = p->d_tmpT2;
        a.v = fdx;
        a.N = p->N;
        a.beta = f;
        CK(launch_td(TD_APPLY, a, p->st));
        return enq_K(p, p->d_tmp2, p->d_tmpT2, kx);
    };
    CK(cudaMemsetAsync(lu, 0, m * sizeof(float), p->st));
    CK(cudaMemsetAsync(lv, 0, nv * sizeof(float), p->st));
    CKS(apply_A(x));
    const int T = p->opt.check_every > 0 ? p->opt.check_every : 10;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, p->st));
    int it = 0, status = NCS_NOT_CONVERGED, rc = NCS_OK;
    double fval = std::numeric_limits<double>::quiet_NaN(), f_prev = fval, gap = fval;
    while (it < max_outer && rc == NCS_OK) {
        // z+ and the x-update's right-hand side A^T (z+ + b + lambda)
        if (launch_admm_z(kx, b, lu, zu, yu, m, inv1pia, fdx, lv, zv, yv, p->N, thr, p->iso ? 1 : 0, p->st) !=
            cudaSuccess) { rc = NCS_ERR_CUDA; break; }
        if ((rc = enq_gather(p, GATHER_R, yu, yv, f, nullptr, 0.f, rhs, nullptr, nullptr, 0.f, p->na)) != NCS_OK) break;
        // PCG from x
        if ((rc = enq_AtA(p, x, yk, vb, sb, w)) != NCS_OK) break;
        if (cudaMemcpyAsync(r, rhs, n * sizeof(float), cudaMemcpyDeviceToDevice, p->st) != cudaSuccess ||
            launch_axpy(-1.0f, w, r, n, p->st) != cudaSuccess) { rc = NCS_ERR_CUDA; break; }
        if ((rc = enq_solve(p, r, p->d_invmu, 1, nullptr, nullptr, sv)) != NCS_OK) break;
        if (cudaMemcpyAsync(pd, sv, n * sizeof(float), cudaMemcpyDeviceToDevice, p->st) != cudaSuccess) {
            rc = NCS_ERR_CUDA;
            break;
        }
        if ((rc = enq_dot(p, r, sv, n, 0)) != NCS_OK || (rc = read_scalars(p, 1)) != NCS_OK) break;
        double rs = p->h_pin[0];
        for (int j = 0; j < n_cg && rs > 0.0 && rc == NCS_OK; ++j) {
            if ((rc = enq_AtA(p, pd, yk, vb, sb, q)) != NCS_OK) break;
            if ((rc = enq_dot(p, pd, q, n, 0)) != NCS_OK || (rc = read_scalars(p, 1)) != NCS_OK) break;
            const double pq = p->h_pin[0];
            if (!(pq > 0.0)) break;
            const float step = (float)(rs / pq);
            if (launch_axpy(step, pd, x, n, p->st) != cudaSuccess || launch_axpy(-step, q, r, n, p->st) != cudaSuccess) {
                rc = NCS_ERR_CUDA;
                break;
            }
            if ((rc = enq_solve(p, r, p->d_invmu, 1, nullptr, nullptr, sv)) != NCS_OK) break;
            if ((rc = enq_dot(p, r, sv, n, 0)) != NCS_OK || (rc = read_scalars(p, 1)) != NCS_OK) break;
            const double rs_new = p->h_pin[0];
            if (launch_xpby(sv, (float)(rs_new / rs), pd, n, p->st) != cudaSuccess) { rc = NCS_ERR_CUDA; break; }
            rs = rs_new;
        }
        if (rc != NCS_OK) break;
        // A x+ and lambda+
        if ((rc = apply_A(x)) != NCS_OK) break;
        if (launch_admm_lambda(lu, zu, kx, b, m, lv, zv, fdx, nv, p->st) != cudaSuccess) { rc = NCS_ERR_CUDA; break; }
        ++it;
        if (it % T == 0 || it == max_outer) {
            if ((rc = enq_objective(p, x, b, nullptr, 0)) != NCS_OK || (rc = read_scalars(p, 1)) != NCS_OK) break;
            fval = p->h_pin[0];
            if (!std::isfinite(fval)) { status = NCS_ERR_DIVERGED; break; }
            gap = solve_gap(fval, f_prev, f_star);
            if (std::isfinite(gap) && gap <= tol) { status = NCS_OK; break; }
            f_prev = fval;
        }
    }
    cudaEventRecord(e1, p->st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != NCS_OK) return rc;
    if (rep) {
        rep->iters = it;
        rep->status = status;
        rep->time_ms = ms;
        rep->f = fval;
        rep->gap = gap;
        rep->rho = (double)n_cg;
    }
    return status;
}

}  // namespace

// ======================================================================= C ABI

extern "C" void ncs_options_default(ncs_options* o);

namespace {

// Validate the sizes and options shared by every plan and fill a new plan's scalars.
int new_plan(int nx, int ny, int n_angles, int n_det, double lambda, double alpha, const ncs_options* opt,
             ncs_plan** out)
{
    if (nx != ny || nx < 8 || n_angles < 1 || n_det < 1) return NCS_ERR_BADARG;
    if (!(lambda >= 0.0) || !(alpha > 0.0)) return NCS_ERR_BADARG;
    ncs_options o;
    if (opt) o = *opt;
    else ncs_options_default(&o);
    if (o.prec != NCS_FP32 && o.prec != NCS_BF16_STORE && o.prec != NCS_BF16_DUALS) return NCS_ERR_BADARG;
    if (o.nonneg && o.data != NCS_DATA_KL) return NCS_ERR_BADARG;
    if (o.warm_dual && o.prec != NCS_FP32) return NCS_ERR_BADARG;
    if (o.power_max_iter < 1 || !(o.power_tol >= 0.0)) return NCS_ERR_BADARG;
    if (o.pdhg_only != 0 && o.pdhg_only != 1) return NCS_ERR_BADARG;
    RadixPlan rp;
    if (nx % 2 != 0 || nx > 4096 || !factor_radices(nx, &rp)) return NCS_ERR_UNSUPPORTED;
    ncs_plan* p = new (std::nothrow) ncs_plan();
    if (!p) return NCS_ERR_NOMEM;
    p->N = nx;
    p->na = n_angles;
    p->nd = n_det;
    p->lam = lambda;
    p->alpha = alpha;
    p->beta = std::isnan(o.beta) ? alpha : o.beta;
    p->gamma = o.gamma;
    p->kappa = o.kappa;
    p->c_r = o.c_r;
    p->h_dc = o.h_dc;
    p->kl = o.data == NCS_DATA_KL;
    p->iso = o.tv == NCS_TV_ISO;
    p->nonneg = o.nonneg != 0;
    p->bf = o.prec != NCS_FP32;
    p->bf_img = o.prec == NCS_BF16_STORE;
    p->opt = o;
    p->rp = rp;
    if (!(p->beta > 0.0) || !(p->gamma >= 0.0) || (p->nonneg && !(p->kappa > 0.0))) {
        delete p;
        return NCS_ERR_BADARG;
    }
    *out = p;
    return NCS_OK;
}

}  // namespace

extern "C" {

void ncs_options_default(ncs_options* o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    const double nan = std::numeric_limits<double>::quiet_NaN();
    o->beta = nan;
    o->gamma = 0.0;
    o->h_dc = nan;
    o->c_r = nan;
    o->kappa = 1.0;
    o->data = NCS_DATA_L2;
    o->tv = NCS_TV_ANISO;
    o->nonneg = 0;
    o->prec = NCS_FP32;
    o->a3_margin = 1e-2;
    o->power_max_iter = 500;
    o->power_tol = 1e-6;
    o->power_seed = 0;
    o->check_every = 10;
    o->cuda_stream = nullptr;
    o->autotune = 0;
    o->warm_dual = 0;
    o->h_probes = 0;
    o->fan_gather = 0;
    o->pdhg_only = 0;
    o->fwd_kernel = 0;
}

int ncs_plan_create(const ncs_geometry* geom, int nx, int ny, double lambda, double alpha, const ncs_options* opt,
                    ncs_plan** out)
{
    if (!out) return NCS_ERR_BADARG;
    *out = nullptr;
    if (!geom) return NCS_ERR_BADARG;
    ncs_plan* p = nullptr;
    CKS(new_plan(nx, ny, geom->n_angles, geom->n_det, lambda, alpha, opt, &p));
    int rc = NCS_OK;
    if (geom->det_spacing != 0.0 && !(geom->det_spacing >= 1.0)) rc = NCS_ERR_UNSUPPORTED;
    if (rc == NCS_OK && geom->angles)
        for (int a = 0; a < geom->n_angles; ++a)
            if (!std::isfinite(geom->angles[a])) rc = NCS_ERR_BADARG;
    if (rc != NCS_OK) {
        delete p;
        return rc;
    }
    rc = build_plan(p, geom);
    if (rc != NCS_OK) {
        free_plan(p);
        delete p;
        return rc;
    }
    *out = p;
    return NCS_OK;
}

int ncs_plan_create_fan(const ncs_fan_geometry* geom, int nx, int ny, double lambda, double alpha,
                        const ncs_options* opt, ncs_plan** out)
{
    if (!out) return NCS_ERR_BADARG;
    *out = nullptr;
    if (!geom || !(geom->pitch > 0.0) || !std::isfinite(geom->pitch) || !std::isfinite(geom->offset) ||
        !std::isfinite(geom->src_dist))
        return NCS_ERR_BADARG;
    // the source must lie outside the image's circumscribed circle with room to spare (the gather's
    // channel window assumes every pixel centre is at least 2 pixels from the source)
    if (nx >= 8 && !(geom->src_dist >= 0.5 * (nx - 1) * std::sqrt(2.0) + 3.0)) return NCS_ERR_BADARG;
    if (geom->views)
        for (int a = 0; a < geom->n_views; ++a)
            if (!std::isfinite(geom->views[a])) return NCS_ERR_BADARG;
    ncs_options o;
    if (opt) o = *opt;
    else ncs_options_default(&o);
    // the fan beam has no closed-form H_R; with fewer probes the estimate's noise leaves some
    // frequencies far too low (512x512 fan: rho(M^{-1} alpha A^T A) 47 with 32 probes, 8.7 with 128)
    if (o.h_probes == 0) o.h_probes = 128;
    if (o.fan_gather < 0 || o.fan_gather > 2) return NCS_ERR_BADARG;
    if (o.fwd_kernel < 0 || o.fwd_kernel > 2) return NCS_ERR_BADARG;
    ncs_plan* p = nullptr;
    CKS(new_plan(nx, ny, geom->n_views, geom->n_det, lambda, alpha, &o, &p));
    p->fan_lines = o.fan_gather != 1;
    int rc = open_stream(p);
    if (rc == NCS_OK) rc = build_fan_tables(p, geom);
    if (rc == NCS_OK) rc = build_common(p);
    if (rc != NCS_OK) {
        free_plan(p);
        delete p;
        return rc;
    }
    *out = p;
    return NCS_OK;
}

void ncs_plan_destroy(ncs_plan* p)
{
    if (!p) return;
    cudaSetDevice(p->dev);
    if (p->st) cudaStreamSynchronize(p->st);
    free_plan(p);
    delete p;
}

int ncs_step(ncs_plan* p, float* x, float* u, float* v, float* s, const float* b, const float* bg, int n_iter)
{
    CKS(check_plan_m(p));
    if (!x || !u || !v || !b || n_iter < 1) return NCS_ERR_BADARG;
    if (p->nonneg && !s) return NCS_ERR_BADARG;
    if (!p->kl && bg) return NCS_ERR_BADARG;
    CK(cudaSetDevice(p->dev));
    for (int k = 0; k < n_iter; ++k) CKS(enq_ncs_iter(p, x, u, v, s, b, bg));
    return NCS_OK;
}

int pdhg_step(ncs_plan* p, float* x, float* u, float* v, float* s, const float* b, const float* bg, int n_iter)
{
    CKS(check_plan(p));
    if (!x || !u || !v || !b || n_iter < 1) return NCS_ERR_BADARG;
    if (p->nonneg && !s) return NCS_ERR_BADARG;
    if (!p->kl && bg) return NCS_ERR_BADARG;
    CK(cudaSetDevice(p->dev));
    CKS(ensure_gamma_p(p));
    for (int k = 0; k < n_iter; ++k) CKS(enq_pdhg_iter(p, x, u, v, s, b, bg));
    return NCS_OK;
}

int ncs_solve(ncs_plan* p, const float* b, const float* bg, float* x, double tol, int max_iter, double f_star,
              ncs_report* rep)
{
    CKS(check_plan_m(p));
    return solve_common(p, 0, b, bg, x, tol, max_iter, f_star, rep);
}

int pdhg_solve(ncs_plan* p, const float* b, const float* bg, float* x, double tol, int max_iter, double f_star,
               ncs_report* rep)
{
    CKS(check_plan(p));
    return solve_common(p, 1, b, bg, x, tol, max_iter, f_star, rep);
}

int admm_solve(ncs_plan* p, const float* b, float* x, double tol, int max_outer, int n_cg, double f_star,
               ncs_report* rep)
{
    CKS(check_plan_m(p));
    return admm_common(p, b, x, tol, max_outer, n_cg, f_star, rep);
}

int ncs_power_bound(ncs_plan* p, double* lambda_max_AtA, double* rho_M)
{
    CKS(check_plan(p));
    CK(cudaSetDevice(p->dev));
    if (lambda_max_AtA) {
        if (!std::isfinite(p->lmax)) CKS(power_lmax(p, &p->lmax));
        *lambda_max_AtA = p->lmax;
    }
    if (rho_M) *rho_M = p->rho;
    return NCS_OK;
}

int ncs_apply_K(ncs_plan* p, const float* x, float* y)
{
    CKS(check_plan(p));
    if (!x || !y) return NCS_ERR_BADARG;
    CK(cudaSetDevice(p->dev));
    CKS(enq_pairs(p, x, p->d_tmp2, p->d_tmpT2));
    return enq_K(p, p->d_tmp2, p->d_tmpT2, y);
}

int ncs_apply_KT(ncs_plan* p, const float* y, float* x)
{
    CKS(check_plan(p));
    if (!x || !y) return NCS_ERR_BADARG;
    CK(cudaSetDevice(p->dev));
    return enq_gather(p, GATHER_R, y, nullptr, 0.f, nullptr, 0.f, x, nullptr, nullptr, 0.f, p->na);
}

int ncs_apply_K_bf16(ncs_plan* p, const float* x, float* y)
{
    CKS(check_plan(p));
    if (!x || !y) return NCS_ERR_BADARG;
    CK(cudaSetDevice(p->dev));
    const size_t half = pair_elems(p) * 2 * sizeof(__nv_bfloat16);      // one bfloat16 pair image
    if (!p->d_bfpair) {
        if (cudaMalloc(&p->d_bfpair, 2 * half) != cudaSuccess) {
            cudaGetLastError();
            return NCS_ERR_NOMEM;
        }
        CK(cudaMemsetAsync(p->d_bfpair, 0, 2 * half, p->st));         // the zero border
    }
    void* x2 = p->d_bfpair;
    void* xT2 = static_cast<char*>(p->d_bfpair) + half;
    TdArgs a{};
    a.x = x;
    a.x2 = x2;
    a.xT2 = xT2;
    a.N = p->N;
    a.pair_bf = 1;
    CKP(NCS_KERNEL_TD, launch_td(TD_TRANSPOSE, a, p->st));
    FwdArgs f = fwd_args(p);
    f.img2 = x2;
    f.imgT2 = xT2;
    f.pair_bf = 1;
    f.y = y;
    CKPN(NCS_KERNEL_FWD, fwd_kernels(f), launch_fwd(FWD_PLAIN, f, p->st));
    return NCS_OK;
}

int ncs_apply_KT_bf16(ncs_plan* p, const void* y, float* x)
{
    CKS(check_plan(p));
    if (!x || !y) return NCS_ERR_BADARG;
    CK(cudaSetDevice(p->dev));
    return enq_gather(p, GATHER_R, y, nullptr, 0.f, nullptr, 0.f, x, nullptr, nullptr, 0.f, p->na, true, false);
}

int ncs_apply_D(ncs_plan* p, const float* x, float* v)
{
    CKS(check_plan(p));
    if (!x || !v) return NCS_ERR_BADARG;
    CK(cudaSetDevice(p->dev));
    TdArgs a{};
    a.x = x;
    a.v = v;
    a.N = p->N;
    a.beta = 1.0f;
    CK(launch_td(TD_APPLY, a, p->st));
    return NCS_OK;
}

int ncs_apply_DT(ncs_plan* p, const float* v, float* x)
{
    CKS(check_plan(p));
    if (!x || !v) return NCS_ERR_BADARG;
    CK(cudaSetDevice(p->dev));
    // the gather with no angles is D^T v alone
    return enq_gather(p, GATHER_R, nullptr, v, 1.0f, nullptr, 0.f, x, nullptr, nullptr, 0.f, 0);
}

int ncs_fbp(ncs_plan* p, const float* b, float* x)
{
    CKS(check_plan(p));
    if (!b || !x) return NCS_ERR_BADARG;
    if (p->fan) return NCS_ERR_UNSUPPORTED;
    CK(cudaSetDevice(p->dev));
    if (!p->d_q) CKS(dalloc(&p->d_q, MM(p)));
    CK(launch_ramp(b, p->d_q, p->na, p->nd, (float)p->ds, p->st));
    CKS(enq_gather(p, GATHER_R, p->d_q, nullptr, 0.f, nullptr, 0.f, x, nullptr, nullptr, 0.f, p->na));
    CK(launch_scale(x, NN(p), (float)(M_PI / p->na), p->st));
    return NCS_OK;
}

int ncs_apply_Minv(ncs_plan* p, const float* r, float* out)
{
    CKS(check_plan_m(p));
    if (!r || !out) return NCS_ERR_BADARG;
    CK(cudaSetDevice(p->dev));
    return enq_solve(p, r, p->d_invmu, 1, nullptr, nullptr, out);
}

int ncs_objective(ncs_plan* p, const float* x, const float* b, const float* bg, double* f)
{
    CKS(check_plan(p));
    if (!x || !b || !f) return NCS_ERR_BADARG;
    if (!p->kl && bg) return NCS_ERR_BADARG;
    CK(cudaSetDevice(p->dev));
    CKS(enq_objective(p, x, b, bg, 0));
    CKS(read_scalars(p, 1));
    *f = p->h_pin[0];
    return NCS_OK;
}

int ncs_get_mu(ncs_plan* p, double* mu_host)
{
    CKS(check_plan_m(p));
    if (!mu_host) return NCS_ERR_BADARG;
    memcpy(mu_host, p->mu.data(), p->mu.size() * sizeof(double));
    return NCS_OK;
}

int ncs_plan_sizes(const ncs_plan* p, int* N, int* n_angles, int* n_det)
{
    CKS(check_plan(p));
    if (N) *N = p->N;
    if (n_angles) *n_angles = p->na;
    if (n_det) *n_det = p->nd;
    return NCS_OK;
}

int ncs_plan_info(const ncs_plan* p, int* gather_parts, int* fft_radices, int* n_radices)
{
    CKS(check_plan(p));
    if (gather_parts) *gather_parts = p->gparts;
    if (n_radices) *n_radices = p->rp.n;
    if (fft_radices)
        for (int k = 0; k < p->rp.n; ++k) fft_radices[k] = p->rp.r[k];
    return NCS_OK;
}

int ncs_plan_fwd_strips(const ncs_plan* p, int* n_strip, int* strip_rows)
{
    CKS(check_plan(p));
    if (n_strip) *n_strip = p->d_spart ? p->n_strip : 0;
    if (strip_rows) *strip_rows = p->d_spart ? p->strip_rows : 0;
    return NCS_OK;
}

int ncs_batch_create(ncs_plan* const* plans, int n_plans, ncs_batch** out)
{
    if (!out) return NCS_ERR_BADARG;
    *out = nullptr;
    if (!plans || n_plans < 1) return NCS_ERR_BADARG;
    for (int i = 0; i < n_plans; ++i) {
        if (!plans[i]) return NCS_ERR_BADARG;
        if (plans[i]->opt.pdhg_only) return NCS_ERR_UNSUPPORTED;
        if (plans[i]->dev != plans[0]->dev) return NCS_ERR_BADARG;
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return NCS_ERR_BADARG;
    }
    ncs_batch* B = new (std::nothrow) ncs_batch();
    if (!B) return NCS_ERR_NOMEM;
    B->dev = plans[0]->dev;
    B->plans.assign(plans, plans + n_plans);
    B->join.assign(n_plans, nullptr);
    bool ok = cudaSetDevice(B->dev) == cudaSuccess &&
              cudaStreamCreateWithFlags(&B->main, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; ok && i < n_plans; ++i)
        ok = cudaEventCreateWithFlags(&B->join[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        ncs_batch_destroy(B);
        return NCS_ERR_CUDA;
    }
    *out = B;
    return NCS_OK;
}

int ncs_batch_set_lanes(ncs_batch* B, int lanes)
{
    if (!B || lanes < 0) return NCS_ERR_BADARG;
    B->lanes = lanes;
    return NCS_OK;
}

int ncs_batch_tune_lanes(ncs_batch* B, const float* const* b, const float* const* bg, float* const* x, int iters,
                         int* lanes_out)
{
    if (!B || !b || !x || iters < 1) return NCS_ERR_BADARG;
    const int n = (int)B->plans.size();
    std::vector<int> cand = {0};
    for (int l = 1; l < n && l <= 16; l *= 2) cand.push_back(l);
    std::vector<ncs_report> rep(n);
    const double nan = std::numeric_limits<double>::quiet_NaN();
    std::vector<double> fs(n, nan);
    int best = 0;
    double best_ms = std::numeric_limits<double>::infinity();
    for (int l : cand) {
        B->lanes = l;
        // a first short solve builds and warms the graph; the second is timed
        int rc = ncs_batch_solve(B, b, bg, x, 0.0, iters, fs.data(), rep.data());
        if (rc == NCS_OK || rc == NCS_NOT_CONVERGED) rc = ncs_batch_solve(B, b, bg, x, 0.0, iters, fs.data(), rep.data());
        if (rc != NCS_OK && rc != NCS_NOT_CONVERGED) return rc;
        if (rep[0].time_ms < best_ms) { best_ms = rep[0].time_ms; best = l; }
    }
    B->lanes = best;
    if (lanes_out) *lanes_out = best;
    return NCS_OK;
}

void ncs_batch_destroy(ncs_batch* B)
{
    if (!B) return;
    cudaSetDevice(B->dev);
    if (B->main) cudaStreamSynchronize(B->main);
    for (auto e : B->join)
        if (e) cudaEventDestroy(e);
    if (B->fork) cudaEventDestroy(B->fork);
    if (B->main) cudaStreamDestroy(B->main);
    delete B;
}

int ncs_batch_solve(ncs_batch* B, const float* const* b, const float* const* bg, float* const* x, double tol,
                    int max_iter, const double* f_star, ncs_report* reports)
{
    if (!B || !b || !x || max_iter < 1 || !(tol >= 0.0)) return NCS_ERR_BADARG;
    const int n = (int)B->plans.size();
    for (int i = 0; i < n; ++i) {
        if (!b[i] || !x[i]) return NCS_ERR_BADARG;
        if (!B->plans[i]->kl && bg && bg[i]) return NCS_ERR_BADARG;
    }
    CK(cudaSetDevice(B->dev));
    const double nan = std::numeric_limits<double>::quiet_NaN();
    std::vector<int> status(n, NCS_NOT_CONVERGED), iters(n, 0), active;
    std::vector<double> f(n, nan), f_prev(n, nan), gap(n, nan);
    for (int i = 0; i < n; ++i) {
        ncs_plan* p = B->plans[i];
        CKS(prepare_solve(p, 0, b[i], x[i]));
        CK(cudaEventRecord(B->join[i], p->st));
        CK(cudaStreamWaitEvent(B->main, B->join[i], 0));
        active.push_back(i);
    }
    const int T = B->plans[0]->opt.check_every > 0 ? B->plans[0]->opt.check_every : 10;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, B->main));
    cudaGraphExec_t exec = nullptr;
    std::vector<int> graph_set;
    int graph_nit = 0, done = 0, rc = NCS_OK;
    while (!active.empty() && rc == NCS_OK) {
        const int n_it = std::min(T, max_iter - done);
        if (!exec || graph_set != active || graph_nit != n_it) {
            // one graph: a branch per active slice, forked from and joined into the batch stream
            if (exec) { cudaGraphExecDestroy(exec); exec = nullptr; }
            cudaGraph_t graph = nullptr;
            CK(cudaStreamBeginCapture(B->main, cudaStreamCaptureModeThreadLocal));
            cudaEventRecord(B->fork, B->main);
            // With a lane limit each slice waits for the previous slice of its lane
            // (lanes filled largest slice first, each to the least loaded lane).
            std::vector<int> order(active), after(n, -1);
            if (B->lanes > 0 && (int)active.size() > B->lanes) {
                auto cost = [&](int i) { return (double)NN(B->plans[i]) + (double)MM(B->plans[i]); };
                std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost(a) > cost(c); });
                std::vector<double> load(B->lanes, 0.0);
                std::vector<int> last(B->lanes, -1);
                for (int i : order) {
                    const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
                    after[i] = last[l];
                    last[l] = i;
                    load[l] += cost(i);
                }
            }
            for (int i : order) {
                ncs_plan* p = B->plans[i];
                p->capturing = true;
                cudaEvent_t dep = after[i] >= 0 ? B->join[after[i]] : B->fork;
                if (cudaStreamWaitEvent(p->st, dep, 0) != cudaSuccess) rc = NCS_ERR_CUDA;
                if (rc == NCS_OK) rc = enq_solve_block(p, 0, b[i], bg ? bg[i] : nullptr, x[i], n_it);
                p->capturing = false;
                if (rc == NCS_OK && (cudaEventRecord(B->join[i], p->st) != cudaSuccess ||
                                     cudaStreamWaitEvent(B->main, B->join[i], 0) != cudaSuccess))
                    rc = NCS_ERR_CUDA;
                if (rc != NCS_OK) break;
            }
            cudaError_t e = cudaStreamEndCapture(B->main, &graph);
            if (rc != NCS_OK || e != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                cudaGetLastError();
                if (rc == NCS_OK) rc = NCS_ERR_CUDA;
                break;
            }
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) { cudaGetLastError(); rc = NCS_ERR_CUDA; break; }
            graph_set = active;
            graph_nit = n_it;
        }
        if (cudaGraphLaunch(exec, B->main) != cudaSuccess || cudaStreamSynchronize(B->main) != cudaSuccess) {
            cudaGetLastError();
            rc = NCS_ERR_CUDA;
            break;
        }
        done += n_it;
        std::vector<int> still;
        for (int i : active) {
            ncs_plan* p = B->plans[i];
            iters[i] = done;
            f[i] = p->h_pin[0];
            if (!std::isfinite(f[i])) { status[i] = NCS_ERR_DIVERGED; continue; }
            gap[i] = solve_gap(f[i], f_prev[i], f_star ? f_star[i] : nan);
            if (std::isfinite(gap[i]) && gap[i] <= tol) { status[i] = NCS_OK; continue; }
            f_prev[i] = f[i];
            if (done < max_iter) still.push_back(i);
        }
        active.swap(still);
    }
    if (exec) cudaGraphExecDestroy(exec);
    cudaEventRecord(e1, B->main);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != NCS_OK) return rc;
    int worst = NCS_OK;
    for (int i = 0; i < n; ++i) {
        if (reports) {
            reports[i].iters = iters[i];
            reports[i].status = status[i];
            reports[i].time_ms = ms;
            reports[i].f = f[i];
            reports[i].gap = gap[i];
            reports[i].rho = B->plans[i]->rho;
        }
        if (status[i] < 0) worst = status[i];
        else if (worst == NCS_OK && status[i] != NCS_OK) worst = status[i];
    }
    return worst;
}

int ncs_profile_enable_mask(ncs_plan* p, unsigned mask)
{
    CKS(check_plan(p));
    CK(cudaSetDevice(p->dev));
    CK(cudaStreamSynchronize(p->st));
    for (auto& r : p->recs) { p->ev_pool.push_back(r.a); p->ev_pool.push_back(r.b); }
    p->recs.clear();
    p->prof = mask & ((1u << NCS_KERNEL_COUNT) - 1u);
    return NCS_OK;
}

int ncs_profile_enable(ncs_plan* p, int on)
{
    return ncs_profile_enable_mask(p, on ? ~0u : 0u);
}

int ncs_profile_read(ncs_plan* p, double* ms, int* launches, int* kernels)
{
    CKS(check_plan(p));
    if (!ms || !launches) return NCS_ERR_BADARG;
    CK(cudaSetDevice(p->dev));
    CK(cudaStreamSynchronize(p->st));
    for (int k = 0; k < NCS_KERNEL_COUNT; ++k) {
        ms[k] = 0.0;
        launches[k] = 0;
        if (kernels) kernels[k] = 0;
    }
    int rc = NCS_OK;
    for (auto& r : p->recs) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) { cudaGetLastError(); rc = NCS_ERR_CUDA; }
        ms[r.cls] += t;
        launches[r.cls] += 1;
        if (kernels) kernels[r.cls] += r.n;
        p->ev_pool.push_back(r.a);
        p->ev_pool.push_back(r.b);
    }
    p->recs.clear();
    return rc;
}

const char* ncs_kernel_name(int k)
{
    switch (k) {
        case NCS_KERNEL_GATHER: return "joseph_gather";
        case NCS_KERNEL_ROWS_FWD: return "fft_rows_fwd";
        case NCS_KERNEL_COLS_SOLVE: return "fft_cols_solve";
        case NCS_KERNEL_ROWS_INV: return "fft_rows_inv";
        case NCS_KERNEL_TD: return "tv_prox_transpose";
        case NCS_KERNEL_FWD: return "joseph_fwd";
        case NCS_KERNEL_FWD_RESID: return "joseph_fwd_resid";
        case NCS_KERNEL_REDUCE: return "reduce_fp64";
        default: return "unknown";
    }
}

int ncs_plan_nnz(ncs_plan* p, double* nnz)
{
    CKS(check_plan(p));
    if (!nnz) return NCS_ERR_BADARG;
    if (p->nnz_K < 0.0) {
        // count the nonzero weights of K exactly as the kernels evaluate them
        const int N = p->N;
        double cnt = 0.0;
        for (size_t r = 0; r < p->h_rays.size(); ++r) {
            const FanRay& q = p->h_rays[r];
            if (p->h_rayw[r] == 0.0f) continue;          // a ray that passes no pixel
            for (int j = 0; j < N; ++j) {
                const float jf = (float)j;
                const float H = std::fma(q.x, jf, q.z);
                const float L = std::fma(q.y, jf, q.w);
                const float Hi = std::floor(H);
                const float fr = (H - Hi) + L;
                const float fl = std::floor(fr);
                const float w = fr - fl;
                const int i0 = (int)(Hi + fl);
                if (i0 >= 0 && i0 < N && 1.0f - w != 0.0f) cnt += 1.0;
                if (i0 + 1 >= 0 && i0 + 1 < N && w != 0.0f) cnt += 1.0;
            }
        }
        for (int a = 0; a < (p->fan ? 0 : p->na); ++a) {
            const AngleParam& q = p->h_ap[a];
            for (int t = 0; t < p->nd; ++t) {
                for (int j = 0; j < N; ++j) {
                    int i0;
                    const float w = fix_weight(q.Ai * t + q.Bi * j + q.Ci, i0);
                    if (i0 >= 0 && i0 < N && 1.0f - w != 0.0f) cnt += 1.0;
                    if (i0 + 1 >= 0 && i0 + 1 < N && w != 0.0f) cnt += 1.0;
                }
            }
        }
        p->nnz_K = cnt;
    }
    *nnz = p->nnz_K;
    return NCS_OK;
}

const char* ncs_status_string(int s)
{
    switch (s) {
        case NCS_OK: return "ok";
        case NCS_NOT_CONVERGED: return "not converged within max_iter";
        case NCS_ERR_BADARG: return "bad argument";
        case NCS_ERR_UNSUPPORTED: return "unsupported size or option";
        case NCS_ERR_CUDA: return "CUDA error";
        case NCS_ERR_NOMEM: return "out of device memory";
        case NCS_ERR_DIVERGED: return "diverged (non-finite objective)";
        case NCS_ERR_TIMEOUT: return "device wait timed out";
        default: return "unknown status";
    }
}

}  // extern "C"
