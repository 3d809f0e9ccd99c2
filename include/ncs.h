/*
 * ncs.h - C ABI of the GB300 (sm_103a) near-circulant splitting library.
 *
 * Near-circulant splitting (NCS), Ryu, Ko, Won, "Splitting with
 * Near-Circulant Linear Systems: Applications to Total Variation CT and PET"
 * (arXiv 1810.13100), solves  min_x g(Ax - b)  (Sec. 1, eq. (RCP)) with
 *
 *     x+   = x - M^+ A^T u                                  (eq. (NCS))
 *     u+   = prox_{alpha g*}(u + alpha (A (2x+ - x) - b))
 *
 * for the TV-CT problem of Sec. 4.1, A = [K; (beta/alpha) D], and the TV-PET
 * problem of Sec. 4.2, A = [K; (beta/alpha) D; kappa I] (the nonnegativity row of
 * its remark).  K is a parallel-beam (or fan-beam) Joseph projector, D the 2-D forward
 * difference operator (Sec. 2), and M = gamma I + alpha C is the circulant
 * matrix whose eigenvalues come from eqs. (circ_R) and (circ_D), solved with a
 * real 2-D FFT.  PDHG (eq. (PDHG)) is provided on the same kernels.
 *
 * Conventions shared by every entry point
 *   - Image x: N x N float32, row-major, x[j*N + i]; row j, column i; pixel
 *     centre (u, v) = (i - (N-1)/2, (N-1)/2 - j) in pixel units.
 *   - Sinogram y: n_angles x n_det float32, row-major, y[a*n_det + t]; the ray
 *     of bin t at angle theta_a is u cos + v sin = s_t (Sec. 2, eq. (radon-def)),
 *     s_t = (t - (n_det-1)/2) * det_spacing + det_offset.
 *   - TV dual v: 2 x N x N float32; v[0..N*N) holds the horizontal block
 *     (D_h x)[j][i] = x[j][i] - x[j][i+1], v[N*N..2*N*N) the vertical block
 *     (D_v x)[j][i] = x[j][i] - x[j+1][i]; the last column of the first block
 *     and the last row of the second are not part of D (kept at zero).
 *   - Nonnegativity dual s: N x N float32 (PET with nonneg only, else NULL).
 *   - All array pointers are DEVICE pointers unless a name says host, and are
 *     owned by the caller.  Work is enqueued on the plan's stream
 *     (ncs_options.cuda_stream, or a stream the plan creates); calls return
 *     after enqueueing unless documented as synchronising.
 *   - Return value: NCS_OK (0) on success, a positive status for a normal
 *     outcome that is not success (NCS_NOT_CONVERGED), a negative NCS_ERR_* on
 *     failure.  No C++ exception crosses this boundary.
 *   - One plan is used by one host thread at a time.
 */
#ifndef NCS_H_
#define NCS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NCS_OK                 0
#define NCS_NOT_CONVERGED      1   /* solve stopped at max_iter above tolerance */
#define NCS_ERR_BADARG        -1   /* null pointer, bad size or parameter */
#define NCS_ERR_UNSUPPORTED   -2   /* e.g. N not of the form 2^a 3^b, N > 4096 */
#define NCS_ERR_CUDA          -3   /* a CUDA runtime call failed */
#define NCS_ERR_NOMEM         -4   /* device allocation failed */
#define NCS_ERR_DIVERGED      -5   /* objective became NaN/Inf */
#define NCS_ERR_TIMEOUT       -6   /* a bounded device wait ran out */

/* Parallel-beam geometry (Sec. 2, eq. (radon-def)). */
typedef struct {
    int n_angles;          /* number of projection angles, >= 1 */
    int n_det;             /* detector bins per angle, >= 1 */
    double det_spacing;    /* bin pitch in pixel units, >= 1 (0 -> 1) */
    double det_offset;     /* shift of the bin centres, pixel units */
    const double* angles;  /* host array of n_angles radians, or NULL for theta_a = a*pi/n_angles */
} ncs_geometry;

typedef enum { NCS_DATA_L2 = 0, NCS_DATA_KL = 1 } ncs_data_term;
typedef enum { NCS_TV_ANISO = 0, NCS_TV_ISO = 1 } ncs_tv_kind;
/* Storage of the iteration state (arithmetic is FP32 and reductions FP64 in all three):
 * NCS_FP32: everything float32;
 * NCS_BF16_STORE: the duals u, v, s and the projector's internal images of xbar in bfloat16;
 * NCS_BF16_DUALS: only the duals u, v, s in bfloat16.
 * x, b and bg are float32 in every mode. */
typedef enum { NCS_FP32 = 0, NCS_BF16_STORE = 1, NCS_BF16_DUALS = 2 } ncs_precision;

/* Solver options.  Fill with ncs_options_default() and change what you need. */
typedef struct {
    double beta;           /* TV scaling beta of Sec. 4.1 (default alpha) */
    double gamma;          /* gamma of M = gamma I + alpha C (default 0) */
    double h_dc;           /* DC entry of H_R (eq. (circ_R)); NaN -> ||K 1||^2 / ||1||^2 */
    double c_r;            /* C_R of eq. (circ_R); NaN -> n_angles * N / pi */
    double kappa;          /* weight of the nonnegativity row (PET, nonneg = 1); default 1 */
    ncs_data_term data;    /* NCS_DATA_L2: 1/2||Kx - b||^2; NCS_DATA_KL: Poisson likelihood (Sec. 4.2) */
    ncs_tv_kind tv;        /* anisotropic box (Sec. 4.1) or isotropic per-pixel ball */
    int nonneg;            /* 1: add the row kappa I with delta_{R+} (Sec. 4.2 remark); KL only */
    ncs_precision prec;    /* storage of the iteration state (see ncs_precision) */
    double a3_margin;      /* M is rescaled to rho(M^{-1} alpha A^T A) = 1/(1+margin); default 1e-2; <0 disables */
    int power_max_iter;    /* power iteration cap (default 500) */
    double power_tol;      /* power iteration relative-change stop (default 1e-6: rho then lies within
                              ~1e-5 of its limit, far inside the 1e-2 (A3) margin) */
    uint64_t power_seed;   /* seed of the SplitMix64 start vector (default 0) */
    int check_every;       /* objective evaluated every T iterations in the solves (default 10) */
    void* cuda_stream;     /* cudaStream_t to run on, or NULL for a plan-owned stream */
    int autotune;          /* 1: time the gather's angle slicing and the FFT radix orders at plan
                              creation and keep the fastest (default 0) */
    int warm_dual;         /* 1: the solves start the data dual at u^0 = K x^0 - b, consistent with the
                              given x^0 (L2 data term, FP32 storage); 0: zero duals (default) */
    int h_probes;          /* 0 (default): the projector part of M from eq. (circ_R), C_R / |nu|;
                              P > 0: from eq. (H-fan) in least-squares form over P probe images v
                              (SplitMix64 seeds power_seed + 1 .. power_seed + P, uniform in
                              [-1, 1)): sum_v Re((F K^T K v) conj(F v)) / sum_v |F v|^2, clamped at
                              0; the DC entry stays h_dc either way */
    int fan_gather;        /* fan-beam plans only, the K^T kernel: 0 (default) or 2: ray-driven 32 x 32 tiles,
                              1: pixel-driven 2 x 2 quads (both exact transposes); with autotune = 1 the plan
                              times both and keeps the faster */
    int pdhg_only;         /* 1: the plan serves PDHG (eq. (PDHG)) and the operator entry points only: M's
                              eigenvalues, the probes of eq. (H-fan) and the (A3) power iteration are
                              skipped at creation (PDHG needs only lambda_max(A^T A)); ncs_step, ncs_solve,
                              admm_solve, ncs_apply_Minv, ncs_get_mu and ncs_batch_create then return
                              NCS_ERR_UNSUPPORTED for it, and its report's rho is NaN.  0 (default): full plan */
    int fwd_kernel;        /* parallel-beam plans, the K kernel (both evaluate the same matrix, summed in a
                              different order): 0 (default): image strips staged in shared memory (N <= 864),
                              else the row walk; 1: the row walk (each ray reads its rows from L2); 2: strips,
                              NCS_ERR_UNSUPPORTED if the image is too large for them.  The strip form holds
                              n_strip * n_angles * n_det floats of scratch (at 512 x 512 with 720 x 730: 5
                              strips of 103 rows, 10.5 MB) */
} ncs_options;

/* Result of ncs_solve / pdhg_solve. */
typedef struct {
    int iters;             /* iterations run */
    int status;            /* NCS_OK, NCS_NOT_CONVERGED or an error */
    double time_ms;        /* wall time of the iteration loop on the plan's stream */
    double f;              /* FP64 objective at the returned x */
    double gap;            /* (f - f_star)/|f_star|, or the last relative change of f if f_star is NaN */
    double rho;            /* rho(M^{-1} alpha A^T A) before the rescale (NCS) or gamma_P (PDHG) */
} ncs_report;

typedef struct ncs_plan ncs_plan;   /* opaque; owns its workspace, tables and solver state */

/* Defaults: beta = NaN (-> alpha), gamma = 0, h_dc = c_r = NaN, kappa = 1, L2 data,
 * anisotropic TV, nonneg 0, FP32, a3_margin 1e-2, power 500 / 1e-6 / seed 0,
 * check_every 10, NULL stream, autotune 0, warm_dual 0, h_probes 0, fan_gather 0, pdhg_only 0,
 * fwd_kernel 0. */
void ncs_options_default(ncs_options* opt);

/* Build a plan for an N x N image (nx == ny == N, N even, N = 2^a 3^b, 8 <= N <= 4096).
 * Computes the per-angle Joseph coefficients and the eigenvalues of M (eqs.
 * (circ_R), (circ_D)) on the host in FP64, then on the GPU the power-iteration
 * bound rho = lambda_max(M^{-1} alpha A^T A) of assumption (A3) (Sec. 3) with FP64
 * reductions, and rescales M so that (A3) holds with the margin.  Synchronises.
 * lambda > 0 is the TV weight, alpha > 0 the dual step.
 * Errors: NCS_ERR_BADARG, NCS_ERR_UNSUPPORTED (also for a user angle whose ray spacing
 * along the stepped axis, det_spacing / max(|cos|, |sin|), exceeds 1 by less than twice
 * the FP32 rounding of a crossing difference, ~3e-7 at N = 512: the exact-transpose
 * gather's two-phase shared-memory sums need rays at least one pixel apart in FP32),
 * NCS_ERR_NOMEM, NCS_ERR_CUDA. */
int ncs_plan_create(const ncs_geometry* geom, int nx, int ny, double lambda, double alpha,
                    const ncs_options* opt, ncs_plan** out);

/* Fan-beam geometry with an equiangular (arc) detector (Sec. 4, "fan beam and cone beam
 * geometry": X-rays leave a point source and are received over a fan of angles; source and
 * detector circle the object).  Pixel coordinates as above.  View a puts the source at
 * S_a = R (-sin beta_a, cos beta_a), R = src_dist.  Channel t receives the ray leaving S_a at
 * the fan angle gamma_t = (t - (n_det-1)/2) * pitch + offset, counted counter-clockwise from
 * the central ray (S_a towards the rotation centre); it is the line
 * u cos(beta_a + gamma_t) + v sin(beta_a + gamma_t) = R sin(gamma_t) of eq. (radon-def).
 * The sinogram is y[a*n_det + t]. */
typedef struct {
    int n_views;           /* source positions, >= 1 */
    int n_det;             /* channels per view, >= 1 */
    double src_dist;       /* R in pixel units, >= (N-1)/sqrt(2) + 3 (source outside the image's circle) */
    double pitch;          /* fan angle between adjacent channels, radians, > 0 */
    double offset;         /* fan angle of the detector centre, radians */
    const double* views;   /* host array of n_views source angles beta_a (radians), or NULL for 2 pi a / n_views */
} ncs_fan_geometry;

/* Build a plan for the fan beam: the same solver, options and entry points as
 * ncs_plan_create, with K the Joseph projector of the fan's rays (each ray stepped over the
 * rows or the columns of the image by the parallel beam's rule, ties to rows) and K^T its
 * exact transpose.  The projector part of M comes from eq. (H-fan) (least-squares form over
 * ncs_options.h_probes probe images; 0 selects 128), since eq. (circ_R) is for the parallel
 * beam; c_r is ignored.  ncs_fbp is not available for a fan plan (NCS_ERR_UNSUPPORTED).
 * Errors as ncs_plan_create, and NCS_ERR_BADARG for a non-positive pitch, non-finite
 * values or a source inside the image's circumscribed circle (plus a 3-pixel margin).
 * Synchronises. */
int ncs_plan_create_fan(const ncs_fan_geometry* geom, int nx, int ny, double lambda, double alpha,
                        const ncs_options* opt, ncs_plan** out);

/* Release the plan and everything it owns (NULL is a no-op). */
void ncs_plan_destroy(ncs_plan* plan);

/* Run n_iter >= 1 NCS iterations (eq. (NCS); explicit updates of Sec. 4.1 / 4.2) in
 * place on the caller's state: x (N*N), u (n_angles*n_det), v (2*N*N), s (N*N, PET
 * with nonneg only, else NULL); b is the measured sinogram (CT) or the counts
 * (PET); bg is the PET background sinogram or NULL (CT: must be NULL).
 * x, b and bg are float32.  With prec = NCS_BF16_STORE or NCS_BF16_DUALS, u, v and s
 * point to bfloat16 arrays of the same element counts (the float* type is kept for
 * the ABI).
 * Asynchronous on the plan's stream. */
int ncs_step(ncs_plan* plan, float* x, float* u, float* v, float* s,
             const float* b, const float* bg, int n_iter);

/* Same as ncs_step for PDHG (eq. (PDHG)): x+ = x - gamma_P^{-1} A^T u with
 * gamma_P = alpha lambda_max(A^T A)(1 + margin) (computed on first use). */
int pdhg_step(ncs_plan* plan, float* x, float* u, float* v, float* s,
              const float* b, const float* bg, int n_iter);

/* Solve with NCS from x (in: x^0, out: the result; device, float32) and zero duals (or the
 * consistent data dual of ncs_options.warm_dual), until
 * (f - f_star)/|f_star| <= tol (f_star finite) or the relative change of f over
 * one check interval <= tol (f_star NaN), or max_iter iterations.  The FP64
 * objective is evaluated every check_every iterations on the GPU; the loop runs
 * as CUDA graphs of check_every iterations.  Synchronises.  report may be NULL.
 * Returns NCS_OK, NCS_NOT_CONVERGED or an error. */
int ncs_solve(ncs_plan* plan, const float* b, const float* bg, float* x,
              double tol, int max_iter, double f_star, ncs_report* report);

/* Same as ncs_solve with PDHG updates. */
int pdhg_solve(ncs_plan* plan, const float* b, const float* bg, float* x,
               double tol, int max_iter, double f_star, ncs_report* report);

/* The ADMM comparator (Ramani and Fessler's scheme, Sec. 1.3; the textbook ADMM of the
 * Appendix with A = [K; (beta/alpha) D]): per outer step z+ = prox_{(1/alpha) g}(A x - b -
 * lambda), then n_cg steps of conjugate gradients on A^T A x = A^T (z+ + b + lambda)
 * preconditioned by the plan's circulant M and started from the current x, then
 * lambda+ = lambda + z+ - A x+ + b.  L2 data, FP32 storage, no nonnegativity row (else
 * NCS_ERR_UNSUPPORTED).  x (device, N*N) holds x^0 on entry and the result on exit; tol,
 * f_star and the check every check_every outer steps as in ncs_solve; max_outer bounds the
 * outer steps.  report->iters counts outer steps and report->rho holds n_cg.  Synchronises
 * (each conjugate-gradient step reads two dot products on the host). */
int admm_solve(ncs_plan* plan, const float* b, float* x, double tol, int max_outer, int n_cg, double f_star,
               ncs_report* report);

/* Host-side results of the setup power iterations: lambda_max(A^T A) (computed
 * now if not yet) and rho = lambda_max(M^{-1} alpha A^T A) before the rescale.
 * Synchronises. */
int ncs_power_bound(ncs_plan* plan, double* lambda_max_AtA, double* rho_M);

/* ---- Cone beam (3-D) operators ---- */

/* Cone beam on a circular orbit (Sec. 4, "fan beam and cone beam geometry": the 3-D
 * divergent-beam transform).  Volume x[k*N*N + j*N + i]: Nz slices of N x N, voxel centre
 * (i - (N-1)/2, (N-1)/2 - j, k - (Nz-1)/2).  Sinogram y[(a*n_rows + r)*n_det + t].  The source
 * of view a is that of the fan beam (ncs_fan_geometry) in the plane w = 0; channel t has the fan
 * beam's fan angle, and detector row r (a cylindrical detector) holds the rays whose slope
 * sigma_r = (r - (n_rows-1)/2) * row_pitch + row_offset is the rise in w per unit of in-plane
 * distance from the source.  K is Joseph's method along the ray's in-plane trace (rows or
 * columns, the fan beam's rule), bilinear in (in-plane position, slice), weighted by the path
 * length per step sqrt(1 + sigma^2)/|cos| (or /|sin|); voxels outside the volume are zero. */
typedef struct {
    int n_views;           /* source positions, >= 1 */
    int n_rows;            /* detector rows, >= 1 */
    int n_det;             /* channels per row, >= 1 */
    double src_dist;       /* R in voxel units, >= (N-1)/sqrt(2) + 3 */
    double pitch;          /* fan angle between adjacent channels, radians, > 0 */
    double offset;         /* fan angle of the channel centre, radians */
    double row_pitch;      /* slope step between adjacent rows, > 0 */
    double row_offset;     /* slope of the row centre; every |sigma_r| < 1/sqrt(2) */
    const double* views;   /* host array of n_views source angles, or NULL for 2 pi a / n_views */
} ncs_cone_geometry;

typedef struct ncs_cone ncs_cone;   /* opaque; owns the projector's device tables */

/* Build the cone-beam operator pair for an N x N x Nz volume (N even, 8 <= N <= 4096,
 * 1 <= Nz <= 4096) whose calls run on cuda_stream (NULL: the default stream).  Synchronises.
 * Errors: NCS_ERR_BADARG (sizes, non-positive pitches, a slope of magnitude >= 1/sqrt(2), a
 * source inside the image's circle plus 3 pixels, non-finite values), NCS_ERR_UNSUPPORTED, NCS_ERR_NOMEM,
 * NCS_ERR_CUDA. */
int ncs_cone_create(const ncs_cone_geometry* geom, int N, int Nz, void* cuda_stream, ncs_cone** out);

/* Release it (NULL is a no-op); waits for its stream. */
void ncs_cone_destroy(ncs_cone* cone);

/* y = K x (device pointers, float32; x: N*N*Nz, y: n_views*n_rows*n_det).  Asynchronous. */
int ncs_cone_apply_K(ncs_cone* cone, const float* x, float* y);

/* x = K^T y, the exact transpose (gather, no atomics; deterministic).  Asynchronous. */
int ncs_cone_apply_KT(ncs_cone* cone, const float* y, float* x);

/* ---- Cone beam (3-D) NCS ---- */

/* NCS (eq. (NCS), the updates of Sec. 4.1 in 3-D) for min 1/2 ||K x - b||^2 + lambda TV(x)
 * on the cone beam, A = [K; (beta/alpha) D] with D the forward differences along x, y and z
 * (Sec. 2 per axis).  Layouts as for ncs_cone; the TV dual v is three N*N*Nz blocks (the x, y
 * and z differences, zero at the last index of their axis).  TV is anisotropic (the box of
 * radius lambda alpha/beta per component) or isotropic (the ball of that radius per voxel).
 * M = gamma I + alpha C is circulant on the periodic N x N x Nz grid: its projector part comes
 * from eq. (H-fan) in least-squares form over ncs_options.h_probes SplitMix64 probe volumes
 * (0 selects 128; seeds power_seed + 1 ..), the DC entry from ||K 1||^2 / ||1||^2 (or
 * ncs_options.h_dc), the difference part from the 3-D periodic Laplacian
 * 4 (sin^2(pi l/Nz) + sin^2(pi p/N) + sin^2(pi q/N)); M is rescaled for (A3) as for the 2-D
 * plans.  Its solve is a real 3-D FFT: per-slice row and column transforms and a direct
 * transform along z (Nz <= 64).  Options used: beta, gamma, h_dc, tv, h_probes, a3_margin,
 * power_max_iter, power_tol, power_seed, check_every, cuda_stream; the others must keep
 * their defaults (NCS_ERR_UNSUPPORTED otherwise: L2 data, FP32 only).  Synchronises.
 * Errors: NCS_ERR_BADARG (as ncs_cone_create, lambda < 0, alpha <= 0, Nz < 2),
 * NCS_ERR_UNSUPPORTED (N not of the form 2^a 3^b, Nz > 64), NCS_ERR_NOMEM, NCS_ERR_CUDA. */
typedef struct ncs_cone_plan ncs_cone_plan;
int ncs_cone_plan_create(const ncs_cone_geometry* geom, int N, int Nz, double lambda, double alpha,
                         const ncs_options* opt, ncs_cone_plan** out);

/* Release the plan (NULL is a no-op); waits for its stream. */
void ncs_cone_plan_destroy(ncs_cone_plan* plan);

/* n_iter >= 1 NCS iterations in place on the caller's state: x (N*N*Nz), u
 * (n_views*n_rows*n_det), v (3*N*N*Nz); b is the measured sinogram.  Asynchronous. */
int ncs_cone_step(ncs_cone_plan* plan, float* x, float* u, float* v, const float* b, int n_iter);

/* Solve from x (in: x^0, out: the result) with zero duals until the FP64 objective gap
 * (f - f_star)/|f_star| <= tol (or the relative change of f over one check interval if
 * f_star is NaN), or max_iter iterations; CUDA graphs of check_every iterations, the data term
 * from a running K x.  Synchronises.  Returns NCS_OK, NCS_NOT_CONVERGED or an error. */
int ncs_cone_solve(ncs_cone_plan* plan, const float* b, float* x, double tol, int max_iter, double f_star,
                   ncs_report* report);

/* *f = 1/2 ||K x - b||^2 + lambda TV(x) with FP64 reductions.  Synchronises. */
int ncs_cone_objective(ncs_cone_plan* plan, const float* x, const float* b, double* f);

/* *n = the CUDA kernels the plan has enqueued on its stream since creation (an iteration of
 * ncs_cone_step is 8: the gather, five of the 3-D circulant solve, the forward pass with the
 * data prox, the TV prox; ncs_cone_objective is 3).  A solve's CUDA graph is counted once, when
 * it is captured, not per replay. */
int ncs_cone_kernels(const ncs_cone_plan* plan, long long* n);

/* out = M^{-1} r (the plan's 3-D circulant solve; N*N*Nz).  Asynchronous. */
int ncs_cone_apply_Minv(ncs_cone_plan* plan, const float* r, float* out);

/* The eigenvalues of M after the (A3) rescale, host array of Nz*N*N doubles [l][p][q]
 * (frequencies along z, y, x). */
int ncs_cone_get_mu(ncs_cone_plan* plan, double* mu_host);

/* *rho = lambda_max(M^{-1} alpha A^T A) before the rescale (NaN if a3_margin < 0). */
int ncs_cone_power_bound(ncs_cone_plan* plan, double* rho);

/* ---- Batches of independent slices ---- */

typedef struct ncs_batch ncs_batch;   /* opaque; a set of plans solved together */

/* Group n_plans distinct plans (any sizes and geometries, same device) into a batch.
 * The plans stay owned by the caller and must outlive the batch. */
int ncs_batch_create(ncs_plan* const* plans, int n_plans, ncs_batch** out);

/* Release the batch (not its plans; NULL is a no-op). */
void ncs_batch_destroy(ncs_batch* batch);

/* At most `lanes` slices of the batch in flight at once (0, the default: all).  Each
 * launch then chains the slices into `lanes` sequences, largest slice first onto the
 * least loaded sequence, so fewer slices share the L2 cache at a time.  Errors:
 * NCS_ERR_BADARG for a negative count. */
int ncs_batch_set_lanes(ncs_batch* batch, int lanes);

/* Times `iters` NCS iterations of every slice (after one untimed solve of the same
 * length that builds the graph) with 0 (all), 1, 2, 4, 8 and 16 lanes (those below the
 * slice count), keeps the fastest as the batch's lane count and returns it in
 * *lanes_out (may be NULL).  The solves start from and overwrite x; reset x before the
 * real solve.  Synchronises.  Errors: those of ncs_batch_solve. */
int ncs_batch_tune_lanes(ncs_batch* batch, const float* const* b, const float* const* bg, float* const* x,
                         int iters, int* lanes_out);

/* Solve every slice with NCS from its x[i] (in: x^0, out: the result) and zero duals,
 * as ncs_solve does for one plan, with all slices in flight at once: each launch is one
 * CUDA graph holding a branch per active slice (check_every iterations of plans[0] and
 * the FP64 objective), forked from and joined into a batch-owned stream, so the slices'
 * kernels run concurrently.  A slice leaves the batch when it reaches tol (against
 * f_star[i], or the relative change when f_star is NULL or f_star[i] is NaN), diverges,
 * or reaches max_iter; the graph is rebuilt for the remaining slices.  b[i], x[i]:
 * device pointers per slice; bg: NULL or per-slice PET backgrounds (entries NULL for
 * CT).  reports[i] (may be NULL) gets each slice's iterations, status, f, gap; time_ms is
 * the batch's wall time.  Synchronises.  Returns NCS_OK if every slice converged, else
 * an error of a slice, else NCS_NOT_CONVERGED. */
int ncs_batch_solve(ncs_batch* batch, const float* const* b, const float* const* bg, float* const* x,
                    double tol, int max_iter, const double* f_star, ncs_report* reports);

/* ---- Operators of the plan (device pointers, asynchronous) ---- */

/* y = K x, the Joseph forward projection (N*N -> n_angles*n_det). */
int ncs_apply_K(ncs_plan* plan, const float* x, float* y);

/* x = K^T y, computed as a per-pixel gather with the same FP32 weights as K. */
int ncs_apply_KT(ncs_plan* plan, const float* y, float* x);

/* y = K x with x held as bfloat16 pair images (each value rounded to nearest once), as the
 * NCS_BF16_STORE iterations hold xbar; the taps are read as bfloat16 and accumulated in FP32.
 * x, y: float32, N*N and n_angles*n_det.  Allocates its two bfloat16 images on the first call
 * (NCS_ERR_NOMEM if that fails).  Errors: NCS_ERR_BADARG. */
int ncs_apply_K_bf16(ncs_plan* plan, const float* x, float* y);

/* x = K^T y for a bfloat16 sinogram y (n_angles*n_det), as the bfloat16-storage iterations
 * read their data dual; FP32 accumulation, float32 x (N*N).  Errors: NCS_ERR_BADARG. */
int ncs_apply_KT_bf16(ncs_plan* plan, const void* y, float* x);

/* v = D x (2*N*N layout above) and x = D^T v. */
int ncs_apply_D(ncs_plan* plan, const float* x, float* v);
int ncs_apply_DT(ncs_plan* plan, const float* v, float* x);

/* Filtered backprojection (not in the paper; a warm start for the solves):
 * x = (pi / n_angles) K^T q with q = tau (h * b) row by row, h the Ram-Lak kernel of
 * Kak and Slaney for bin pitch tau (h(0) = 1/(4 tau^2), h(n) = -1/(n^2 pi^2 tau^2) for odd n,
 * 0 for even n != 0).  b: n_angles*n_det, x: N*N, float32 device pointers.  Asynchronous. */
int ncs_fbp(ncs_plan* plan, const float* b, float* x);

/* out = M^{-1} r = F^{-1} diag(mu)^{-1} F r with the plan's (rescaled) mu (Sec. 2). */
int ncs_apply_Minv(ncs_plan* plan, const float* r, float* out);

/* FP64 objective at x: 1/2||Kx - b||^2 + lambda TV(x) (L2), or
 * KL(b, K x+ + bg) + lambda TV(x+) with x+ = max(x, 0) (KL).  Synchronises;
 * writes the host double *f. */
int ncs_objective(ncs_plan* plan, const float* x, const float* b, const float* bg, double* f);

/* Copy the plan's eigenvalue table of M (after the (A3) rescale), N x N row-major
 * in FP64, mu[p*N + q] for frequency p along rows and q along columns, to the
 * host array mu_host.  Synchronises. */
int ncs_get_mu(ncs_plan* plan, double* mu_host);

/* Tuning of the plan: the gather's angle slices per tile (32 x 32 pixels; for a fan plan the
 * view slices of its K^T kernel, whose tiles are 32 x 32 or, with pixel quads, 32 x 16) and
 * the FFT radix order (fft_radices: host array of at least 12 ints; any pointer may be NULL). */
int ncs_plan_info(const ncs_plan* plan, int* gather_parts, int* fft_radices, int* n_radices);

/* The plan's K kernel (the fwd_kernel option): *n_strip image strips of *strip_rows rows each
 * (the last may be shorter) for the strip form, 0 and 0 for the row walk (a fan-beam plan, an
 * image too large for strips, or fwd_kernel 1).  Either pointer may be NULL. */
int ncs_plan_fwd_strips(const ncs_plan* plan, int* n_strip, int* strip_rows);

/* Plan sizes: N, n_angles, n_det. */
int ncs_plan_sizes(const ncs_plan* plan, int* N, int* n_angles, int* n_det);

/* ---- Measurement ---- */

/* Kernel classes reported by ncs_profile_read. */
#define NCS_KERNEL_GATHER      0   /* K^T gather (+ D^T, nonneg row, PDHG update) */
#define NCS_KERNEL_ROWS_FWD    1   /* FFT solve: row transforms */
#define NCS_KERNEL_COLS_SOLVE  2   /* FFT solve: column transforms and 1/mu */
#define NCS_KERNEL_ROWS_INV    3   /* FFT solve: inverse rows and primal update */
#define NCS_KERNEL_TD          4   /* D x, TV / nonneg dual prox, transposes, TV sums */
#define NCS_KERNEL_FWD         5   /* K forward projection with the data prox (strip pass + strip sum, or row walk) */
#define NCS_KERNEL_FWD_RESID   6   /* K forward projection with the FP64 data-term sum (the same kernels) */
#define NCS_KERNEL_REDUCE      7   /* FP64 reductions */
#define NCS_KERNEL_COUNT       8

/* Turn per-kernel timing on (1) or off (0) and clear what was recorded.  While
 * on, every kernel the plan enqueues outside graph capture is bracketed by
 * CUDA events on the plan's stream (at most 2^18 launches are kept).
 * Synchronises. */
int ncs_profile_enable(ncs_plan* plan, int on);

/* As ncs_profile_enable, for the kernel classes whose bit (1 << NCS_KERNEL_*) is set in
 * mask only (0: off), so a timed region can carry the events of one kernel alone.
 * Synchronises. */
int ncs_profile_enable_mask(ncs_plan* plan, unsigned mask);

/* Sum of the recorded durations (ms) and the number of recorded launches per class into
 * ms[NCS_KERNEL_COUNT] and launches[NCS_KERNEL_COUNT] (host arrays), and, if kernels is not
 * NULL, the CUDA kernels those launches enqueued into kernels[NCS_KERNEL_COUNT] (a strip-form
 * forward projection is one launch of two kernels), then clear the record.  Synchronises. */
int ncs_profile_read(ncs_plan* plan, double* ms, int* launches, int* kernels);

/* Name of a kernel class (static string). */
const char* ncs_kernel_name(int kernel_class);

/* Number of nonzero weights of the plan's K, counted on the host with the same
 * FP32 arithmetic the kernels use (the work of one application of K or K^T is
 * 2 * nnz flops).  Computed once per plan. */
int ncs_plan_nnz(ncs_plan* plan, double* nnz);

/* ---- Learned warm start (not in the paper; only x^0 changes, so convergence is untouched) ---- */

typedef struct ncs_unet ncs_unet;   /* opaque U-Net for one H x W single-channel image */

/* A U-Net with `levels` resolution levels (channels base, 2 base, ... per level; two 3x3
 * convolutions + ReLU per level and side; 2x2 average pooling down, nearest 2x upsampling and
 * concatenation with the skip connection up; a 1x1 head) whose output is added to its input:
 * y = x + net(x).  Convolutions run on the tensor cores with bfloat16 operands and FP32
 * accumulation; weights are kept in FP32 and initialised with He's normal from `seed`.
 * H and W must be multiples of 2^(levels-1).  Errors: NCS_ERR_BADARG, NCS_ERR_UNSUPPORTED,
 * NCS_ERR_NOMEM. */
int ncs_unet_create(int H, int W, int levels, int base_channels, uint64_t seed, ncs_unet** out);
void ncs_unet_destroy(ncs_unet* net);

/* Number of parameters.  Order: per convolution in creation order (encoder levels top down,
 * two convolutions each; decoder levels bottom up, two each) the weights [Cout][3][3][Cin]
 * then the biases [Cout]; last the head weights [base] and its bias. */
size_t ncs_unet_num_params(const ncs_unet* net);

/* Copy the FP32 parameters to (set = 0) or from (set = 1) the host array (num_params floats).
 * Synchronises. */
int ncs_unet_params(ncs_unet* net, float* host, int set);

/* y = x + net(x) for one image (device float32 arrays of H*W).  Synchronises. */
int ncs_unet_forward(ncs_unet* net, const float* x, float* y);

/* Loss mean((x + net(x) - target)^2) and its gradient with respect to every parameter
 * (grad_host: num_params floats, may be NULL).  Synchronises. */
int ncs_unet_gradient(ncs_unet* net, const float* x, const float* target, double* loss, float* grad_host);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the loss of one (x, target) pair;
 * *loss (if not NULL) gets the loss before the step (then synchronises). */
int ncs_unet_train_step(ncs_unet* net, const float* x, const float* target, float lr, double* loss);

/* Which kernel computes the 3x3 convolutions (forward and data gradient): 1 (the default)
 * the tcgen05 tensor-core path (accumulators in tensor memory) for every convolution whose
 * input and output channel counts are multiples of 16, the mma.sync path for the others;
 * 0 the mma.sync path for all.  The weight gradient always uses mma.sync.  Forward,
 * gradient and train step return NCS_ERR_TIMEOUT if a tensor-core completion wait gave up
 * (the results of that call are then invalid).  Errors: NCS_ERR_BADARG. */
int ncs_unet_set_conv_path(ncs_unet* net, int tensor_cores);

/* Failure-path test: the tensor-core convolutions of the next forward, gradient or train
 * step issue no MMAs and give up their completion waits after 4096 polls, so that call
 * returns NCS_ERR_TIMEOUT with invalid results; the device context stays usable and later
 * calls are unaffected.  (Nothing else arms this.)  Errors: NCS_ERR_BADARG. */
int ncs_unet_inject_wait_timeout(ncs_unet* net);

/* ---- Backprojection without device allocation ---- */

/* Largest sizes ncs_apply_KT_static accepts. */
#define NCS_STATIC_MAX_N       512
#define NCS_STATIC_MAX_ANGLES  2048

/* x = K^T y for the geometry and an N x N image, without a plan and without
 * allocating any device memory.  The paper has no counterpart: this is for
 * callers that cannot allocate device memory when they need a backprojection
 * (a process whose memory pool owns the whole GPU, a framework whose allocator
 * must not be bypassed, code that reserved all memory up front).  It runs the
 * same tiled gather kernel as ncs_apply_KT with its working memory (angle
 * table, per-tile counters, partial sums of the angle slices) taken from one
 * file-scope device array of about 4.1 MiB that every GPU loading the library
 * holds until the process exits.  y: n_angles*n_det, x: N*N, both device
 * pointers owned by the caller; cuda_stream: a cudaStream_t or NULL (legacy
 * default stream).  Asynchronous, apart from the host-to-device copy of the
 * angle table, which returns once the table is staged.
 * Sizes N > NCS_STATIC_MAX_N or n_angles > NCS_STATIC_MAX_ANGLES return
 * NCS_ERR_UNSUPPORTED, and so do a det_spacing in (0, 1) and the geometries that
 * ncs_plan_create rejects with NCS_ERR_UNSUPPORTED; N < 8, null pointers or an
 * empty geometry return NCS_ERR_BADARG.  All calls share the array: calls whose work overlaps on the
 * GPU (several streams or host threads) race and must be serialised by the
 * caller.  The call cannot be captured into a CUDA graph (it copies the angle
 * table from host memory it owns): on a capturing stream it returns
 * NCS_ERR_UNSUPPORTED and enqueues nothing. */
int ncs_apply_KT_static(const ncs_geometry* geom, int N, const float* y, float* x, void* cuda_stream);

/* Human-readable name of a status code (static string). */
const char* ncs_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* NCS_H_ */
