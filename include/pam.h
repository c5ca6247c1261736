/*
 * pam.h -- C ABI of libpam, the GB300 (sm_103a) implementation of the PAM
 * fitting path: Parallel and Adaptive Mesh-free approximation of cellwise
 * constant coefficient data by Shepard-normalised Gaussian RBFs, fitted per
 * subdomain by an Elastic Net with residual-driven refinement.
 *
 * The calls follow the paper's statement of the method (section 2):
 *   pam_partition        Step 1   split the grid into subdomains
 *   pam_fit_subdomains   Step 2   assemble, Gram products, Elastic Net solve
 *   pam_refine           Step 3   indicators, marking, enrichment, re-solve
 *                                 (Algorithm 1, repeated n_levels times)
 *   pam_eval             Step 4   evaluate the piecewise surrogate anywhere
 *   pam_eval_glued       Step 4   the same, blended across subdomain interfaces
 *   pam_errors                    relative L1/L2 errors over the source cells
 *
 * Conventions shared by every call:
 *  - Grid: dim in {1,2,3}; n_cells[a] cells per axis (axes >= dim are 1);
 *    isotropic cells of side h = 1/max_a n_cells[a]; cell (i,j,k) has the
 *    centroid ((i+1/2)h, (j+1/2)h, (k+1/2)h) and global index
 *    i + n_x (j + n_y k) (x fastest). Field arrays follow that order.
 *  - Pointers named d_* are DEVICE pointers, h_* HOST pointers. Every
 *    buffer is owned by the caller; the library allocates no memory.
 *    Scratch comes from a caller workspace of pam_plan.workspace_bytes.
 *    (The mixed form's subdomain groups, pam_tuning.level_groups, create
 *    one stream and two events per host thread and device on first use and
 *    keep them for the process.)
 *  - Device work is enqueued on `stream` (a cudaStream_t, NULL = legacy
 *    default stream). Calls that return device-side status synchronise
 *    that stream once before returning; this is stated per call.
 *  - Errors: arguments are validated on the host before any launch; an
 *    invalid one returns PAM_ERR_INVALID_ARG and enqueues nothing. Device
 *    code never traps: per-subdomain problems are reported in the info
 *    array of the model (PAM_FLAG_*), and input faults through the status.
 *  - Thread safety: calls on different workspaces/models may run
 *    concurrently on different streams; calls sharing a workspace must be
 *    ordered on one stream.
 */
#ifndef PAM_H
#define PAM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PAM_MAX_DIM 3
#define PAM_MAX_M 1024         /* largest dictionary capacity per subdomain */
#define PAM_INFO_N 8           /* int32 entries per subdomain in pam_model.info */

typedef enum {
    PAM_OK = 0,
    PAM_ERR_INVALID_ARG = 1,   /* bad pointer, size, or parameter */
    PAM_ERR_NONPOSITIVE_K = 2, /* a cell value is <= 0, NaN or Inf (the paper assumes 0 < K_min) */
    PAM_ERR_CUDA = 3,          /* a CUDA runtime call failed */
    PAM_ERR_WORKSPACE = 4,     /* workspace smaller than pam_plan.workspace_bytes */
    PAM_ERR_NOT_CONVERGED = 5, /* some subdomain's solve was not certified (see info) */
    PAM_ERR_UNSUPPORTED = 6,   /* a valid request the library does not serve */
    PAM_ERR_TIMEOUT = 7        /* a bounded device wait gave up (tensor-core pipeline) */
} pam_status;

typedef enum {
    PAM_PREC_FP64 = 0,   /* plain form: every step in binary64 */
    PAM_PREC_MIXED = 1   /* Gram on tensor cores (bf16 hi/lo split, fp32 accumulate),
                            fp32 active-set solve with iterative refinement,
                            fp64 residual and error accumulation */
} pam_precision;

/* Per-subdomain info entries (pam_model.info[s * PAM_INFO_N + k]). */
enum {
    PAM_INFO_M = 0,        /* current dictionary size M_i */
    PAM_INFO_SUPPORT = 1,  /* nonzero coefficients */
    PAM_INFO_LEVELS = 2,   /* enrichment rounds done */
    PAM_INFO_ITERS = 3,    /* iterations of the last solve (mixed: active-set + 100 x refinement) */
    PAM_INFO_FLAGS = 4,    /* PAM_FLAG_* bits */
    PAM_INFO_STOPPED = 5,  /* 1 once Algorithm 1 stopped for this subdomain */
    PAM_INFO_N_CELLS = 6,  /* patch cells N_i */
    PAM_INFO_MARKED = 7    /* cells marked in the last round */
};

enum {
    PAM_FLAG_NOT_CERTIFIED = 1, /* the last solve did not pass the optimality check */
    PAM_FLAG_CHOLESKY = 2,      /* a non-positive pivot (never expected: lambda2 > 0) */
    PAM_FLAG_REFINE_DIVERGED = 4/* mixed form: the fp32 solve of this subdomain did not pass the
                                   optimality check and the subdomain was solved again in binary64
                                   (assembly, Gram and active-set solve of the plain form, so it
                                   meets the plain form's certificate; NOT_CERTIFIED and CHOLESKY
                                   then describe that solve). At most 32 subdomains per mixed solve
                                   take this path; any others keep NOT_CERTIFIED. The cross-
                                   validation fold solves of pam_lambda_cv never do (its refit does). */
};

/* The problem: grid, decomposition and initial dictionary (section 2 Step 1;
 * Algorithm 1 inputs). */
typedef struct {
    int dim;
    int n_cells[PAM_MAX_DIM];
    int n_sub[PAM_MAX_DIM];   /* subdomains per axis; cores split axis a as
                                 [floor(j n / p), floor((j+1) n / p)) */
    int overlap;              /* patch = core grown by `overlap` cells, clipped */
    int g_init[PAM_MAX_DIM];  /* initial uniform lattice per subdomain core */
} pam_problem;

/* Algorithm 1 parameters. */
typedef struct {
    double lambda1_hat;  /* Elastic Net weights per sample: lambda_k = N_i * lambda_k_hat */
    double lambda2_hat;  /*   (Eq. (2); Example 2 prints 4.59e-4 and 4.64e-6) */
    double eps_tol_rel;  /* eps_tol = |T| (eps_tol_rel * max_{T in patch} K_T)^2;
                            negative: no tolerance, always mark k_top cells */
    double eta;          /* width ratio of new centres, in (0,1) (section 3.4) */
    int k_top;           /* cells marked per round (Algorithm 1 K_top) */
    int m_max;           /* at most m_max centres added per subdomain (M_max) */
    int levels;          /* enrichment rounds planned (sizes the capacity) */
    int max_iters;       /* active-set iteration cap per solve (0: default 200) */
    int precision;       /* pam_precision */
    int warm_start;      /* pam_fit_subdomains: 1 = start the solve from the caller's
                            model->beta[s][0..m0) (e.g. a learned prediction; its
                            nonzero pattern and signs seed the active set), 0 = from 0 */
    int quad;            /* quadrature of the indicators R_T (Eq. (4)): 0 = midpoint
                            (one node, the centroid), 1 = tensor two-point
                            Gauss-Legendre (2^dim nodes x_T +- h / (2 sqrt 3) per
                            axis, weight |T| / 2^dim each) */
    int deferred_status; /* pam_fit_subdomains / pam_refine: 0 = synchronise once and
                            return the device status; 1 = no host synchronisation
                            (the calls can be captured in a CUDA graph): they return
                            PAM_OK after the launches, fit even when some K_T is
                            invalid, and the status accumulates in the workspace
                            until pam_status_read */
    void *warm_start_event; /* pam_fit_subdomains / pam_fit_cells with warm_start = 1: a
                            cudaEvent_t or NULL. When set, the stream waits on the event
                            (cudaStreamWaitEvent) just before the level-0 solve, the first
                            kernel that reads model->beta; the partition, the dictionary
                            set-up (which leaves beta[s][0..m0) alone in warm-start mode),
                            the cell data and the Gram products are enqueued before the
                            wait. So a warm start written on another stream (pam_nn_seed)
                            and followed by a record of this event overlaps them.
                            pam_fit_cells waits before the dictionary set-up instead (it
                            zeroes the coefficients of a patch without elements). Ignored
                            otherwise and by the other calls. An invalid event gives
                            PAM_ERR_CUDA. */
    /* pam_fit_subdomains / pam_fit_cells: fit only the subdomains [sub_begin,
       sub_end) (0, 0 = all). The others get the initial lattice with beta = 0
       and are marked stopped (info STOPPED = 1): no solve, no refinement. One
       field sharded over several GPUs (section 2's subdomains are independent):
       each rank fits a contiguous range, evaluates the points its range owns
       and adds up the sums of pam_error_sums. PAM_ERR_INVALID_ARG unless
       0 <= sub_begin <= sub_end <= S. */
    int sub_begin;
    int sub_end;
} pam_params;

/* Sizes derived from a problem and parameters by pam_plan_create. */
typedef struct {
    int n_subdomains;
    int max_patch_cells;     /* max_i N_i */
    int m0;                  /* initial dictionary size prod g_init */
    int m_cap;               /* dictionary capacity per subdomain (<= PAM_MAX_M) */
    int64_t n_grid_cells;
    size_t workspace_bytes;  /* device scratch the fit/refine/error calls need; in the mixed
                                form it includes the binary64 fallback's min(S, 32) slots
                                (E, G and factor of one subdomain each) */
} pam_plan;

/* Device model, caller-owned (sizes from pam_plan):
 *   boxes   int32  [S][12]  core_lo[3], core_hi[3], patch_lo[3], patch_hi[3]
 *   centres double [S][m_cap][4]  (c_x, c_y, c_z, sigma); unused axes 0
 *   beta    double [S][m_cap]     coefficients (log space), zero past M_i
 *   info    int32  [S][PAM_INFO_N]  */
typedef struct {
    int32_t *boxes;
    double *centres;
    double *beta;
    int32_t *info;
} pam_model;

/* Library version string (static storage). */
const char *pam_version(void);

/* Sizes in bytes of the ABI's structs as this library was compiled, for a
 * binding to check its own layouts against: out[0..5] = sizeof pam_problem,
 * pam_params, pam_plan, pam_model, pam_cells, pam_tuning (n >= 6; fewer are
 * written when n is smaller). Host only; returns the number of sizes the
 * library knows (6). */
int pam_struct_sizes(size_t *out, int n);

/* Human-readable name of a status (static storage). */
const char *pam_status_string(pam_status s);

/*
 * Sizes for `prob` and `par` (host only, no device work).
 * m_cap = min(prod g_init + levels (dim+1) k_top, prod g_init + m_max),
 * rounded up to a multiple of 64; PAM_ERR_UNSUPPORTED if it exceeds
 * PAM_MAX_M, or if levels > 0 and a patch holds more than 16,384 cells
 * (marking keeps a patch's indicator keys in shared memory). Returns PAM_ERR_INVALID_ARG for an inconsistent problem
 * (dim outside 1..3, n_sub[a] outside 1..n_cells[a], overlap < 0,
 * g_init < 1, lambda's < 0 or lambda2_hat == 0, eta outside (0,1),
 * k_top < 0, m_max < 0, levels < 0, precision unknown).
 */
pam_status pam_plan_create(const pam_problem *prob, const pam_params *par, pam_plan *out);

/*
 * Step 1 (section 2) on the host: core and patch boxes of every subdomain,
 * h_boxes [S][12] (layout of pam_model.boxes). Cores are non-overlapping and
 * every cell belongs to exactly one (the half-open decomposition of
 * Experiment 1.2); patches add `overlap` cells of fit data around a core.
 */
pam_status pam_partition(const pam_problem *prob, int32_t *h_boxes);

/*
 * Step 2 (section 2) for every subdomain: copy the partition into
 * model->boxes, lay down the initial dictionary (uniform g_init lattice over
 * each core box, cell-centred, sigma = lattice spacing), then assemble the
 * Shepard-normalised feature matrix W (Eq. (10)) of the Gaussians (Eq. (6))
 * at the patch centroids, form G = W^T W and b = W^T ln K, and solve the
 * Elastic Net (Eq. (2)) on ln K (Remark on log K, section 3.3) from beta = 0.
 * d_K: device double [n_grid_cells], the cell values, all > 0 and finite.
 * Synchronises `stream` once (to read the input check and the certificates).
 * Returns PAM_ERR_NONPOSITIVE_K if some K_T <= 0, NaN or Inf (nothing is
 * fitted then), PAM_ERR_NOT_CONVERGED if a subdomain's solve was not
 * certified (its info carries PAM_FLAG_NOT_CERTIFIED), else PAM_OK.
 */
pam_status pam_fit_subdomains(const pam_problem *prob, const pam_params *par,
                              const pam_plan *plan, const double *d_K,
                              pam_model *model, void *d_workspace,
                              size_t workspace_bytes, void *stream);

/*
 * Per-subdomain choice of the Elastic Net weights by k-fold cross-validation
 * (section 5, Experiment 1.2 chooses (lambda1, lambda2) on each subdomain
 * independently without stating the rule; this is the rule here). On the
 * model's current dictionary (after pam_fit_subdomains / pam_refine), cell t
 * of each patch (local row-major index, x fastest) is in fold t mod n_folds.
 * For every grid pair q and fold f the Elastic Net of Eq. (2) is solved on the
 * other folds' cells with lambda_k = N_train h_grid[q][k] and the squared
 * log-residuals (ln K_t - ln K*(x_t))^2 of the held-out cells summed;
 * d_cv[s][q] = that sum over the folds / N_i. d_choice[s] = the first q of
 * least d_cv[s][q]; model->beta and the support, iteration and flag entries
 * of model->info are then refit on all N_i cells with that pair (the
 * dictionary is kept).
 *   h_grid        host [n_grid][2] (lambda1_hat >= 0, lambda2_hat > 0), 1 <= n_grid <= 32
 *   n_folds       2 ... 1024 (a fold with no cell contributes nothing)
 *   d_cv          device [S][n_grid] binary64, written; d_choice device [S] int32, written
 *   d_workspace   the fit workspace of `plan`; d_cv_workspace: pam_lambda_cv_workspace_size bytes
 * par->precision selects the form (the plan made from the same problem and
 * parameters): PAM_PREC_FP64, binary64 Gram and solves; PAM_PREC_MIXED, the
 * tensor-core Gram of the training rows and the mixed solve, whose exact
 * pass also gives the held-out residuals (PAM_ERR_UNSUPPORTED where the mixed
 * fit is). Synchronises once (unless par->deferred_status) and returns
 * PAM_ERR_NONPOSITIVE_K, PAM_ERR_NOT_CONVERGED (some solve not certified) or
 * PAM_OK.
 */
pam_status pam_lambda_cv_workspace_size(const pam_plan *plan, size_t *bytes);
pam_status pam_lambda_cv(const pam_problem *prob, const pam_params *par, const pam_plan *plan,
                         const double *d_K, pam_model *model, const double *h_grid, int n_grid,
                         int n_folds, double *d_cv, int32_t *d_choice, void *d_workspace,
                         size_t workspace_bytes, void *d_cv_workspace, size_t cv_workspace_bytes,
                         void *stream);

/*
 * Status of the pam_fit_subdomains / pam_refine calls made with
 * deferred_status = 1 on this workspace since the last pam_fit_subdomains:
 * synchronises `stream` and returns PAM_ERR_NONPOSITIVE_K (some K_T <= 0,
 * NaN or Inf: the results are meaningless), PAM_ERR_TIMEOUT,
 * PAM_ERR_NOT_CONVERGED (some solve not certified) or PAM_OK.
 */
pam_status pam_status_read(const pam_plan *plan, void *d_workspace, size_t workspace_bytes, void *stream);

/*
 * Step 3 (section 2; Algorithm 1 (2)-(5)) n_levels times on every
 * subdomain still running: residual indicators R_T (Eq. (4), midpoint
 * rule), marking of the k_top largest R_T >= eps_tol, d+1 new centres per
 * marked cell at width eta * sigma_parent, zero extension of beta, and the
 * re-assembly and re-solve on the enlarged dictionary. A subdomain stops
 * when nothing is marked or its size reaches m0 + m_max (info STOPPED).
 * Must follow pam_fit_subdomains on the same model, workspace and d_K.
 * Synchronises `stream` once; returns as pam_fit_subdomains.
 */
pam_status pam_refine(const pam_problem *prob, const pam_params *par,
                      const pam_plan *plan, const double *d_K, pam_model *model,
                      int n_levels, void *d_workspace, size_t workspace_bytes,
                      void *stream);

/*
 * Normal-equation data of the Elastic Net (Eq. (2) with the Shepard matrix W
 * of Eq. (10) in place of Phi) for the model's CURRENT dictionaries, every
 * subdomain: d_G [S][m_cap][m_cap] = W^T W (both triangles; zero past M_i)
 * and d_b [S][m_cap] = W^T ln K, as device doubles. The building block that
 * pam_fit_subdomains and pam_refine use before each solve, exposed for
 * inspection: PAM_PREC_FP64 forms it in binary64; PAM_PREC_MIXED on the
 * tensor cores (W split into bf16 hi + lo, three products, fp32
 * accumulation; about 2^-16 relative per entry). Needs a model set up by
 * pam_fit_subdomains. The workspace of a plan of either precision serves
 * (no solve runs, so the mixed form's fallback slots are not needed).
 * Synchronises `stream` once; PAM_ERR_TIMEOUT if the tensor-core pipeline
 * stalled (no result then).
 */
pam_status pam_gram(const pam_problem *prob, const pam_params *par, const pam_plan *plan,
                    const double *d_K, const pam_model *model, double *d_G, double *d_b,
                    void *d_workspace, size_t workspace_bytes, void *stream);

/*
 * Device scratch pam_eval needs for n_pts points (owner keys, ranks and the
 * bucketed point order: 12 bytes per point plus 8 per subdomain).
 * PAM_ERR_UNSUPPORTED above 2^31 - 1 points.
 */
pam_status pam_eval_workspace_size(const pam_plan *plan, int64_t n_pts, size_t *bytes);

/*
 * Step 4 (section 2): K*(x) = exp(sum_m beta_m w_m(x)) with the Shepard
 * weights w_m (Eq. (9)) over the whole dictionary of the subdomain whose
 * core contains x (half-open cores, outer face of the grid closed).
 * d_pts: device double [n_pts][dim]; d_out: device double [n_pts], K*(x),
 * or the log-space value when log_space != 0; NaN for points outside the
 * grid. The points are bucketed by owner in d_workspace (at least
 * pam_eval_workspace_size bytes). PAM_PREC_FP64 evaluates in binary64;
 * PAM_PREC_MIXED evaluates the Gaussians, their weighted sums and the final
 * exp in fp32 (local coordinates, 2^x on the special-function unit).
 * Asynchronous (no synchronisation); n_pts == 0 is a no-op.
 */
pam_status pam_eval(const pam_problem *prob, const pam_plan *plan,
                    const pam_model *model, const double *d_pts, int64_t n_pts,
                    double *d_out, int log_space, int precision, void *d_workspace,
                    size_t workspace_bytes, void *stream);

/*
 * pam_eval in two calls. pam_eval_bucket buckets the points by owner core in
 * d_workspace and writes NaN to d_out for the points outside the grid; it
 * reads no model, so it may run before or beside the fit (on another stream).
 * pam_eval_bucketed then evaluates the model at the bucketed points into the
 * other entries of d_out: the same values as pam_eval, bit for bit. Between
 * the two calls the caller keeps d_pts, d_out and d_workspace unchanged and
 * orders the second after the first (same stream, or an event); the same
 * arguments and checks as pam_eval, the bucketing's precision irrelevant.
 */
pam_status pam_eval_bucket(const pam_problem *prob, const pam_plan *plan, const double *d_pts,
                           int64_t n_pts, double *d_out, void *d_workspace, size_t workspace_bytes,
                           void *stream);
pam_status pam_eval_bucketed(const pam_problem *prob, const pam_plan *plan,
                             const pam_model *model, const double *d_pts, int64_t n_pts,
                             double *d_out, int log_space, int precision, void *d_workspace,
                             size_t workspace_bytes, void *stream);

/*
 * Glued evaluation (section 2, Step 4 remark: the piecewise surrogate of
 * pam_eval is discontinuous across subdomain interfaces, and a gluing or
 * averaging of neighbouring local surrogates makes it continuous; the paper
 * leaves the procedure open, this is the one here). The local log-surrogates
 * u_i(x) = sum_m beta_m w_m(x) of Eq. (9) are blended by a tensor-product
 * partition of unity that ramps across every interior core face over a band
 * of half-width delta = band * h:
 *   psi_i(x) = prod_a r((x_a - lo_a + delta) / (2 delta)) r((hi_a + delta - x_a) / (2 delta))
 * with r(t) = t^2 (3 - 2 t) on [0, 1] (clamped outside; r(t) + r(1 - t) = 1)
 * and a factor of 1 at the outer faces of the grid; then
 *   ln K*(x) = sum_i psi_i(x) u_i(x) / sum_i psi_i(x).
 * Farther than delta from every interior face this equals pam_eval; the
 * result is continuous (C^1 in the weights) across the interfaces.
 *   band        half-width of the ramp in cells, 0 < band <= half the
 *               narrowest core of any axis with more than one subdomain
 *               (then at most 2^dim subdomains carry weight at a point);
 *               PAM_ERR_INVALID_ARG otherwise
 *   d_pts       device double [n_pts][dim]; d_out device double [n_pts]:
 *               K*(x), or ln K*(x) when log_space != 0; NaN outside the grid
 *   precision   PAM_PREC_FP64 (binary64 throughout) or PAM_PREC_MIXED (the
 *               local surrogates in fp32 as in pam_eval, the blend in
 *               binary64, the final exp in fp32)
 *   d_workspace at least pam_eval_glued_workspace_size bytes (2^dim
 *               (point, subdomain) slots per point, 28 bytes each: local
 *               value, weight, subdomain, rank, bucket entry; one byte per
 *               point and 8 per subdomain)
 * The per-point sum runs over the subdomains in ascending index order
 * (deterministic). PAM_ERR_UNSUPPORTED above (2^31 - 1) / 2^dim points.
 * Asynchronous (no synchronisation); n_pts == 0 is a no-op.
 */
pam_status pam_eval_glued_workspace_size(const pam_problem *prob, const pam_plan *plan, int64_t n_pts,
                                         size_t *bytes);
pam_status pam_eval_glued(const pam_problem *prob, const pam_plan *plan, const pam_model *model,
                          const double *d_pts, int64_t n_pts, double band, double *d_out, int log_space,
                          int precision, void *d_workspace, size_t workspace_bytes, void *stream);

/*
 * Relative errors of the reconstruction over the source cells, each cell
 * measured with its owner's surrogate at its centroid (quad = 0) or at the
 * 2^dim Gauss-Legendre nodes of pam_params.quad = 1 (weight 1/2^dim of the
 * cell each):
 * d_err[0] = sum |K_T - K*| / sum |K_T|, d_err[1] = (Eq. (12))
 * (sum (K_T - K*)^2 / sum K_T^2)^(1/2), d_err[2] = sum |ln K_T - ln K*| /
 * sum |ln K_T|, d_err[3] = max over the nodes of |log10 K_T - log10 K*(x)|;
 * fp64 accumulation in a fixed order (deterministic). precision selects how
 * the Gaussians are evaluated (as pam_eval). d_err: device double [4]. Uses
 * the fit workspace. PAM_ERR_INVALID_ARG for quad outside {0, 1}.
 * Asynchronous.
 */
pam_status pam_errors(const pam_problem *prob, const pam_plan *plan,
                      const pam_model *model, const double *d_K, double *d_err,
                      int precision, int quad, void *d_workspace, size_t workspace_bytes,
                      void *stream);

/*
 * The sums behind pam_errors over the cells owned by the subdomains
 * [sub_begin, sub_end) only, for one field sharded over several GPUs
 * (section 2: the subdomains are independent; each rank fits its range with
 * pam_params.sub_begin/sub_end): d_sums (device double [8]) receives
 * sum |K - K*|, sum |K|, sum (K - K*)^2, sum K^2, sum |ln K - ln K*|,
 * sum |ln K|, max |ln K - ln K*| and 0. Added over the ranks (the maximum
 * taken for entry 6) they give pam_errors' measures: L1 = s0 / s1,
 * L2 = sqrt(s2 / s3), log-L1 = s4 / s5, max log10 = s6 / ln 10. Arguments
 * and workspace as pam_errors; PAM_ERR_INVALID_ARG unless
 * 0 <= sub_begin <= sub_end <= S. Asynchronous.
 */
pam_status pam_error_sums(const pam_problem *prob, const pam_plan *plan, const pam_model *model,
                          const double *d_K, double *d_sums, int precision, int quad, int sub_begin,
                          int sub_end, void *d_workspace, size_t workspace_bytes, void *stream);

/*
 * pam_errors without a workspace and without allocating device memory.
 * The paper has no counterpart: this exists for callers that cannot
 * allocate on the GPU or hand the library scratch space -- host programs
 * that reserve all device memory in their own pool at start-up, or
 * real-time loops where an allocation's latency or failure is not
 * acceptable. It computes the same four measures into d_err (device
 * double [4]) as pam_errors with PAM_PREC_FP64 and quad = 0: each cell is
 * measured at its centroid (the Gauss-Legendre rule, quad = 1, is not
 * offered here), summing fixed chunks of 4096 grid cells. It reads the
 * dictionary from global memory per cell, so it is slower than pam_errors.
 * Scratch: a file-scope device array of 4096 x 8 doubles (256 KiB) that
 * every GPU loading the library holds until the process exits; grids of
 * more than 16,777,216 cells return PAM_ERR_UNSUPPORTED. The first call on
 * each device looks up the array's device address with that device
 * current (again after the device's context was replaced, e.g. by
 * cudaDeviceReset); make that first call before any stream capture. Every call
 * writes all the partial sums it reads, so no state carries over, but all
 * calls share the one array: calls that overlap on the GPU (different
 * streams, or different host threads on one device) race and must be
 * serialised by the caller. Asynchronous on `stream`.
 */
pam_status pam_errors_noalloc(const pam_problem *prob, const pam_plan *plan,
                              const pam_model *model, const double *d_K, double *d_err,
                              void *stream);

/*
 * Checkpoint and resume (no counterpart in the paper, which fits in one
 * run). A model serialises as one flat host blob: a header (magic
 * "PAMMODEL", version 1, dim, n_cells, n_sub, overlap, g_init, S, m_cap)
 * followed by boxes int32 [S][12], centres double [S][m_cap][4], beta
 * double [S][m_cap] and info int32 [S][PAM_INFO_N], in host byte order.
 *   pam_model_save  h_buf NULL: *size receives the blob size; otherwise
 *                   *size must be at least that (else PAM_ERR_INVALID_ARG
 *                   with *size set) and the blob is written; synchronises
 *                   `stream` once.
 *   pam_model_load  checks the header against the problem and plan, the
 *                   boxes against pam_partition and every M_i against the
 *                   capacity (PAM_ERR_INVALID_ARG on any mismatch, nothing
 *                   copied), then copies the blob into the device model;
 *                   synchronises once.
 *   pam_resume      makes a workspace ready for pam_refine on a loaded
 *                   model: prepares the cell data of d_K and solves every
 *                   subdomain still running (info STOPPED = 0) from the
 *                   model's coefficients (the same unique minimiser, so the
 *                   coefficients are those of the saved fit up to the solve's
 *                   rounding), which also recomputes the indicators. Returns
 *                   as pam_fit_subdomains. pam_resume_cells: the same for a
 *                   mesh given as cells.
 * The network weights of the learned warm start are the caller's fp32
 * arrays (pam_nn_*) and are saved by the caller.
 */
pam_status pam_model_save(const pam_problem *prob, const pam_plan *plan, const pam_model *model, void *h_buf,
                          size_t *size, void *stream);
pam_status pam_model_load(const pam_problem *prob, const pam_plan *plan, const void *h_buf, size_t size,
                          pam_model *model, void *stream);
pam_status pam_resume(const pam_problem *prob, const pam_params *par, const pam_plan *plan, const double *d_K,
                      pam_model *model, void *d_workspace, size_t workspace_bytes, void *stream);

/*
 * General meshes given as cells (section 2: the data are piecewise constant
 * on the elements T of a shape-regular partition -- intervals, triangles,
 * quadrilaterals, ... -- each with a sampling point x_T in T, e.g. its
 * centroid, a value K_T and a measure |T|). The problem's grid fields
 * (n_cells, n_sub, overlap, g_init) keep their meaning for the domain and
 * its decomposition only: the domain is the box [0, n_cells[a] h] (h =
 * 1 / max n_cells), subdomain s owns the core box of pam_partition, and the
 * initial dictionary is the same lattice over it. An element belongs to the
 * core that holds its sampling point (the owner rule of pam_eval: half-open
 * boxes, the outer face closed), and to the patch of every subdomain whose
 * core grown by `overlap` h (clipped to the domain) holds it; a patch lists
 * its elements in ascending index, the local order of the fit. Every step
 * then runs as on a grid, with the element's own measure in R_T = |T| (K*(x_T)
 * - K_T)^2 and in the marking tolerance eps_T = |T| (eps_tol_rel max K)^2.
 * The midpoint rule only (pam_params.quad = 1 needs the element shapes:
 * PAM_ERR_UNSUPPORTED). pam_eval and pam_eval_glued evaluate the model as
 * for a grid.
 */
typedef struct {
    int64_t n_cells;             /* elements n (< 2^31) */
    const double *x;             /* device [n][dim] sampling points, inside the domain box */
    const double *vol;           /* device [n] measures |T| > 0 */
    const int32_t *patch_start;  /* device [S + 1]: patch s holds patch_cells[patch_start[s] ..
                                    patch_start[s + 1]) */
    const int32_t *patch_cells;  /* device: element indices, ascending within each patch */
} pam_cells;

/*
 * Step 1 for a mesh given as cells, on the host: the patch lists of the
 * elements with sampling points h_x [n_cells][dim] (host). Writes
 * h_patch_start [S + 1] (offsets) and, when h_patch_cells is not NULL, the
 * lists into h_patch_cells [h_patch_start[S]] (call once with NULL to size
 * it). PAM_ERR_INVALID_ARG for a point outside the domain box (or NaN).
 */
pam_status pam_partition_cells(const pam_problem *prob, const double *h_x, int64_t n_cells,
                               int32_t *h_patch_start, int32_t *h_patch_cells);
/* pam_plan_create for a mesh given as cells: the patch size comes from the
 * host patch offsets h_patch_start [S + 1]; workspace_bytes adds 32 bytes
 * per patch-cell slot for the gathered points and measures. */
pam_status pam_plan_create_cells(const pam_problem *prob, const pam_params *par, int64_t n_cells,
                                 const int32_t *h_patch_start, pam_plan *out);
/* pam_fit_subdomains / pam_refine on a mesh given as cells; d_K: device
 * [n_cells] element values. A measure <= 0, NaN or Inf is reported like a bad
 * K (PAM_ERR_NONPOSITIVE_K). Same synchronisation and status as the grid
 * calls. */
pam_status pam_fit_cells(const pam_problem *prob, const pam_params *par, const pam_plan *plan,
                         const pam_cells *cells, const double *d_K, pam_model *model, void *d_workspace,
                         size_t workspace_bytes, void *stream);
pam_status pam_refine_cells(const pam_problem *prob, const pam_params *par, const pam_plan *plan,
                            const pam_cells *cells, const double *d_K, pam_model *model, int n_levels,
                            void *d_workspace, size_t workspace_bytes, void *stream);
/* pam_errors over the elements, each measured with its owner's surrogate at
 * its sampling point and weighted by |T|: d_err[0] = sum |T| |K_T - K*| /
 * sum |T| |K_T|, d_err[1] = (sum |T| (K_T - K*)^2 / sum |T| K_T^2)^(1/2)
 * (Eq. (12)), d_err[2] the first in log space, d_err[3] = max |log10 K_T -
 * log10 K*|. Asynchronous. */
pam_status pam_errors_cells(const pam_problem *prob, const pam_plan *plan, const pam_model *model,
                            const pam_cells *cells, const double *d_K, double *d_err, int precision,
                            void *d_workspace, size_t workspace_bytes, void *stream);
pam_status pam_resume_cells(const pam_problem *prob, const pam_params *par, const pam_plan *plan,
                            const pam_cells *cells, const double *d_K, pam_model *model, void *d_workspace,
                            size_t workspace_bytes, void *stream);

/*
 * Learned warm start (an addition: the paper has no learned part).
 * A convolutional network maps a subdomain patch of log10(K)/3 (clipped to
 * [-1, 1], NHWC) to n_out support logits and n_out coefficients / 4 of the
 * patch's initial dictionary. Two architectures (arch):
 *   PAM_NN_PATCH2D   input [32][32][1] (a 32 x 32 patch), n_out = 256 (its
 *                    16 x 16 dictionary): conv3x3 stride 2 (1->32),
 *                    (32->64), (64->128), conv3x3 stride 1 (128->128),
 *                    dense 2048->256, dense 256->512;
 *   PAM_NN_LAYERED3D input [16][16][8] (a 3-D patch of up to 16 x 16 x 8
 *                    cells, x and y as pixels, z layers as channels),
 *                    n_out = 32 (a 4 x 4 x 2 lattice): conv3x3 stride 2
 *                    (8->32), (32->64), conv3x3 stride 1 (64->64),
 *                    (64->64), dense 1024->128, dense 128->64;
 * ReLU after every layer but the last. Parameters are fp32 (flat, layout
 * from pam_nn_layer_offsets: per layer weight offset, bias offset, rows,
 * cols, with W[row][col] and conv columns (ky*3+kx)*cin+c, zero-padded to a
 * multiple of 32); the passes run in bf16 on the tensor cores with fp32
 * accumulation. batch: a multiple of 32. PAM_ERR_INVALID_ARG for an
 * unknown arch.
 */
enum { PAM_NN_PATCH2D = 0, PAM_NN_LAYERED3D = 1 };
pam_status pam_nn_sizes(int arch, int batch, int64_t *n_params, size_t *workspace_bytes);
/* h_geo [3] = (input pixels per side, input channels, n_out). */
pam_status pam_nn_geometry(int arch, int32_t *h_geo);
pam_status pam_nn_layer_offsets(int arch, int64_t *h_offsets /* [6][4] */);
/* d_x [batch][h][h][c] fp32; d_out [batch][2 n_out] fp32 (logits | beta/4).
 * Convolutions with a power-of-two input channel count >= 8 read their input
 * directly (no im2col matrix); the sums are those of the training pass. */
pam_status pam_nn_forward(int arch, const float *d_params, const float *d_x, int batch, float *d_out,
                          void *d_workspace, size_t workspace_bytes, void *stream);
/* Forward + loss + backward: d_grads (same layout as the parameters) and
 * d_loss [2] = (mean BCE of the support logits against d_support in {0,1},
 * mean squared error of beta/4 against d_beta / 4), both [batch][n_out]. */
pam_status pam_nn_gradients(int arch, const float *d_params, const float *d_x, const float *d_support,
                            const float *d_beta, int batch, float *d_grads, float *d_loss,
                            void *d_workspace, size_t workspace_bytes, void *stream);
/*
 * PAM_NN_LAYERED3D inputs of every subdomain of a 3-D problem, from its
 * patch (the pam_partition layout) and the cell values d_K:
 * d_x [n_rows][16][16][8] fp32, row s = subdomain s, entry [iy][ix][iz]
 * = clip(log10 K / 3, -1, 1) at patch cell (ix, iy, iz), zero outside the
 * patch and in rows s >= S. n_rows >= S (the network batch). Returns
 * PAM_ERR_UNSUPPORTED if a patch exceeds 16 x 16 x 8 cells, and
 * PAM_ERR_INVALID_ARG for a problem that is not 3-D. Asynchronous.
 */
pam_status pam_nn_layered_inputs(const pam_problem *prob, const pam_plan *plan, const double *d_K,
                                 float *d_x, int n_rows, void *stream);
/*
 * The same for either network: arch PAM_NN_LAYERED3D as above, or
 * PAM_NN_PATCH2D for a 2-D problem whose patches are at most 32 x 32 cells
 * (d_x [n_rows][32][32][1], entry [iy][ix] = clip(log10 K / 3, -1, 1) at patch
 * cell (ix, iy), zero outside the patch and in rows s >= S): the learned warm
 * start's inputs gathered on the device from the field itself.
 */
pam_status pam_nn_inputs(int arch, const pam_problem *prob, const pam_plan *plan, const double *d_K, float *d_x,
                         int n_rows, void *stream);
/*
 * Seeds the active set from a network output d_out [>= S][2 n_out]: for
 * every subdomain s and initial dictionary entry j < n_out,
 * model->beta[s][j] = b if |b| > threshold else 0, b = 4 d_out[s][n_out + j]
 * (the coefficients the network predicts large; their signs seed the
 * support of the next pam_fit_subdomains call with warm_start = 1). The
 * plan's initial dictionary must hold exactly n_out entries. Asynchronous.
 */
pam_status pam_nn_seed(const pam_plan *plan, int arch, const float *d_out, float threshold,
                       pam_model *model, void *stream);
/* One AdamW step (decoupled weight decay) on n fp32 parameters; step >= 1. */
pam_status pam_nn_adamw(float *d_params, const float *d_grads, float *d_m, float *d_v, int64_t n,
                        float lr, float beta1, float beta2, float eps, float weight_decay, int step,
                        void *stream);

/*
 * Launch tuning and the autotuner (tile and launch shapes; no counterpart in
 * the paper). Five process-wide choices change the speed of the kernels
 * but not their results:
 *   factor_kb    shared-memory budget (KiB) of the mixed solve's packed
 *                support factor; larger supports keep their factor in global
 *                memory, and the budget sets how many CTAs fit per SM
 *                (0: the largest budget up to 64 KiB with two CTAs per SM)
 *   gram_stages  pipeline depth of the tensor-core Gram, 2 or 3 (0: 3 where
 *                shared memory allows)
 *   eval_block   threads per block of the evaluation kernels, 128, 256, 512
 *                or 1024 (0: 256)
 *   solve_persistent  the mixed solve's launch: 0 one CTA per subdomain in
 *                longest-first order (the built-in), 1 one CTA per resident
 *                slot (two per SM), each taking the next subdomain of the
 *                same order from a device counter until none is left; a
 *                solve of one subdomain group (level_groups) always takes
 *                the first form
 *   level_groups the mixed form's levels (the initial lattices' statistics,
 *                Gram and solve in pam_fit_subdomains / pam_fit_cells, the
 *                refinement levels in pam_refine / pam_refine_cells; each
 *                call forks and joins): 1 one pipeline of launches over every
 *                subdomain, 2 the subdomains in two groups (even and odd
 *                index), each running its levels on its own stream (the
 *                caller's and one the library creates per host thread and
 *                device, joined to the caller's stream before the call
 *                returns), so that one group's solve tail overlaps the other
 *                group's work; each group then has its share of the
 *                binary64 fallback's slots (the even group the larger half),
 *                and the results are the same bits as one pipeline's unless
 *                a group runs out of slots where the one list would not.
 *                0: two groups from 1,024 subdomains up (one pipeline
 *                while the phase profiler is on). The autotuner does not
 *                choose it.
 * pam_tuning_set (NULL: all built-in) applies to every later launch of the
 * process; it is not synchronised with launches in flight on other threads.
 * pam_autotune measures, on a fitted model (after pam_fit_subdomains /
 * pam_refine on the same workspace), each candidate with CUDA events on
 * `stream` (median of three runs after one warm-up): the stages on the
 * tensor-core Gram of every subdomain, then the factor budgets {built-in, 64,
 * 48, 32, 24, 16} on the mixed solve of every subdomain from its current
 * coefficients (the same minimiser: the coefficients are re-solved, as by
 * pam_resume, and the indicators rewritten), then the block sizes on
 * pam_eval of d_pts [n_pts][dim] into d_out [n_pts] (skipped when n_pts ==
 * 0; d_eval_workspace as for pam_eval), then the solve's launch {0, 1}. The
 * binary64 form tunes the evaluation only. Within each choice a candidate
 * replaces the built-in (or the candidate kept so far) only when it measures
 * at least 2 % faster (equivalent launches differ by about 1 % between
 * runs); the choices become the process tuning and *out (eval_block 0 when
 * the built-in 256 is kept); h_ms (optional, [14]) receives the medians in
 * ms in that order (stages 3, 2; budgets; blocks; launches), -1 where a
 * candidate was not run.
 * Synchronises `stream`; not to be captured in a CUDA graph.
 */
typedef struct {
    int factor_kb;
    int gram_stages;
    int eval_block;
    int solve_persistent;
    int level_groups;
    int reserved[3];
} pam_tuning;
pam_status pam_tuning_set(const pam_tuning *t);
pam_status pam_tuning_get(pam_tuning *t);
/*
 * Host only: the subdomain groups the mixed form's levels would run in for
 * a problem of n_subdomains subdomains under the current tuning (the phase
 * profiler off). Returns the number of groups (1 or 2), or -1 for
 * n_subdomains < 1. For each group q, out[7 q .. 7 q + 6] (caller-owned,
 * 14 entries) = its first subdomain, the stride between its subdomains,
 * their count, the offset of its solve order in the workspace's order
 * region (entries), the offset of its fallback list in the list region
 * (int32 words: two counters, then the slots' subdomains), its number of
 * binary64 fallback slots and the first of them. One group: the whole
 * range, offsets 0 and min(n_subdomains, 32) slots.
 */
int pam_group_layout(int n_subdomains, int32_t *out);
pam_status pam_autotune(const pam_problem *prob, const pam_params *par, const pam_plan *plan, const double *d_K,
                        pam_model *model, void *d_workspace, size_t workspace_bytes, const double *d_pts,
                        int64_t n_pts, double *d_out, void *d_eval_workspace, size_t eval_workspace_bytes,
                        void *stream, pam_tuning *out, double *h_ms);
/* The same on a model fitted on a mesh given as cells (pam_fit_cells). */
pam_status pam_autotune_cells(const pam_problem *prob, const pam_params *par, const pam_plan *plan,
                              const pam_cells *cells, const double *d_K, pam_model *model, void *d_workspace,
                              size_t workspace_bytes, const double *d_pts, int64_t n_pts, double *d_out,
                              void *d_eval_workspace, size_t eval_workspace_bytes, void *stream, pam_tuning *out,
                              double *h_ms);

/*
 * Failure-detection self-test (no counterpart in the paper). One block waits
 * on an mbarrier with the same bounded wait (a clock64 budget) that the
 * tensor-core pipeline's waits use. arrive = 0: nothing ever arrives, so the
 * wait gives up after about budget_cycles clocks (1,000 ... 4e9), the kernel
 * writes 1 into d_flag (device int32) and returns -- no trap, no hang, the
 * context stays usable -- and the call returns PAM_ERR_TIMEOUT; arrive = 1:
 * the barrier completes at once, d_flag = 0, PAM_OK. Synchronises `stream`.
 */
pam_status pam_selftest_wait(int arrive, long long budget_cycles, int32_t *d_flag, void *stream);

/*
 * Optional kernel timing. When enabled, every kernel family below records a
 * CUDA event pair around its launches on the caller's stream; reading sums
 * the elapsed times per family (and synchronises on the recorded events).
 * Families: PAM_PHASE_* (prepare, assemble, gram, solve, residual, mark,
 * eval, errors, stats, gram_tc, refine, eval_kernel: the evaluation's
 * per-owner kernel alone, inside eval, which adds the owner lookup, scan and
 * scatter). Not thread-safe against concurrent
 * enable/reset; intended for benchmarks. No counterpart in the paper.
 * Calls made while `stream` is being captured into a CUDA graph record the
 * pairs as event-record nodes of the graph: each replay re-records them, so
 * pam_timing_read after a replay returns that replay's times, and
 * pam_timing_reset (which destroys the events) must wait until the graph is
 * destroyed. pam_kernel_launches counts a captured launch once, at capture.
 */
enum {
    PAM_PHASE_PREPARE = 0, PAM_PHASE_ASSEMBLE, PAM_PHASE_GRAM, PAM_PHASE_SOLVE,
    PAM_PHASE_RESIDUAL, PAM_PHASE_MARK, PAM_PHASE_EVAL, PAM_PHASE_ERRORS,
    PAM_PHASE_STATS, PAM_PHASE_GRAM_TC, PAM_PHASE_REFINE, PAM_PHASE_EVAL_KERNEL, PAM_PHASE_COUNT
};
void pam_timing_enable(int on);
/* Kernels this library has launched since it was loaded (host-side count). */
long long pam_kernel_launches(void);
void pam_timing_reset(void);
pam_status pam_timing_read(int phase, double *h_total_ms, int *h_count);

#ifdef __cplusplus
}
#endif

#endif /* PAM_H */
