// pam_internal.cuh -- declarations shared by libpam's translation units:
// workspace layout, the kernel-side view of a problem, and small device
// helpers. Internal to the library (the public ABI is include/pam.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pam.h"

namespace pam {

constexpr int kInfoN = PAM_INFO_N;

// 32-byte aligned four-double vector (a centre: c_x, c_y, c_z, sigma).
using dvec4 = double4_32a;

// Kernel-side copy of the problem and parameters (passed by value).
struct Geo {
    int dim;
    int n[3];       // cells per axis (unused axes 1)
    int p[3];       // subdomains per axis (unused axes 1)
    int overlap;
    int g[3];       // initial lattice (unused axes 1)
    int nmax;       // max_a n[a]
    double h;       // 1 / nmax
    double vol;     // h^dim
    int S;          // subdomains
    int n_max;      // max patch cells (padded stride of per-cell arrays)
    int m0, m_cap;
    int prec;       // pam_precision of the fit calls (sizes the workspace)
    int sub_lo, sub_hi;  // the subdomains a fit solves (the others start stopped)
    // the subdomains a launch of the refinement levels covers: gb + i gs for
    // 0 <= i < gn (gn 0: all S); a group of them runs its levels on its own
    // stream, beside the other groups
    int gb = 0, gs = 1, gn = 0;
    // a general mesh given as cells (section 2: elements with a sampling
    // point, a value and a measure); all NULL / 0 for a structured grid
    int cells;               // 1: the patches are element lists
    const double *cx;        // [n][dim] sampling points x_T
    const double *cvol;      // [n] measures |T|
    const int32_t *pstart;   // [S+1] offsets of the patch lists
    const int32_t *pcells;   // element indices, ascending within a patch
    const double4_32a *cxv;  // workspace [S][n_max]: (x, y, z, |T|) of each patch cell
};

__host__ __device__ __forceinline__ int group_count(const Geo &g) { return g.gn > 0 ? g.gn : g.S; }
__host__ __device__ __forceinline__ int group_sub(const Geo &g, int i) { return g.gb + i * g.gs; }

struct Par {
    double lam1_hat, lam2_hat, eps_tol_rel, eta;
    int k_top, m_max, levels, max_iters;
    int quad;  // 0 midpoint, 1 Gauss-Legendre indicators
    int cv_folds, cv_fold;  // cross-validation fold of a solve (0: all rows)
};

// Workspace carve-up. Every region is 256-byte aligned.
struct Ws {
    double *y;        // [S][n_max]   ln K of patch cells (row-major over the patch)
    double *kv;       // [S][n_max]   K of patch cells
    double *inv_s;    // [S][n_max]   1 / Shepard sum of the max-shifted exps of each row
    double *E;        // [S][m_cap][n_max] exp(l - l*) (fp64 form; W = E * inv_s)
    double *G;        // [S][m_cap][m_cap] Gram W^T W (fp64 form)
    double *b;        // [S][m_cap]   W^T y
    double *R;        // [S][n_max]   residual indicators
    double *L;        // [S][m_cap (m_cap+1)/2] packed fp64 Cholesky factor when it exceeds shared memory
    float *Lf;        // the same region as fp32 factors (mixed form), same per-subdomain stride in elements
    float *Gf;        // [S][m_cap][m_cap] Gram in fp32 (mixed form)
    float *rowmax;    // [S][n_max]   row maximum of the logits (mixed form)
    float *rowinv;    // [S][n_max]   1 / Shepard sum (mixed form)
    float *wsum;      // [S][m_cap]   sum_t W_tj of each centre (mixed form: bounds of the exact gradient)
    double *err_part; // [err_blocks][4] per-block partial sums of the error measures
    unsigned long long *kmax_bits; // [S] max K of each patch as ordered bits
    int32_t *status;  // [8] device status words
    uint32_t *cost;   // [S] clock cycles of each subdomain's last mixed solve (a scheduling hint)
    int32_t *order;   // [S] subdomains in decreasing cost, the mixed solve's block order
    double4_32a *cxv; // [S][n_max] gathered (x, y, z, |T|) of patch cells (element-list meshes only)
    // binary64 fallback of the mixed form: the subdomains whose fp32 solve
    // did not certify are solved again in binary64 on fb_slots slots
    int32_t *fb;      // [2 + fb_slots]: fb[0] = subdomains listed, fb[1] = the persistent
                      // solve's counter, fb[2 + i] = the i-th (two more words are carved:
                      // a group's view starts its own list after the first group's slots)
    double *fbE;      // [fb_slots][m_cap][n_max] exp(l - l*) of the listed subdomains
    double *fbG;      // [fb_slots][m_cap][m_cap] their binary64 Gram
    double *fbL;      // [fb_slots][m_cap (m_cap+1)/2] their binary64 factors beyond shared memory
    int fb_slots;     // 0 in the binary64 form
    size_t bytes;
    size_t bytes_no_fb;  // the regions before the fallback's (all that pam_gram uses)
};

// Slots of the binary64 fallback: at most this many subdomains of one mixed
// solve are solved again in binary64 (the rest stay flagged NOT_CERTIFIED).
constexpr int kFbSlots = 32;


enum StatusWord { kStBadK = 0, kStUncertified = 1, kStCholesky = 2, kStTimeout = 3 };

constexpr int kErrBlocks = 1024;
constexpr int kMixedMaxM = 512;  // dictionary capacity limit of the tensor-core Gram

Ws carve_workspace(const Geo &g, void *base);
bool make_geo(const pam_problem *prob, const pam_params *par, Geo *g, Par *p, pam_status *st);

// Launchers implemented in the kernel translation units.
void launch_partition(const Geo &g, int32_t *boxes, cudaStream_t st);
void launch_prepare(const Geo &g, const int32_t *boxes, const double *K, const Ws &w, cudaStream_t st);
void launch_errors_cells(const Geo &g, const int32_t *boxes, const double *centres, const double *beta,
                         const int32_t *info, const double *K, double *err, int precision, const Ws &w,
                         cudaStream_t st);
void launch_init_dictionary(const Geo &g, const int32_t *boxes, double *centres, double *beta,
                            int32_t *info, cudaStream_t st, int keep_beta);
// before_solve: an event the stream waits on between the Gram products and
// the solve (the first kernel of a level that reads beta), or null.
void launch_solve_level_f64(const Geo &g, const Par &p, const int32_t *boxes, const double *centres,
                            double *beta, int32_t *info, const Ws &w, cudaStream_t st,
                            cudaEvent_t before_solve = nullptr);
// m_bound: an upper bound on every dictionary size of the launch (0: the
// capacity); at most 64 takes the CUDA-core Gram of the initial lattices.
void launch_stats_gram_tc(const Geo &g, const int32_t *boxes, const double *centres,
                          const int32_t *info, const Ws &w, cudaStream_t st, int all, int m_bound = 0);
void launch_assemble_gram_f64(const Geo &g, const int32_t *boxes, const double *centres,
                              const int32_t *info, const Ws &w, cudaStream_t st, int all);
void launch_bgram_f64(const Geo &g, const int32_t *info, const Ws &w, cudaStream_t st, int all, int folds,
                      int fold);
void launch_solve_f64(const Geo &g, const Par &p, double *beta, int32_t *info, const Ws &w,
                      const double *lam_tab, int all, cudaStream_t st);
void launch_fallback_f64(const Geo &g, const Par &p, const int32_t *boxes, const double *centres,
                         double *beta, int32_t *info, const Ws &w, const double *lam_tab, cudaStream_t st);
void launch_stats_f32(const Geo &g, const int32_t *boxes, const double *centres, const int32_t *info,
                      const Ws &w, cudaStream_t st, int all);
void launch_gram_tc(const Geo &g, const int32_t *boxes, const double *centres, const int32_t *info,
                    const Ws &w, cudaStream_t st, int all, int folds, int fold);
void launch_solve_mixed(const Geo &g, const Par &p, const int32_t *boxes, const double *centres,
                        double *beta, int32_t *info, const Ws &w, const double *lam_tab, int all, double *cv,
                        int cv_stride, cudaStream_t st, int fallback, int m_bound = 0);
void launch_copy_gram_f32(const Geo &g, const int32_t *info, const Ws &w, double *G_out,
                          double *b_out, cudaStream_t st);
void launch_copy_gram_f64(const Geo &g, const int32_t *info, const Ws &w, double *G_out,
                          double *b_out, cudaStream_t st);
void launch_solve_level_mixed(const Geo &g, const Par &p, const int32_t *boxes, const double *centres,
                              double *beta, int32_t *info, const Ws &w, cudaStream_t st,
                              cudaEvent_t before_solve = nullptr, int m_bound = 0);
void launch_refine_round(const Geo &g, const Par &p, int precision, const int32_t *boxes,
                         double *centres, double *beta, int32_t *info, const Ws &w, cudaStream_t st);
void launch_eval_bucket(const Geo &g, const double *pts, int64_t n_pts, double *out, void *ws, cudaStream_t st);
void launch_eval_bucketed(const Geo &g, const int32_t *boxes, const double *centres, const double *beta,
                          const int32_t *info, const double *pts, int64_t n_pts, double *out, int log_space,
                          int precision, void *ws, cudaStream_t st);
void launch_eval(const Geo &g, const int32_t *boxes, const double *centres, const double *beta,
                 const int32_t *info, const double *pts, int64_t n_pts, double *out, int log_space,
                 int precision, void *ws, cudaStream_t st);
size_t eval_workspace_bytes(int S, int64_t n_pts);
void launch_eval_glued(const Geo &g, const int32_t *boxes, const double *centres, const double *beta,
                       const int32_t *info, const double *pts, int64_t n_pts, double band, double *out,
                       int log_space, int precision, void *ws, cudaStream_t st);
size_t glue_workspace_bytes(int S, int dim, int64_t n_pts);
void launch_errors(const Geo &g, const int32_t *boxes, const double *centres, const double *beta,
                   const int32_t *info, const double *K, double *err, int precision, int quad,
                   const Ws &w, cudaStream_t st, int row0 = 0, int row1 = -1);
void launch_residual_quad(const Geo &g, int precision, const int32_t *boxes, const double *centres,
                          const double *beta, const int32_t *info, const Ws &w, cudaStream_t st);
bool mixed_solve_fits(const Geo &g);
void launch_wait_selftest(int arrive, long long budget, int32_t *flag, cudaStream_t st);

// Grid of (lambda1_hat, lambda2_hat) pairs of the cross-validation (by value).
constexpr int kCvMaxGrid = 32;
struct CvGrid {
    int n;
    double lam[kCvMaxGrid][2];
};
size_t cv_workspace_bytes(const Geo &g);
void launch_lambda_cv(const Geo &g, const Par &p, int precision, const int32_t *boxes, const double *centres,
                      double *beta, int32_t *info, const Ws &w, const CvGrid &grid, int folds, double *cv,
                      int32_t *choice, void *cv_ws, cudaStream_t st);

// Process-wide launch tuning (pam_tuning_set / pam_autotune); zero fields
// take the built-in choices.
const pam_tuning &tuning();

// Kernel families timed by the optional event profiler (pam_timing_*).
enum Phase {
    kPhPrepare = 0, kPhAssemble, kPhGram, kPhSolve, kPhResidual, kPhMark, kPhEval, kPhErrors,
    kPhStats, kPhGramTC, kPhRefine, kPhEvalKernel, kPhCount
};

// Counts kernel launches issued by the library (host side).
void count_launches(int n);

// Records a CUDA event pair around the launches of its scope on `st` when
// the profiler is on (one pair per scope); a no-op otherwise.
struct PhaseScope {
    PhaseScope(int phase, cudaStream_t st);
    ~PhaseScope();
    int phase_;
    cudaStream_t st_;
    cudaEvent_t stop_;
    bool on_;
    bool capturing_;
};

// ---------------------------------------------------------------- device ---

// Patch extent w[a] = patch_hi - patch_lo of subdomain s.
__device__ __forceinline__ void patch_extent(const int32_t *box, int w[3]) {
    w[0] = box[9] - box[6];
    w[1] = box[10] - box[7];
    w[2] = box[11] - box[8];
}

// Centroid of local patch cell t (row-major over the patch, x fastest).
// (i + 1/2) h is one exact add and one rounded multiply, no contraction.
__device__ __forceinline__ void patch_cell(const Geo &g, const int32_t *box, int t, double x[3],
                                          int64_t *gidx) {
    int w[3];
    patch_extent(box, w);
    int i = box[6] + t % w[0];
    int j = box[7] + (t / w[0]) % w[1];
    int k = box[8] + t / (w[0] * w[1]);
    x[0] = __dmul_rn((double)i + 0.5, g.h);
    x[1] = g.dim > 1 ? __dmul_rn((double)j + 0.5, g.h) : 0.0;
    x[2] = g.dim > 2 ? __dmul_rn((double)k + 0.5, g.h) : 0.0;
    *gidx = (int64_t)i + (int64_t)g.n[0] * ((int64_t)j + (int64_t)g.n[1] * (int64_t)k);
}

// Sampling point of local patch cell t of subdomain s: the gathered element
// point for a mesh given as cells, else the grid centroid.
__device__ __forceinline__ void cell_point(const Geo &g, int s, const int32_t *box, int t, double x[3]) {
    if (g.cxv) {
        const double4_32a v = g.cxv[(size_t)s * g.n_max + t];
        x[0] = v.x;
        x[1] = v.y;
        x[2] = v.z;
    } else {
        int64_t gi;
        patch_cell(g, box, t, x, &gi);
    }
}

// Measure |T| of local patch cell t of subdomain s.
__device__ __forceinline__ double cell_measure(const Geo &g, int s, int t) {
    return g.cxv ? g.cxv[(size_t)s * g.n_max + t].w : g.vol;
}

// Core j of cell i along an axis of n cells split into p cores ([j n / p,
// (j + 1) n / p) in floor division): j0 = floor(i p / n), plus one where
// floor((j0 + 1) n / p) <= i, i.e. (j0 + 1) n < (i + 1) p. One integer
// division, 32-bit where i p fits (always, below 2^16 cells per axis).
__device__ __forceinline__ int core_of(int i, int n, int p) {
    const uint64_t ip = (uint64_t)i * (uint64_t)p;
    int j = ip <= 0xffffffffull ? (int)((uint32_t)ip / (uint32_t)n) : (int)(ip / (uint64_t)n);
    if (j + 1 < p && (uint64_t)(j + 1) * (uint64_t)n < ip + (uint64_t)p) ++j;
    return j;
}

// Owner subdomain of a point (half-open cores, outer face closed), -1 outside
// or NaN. The cell index is floor(x n_max) in binary64; past the sign test
// the range test is made on it in integers (u in [0, n] <=> i in [0, n), or
// i = n with u = n), which spares the narrow binary64 pipe a comparison.
__device__ __forceinline__ int owner_of_point(const Geo &g, const double x[3]) {
    int j[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a >= g.dim) break;
        // fp32 first: uf differs from the binary64 u = x n_max by at most
        // 2^-22 |u| (the rounding of x to fp32 and of the product), so away
        // from the integers and from both ends of the grid (margin d, twice
        // that bound and more) floor(uf) is floor(u); the few points within
        // d of one take the binary64 path. NaN fails every test and goes
        // there too.
        const float uf = (float)x[a] * (float)g.nmax;
        const float fl = floorf(uf), d = fmaf(uf, 4.8e-7f, 1e-6f);
        int i;
        if (uf - fl >= d && fl + 1.f - uf >= d && uf >= d && uf <= (float)g.n[a] - d) {
            i = (int)fl;
        } else {
            const double u = x[a] * (double)g.nmax;
            if (!(u >= 0.0)) return -1;
            i = __double2int_rd(u);  // beyond the int range: INT_MAX
            if (i > g.n[a]) return -1;
            if (i == g.n[a]) {
                if (u != (double)g.n[a]) return -1;
                i = g.n[a] - 1;
            }
        }
        j[a] = core_of(i, g.n[a], g.p[a]);
    }
    return j[0] + g.p[0] * (j[1] + g.p[1] * j[2]);
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

}  // namespace pam

#define PAM_CUDA_TRY(expr)                                      \
    do {                                                        \
        cudaError_t e_ = (expr);                                \
        if (e_ != cudaSuccess) return PAM_ERR_CUDA;             \
    } while (0)
