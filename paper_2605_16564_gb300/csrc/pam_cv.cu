// pam_cv.cu -- per-subdomain choice of the Elastic Net weights by k-fold
// cross-validation (section 5, Experiment 1.2: the weights are chosen on
// each subdomain independently; the paper does not state the rule).
//
// On the subdomain's current dictionary, cell t of the patch (local
// row-major index) belongs to fold t mod k. For every grid pair
// (lambda1_hat, lambda2_hat) and fold f the Elastic Net of Eq. (2) is solved
// on the other folds' cells with lambda_k = N_train lambda_k_hat (the binary64
// active-set solver on the masked Gram), and the squared log-residuals
// (y_t - (W beta)_t)^2 of the held-out cells are summed; cv = the sum over all
// folds / N. The least cv (first grid index on ties) is chosen and the
// coefficients are refit on all N cells with it.
//
// Binary64 form: E (exp(l - l*), [S][m_cap][n_max]) and 1 / Shepard sum are
// assembled once for all folds; per fold the masked b and G are formed, and
// per grid pair a scratch copy of the model's coefficients is solved in
// place, then its held-out residuals are summed by one block per subdomain in
// a fixed order (cv is bitwise reproducible). Mixed form: the row statistics
// once, per fold the tensor-core Gram of the training rows, and per grid pair
// the mixed solve in its cross-validation form, which sums the held-out
// residuals of its final coefficients itself (fixed order too).
#include <cfloat>

#include "pam_internal.cuh"

namespace pam {

// One block per subdomain: cv[s][gi] += sum over the held-out cells t of fold
// `fold` of (y_t - inv_s_t sum_m E_mt beta_m)^2.
__global__ void __launch_bounds__(256) k_cv_heldout(Geo g, int folds, int fold, const double *beta,
                                                    const int32_t *info, Ws w, double *cv, int n_grid,
                                                    int gi) {
    const int s = blockIdx.x;
    const int32_t *inf = info + s * kInfoN;
    const int M = inf[PAM_INFO_M], N = inf[PAM_INFO_N_CELLS];
    __shared__ double part[8];
    const double *E = w.E + (size_t)s * g.m_cap * g.n_max;
    const double *iv = w.inv_s + (size_t)s * g.n_max;
    const double *y = w.y + (size_t)s * g.n_max;
    const double *b = beta + (size_t)s * g.m_cap;
    double acc = 0.0;
    for (int t = fold + folds * (int)threadIdx.x; t < N; t += folds * (int)blockDim.x) {
        double v = 0.0;
        for (int m = 0; m < M; ++m) v += E[(size_t)m * g.n_max + t] * b[m];
        const double r = y[t] - iv[t] * v;
        acc += r * r;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot += part[q];
        cv[(size_t)s * n_grid + gi] += tot;
    }
}

// A scratch copy of the model's coefficients and diagnostics for one solve.
__global__ void k_cv_scratch(int n_beta, const double *beta, double *beta_s, int n_info,
                             const int32_t *info, int32_t *info_s) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_beta; i += gridDim.x * blockDim.x)
        beta_s[i] = beta[i];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_info; i += gridDim.x * blockDim.x)
        info_s[i] = info[i];
}

// cv /= N, the first least entry chosen, its pair written to lam_tab.
__global__ void k_cv_choose(int S, CvGrid grid, const int32_t *info, double *cv, int32_t *choice,
                            double *lam_tab) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const int N = info[s * kInfoN + PAM_INFO_N_CELLS];
    double best = 0.0;
    int bi = 0;
    for (int q = 0; q < grid.n; ++q) {
        const double v = cv[(size_t)s * grid.n + q] / (double)(N > 0 ? N : 1);
        cv[(size_t)s * grid.n + q] = v;
        if (q == 0 || v < best) { best = v; bi = q; }
    }
    choice[s] = bi;
    lam_tab[2 * s] = grid.lam[bi][0];
    lam_tab[2 * s + 1] = grid.lam[bi][1];
}

size_t cv_workspace_bytes(const Geo &g) {
    const size_t S = (size_t)g.S;
    return ((S * g.m_cap * sizeof(double) + 255) / 256) * 256 + ((S * kInfoN * 4 + 255) / 256) * 256 +
           S * 2 * sizeof(double);
}

void launch_lambda_cv(const Geo &g, const Par &p, int precision, const int32_t *boxes, const double *centres,
                      double *beta, int32_t *info, const Ws &w, const CvGrid &grid, int folds, double *cv,
                      int32_t *choice, void *cv_ws, cudaStream_t st) {
    const size_t S = (size_t)g.S;
    const bool mixed = precision == PAM_PREC_MIXED;
    char *base = (char *)cv_ws;
    double *beta_s = (double *)base;
    int32_t *info_s = (int32_t *)(base + ((S * g.m_cap * sizeof(double) + 255) / 256) * 256);
    double *lam_tab = (double *)((char *)info_s + ((S * kInfoN * 4 + 255) / 256) * 256);
    // once for all folds: E and 1 / Shepard sum (binary64 form), or the row
    // statistics of the Shepard rows (mixed form)
    if (mixed) launch_stats_f32(g, boxes, centres, info, w, st, 1);
    else launch_assemble_gram_f64(g, boxes, centres, info, w, st, 1);
    cudaMemsetAsync(cv, 0, S * grid.n * sizeof(double), st);
    const int nb = (int)S * g.m_cap, ni = (int)S * kInfoN;
    for (int f = 0; f < folds; ++f) {
        if (mixed) launch_gram_tc(g, boxes, centres, info, w, st, 1, folds, f);
        else launch_bgram_f64(g, info, w, st, 1, folds, f);
        Par pf = p;
        pf.cv_folds = folds;
        pf.cv_fold = f;
        for (int q = 0; q < grid.n; ++q) {
            pf.lam1_hat = grid.lam[q][0];
            pf.lam2_hat = grid.lam[q][1];
            k_cv_scratch<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(nb, beta, beta_s, ni, info, info_s);
            count_launches(1);
            if (mixed) {
                launch_solve_mixed(g, pf, boxes, centres, beta_s, info_s, w, nullptr, 1, cv + q, grid.n, st, 0);
            } else {
                launch_solve_f64(g, pf, beta_s, info_s, w, nullptr, 1, st);
                k_cv_heldout<<<(unsigned)S, 256, 0, st>>>(g, folds, f, beta_s, info_s, w, cv, grid.n, q);
                count_launches(1);
            }
        }
    }
    k_cv_choose<<<(unsigned)((S + 127) / 128), 128, 0, st>>>((int)S, grid, info, cv, choice, lam_tab);
    count_launches(1);
    // refit on all cells with each subdomain's chosen pair
    if (mixed) {
        launch_gram_tc(g, boxes, centres, info, w, st, 1, 0, 0);
        launch_solve_mixed(g, p, boxes, centres, beta, info, w, lam_tab, 1, nullptr, 0, st, 1);
    } else {
        launch_bgram_f64(g, info, w, st, 1, 0, 0);
        launch_solve_f64(g, p, beta, info, w, lam_tab, 1, st);
    }
}

}  // namespace pam
