/*
 * pam_oracle.c -- plain, slow, FP64 CPU oracle for the PAM fitting path.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg load this library; the product path never
 * does, and shares no code, header, table or constant with it.
 *
 * What it computes (PAM = Parallel and Adaptive Mesh-free approximation):
 *   Step 1 (section 2)  split the cell grid into subdomains;
 *   Step 2 (section 2, sections 3.1-3.3) on each subdomain build the Gaussian
 *          RBF feature matrix, Shepard-normalise its rows, and solve the
 *          Elastic Net for the coefficients on the log of the data;
 *   Step 3 (section 2, Algorithm 1) residual indicators, marking, enrichment,
 *          repeated;
 *   Step 4 (section 2) evaluate the piecewise surrogate anywhere.
 *
 * Everything is written from its definition, in naive ordered loops, in
 * IEEE binary64 with no fused multiply-add (build with -ffp-contract=off).
 * Readings of the paper where it is silent are marked "Reading:" below.
 *
 * Parity status: every function here is pinned by a test against something
 * other than itself (closed forms, brute force, library routines, printed
 * counts); see the test files for the pin of each function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXD 3

/* ------------------------------------------------------------------------ */
/* Step 1: partition.                                                        */
/* ------------------------------------------------------------------------ */

/*
 * Core boxes split each axis a of n_cells[a] cells into n_sub[a] pieces
 * [floor(j n / p), floor((j+1) n / p)); subdomain s = sx + px*(sy + py*sz).
 * The paper's subdomains are non-overlapping (Step 1, section 2) and every cell
 * belongs to exactly one (half-open decomposition, Experiment 1.2).
 * Reading: a patch is the core grown by `overlap` cells on every side and
 * clipped to the grid; patch cells are the regression data, while ownership
 * and evaluation use the non-overlapping cores only.
 * boxes[s*12 + 0..2] core_lo, 3..5 core_hi, 6..8 patch_lo, 9..11 patch_hi
 * (cell indices, hi exclusive; axes >= dim are [0,1)).
 */
int orc_partition(int dim, const int *n_cells, const int *n_sub, int overlap,
                  int32_t *boxes)
{
    int p[ORC_MAXD] = {1, 1, 1}, n[ORC_MAXD] = {1, 1, 1};
    for (int a = 0; a < dim; ++a) { p[a] = n_sub[a]; n[a] = n_cells[a]; }
    int S = p[0] * p[1] * p[2];
    for (int s = 0; s < S; ++s) {
        int j[ORC_MAXD] = {s % p[0], (s / p[0]) % p[1], s / (p[0] * p[1])};
        for (int a = 0; a < ORC_MAXD; ++a) {
            int lo = (int)(((int64_t)j[a] * n[a]) / p[a]);
            int hi = (int)(((int64_t)(j[a] + 1) * n[a]) / p[a]);
            int ov = (a < dim) ? overlap : 0;
            int plo = lo - ov < 0 ? 0 : lo - ov;
            int phi = hi + ov > n[a] ? n[a] : hi + ov;
            boxes[s * 12 + a] = lo;
            boxes[s * 12 + 3 + a] = hi;
            boxes[s * 12 + 6 + a] = plo;
            boxes[s * 12 + 9 + a] = phi;
        }
    }
    return S;
}

/* Number of cells in box [lo, hi). */
static int64_t box_count(const int32_t *lo, const int32_t *hi)
{
    int64_t c = 1;
    for (int a = 0; a < ORC_MAXD; ++a) c *= (int64_t)(hi[a] - lo[a]);
    return c;
}

/*
 * Gather the cells of box [lo, hi) in row-major order (x fastest).
 * Sampling point x_T = cell centroid (Step 2, section 2), h = 1/max(n_cells);
 * data y_T = natural log of K_T (Remark on log K, section 3.3).
 * Returns the number of cells; x is [N][3], y, kv are [N].
 */
int64_t orc_box_cells(int dim, const int *n_cells, const int32_t *lo,
                      const int32_t *hi, const double *K, double *x, double *y,
                      double *kv)
{
    int n[ORC_MAXD] = {1, 1, 1};
    int nmax = 1;
    for (int a = 0; a < dim; ++a) { n[a] = n_cells[a]; if (n[a] > nmax) nmax = n[a]; }
    double h = 1.0 / (double)nmax;
    int64_t t = 0;
    for (int k = lo[2]; k < hi[2]; ++k)
        for (int j = lo[1]; j < hi[1]; ++j)
            for (int i = lo[0]; i < hi[0]; ++i) {
                int64_t g = (int64_t)i + (int64_t)n[0] * ((int64_t)j + (int64_t)n[1] * k);
                int idx[ORC_MAXD] = {i, j, k};
                for (int a = 0; a < ORC_MAXD; ++a)
                    x[t * 3 + a] = (a < dim) ? ((double)idx[a] + 0.5) * h : 0.0;
                kv[t] = K[g];
                y[t] = log(K[g]);
                ++t;
            }
    return t;
}

/*
 * Initial dictionary (Algorithm 1 input D): a uniform g[0] x ... lattice over
 * the core box, cell-centred: c_a = lo_a + (j + 1/2) L_a / g_a, and the width
 * sigma = the lattice spacing L_a / g_a (largest over the axes).
 * Reading: the paper puts centres on a uniform g x g lattice over the domain
 * with width tied to g (Experiment 1, Table 1: sigma = 1/g for g = 16, 32).
 * c is [M][4] = (c_x, c_y, c_z, sigma); returns M.
 */
int orc_initial_dictionary(int dim, const int *n_cells, const int32_t *core_lo,
                           const int32_t *core_hi, const int *g, double *c)
{
    int nmax = 1;
    for (int a = 0; a < dim; ++a) if (n_cells[a] > nmax) nmax = n_cells[a];
    double h = 1.0 / (double)nmax;
    int gg[ORC_MAXD] = {1, 1, 1};
    double lo[ORC_MAXD] = {0, 0, 0}, sp[ORC_MAXD] = {0, 0, 0};
    double sigma = 0.0;
    for (int a = 0; a < dim; ++a) {
        gg[a] = g[a];
        lo[a] = (double)core_lo[a] * h;
        sp[a] = ((double)(core_hi[a] - core_lo[a]) * h) / (double)g[a];
        if (sp[a] > sigma) sigma = sp[a];
    }
    int m = 0;
    for (int k = 0; k < gg[2]; ++k)
        for (int j = 0; j < gg[1]; ++j)
            for (int i = 0; i < gg[0]; ++i) {
                int idx[ORC_MAXD] = {i, j, k};
                for (int a = 0; a < ORC_MAXD; ++a)
                    c[m * 4 + a] = (a < dim) ? lo[a] + ((double)idx[a] + 0.5) * sp[a] : 0.0;
                c[m * 4 + 3] = sigma;
                ++m;
            }
    return m;
}

/* ------------------------------------------------------------------------ */
/* Step 2: feature matrix, Shepard rows, Gram products.                      */
/* ------------------------------------------------------------------------ */

/*
 * Logit of the Gaussian RBF, Eq. (6): phi_m(x) = exp(l), l = -|x - c_m|^2 /
 * (2 sigma_m^2), computed from the coordinate differences.
 */
static double rbf_logit(int dim, const double *x, const double *c)
{
    double d2 = 0.0;
    for (int a = 0; a < dim; ++a) {
        double d = x[a] - c[a];
        d2 += d * d;
    }
    double s = c[3];
    return -d2 / (2.0 * s * s);
}

/*
 * Shepard-normalised feature matrix, Eq. (10): W_jm = Phi_jm / sum_k Phi_jk.
 * Each row is evaluated as exp(l_jm - l*) / sum_k exp(l_jk - l*) with
 * l* = max_k l_jk, which is the same quotient (the common factor exp(l*)
 * cancels) but stays finite where every raw Phi_jk underflows.
 * The normaliser runs over the whole dictionary. W is [n][m] row-major.
 */
void orc_assemble(int dim, int64_t n, const double *x, int m, const double *c,
                  double *W)
{
    for (int64_t j = 0; j < n; ++j) {
        double *row = W + j * m;
        double lmax = -INFINITY;
        for (int k = 0; k < m; ++k) {
            row[k] = rbf_logit(dim, x + j * 3, c + k * 4);
            if (row[k] > lmax) lmax = row[k];
        }
        double sum = 0.0;
        for (int k = 0; k < m; ++k) {
            row[k] = exp(row[k] - lmax);
            sum += row[k];
        }
        for (int k = 0; k < m; ++k) row[k] = row[k] / sum;
    }
}

/*
 * Normal-equation data of the Elastic Net, Eq. (2), with W in place of Phi:
 * G = W^T W (m x m) and b = W^T y (naive ordered sums over the rows).
 */
void orc_gram(int64_t n, int m, const double *W, const double *y, double *G,
              double *b)
{
    for (int p = 0; p < m; ++p) {
        for (int q = 0; q < m; ++q) {
            double s = 0.0;
            for (int64_t j = 0; j < n; ++j) s += W[j * m + p] * W[j * m + q];
            G[p * m + q] = s;
        }
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) s += W[j * m + p] * y[j];
        b[p] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* Step 2: Elastic Net by coordinate descent (section 3.3), then an exact    */
/* active-set polish certified by the optimality (KKT) conditions.           */
/* ------------------------------------------------------------------------ */

static double soft_threshold(double z, double t)
{
    if (z > t) return z - t;
    if (z < -t) return z + t;
    return 0.0;
}

/* g = b - G beta */
static void gradient(int m, const double *G, const double *b, const double *beta,
                     double *g)
{
    for (int p = 0; p < m; ++p) {
        double s = 0.0;
        for (int q = 0; q < m; ++q) s += G[p * m + q] * beta[q];
        g[p] = b[p] - s;
    }
}

/*
 * Cyclic coordinate descent on
 *   F(beta) = 1/2 |y - W beta|^2 + lambda1 |beta|_1 + lambda2/2 |beta|^2,
 * written with G = W^T W and b = W^T y: coordinate j takes the exact
 * minimiser of F in beta_j with the others fixed,
 *   beta_j = S(b_j - sum_{l != j} G_jl beta_l, lambda1) / (G_jj + lambda2),
 * S the soft threshold; g = b - G beta is kept current after every change.
 * Sweeps j = 0..m-1 until max_j |delta beta_j| (G_jj + lambda2) <= tol.
 * Returns the number of sweeps made.
 */
static int cd_sweeps(int m, const double *G, const double *b, double lam1,
                     double lam2, double *beta, double *g, int max_sweeps,
                     double tol)
{
    int s;
    (void)b; /* enters through g = b - G beta, which the caller forms */
    for (s = 0; s < max_sweeps; ++s) {
        double maxd = 0.0;
        for (int j = 0; j < m; ++j) {
            double gjj = G[j * m + j];
            double z = g[j] + gjj * beta[j];
            double nb = soft_threshold(z, lam1) / (gjj + lam2);
            double d = nb - beta[j];
            if (d != 0.0) {
                for (int k = 0; k < m; ++k) g[k] -= d * G[k * m + j];
                beta[j] = nb;
                double a = fabs(d) * (gjj + lam2);
                if (a > maxd) maxd = a;
            }
        }
        if (maxd <= tol) return s + 1;
    }
    return s;
}

/* In-place Cholesky of the s x s SPD matrix A (lower triangle); 0 on success. */
static int cholesky(int s, double *A)
{
    for (int j = 0; j < s; ++j) {
        double d = A[j * s + j];
        for (int k = 0; k < j; ++k) d -= A[j * s + k] * A[j * s + k];
        if (!(d > 0.0)) return -1;
        double l = sqrt(d);
        A[j * s + j] = l;
        for (int i = j + 1; i < s; ++i) {
            double v = A[i * s + j];
            for (int k = 0; k < j; ++k) v -= A[i * s + k] * A[j * s + k];
            A[i * s + j] = v / l;
        }
    }
    return 0;
}

/* Solve L L^T x = r in place. */
static void cholesky_solve(int s, const double *L, double *r)
{
    for (int i = 0; i < s; ++i) {
        double v = r[i];
        for (int k = 0; k < i; ++k) v -= L[i * s + k] * r[k];
        r[i] = v / L[i * s + i];
    }
    for (int i = s - 1; i >= 0; --i) {
        double v = r[i];
        for (int k = i + 1; k < s; ++k) v -= L[k * s + i] * r[k];
        r[i] = v / L[i * s + i];
    }
}

/*
 * Optimality of the Elastic Net (Eq. (2)) for lambda2 > 0, where F is
 * strictly convex and its minimiser unique: beta is the minimiser iff with
 * g = b - G beta,
 *   g_j - lambda2 beta_j = lambda1 sign(beta_j)   where beta_j != 0,
 *   |g_j| <= lambda1                              where beta_j == 0.
 * Polish: take the support S and signs s of the current iterate, solve
 *   (G_SS + lambda2 I) beta_S = b_S - lambda1 s_S
 * by Cholesky, and accept only if the result keeps the signs s on S and
 * satisfies |g_j| <= lambda1 (1 + kkt_rtol) off S. On success beta is
 * overwritten with the certified minimiser and *margin receives
 * min_{j not in S} (lambda1 - |g_j|) / lambda1 (1 if S is everything).
 */
static int polish(int m, const double *G, const double *b, double lam1, double lam2,
                  double *beta, double kkt_rtol, double *margin)
{
    int *S = (int *)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
    int s = 0;
    for (int j = 0; j < m; ++j) if (beta[j] != 0.0) S[s++] = j;
    double *A = (double *)malloc(sizeof(double) * (size_t)(s > 0 ? s * s : 1));
    double *r = (double *)malloc(sizeof(double) * (size_t)(s > 0 ? s : 1));
    double *full = (double *)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
    double *g = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    int ok = 1;
    for (int p = 0; p < s; ++p) {
        for (int q = 0; q < s; ++q) A[p * s + q] = G[S[p] * m + S[q]];
        A[p * s + p] += lam2;
        double sg = beta[S[p]] > 0.0 ? 1.0 : -1.0;
        r[p] = b[S[p]] - lam1 * sg;
    }
    if (s > 0 && cholesky(s, A) != 0) ok = 0;
    if (ok && s > 0) cholesky_solve(s, A, r);
    if (ok) {
        for (int p = 0; p < s; ++p) {
            double sg = beta[S[p]] > 0.0 ? 1.0 : -1.0;
            if (!(r[p] * sg > 0.0)) { ok = 0; break; }
            full[S[p]] = r[p];
        }
    }
    double mg = 1.0;
    if (ok) {
        gradient(m, G, b, full, g);
        for (int j = 0; j < m; ++j) {
            if (full[j] != 0.0) continue;
            double mj = (lam1 - fabs(g[j])) / lam1;
            if (mj < mg) mg = mj;
            if (fabs(g[j]) > lam1 * (1.0 + kkt_rtol)) { ok = 0; break; }
        }
    }
    if (ok) {
        memcpy(beta, full, sizeof(double) * (size_t)m);
        *margin = mg;
    }
    free(S); free(A); free(r); free(full); free(g);
    return ok;
}

/*
 * Elastic Net minimiser of Eq. (2) in normal-equation form.
 * beta: in = warm start (Algorithm 1: zero, or the previous coefficients
 * extended by zeros), out = the minimiser.
 * Coordinate descent (section 3.3) runs with a tolerance that tightens by a
 * factor 100 per attempt; after each run the polish is tried, and the first
 * polish that passes the optimality check ends the solve.
 * info[0] = sweeps, info[1] = polish attempts, info[2] = KKT margin,
 * info[3] = 1 if certified, info[4] = support size.
 * Returns 0 when certified, 1 otherwise (beta then holds the CD iterate).
 */
int orc_enet(int m, const double *G, const double *b, double lam1, double lam2,
             double *beta, int max_sweeps, double *info)
{
    double *g = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double bmax = 1.0;
    for (int j = 0; j < m; ++j) if (fabs(b[j]) > bmax) bmax = fabs(b[j]);
    double tol = 1e-6 * bmax;
    int sweeps = 0, attempts = 0, ok = 0;
    double margin = 0.0;
    double *trial = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    gradient(m, G, b, beta, g);
    while (sweeps < max_sweeps) {
        sweeps += cd_sweeps(m, G, b, lam1, lam2, beta, g, max_sweeps - sweeps, tol);
        gradient(m, G, b, beta, g); /* drop the drift of the running update */
        memcpy(trial, beta, sizeof(double) * (size_t)m);
        ++attempts;
        if (polish(m, G, b, lam1, lam2, trial, 1e-9, &margin)) {
            memcpy(beta, trial, sizeof(double) * (size_t)m);
            ok = 1;
            break;
        }
        if (tol < 1e-15 * bmax) {
            /* converged as far as CD can go: keep sweeping at this tolerance */
            continue;
        }
        tol *= 1e-2;
    }
    int sup = 0;
    for (int j = 0; j < m; ++j) if (beta[j] != 0.0) ++sup;
    if (info) {
        info[0] = sweeps; info[1] = attempts; info[2] = margin;
        info[3] = ok; info[4] = sup;
    }
    free(g); free(trial);
    return ok ? 0 : 1;
}

/* Elastic Net objective, Eq. (2), in normal-equation form (plus the constant
 * 1/2 y^T y, passed as yty). */
double orc_enet_objective(int m, const double *G, const double *b, double yty,
                          double lam1, double lam2, const double *beta)
{
    double quad = 0.0, lin = 0.0, l1 = 0.0, l2 = 0.0;
    for (int p = 0; p < m; ++p) {
        double s = 0.0;
        for (int q = 0; q < m; ++q) s += G[p * m + q] * beta[q];
        quad += beta[p] * s;
        lin += b[p] * beta[p];
        l1 += fabs(beta[p]);
        l2 += beta[p] * beta[p];
    }
    return 0.5 * yty - lin + 0.5 * quad + lam1 * l1 + 0.5 * lam2 * l2;
}

/* ------------------------------------------------------------------------ */
/* Step 3: residual indicators, marking, enrichment (Algorithm 1 (2)-(5)).   */
/* ------------------------------------------------------------------------ */

/*
 * Elementwise indicator, Eq. (4): R_T = sum_l w_T^l (K*(x_T^l) - K_T)^2 with
 * K* = exp(W beta) at the data points.
 * Reading: the quadrature rule is unspecified; this is the one-point
 * midpoint rule (x_T^1 = centroid, w_T^1 = |T|). R_T is taken in K space
 * as written, not in log space.
 */
void orc_residual(int64_t n, int m, const double *W, const double *beta,
                  const double *kv, double vol, double *R)
{
    for (int64_t j = 0; j < n; ++j) {
        double t = 0.0;
        for (int k = 0; k < m; ++k) t += W[j * m + k] * beta[k];
        double e = exp(t) - kv[j];
        R[j] = vol * (e * e);
    }
}

/*
 * The same indicator for cells of unequal measure: R_T = |T| (K*(x_T) - K_T)^2
 * with |T| = vol[j] (the midpoint rule on each cell, Eq. (4)).
 */
void orc_residual_cells(int64_t n, int m, const double *W, const double *beta,
                        const double *kv, const double *vol, double *R)
{
    for (int64_t j = 0; j < n; ++j) {
        double t = 0.0;
        for (int k = 0; k < m; ++k) t += W[j * m + k] * beta[k];
        double e = exp(t) - kv[j];
        R[j] = vol[j] * (e * e);
    }
}

/*
 * Two-point Gauss-Legendre rule per axis on a cell of side h centred at x
 * (the tensor rule has 2^dim nodes, each of weight |T| / 2^dim): node q has
 * x_a + s h / (2 sqrt(3)) on axis a, s = -1 if bit a of q is clear else +1.
 * It integrates every polynomial of degree <= 3 in each variable exactly.
 */
void orc_gl_points(int dim, const double *x, double h, double *pts)
{
    const double off = 0.5 * h / sqrt(3.0);
    for (int q = 0; q < (1 << dim); ++q)
        for (int a = 0; a < dim; ++a)
            pts[q * dim + a] = x[a] + (((q >> a) & 1) ? off : -off);
}

/*
 * Eq. (4) with the 2^dim-point Gauss-Legendre rule instead of the midpoint:
 * R_T = sum_q (|T| / 2^dim) (K*(x_T^q) - K_T)^2, K* = exp(W(x) beta) with the
 * Shepard row W(x) of the subdomain's whole dictionary at each node.
 */
void orc_residual_gl(int dim, int64_t n, const double *x, int m, const double *c,
                     const double *beta, const double *kv, double vol, double h, double *R)
{
    const int nq = 1 << dim;
    double pts[8 * ORC_MAXD];
    double *Wq = (double *)malloc(sizeof(double) * (size_t)nq * (size_t)(m > 0 ? m : 1));
    for (int64_t j = 0; j < n; ++j) {
        orc_gl_points(dim, x + j * 3, h, pts);
        double pq[8 * 3];
        for (int q = 0; q < nq; ++q)
            for (int a = 0; a < 3; ++a) pq[q * 3 + a] = a < dim ? pts[q * dim + a] : 0.0;
        orc_assemble(dim, nq, pq, m, c, Wq);
        double r = 0.0;
        for (int q = 0; q < nq; ++q) {
            double t = 0.0;
            for (int k = 0; k < m; ++k) t += Wq[q * m + k] * beta[k];
            double e = exp(t) - kv[j];
            r += (vol / (double)nq) * (e * e);
        }
        R[j] = r;
    }
    free(Wq);
}

/*
 * Algorithm 1 (3): E_worst = the k_top cells with the largest R_T.
 * Reading: only cells with R_T >= eps_tol are candidates (so "E_worst empty"
 * is reachable and equals the tolerance stop max R_T < eps_tol); cells are
 * ranked by R_T rounded to binary32 and ties go to the lower local cell
 * index, so that a rounding-order difference below 2^-24 relative cannot
 * reorder cells whose indicators agree. marked[] receives the local indices
 * in rank order; returns how many (<= k_top).
 */
static int mark_impl(int64_t n, const double *R, double eps_tol, const double *eps_cell, int k_top,
                     int32_t *marked)
{
    int cnt = 0;
    for (int t = 0; t < k_top; ++t) {
        int64_t best = -1;
        float bk = 0.0f;
        for (int64_t j = 0; j < n; ++j) {
            float kj = (float)R[j];
            float ek = (float)(eps_cell ? eps_cell[j] : eps_tol);
            if (!(kj >= ek)) continue;
            int taken = 0;
            for (int u = 0; u < cnt; ++u) if (marked[u] == j) { taken = 1; break; }
            if (taken) continue;
            if (best < 0 || kj > bk) { best = j; bk = kj; }
        }
        if (best < 0) break;
        marked[cnt++] = (int32_t)best;
    }
    return cnt;
}

int orc_mark(int64_t n, const double *R, double eps_tol, int k_top, int32_t *marked)
{
    return mark_impl(n, R, eps_tol, NULL, k_top, marked);
}

/*
 * The same marking with a threshold per cell, eps_cell[j] (cells of unequal
 * measure: eps_T = |T| (eps_tol_rel max K)^2, so that R_T >= eps_T says
 * |K*(x_T) - K_T| >= eps_tol_rel max K whatever the cell's size).
 */
int orc_mark_cells(int64_t n, const double *R, const double *eps_cell, int k_top, int32_t *marked)
{
    return mark_impl(n, R, 0.0, eps_cell, k_top, marked);
}

/* Unit directions of the new centres, the d+1 vertices of a regular simplex
 * centred at the origin (fixed orientation). */
static void simplex_direction(int dim, int q, double *u)
{
    u[0] = u[1] = u[2] = 0.0;
    if (dim == 1) {
        u[0] = (q == 0) ? 1.0 : -1.0;
    } else if (dim == 2) {
        /* angles 90 + 120 (q+1) degrees: 210, 330, 90 */
        const double c30 = 0.86602540378443864676; /* cos 30 deg = sqrt(3)/2 */
        if (q == 0) { u[0] = -c30; u[1] = -0.5; }
        else if (q == 1) { u[0] = c30; u[1] = -0.5; }
        else { u[0] = 0.0; u[1] = 1.0; }
    } else {
        const double r3 = 0.57735026918962576451; /* 1/sqrt(3) */
        static const int sg[4][3] = {{1, 1, 1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
        for (int a = 0; a < 3; ++a) u[a] = (double)sg[q][a] * r3;
    }
}

/*
 * Algorithm 1 (4)-(5) and the refinement rule of section 3.4: for each marked
 * cell T (in rank order) add new centres near the centre nearest to x_T with
 * width eta * sigma_parent, eta in (0,1).
 * Reading: the paper fixes only the width rule (eta = 1/2 in its
 * experiments) and, through Table 2 (+612 = 3 x 204 per round in 2-D), that
 * every marked cell adds d+1 centres with no de-duplication. The positions
 * are ours: parent p = the current centre nearest to x_T (ties to the lower
 * index; "current" = the dictionary the residuals were computed with), new
 * centres x_T + eta sigma_p u_q on the d+1 simplex directions u_q, each
 * coordinate clipped to the patch extent [plo, phi].
 * c holds m entries on entry and receives the appended ones; at most
 * m_limit entries in total (the cap M_i + M_max of Algorithm 1).
 * Returns the new size.
 */
int orc_enrich(int dim, int m, double *c, int n_marked, const int32_t *marked,
               const double *x, const double *plo, const double *phi, double eta,
               int m_limit)
{
    int m0 = m, mm = m;
    for (int t = 0; t < n_marked; ++t) {
        const double *xt = x + (int64_t)marked[t] * 3;
        int best = 0;
        double bd = INFINITY;
        for (int k = 0; k < m0; ++k) {
            double d2 = 0.0;
            for (int a = 0; a < dim; ++a) {
                double d = xt[a] - c[k * 4 + a];
                d2 += d * d;
            }
            if (d2 < bd) { bd = d2; best = k; }
        }
        double sn = eta * c[best * 4 + 3];
        for (int q = 0; q <= dim; ++q) {
            if (mm >= m_limit) return mm;
            double u[3];
            simplex_direction(dim, q, u);
            for (int a = 0; a < 3; ++a) {
                double v = 0.0;
                if (a < dim) {
                    v = xt[a] + sn * u[a];
                    if (v < plo[a]) v = plo[a];
                    if (v > phi[a]) v = phi[a];
                }
                c[mm * 4 + a] = v;
            }
            c[mm * 4 + 3] = sn;
            ++mm;
        }
    }
    return mm;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 on one subdomain, and on all subdomains.                      */
/* ------------------------------------------------------------------------ */

typedef struct {
    double lambda1_hat, lambda2_hat; /* lambda_k = N_i * lambda_k_hat */
    double eps_tol_rel;              /* eps_tol = |T| (eps_tol_rel max K)^2; <0: no filter */
    double eta;
    int k_top, m_max, levels, max_sweeps;
    int quad; /* R_T quadrature: 0 midpoint, 1 2^dim-point Gauss-Legendre */
} orc_params;

/* Per-subdomain diagnostics written by orc_fit_subdomain. */
#define ORC_NINFO 8 /* M, support, levels done, certified, min margin, sweeps, n cells, max R */

/*
 * Algorithm 1 for subdomain s. Inputs: the grid field K (x fastest), the
 * subdomain's box row, its initial dictionary (c0, m0 entries), params.
 * Outputs: c [m_cap][4] (final dictionary), beta [m_cap], info [ORC_NINFO].
 * Reading on the loop: the coefficients are re-solved after the last
 * enrichment (Table 2 lists the error of every enlarged dictionary), so the
 * loop is  solve -> (stop?) -> indicators -> mark -> enrich -> solve ...
 * and it stops after `levels` enrichments, when nothing is marked, or when
 * the size reaches m0 + m_max.
 * Reading on lambda: the printed values (Example 2) are per-sample weights,
 * lambda_k = N_i * lambda_k_hat for a patch of N_i cells.
 */
/*
 * Algorithm 1 on one patch given as cells: sampling points x [N][3]
 * (unused axes 0), y = ln K, kv = K, measures vol [N] (|T|), the patch
 * extent [ext_lo, ext_hi] that new centres are clipped to, the initial
 * dictionary (c0, m0). quad = 1 (grid cells of side h only) takes the
 * Gauss-Legendre indicators. eps_T = |T| (eps_tol_rel max K)^2 per cell.
 */
static int fit_patch(int dim, int64_t N, const double *x, const double *y, const double *kv,
                     const double *vol, const double *ext_lo, const double *ext_hi, int quad, double h,
                     const double *c0, int m0, const orc_params *P, int m_cap, double *c, double *beta,
                     double *info)
{
    /* Reading: a patch without elements (a mesh with a hole) has no data and,
     * with lambda_k = N lambda_k_hat, no penalty; its coefficients are the
     * limit of the unique minimisers as lambda -> 0+ with G = 0, b = 0, i.e.
     * beta = 0, and Algorithm 1 stops at once. */
    if (N == 0) {
        memset(c, 0, sizeof(double) * (size_t)m_cap * 4);
        memset(beta, 0, sizeof(double) * (size_t)m_cap);
        memcpy(c, c0, sizeof(double) * (size_t)m0 * 4);
        info[0] = m0; info[1] = 0; info[2] = 0; info[3] = 1;
        info[4] = 1.0; info[5] = 0; info[6] = 0; info[7] = 0;
        return 0;
    }
    double kmax = 0.0;
    for (int64_t j = 0; j < N; ++j) if (kv[j] > kmax) kmax = kv[j];
    double *eps = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    for (int64_t j = 0; j < N; ++j)
        eps[j] = P->eps_tol_rel < 0 ? -INFINITY
                                    : vol[j] * (P->eps_tol_rel * kmax) * (P->eps_tol_rel * kmax);
    double lam1 = (double)N * P->lambda1_hat, lam2 = (double)N * P->lambda2_hat;
    int m_limit = m0 + P->m_max;
    if (m_limit > m_cap) m_limit = m_cap;

    memset(c, 0, sizeof(double) * (size_t)m_cap * 4);
    memset(beta, 0, sizeof(double) * (size_t)m_cap);
    memcpy(c, c0, sizeof(double) * (size_t)m0 * 4);
    int m = m0, level = 0, certified = 1, sweeps = 0;
    double min_margin = 1.0, maxR = 0.0;
    double *W = (double *)malloc(sizeof(double) * (size_t)N * (size_t)m_cap);
    double *G = (double *)malloc(sizeof(double) * (size_t)m_cap * (size_t)m_cap);
    double *b = (double *)malloc(sizeof(double) * (size_t)m_cap);
    double *R = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    int32_t *mk = (int32_t *)malloc(sizeof(int32_t) * (size_t)(P->k_top > 0 ? P->k_top : 1));
    for (;;) {
        double inf[5];
        orc_assemble(dim, N, x, m, c, W);
        orc_gram(N, m, W, y, G, b);
        if (orc_enet(m, G, b, lam1, lam2, beta, P->max_sweeps, inf) != 0) certified = 0;
        sweeps += (int)inf[0];
        if (inf[2] < min_margin) min_margin = inf[2];
        if (quad) orc_residual_gl(dim, N, x, m, c, beta, kv, vol[0], h, R);
        else orc_residual_cells(N, m, W, beta, kv, vol, R);
        maxR = 0.0;
        for (int64_t j = 0; j < N; ++j) if (R[j] > maxR) maxR = R[j];
        if (level >= P->levels || m >= m_limit) break;
        int nm = orc_mark_cells(N, R, eps, P->k_top, mk);
        if (nm == 0) break;
        int m_new = orc_enrich(dim, m, c, nm, mk, x, ext_lo, ext_hi, P->eta, m_limit);
        if (m_new == m) break;
        m = m_new; /* beta[m_old..m_new) stays zero: the zero extension */
        ++level;
    }
    int sup = 0;
    for (int k = 0; k < m; ++k) if (beta[k] != 0.0) ++sup;
    info[0] = m; info[1] = sup; info[2] = level; info[3] = certified;
    info[4] = min_margin; info[5] = sweeps; info[6] = (double)N; info[7] = maxR;
    free(eps); free(W); free(G); free(b); free(R); free(mk);
    return certified ? 0 : 1;
}

int orc_fit_subdomain(int dim, const int *n_cells, const double *K,
                      const int32_t *box, const double *c0, int m0,
                      const orc_params *P, int m_cap, double *c, double *beta,
                      double *info)
{
    const int32_t *plo = box + 6, *phi = box + 9;
    int64_t N = box_count(plo, phi);
    int nmax = 1;
    for (int a = 0; a < dim; ++a) if (n_cells[a] > nmax) nmax = n_cells[a];
    double h = 1.0 / (double)nmax, vol = 1.0;
    for (int a = 0; a < dim; ++a) vol *= h;
    double ext_lo[3] = {0, 0, 0}, ext_hi[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) { ext_lo[a] = plo[a] * h; ext_hi[a] = phi[a] * h; }

    double *x = (double *)malloc(sizeof(double) * (size_t)N * 3);
    double *y = (double *)malloc(sizeof(double) * (size_t)N);
    double *kv = (double *)malloc(sizeof(double) * (size_t)N);
    double *vc = (double *)malloc(sizeof(double) * (size_t)N);
    orc_box_cells(dim, n_cells, plo, phi, K, x, y, kv);
    for (int64_t j = 0; j < N; ++j) vc[j] = vol;
    int r = fit_patch(dim, N, x, y, kv, vc, ext_lo, ext_hi, P->quad, h, c0, m0, P, m_cap, c, beta, info);
    free(x); free(y); free(kv); free(vc);
    return r;
}

/*
 * Algorithm 1 on a subdomain whose patch is a list of cells of a general
 * (unstructured) mesh, section 2: each element T contributes its sampling
 * point x_T (e.g. its centroid), its value K_T and its measure |T|.
 * Inputs: all cells' points xs [n][dim], values Ks [n], measures vols [n];
 * the patch's cell indices cells[0..N) (ascending: the local order); the
 * subdomain's box row (core box for the initial dictionary, patch box for
 * the extent of new centres, in units of h = 1/max n_cells).
 */
int orc_fit_cells_subdomain(int dim, const int *n_cells, const double *xs, const double *Ks,
                            const double *vols, const int32_t *cells, int64_t N, const int32_t *box,
                            const double *c0, int m0, const orc_params *P, int m_cap, double *c,
                            double *beta, double *info)
{
    int nmax = 1;
    for (int a = 0; a < dim; ++a) if (n_cells[a] > nmax) nmax = n_cells[a];
    double h = 1.0 / (double)nmax;
    double ext_lo[3] = {0, 0, 0}, ext_hi[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) { ext_lo[a] = box[6 + a] * h; ext_hi[a] = box[9 + a] * h; }
    double *x = (double *)calloc((size_t)(N > 0 ? N : 1) * 3, sizeof(double));
    double *y = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    double *kv = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    double *vc = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    for (int64_t j = 0; j < N; ++j) {
        int64_t t = cells[j];
        for (int a = 0; a < dim; ++a) x[j * 3 + a] = xs[t * dim + a];
        kv[j] = Ks[t];
        y[j] = log(Ks[t]);
        vc[j] = vols[t];
    }
    orc_params Q = *P;
    Q.quad = 0; /* element shapes are not given: the midpoint rule */
    int r = fit_patch(dim, N, x, y, kv, vc, ext_lo, ext_hi, 0, h, c0, m0, &Q, m_cap, c, beta, info);
    free(x); free(y); free(kv); free(vc);
    return r;
}

/*
 * Algorithm 1 on every subdomain (Step 2-3 of section 2); the subdomains are
 * independent, so they are spread over OpenMP threads. Each subdomain starts
 * from the uniform g-lattice of its core box. boxes from orc_partition;
 * the subset `which` (n_which entries, or all when which == NULL) is fitted.
 * Outputs per fitted subdomain s: c[s][m_cap][4], beta[s][m_cap],
 * info[s][ORC_NINFO]. Returns the number that failed to certify.
 */
int orc_fit_all(int dim, const int *n_cells, const double *K, int S,
                const int32_t *boxes, const int *g, const orc_params *P,
                int m_cap, const int32_t *which, int n_which, double *c,
                double *beta, double *info)
{
    int failed = 0;
    int count = which ? n_which : S;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : failed)
    for (int t = 0; t < count; ++t) {
        int s = which ? which[t] : t;
        double *c0 = (double *)malloc(sizeof(double) * (size_t)m_cap * 4);
        int m0 = orc_initial_dictionary(dim, n_cells, boxes + s * 12, boxes + s * 12 + 3, g, c0);
        failed += orc_fit_subdomain(dim, n_cells, K, boxes + s * 12, c0, m0, P, m_cap,
                                    c + (int64_t)s * m_cap * 4, beta + (int64_t)s * m_cap,
                                    info + (int64_t)s * ORC_NINFO);
        free(c0);
    }
    return failed;
}

/*
 * orc_fit_all for a mesh given as cells: patch s holds the cells
 * patch_cells[patch_start[s] .. patch_start[s+1]).
 */
int orc_fit_cells_all(int dim, const int *n_cells, const double *xs, const double *Ks, const double *vols,
                      int S, const int32_t *boxes, const int64_t *patch_start, const int32_t *patch_cells,
                      const int *g, const orc_params *P, int m_cap, const int32_t *which, int n_which,
                      double *c, double *beta, double *info)
{
    int failed = 0;
    int count = which ? n_which : S;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : failed)
    for (int t = 0; t < count; ++t) {
        int s = which ? which[t] : t;
        double *c0 = (double *)malloc(sizeof(double) * (size_t)m_cap * 4);
        int m0 = orc_initial_dictionary(dim, n_cells, boxes + s * 12, boxes + s * 12 + 3, g, c0);
        failed += orc_fit_cells_subdomain(dim, n_cells, xs, Ks, vols, patch_cells + patch_start[s],
                                          patch_start[s + 1] - patch_start[s], boxes + s * 12, c0, m0, P,
                                          m_cap, c + (int64_t)s * m_cap * 4, beta + (int64_t)s * m_cap,
                                          info + (int64_t)s * ORC_NINFO);
        free(c0);
    }
    return failed;
}

/* ------------------------------------------------------------------------ */
/* Step 4: global reconstruction, and the error measures.                    */
/* ------------------------------------------------------------------------ */

/*
 * Owner of point x: K*(x) = K*_{omega_i}(x) for x in omega_i (Step 4).
 * The cores are half-open boxes [lo h, hi h) with the outer face of the grid
 * closed. The cell coordinate u = x * max(n) is floored to a cell index, so
 * the decision uses one exact multiply by an integer. Returns -1 outside
 * the closed domain.
 */
static int owner_of(int dim, const int *n_cells, const int *n_sub, const double *x)
{
    int nmax = 1;
    for (int a = 0; a < dim; ++a) if (n_cells[a] > nmax) nmax = n_cells[a];
    int j[ORC_MAXD] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) {
        double u = x[a] * (double)nmax;
        if (!(u >= 0.0) || u > (double)n_cells[a]) return -1;
        int64_t i = (int64_t)floor(u);
        if (i >= n_cells[a]) i = n_cells[a] - 1;
        int p = n_sub[a];
        int jj = 0;
        for (int q = 0; q < p; ++q) {
            int64_t lo = ((int64_t)q * n_cells[a]) / p, hi = ((int64_t)(q + 1) * n_cells[a]) / p;
            if (i >= lo && i < hi) { jj = q; break; }
        }
        j[a] = jj;
    }
    int p0 = n_sub[0], p1 = dim > 1 ? n_sub[1] : 1;
    return j[0] + p0 * (j[1] + p1 * j[2]);
}

/*
 * Local surrogate on the Shepard basis, Eq. (3) with the weights of Eq. (9):
 * log-space value sum_m beta_m w_m(x) over the whole dictionary of the owner,
 * K*(x) = exp of it (Remark on log K, section 3.3). out[p] = K*(x_p), or the
 * log-space value when log_space != 0; NaN for points outside the domain.
 * owner_out (optional) receives the owner index.
 */
void orc_eval(int dim, const int *n_cells, const int *n_sub, int m_cap,
              const int32_t *M, const double *c, const double *beta, int64_t n_pts,
              const double *pts, int log_space, double *out, int32_t *owner_out)
{
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n_pts; ++p) {
        double xp[3] = {0, 0, 0};
        for (int a = 0; a < dim; ++a) xp[a] = pts[p * dim + a];
        int s = owner_of(dim, n_cells, n_sub, xp);
        if (owner_out) owner_out[p] = s;
        if (s < 0) { out[p] = NAN; continue; }
        const double *cs = c + (int64_t)s * m_cap * 4;
        const double *bs = beta + (int64_t)s * m_cap;
        int m = M[s];
        double lmax = -INFINITY;
        for (int k = 0; k < m; ++k) {
            double l = rbf_logit(dim, xp, cs + k * 4);
            if (l > lmax) lmax = l;
        }
        double num = 0.0, den = 0.0;
        for (int k = 0; k < m; ++k) {
            double e = exp(rbf_logit(dim, xp, cs + k * 4) - lmax);
            num += bs[k] * e;
            den += e;
        }
        double v = num / den;
        out[p] = log_space ? v : exp(v);
    }
}

/*
 * Relative errors of the reconstruction over the source cells, each cell
 * measured with its owner's surrogate, by the midpoint rule (quad = 0: the
 * centroid) or the 2^dim-point Gauss-Legendre rule (quad = 1: the nodes of
 * orc_gl_points, weight 1/2^dim of the cell each, all inside the cell and
 * so owned by the cell's subdomain):
 *   err[0] = L1 in K:   sum_T sum_q w_q |K_T - K*(x_q)| / sum |T| |K_T|
 *   err[1] = L2 in K:   Eq. (12), (sum w_q (K_T - K*)^2 / sum |T| K_T^2)^(1/2)
 *   err[2] = L1 in log: sum w_q |ln K_T - ln K*(x_q)| / sum |T| |ln K_T|
 *   err[3] = max over the points of |log10 K_T - log10 K*(x_q)|
 */
void orc_errors(int dim, const int *n_cells, const int *n_sub, int m_cap,
                const int32_t *M, const double *c, const double *beta,
                const double *K, int quad, double *err)
{
    int n[ORC_MAXD] = {1, 1, 1}, nmax = 1;
    for (int a = 0; a < dim; ++a) { n[a] = n_cells[a]; if (n[a] > nmax) nmax = n[a]; }
    double h = 1.0 / (double)nmax;
    const int nq = quad ? (1 << dim) : 1;
    int64_t total = (int64_t)n[0] * n[1] * n[2];
    double *x = (double *)malloc(sizeof(double) * (size_t)total * (size_t)nq * (size_t)dim);
    double *v = (double *)malloc(sizeof(double) * (size_t)total * (size_t)nq);
    for (int64_t g = 0; g < total; ++g) {
        int64_t idx[3] = {g % n[0], (g / n[0]) % n[1], g / ((int64_t)n[0] * n[1])};
        double xc[ORC_MAXD];
        for (int a = 0; a < dim; ++a) xc[a] = ((double)idx[a] + 0.5) * h;
        if (quad) orc_gl_points(dim, xc, h, x + g * nq * dim);
        else for (int a = 0; a < dim; ++a) x[g * dim + a] = xc[a];
    }
    orc_eval(dim, n_cells, n_sub, m_cap, M, c, beta, total * nq, x, 1, v, NULL);
    double a1 = 0, b1 = 0, a2 = 0, b2 = 0, al = 0, bl = 0, mx = 0;
    for (int64_t g = 0; g < total; ++g) {
        double lk = log(K[g]);
        b1 += fabs(K[g]); b2 += K[g] * K[g]; bl += fabs(lk);
        for (int q = 0; q < nq; ++q) {
            double vq = v[g * nq + q], ks = exp(vq), w = 1.0 / (double)nq;
            a1 += w * fabs(K[g] - ks);
            a2 += w * (K[g] - ks) * (K[g] - ks);
            al += w * fabs(lk - vq);
            double d = fabs(lk - vq) / log(10.0);
            if (d > mx) mx = d;
        }
    }
    err[0] = a1 / b1;
    err[1] = sqrt(a2 / b2);
    err[2] = bl > 0 ? al / bl : al;
    err[3] = mx;
    free(x); free(v);
}

/* Threads of the OpenMP loops over subdomains and points, for timing the
 * oracle on a given number of host cores: n > 0 sets the count for the
 * calling thread's later loops; returns the count in effect. */
int orc_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
