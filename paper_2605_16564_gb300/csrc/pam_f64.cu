// pam_f64.cu -- the plain (binary64) form of the PAM fitting path on sm_103a,
// plus the precision-independent kernels (partition, cell preparation,
// dictionary set-up, marking/enrichment, evaluation, errors).
//
// Data layout in HBM (per subdomain s, strides from the plan):
//   cells:   y = ln K, kv = K, inv_s, R  [S][n_max]   (patch order, x fastest)
//   E        [S][m_cap][n_max]  exp(l_jm - l_j*), transposed so that the
//            cell index is contiguous (coalesced along threads = cells)
//   G        [S][m_cap][m_cap]  W^T W, both triangles
//   b        [S][m_cap]         W^T y
//   model    centres [S][m_cap][4] = (c, sigma), beta [S][m_cap]
#include <cfloat>
#include <cmath>

#include "pam_internal.cuh"

namespace pam {

// --------------------------------------------------------------------------
// Step 1 on the device: core and patch boxes (same rule as pam_partition).
// --------------------------------------------------------------------------
__global__ void k_partition(Geo g, int32_t *boxes) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.S) return;
    int j[3] = {s % g.p[0], (s / g.p[0]) % g.p[1], s / (g.p[0] * g.p[1])};
    for (int a = 0; a < 3; ++a) {
        int lo = (int)(((int64_t)j[a] * g.n[a]) / g.p[a]);
        int hi = (int)(((int64_t)(j[a] + 1) * g.n[a]) / g.p[a]);
        int ov = a < g.dim ? g.overlap : 0;
        boxes[s * 12 + a] = lo;
        boxes[s * 12 + 3 + a] = hi;
        boxes[s * 12 + 6 + a] = lo - ov < 0 ? 0 : lo - ov;
        boxes[s * 12 + 9 + a] = hi + ov > g.n[a] ? g.n[a] : hi + ov;
    }
}

void launch_partition(const Geo &g, int32_t *boxes, cudaStream_t st) {
    k_partition<<<(g.S + 127) / 128, 128, 0, st>>>(g, boxes);
    count_launches(1);
}

// --------------------------------------------------------------------------
// Patch cell data: y = ln K (Remark on log K, section 3.3), K, the patch
// maximum of K, and the input check K > 0 finite.
// --------------------------------------------------------------------------
__global__ void k_prepare(Geo g, const int32_t *boxes, const double *K, Ws w) {
    int s = blockIdx.y;
    const int32_t *box = boxes + s * 12;
    int ext[3];
    patch_extent(box, ext);
    int N = ext[0] * ext[1] * ext[2];
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    double kmax = 0.0;
    if (t < g.n_max) {
        size_t o = (size_t)s * g.n_max + t;
        if (t < N) {
            double x[3];
            int64_t gi;
            patch_cell(g, box, t, x, &gi);
            double k = K[gi];
            if (!(k > 0.0) || !(k <= DBL_MAX)) {
                atomicAdd(&w.status[kStBadK], 1);
                k = 1.0;
            }
            w.kv[o] = k;  // y = ln K: written by k_prepare_log, once per grid cell
            kmax = k;
        } else {
            w.y[o] = 0.0;
            w.kv[o] = 0.0;
        }
    }
    // positive doubles order like their bit patterns
    double m = warp_max(kmax);
    if ((threadIdx.x & 31) == 0 && m > 0.0)
        atomicMax(&w.kmax_bits[s], (unsigned long long)__double_as_longlong(m));
}

// y = ln K of every patch cell, the binary64 log taken once per grid cell
// and written to each patch that holds the cell (the patches overlap, so a
// cell sits in about two on this grid; the log is most of the set-up's cost
// on this part's narrow binary64 pipe). Along axis a the patches holding
// cell i are those of the cores meeting [i - overlap, i + overlap], with the
// boxes of pam_partition (core j: [j n / p, (j + 1) n / p), floor division,
// patch: the core widened by the overlap and clipped). A bad K (<= 0, NaN,
// Inf) gives y = 0, as k_prepare's substitute K = 1 did; k_prepare counts it.
__global__ void k_prepare_log(Geo g, const double *K, Ws w) {
    const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= (int64_t)g.n[0] * g.n[1] * g.n[2]) return;
    const int idx[3] = {(int)(gi % g.n[0]), (int)((gi / g.n[0]) % g.n[1]),
                        (int)(gi / ((int64_t)g.n[0] * g.n[1]))};
    const double k = K[gi];
    const double y = (k > 0.0 && k <= DBL_MAX) ? log(k) : 0.0;
    int jlo[3], jhi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int ov = a < g.dim ? g.overlap : 0;
        jlo[a] = core_of(max(0, idx[a] - ov), g.n[a], g.p[a]);
        jhi[a] = core_of(min(g.n[a] - 1, idx[a] + ov), g.n[a], g.p[a]);
    }
    // the patch box along axis a of core j: [lo, hi) and the cell's offset
    auto patch = [&](int a, int j, int *plo, int *pw) {
        const int ov = a < g.dim ? g.overlap : 0, n = g.n[a], p = g.p[a];
        const int lo = (int)(((int64_t)j * n) / p), hi = (int)(((int64_t)(j + 1) * n) / p);
        *plo = lo - ov < 0 ? 0 : lo - ov;
        *pw = (hi + ov > n ? n : hi + ov) - *plo;
    };
    for (int jz = jlo[2]; jz <= jhi[2]; ++jz) {
        int pz, wz;
        patch(2, jz, &pz, &wz);
        const int oz = idx[2] - pz;
        if (oz < 0 || oz >= wz) continue;
        for (int jy = jlo[1]; jy <= jhi[1]; ++jy) {
            int py, wy;
            patch(1, jy, &py, &wy);
            const int oy = idx[1] - py;
            if (oy < 0 || oy >= wy) continue;
            for (int jx = jlo[0]; jx <= jhi[0]; ++jx) {
                int px, wx;
                patch(0, jx, &px, &wx);
                const int ox = idx[0] - px;
                if (ox < 0 || ox >= wx) continue;
                const int s = jx + g.p[0] * (jy + g.p[1] * jz);
                w.y[(size_t)s * g.n_max + ox + wx * (oy + wy * oz)] = y;
            }
        }
    }
}

// The same for a mesh given as cells: patch cell t of subdomain s is element
// pcells[pstart[s] + t]; its sampling point and measure are gathered into
// the workspace beside y and K (a measure <= 0, NaN or Inf is an input
// fault like a bad K_T).
__global__ void k_prepare_cells(Geo g, const double *K, Ws w) {
    const int s = blockIdx.y;
    const int b = g.pstart[s], N = g.pstart[s + 1] - b;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double kmax = 0.0;
    if (t < g.n_max) {
        const size_t o = (size_t)s * g.n_max + t;
        double4_32a v;
        v.x = v.y = v.z = v.w = 0.0;
        if (t < N) {
            const int64_t e = g.pcells[b + t];
            double k = K[e];
            double vol = g.cvol[e];
            if (!(k > 0.0) || !(k <= DBL_MAX) || !(vol > 0.0) || !(vol <= DBL_MAX)) {
                atomicAdd(&w.status[kStBadK], 1);
                k = 1.0;
                vol = g.vol;
            }
            v.x = g.cx[e * g.dim];
            if (g.dim > 1) v.y = g.cx[e * g.dim + 1];
            if (g.dim > 2) v.z = g.cx[e * g.dim + 2];
            v.w = vol;
            w.y[o] = log(k);
            w.kv[o] = k;
            kmax = k;
        } else {
            w.y[o] = 0.0;
            w.kv[o] = 0.0;
        }
        w.cxv[o] = v;
    }
    double m = warp_max(kmax);
    if ((threadIdx.x & 31) == 0 && m > 0.0)
        atomicMax(&w.kmax_bits[s], (unsigned long long)__double_as_longlong(m));
}

void launch_prepare(const Geo &g, const int32_t *boxes, const double *K, const Ws &w,
                    cudaStream_t st) {
    PhaseScope ps(kPhPrepare, st);
    cudaMemsetAsync(w.kmax_bits, 0, sizeof(unsigned long long) * g.S, st);
    dim3 grid((g.n_max + 255) / 256, g.S);
    if (g.cells) {
        k_prepare_cells<<<grid, 256, 0, st>>>(g, K, w);
        count_launches(1);
    } else {
        const int64_t n = (int64_t)g.n[0] * g.n[1] * g.n[2];
        k_prepare_log<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, K, w);
        k_prepare<<<grid, 256, 0, st>>>(g, boxes, K, w);
        count_launches(2);
    }
}

// --------------------------------------------------------------------------
// Initial dictionary (Algorithm 1 input): a uniform g lattice over each core
// box, cell-centred, sigma = the lattice spacing (largest over the axes).
// --------------------------------------------------------------------------
__global__ void k_init_dictionary(Geo g, const int32_t *boxes, double *centres, double *beta,
                                  int32_t *info, int keep_beta) {
    int s = blockIdx.y;
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t *box = boxes + s * 12;
    if (m < g.m_cap) {
        double *c = centres + ((size_t)s * g.m_cap + m) * 4;
        if (m < g.m0) {
            // the lattice's origin, spacing and width (binary64 divisions:
            // only the lattice's own threads compute them)
            double lo[3] = {0, 0, 0}, sp[3] = {0, 0, 0};
            double sigma = 0.0;
            for (int a = 0; a < g.dim; ++a) {
                lo[a] = __dmul_rn((double)box[a], g.h);
                sp[a] = __ddiv_rn(__dmul_rn((double)(box[3 + a] - box[a]), g.h), (double)g.g[a]);
                sigma = fmax(sigma, sp[a]);
            }
            int idx[3] = {m % g.g[0], (m / g.g[0]) % g.g[1], m / (g.g[0] * g.g[1])};
            for (int a = 0; a < 3; ++a)
                c[a] = a < g.dim ? __dadd_rn(lo[a], __dmul_rn((double)idx[a] + 0.5, sp[a])) : 0.0;
            c[3] = sigma;
        } else {
            c[0] = c[1] = c[2] = c[3] = 0.0;
        }
        // a warm start keeps the caller's coefficients of the initial lattice;
        // a patch without elements (a mesh given as cells, e.g. with a hole)
        // has no data: beta = 0
        const bool empty = g.cells && g.pstart[s + 1] == g.pstart[s];
        if (!keep_beta || m >= g.m0 || empty) beta[(size_t)s * g.m_cap + m] = 0.0;
    }
    if (m == 0) {
        int ext[3];
        patch_extent(box, ext);
        int32_t *inf = info + s * kInfoN;
        inf[PAM_INFO_M] = g.m0;
        inf[PAM_INFO_SUPPORT] = 0;
        inf[PAM_INFO_LEVELS] = 0;
        inf[PAM_INFO_ITERS] = 0;
        inf[PAM_INFO_FLAGS] = 0;
        const int n_cells = g.cells ? g.pstart[s + 1] - g.pstart[s] : ext[0] * ext[1] * ext[2];
        // nothing to fit, or outside the range this call fits: no solve, no refinement
        inf[PAM_INFO_STOPPED] = (n_cells == 0 || s < g.sub_lo || s >= g.sub_hi) ? 1 : 0;
        inf[PAM_INFO_N_CELLS] = n_cells;
        inf[PAM_INFO_MARKED] = 0;
    }
}

void launch_init_dictionary(const Geo &g, const int32_t *boxes, double *centres, double *beta,
                            int32_t *info, cudaStream_t st, int keep_beta) {
    dim3 grid((g.m_cap + 127) / 128, g.S);
    k_init_dictionary<<<grid, 128, 0, st>>>(g, boxes, centres, beta, info, keep_beta);
    count_launches(1);
}

// The slot loop of a kernel that serves both the per-subdomain launch (fb
// null: block row = subdomain = slot, one pass) and the binary64 fallback (fb:
// the listed subdomains; block row `row` of `rows` takes slots row, row +
// rows, ..., so that a launch of a few rows costs next to nothing when the
// list is empty). Items are separated by a barrier: an item's shared-memory
// staging must not overtake the previous item's readers.
template <class F>
__device__ __forceinline__ void for_each_slot(const int32_t *fb, int slots, int row, int rows, F body) {
    const int n = fb ? min(fb[0], slots) : rows;
    for (int slot = row; slot < n; slot += rows) {
        if (slot != row) __syncthreads();
        body(slot, fb ? fb[2 + slot] : slot);
    }
}

// --------------------------------------------------------------------------
// Assembly, Eq. (6) and (10): E_jm = exp(l_jm - l_j*), inv_s_j = 1 / sum_m E_jm,
// so that W_jm = E_jm inv_s_j; l_jm = -|x_j - c_m|^2 / (2 sigma_m^2).
// One thread per patch cell, the dictionary staged in shared memory.
// --------------------------------------------------------------------------
__device__ __forceinline__ void assemble_item(const Geo &g, const int32_t *boxes, const double *centres,
                                              const int32_t *info, const Ws &w, int all, int slot, int s) {
    const int32_t *inf = info + s * kInfoN;
    if (!all && inf[PAM_INFO_STOPPED]) return;
    int M = inf[PAM_INFO_M], N = inf[PAM_INFO_N_CELLS];
    extern __shared__ dvec4 sc[];  // (c_x, c_y, c_z, -1/(2 sigma^2))
    const dvec4 *cg = reinterpret_cast<const dvec4 *>(centres) + (size_t)s * g.m_cap;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        dvec4 c = cg[m];
        c.w = -1.0 / (2.0 * c.w * c.w);
        sc[m] = c;
    }
    __syncthreads();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    double x[3];
    cell_point(g, s, boxes + s * 12, t, x);
    double lmax = -INFINITY;
    for (int m = 0; m < M; ++m) {
        dvec4 c = sc[m];
        double d0 = x[0] - c.x, d1 = x[1] - c.y, d2 = x[2] - c.z;
        double l = (d0 * d0 + d1 * d1 + d2 * d2) * c.w;
        lmax = fmax(lmax, l);
    }
    double sum = 0.0;
    double *E = w.E + (size_t)slot * g.m_cap * g.n_max + t;
    for (int m = 0; m < M; ++m) {
        dvec4 c = sc[m];
        double d0 = x[0] - c.x, d1 = x[1] - c.y, d2 = x[2] - c.z;
        double e = exp((d0 * d0 + d1 * d1 + d2 * d2) * c.w - lmax);
        E[(size_t)m * g.n_max] = e;
        sum += e;
    }
    w.inv_s[(size_t)s * g.n_max + t] = 1.0 / sum;
}

// fb (optional): a fallback list; block row y takes its slots y, y + gridDim.y, ...
// (E indexed by slot).
__global__ void __launch_bounds__(128) k_assemble_f64(Geo g, const int32_t *boxes,
                                                      const double *centres, const int32_t *info,
                                                      Ws w, int all, const int32_t *fb) {
    for_each_slot(fb, w.fb_slots, blockIdx.y, gridDim.y,
                  [&](int slot, int s) { assemble_item(g, boxes, centres, info, w, all, slot, s); });
}

// Row mask of the cross-validation folds: with folds > 0 only the cells t
// with t mod folds != fold enter G and b (the training rows of that fold).
__device__ __forceinline__ bool cv_keep(int t, int folds, int fold) {
    return folds == 0 || t % folds != fold;
}

// b_m = sum_j W_jm y_j, one warp per (subdomain, centre).
__device__ __forceinline__ void bvec_item(const Geo &g, const int32_t *info, const Ws &w, int all, int folds,
                                          int fold, int slot, int s) {
    const int32_t *inf = info + s * kInfoN;
    if (!all && inf[PAM_INFO_STOPPED]) return;
    int M = inf[PAM_INFO_M], N = inf[PAM_INFO_N_CELLS];
    int m = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    int lane = threadIdx.x & 31;
    if (m >= M) return;
    const double *E = w.E + ((size_t)slot * g.m_cap + m) * g.n_max;
    const double *iv = w.inv_s + (size_t)s * g.n_max;
    const double *y = w.y + (size_t)s * g.n_max;
    double acc = 0.0;
    for (int t = lane; t < N; t += 32)
        if (cv_keep(t, folds, fold)) acc += E[t] * iv[t] * y[t];
    acc = warp_sum(acc);
    if (lane == 0) w.b[(size_t)s * g.m_cap + m] = acc;
}

__global__ void k_bvec_f64(Geo g, const int32_t *info, Ws w, int all, int folds, int fold,
                           const int32_t *fb) {
    for_each_slot(fb, w.fb_slots, blockIdx.y, gridDim.y,
                  [&](int slot, int s) { bvec_item(g, info, w, all, folds, fold, slot, s); });
}

// G = W^T W on 64 x 64 tiles of the upper triangle, mirrored; fp64 FMA.
constexpr int kGT = 64, kGK = 16;
__device__ __forceinline__ void gram_item(const Geo &g, const int32_t *info, const Ws &w, int all, int folds,
                                          int fold, int slot, int s) {
    const int32_t *inf = info + s * kInfoN;
    if (!all && inf[PAM_INFO_STOPPED]) return;
    int M = inf[PAM_INFO_M], N = inf[PAM_INFO_N_CELLS];
    int T = g.m_cap / kGT;
    int u = blockIdx.x, ti = 0;
    while (u >= T - ti) { u -= T - ti; ++ti; }
    int tj = ti + u;
    int I0 = ti * kGT, J0 = tj * kGT;
    if (I0 >= M || J0 >= M) return;
    __shared__ double As[kGK][kGT + 1], Bs[kGK][kGT + 1];
    const double *E = w.E + (size_t)slot * g.m_cap * g.n_max;
    const double *iv = w.inv_s + (size_t)s * g.n_max;
    int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
    double acc[4][4] = {};
    for (int t0 = 0; t0 < N; t0 += kGK) {
        for (int e = tid; e < kGT * kGK; e += 256) {
            int row = e / kGK, kk = e % kGK, t = t0 + kk;
            double sc = (t < N && cv_keep(t, folds, fold)) ? iv[t] : 0.0;
            double a = (t < N && I0 + row < M) ? E[(size_t)(I0 + row) * g.n_max + t] * sc : 0.0;
            double b = (t < N && J0 + row < M) ? E[(size_t)(J0 + row) * g.n_max + t] * sc : 0.0;
            As[kk][row] = a;
            Bs[kk][row] = b;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGK; ++kk) {
            double av[4], bv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { av[q] = As[kk][ty + 16 * q]; bv[q] = Bs[kk][tx + 16 * q]; }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
    double *G = w.G + (size_t)slot * g.m_cap * g.m_cap;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            int r = I0 + ty + 16 * i, c = J0 + tx + 16 * j;
            if (r < M && c < M) {
                G[(size_t)r * g.m_cap + c] = acc[i][j];
                G[(size_t)c * g.m_cap + r] = acc[i][j];
            }
        }
}

__global__ void __launch_bounds__(256) k_gram_f64(Geo g, const int32_t *info, Ws w, int all, int folds,
                                                  int fold, const int32_t *fb) {
    for_each_slot(fb, w.fb_slots, blockIdx.y, gridDim.y,
                  [&](int slot, int s) { gram_item(g, info, w, all, folds, fold, slot, s); });
}

// --------------------------------------------------------------------------
// Elastic Net, Eq. (2), in normal-equation form: primal-dual active-set
// iterations. For a guess of the support S and signs s_S, the stationarity
// condition on S is the SPD system (G_SS + lambda2 I) x_S = b_S - lambda1 s_S
// (Cholesky). The guess is corrected until the optimality conditions hold:
// sign(x_S) = s_S and |b_j - G_jS x_S| <= lambda1 (1 + 1e-9) off S, which
// certify the unique minimiser (strict convexity for lambda2 > 0).
// One block per subdomain; the warm start is the previous coefficients
// extended by zeros (Algorithm 1 (5)). After 16 full corrections the
// corrections go one index at a time.
// --------------------------------------------------------------------------
constexpr int kSolveThreads = 256;
constexpr int kFactorSmemBytes = 80 * 1024;

struct SolveShared {
    int cnt, bad, viol, flag, worst;
    double worst_v;
};

// Packed lower-triangular index.
__device__ __forceinline__ size_t tri(int p, int q) { return (size_t)p * (p + 1) / 2 + q; }

__device__ void compact_active(const int *sg, int M, int *idx, int *cnt) {
    // warp 0 scans in chunks of 32 (ascending j)
    if (threadIdx.x < 32) {
        int lane = threadIdx.x, base = 0;
        for (int j0 = 0; j0 < M; j0 += 32) {
            int j = j0 + lane;
            bool on = j < M && sg[j] != 0;
            unsigned bal = __ballot_sync(0xffffffffu, on);
            if (on) idx[base + __popc(bal & ((1u << lane) - 1u))] = j;
            base += __popc(bal);
        }
        if (lane == 0) *cnt = base;
    }
    __syncthreads();
}

// In-place Cholesky of the packed s x s matrix A; sets *flag on a
// non-positive pivot.
__device__ void cholesky_packed(double *A, int s, int *flag, double *inv_piv) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    for (int k = 0; k < s; ++k) {
        if (tid == 0) {
            double d = A[tri(k, k)];
            if (!(d > 0.0)) { *flag = 1; d = 1.0; }
            double l = sqrt(d);
            A[tri(k, k)] = l;
            *inv_piv = 1.0 / l;
        }
        __syncthreads();
        double iv = *inv_piv;
        for (int i = k + 1 + tid; i < s; i += blockDim.x) A[tri(i, k)] *= iv;
        __syncthreads();
        for (int i = k + 1 + warp; i < s; i += nw) {
            double lik = A[tri(i, k)];
            double *row = A + tri(i, 0);
            for (int j = k + 1 + lane; j <= i; j += 32) row[j] -= lik * A[tri(j, k)];
        }
        __syncthreads();
    }
}

// Solves L L^T z = r in place (packed L), by warp 0.
__device__ void cholesky_solve_packed(const double *A, int s, double *r) {
    if (threadIdx.x < 32) {
        int lane = threadIdx.x;
        for (int q = 0; q < s; ++q) {
            double v = r[q] / A[tri(q, q)];
            __syncwarp();
            if (lane == 0) r[q] = v;
            for (int p = q + 1 + lane; p < s; p += 32) r[p] -= A[tri(p, q)] * v;
            __syncwarp();
        }
        for (int q = s - 1; q >= 0; --q) {
            double v = r[q] / A[tri(q, q)];
            __syncwarp();
            if (lane == 0) r[q] = v;
            const double *row = A + tri(q, 0);
            for (int p = lane; p < q; p += 32) r[p] -= row[p] * v;
            __syncwarp();
        }
    }
    __syncthreads();
}

// lam_tab (optional): per-subdomain (lambda1_hat, lambda2_hat) pairs in place
// of p's; all: solve also the subdomains whose refinement has stopped. With
// p.cv_folds > 0 the system is that of the training rows of fold p.cv_fold
// and lambda_k = N_train lambda_k_hat.
__device__ __forceinline__ void solve_item(const Geo &g, const Par &p, double *beta, int32_t *info, const Ws &w,
                                           const double *lam_tab, int all, int slot, int s) {
    int32_t *inf = info + s * kInfoN;
    if (!all && inf[PAM_INFO_STOPPED]) return;
    const int M = inf[PAM_INFO_M], N = inf[PAM_INFO_N_CELLS], mc = g.m_cap;
    const int n_out = (p.cv_folds > 0 && N > p.cv_fold) ? (N - 1 - p.cv_fold) / p.cv_folds + 1 : 0;
    const double n_fit = (double)(N - n_out);
    const double l1h = lam_tab ? lam_tab[2 * s] : p.lam1_hat, l2h = lam_tab ? lam_tab[2 * s + 1] : p.lam2_hat;
    const double lam1 = n_fit * l1h, lam2 = n_fit * l2h;
    const double viol_tol = lam1 * (1.0 + 1e-9);
    extern __shared__ double sm[];
    double *x = sm;          // [mc] full coefficient vector of the current iterate
    double *gr = x + mc;     // [mc] b - G x
    double *bv = gr + mc;    // [mc]
    double *rhs = bv + mc;   // [mc] system on the active list
    int *sg = (int *)(rhs + mc);  // [mc] sign of active coefficients, 0 off the support
    int *idx = sg + mc;           // [mc] active list (ascending)
    double *Asm = (double *)(idx + mc);
    __shared__ SolveShared sh;
    __shared__ double inv_piv;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const double *G = w.G + (size_t)slot * mc * mc;
    const size_t smem_factor_elems = kFactorSmemBytes / sizeof(double);

    for (int j = tid; j < mc; j += blockDim.x) {
        double b0 = j < M ? beta[(size_t)s * mc + j] : 0.0;
        x[j] = b0;
        bv[j] = j < M ? w.b[(size_t)s * mc + j] : 0.0;
        sg[j] = (j < M) ? ((b0 > 0.0) - (b0 < 0.0)) : 0;
    }
    if (tid == 0) { sh.flag = 0; }
    __syncthreads();

    // Up to kPdasFull full primal-dual corrections; then a primal active-set
    // phase from the sign-consistent part of the iterate: step towards the
    // sign-constrained minimiser on the support as far as the signs allow
    // (ratio test; the blocking coefficients leave, a coefficient that joined
    // at zero stays unless its own sign blocks the step), and add all
    // violators once that minimiser is sign-consistent. The objective never
    // increases and every zero-length step shrinks the support, so it ends.
    constexpr int kPdasFull = 12;
    int it = 0, certified = 0, scnt = 0;
    bool primal = false;
    double *A = Asm;
    for (; it < p.max_iters; ++it) {
        compact_active(sg, M, idx, &sh.cnt);
        scnt = sh.cnt;
        A = (tri(scnt, 0) <= smem_factor_elems) ? Asm : w.L + (size_t)slot * ((size_t)mc * (mc + 1) / 2);
        // A = G_SS + lambda2 I (packed lower), rhs = b_S - lambda1 s_S
        for (int pp = warp; pp < scnt; pp += nw) {
            const double *Gr = G + (size_t)idx[pp] * mc;
            for (int q = lane; q <= pp; q += 32)
                A[tri(pp, q)] = Gr[idx[q]] + (q == pp ? lam2 : 0.0);
            if (lane == 0) rhs[pp] = bv[idx[pp]] - lam1 * (double)sg[idx[pp]];
        }
        __syncthreads();
        cholesky_packed(A, scnt, &sh.flag, &inv_piv);
        if (sh.flag) break;
        cholesky_solve_packed(A, scnt, rhs);
        if (!primal) {
            for (int j = tid; j < M; j += blockDim.x) x[j] = 0.0;
            __syncthreads();
            for (int pp = tid; pp < scnt; pp += blockDim.x) x[idx[pp]] = rhs[pp];
            __syncthreads();
        } else {
            // ratio test towards the minimiser rhs on the support
            if (tid == 0) { sh.bad = 0; sh.worst_v = 2.0; }
            __syncthreads();
            for (int pp = tid; pp < scnt; pp += blockDim.x) {
                const int m = idx[pp];
                const double xs = rhs[pp], x0 = x[m], sgn = (double)sg[m];
                if (!(xs * sgn > 0.0)) {
                    const double a = (x0 * sgn > 0.0) ? x0 / (x0 - xs) : 0.0;
                    atomicMin(reinterpret_cast<unsigned long long *>(&sh.worst_v),
                              (unsigned long long)__double_as_longlong(fmax(a, 0.0)));
                    atomicAdd(&sh.bad, 1);
                }
            }
            __syncthreads();
            if (sh.bad) {
                const double alpha = fmin(sh.worst_v, 1.0);
                for (int pp = tid; pp < scnt; pp += blockDim.x) {
                    const int m = idx[pp];
                    const double xs = rhs[pp], x0 = x[m], sgn = (double)sg[m];
                    bool blocking = false;
                    if (!(xs * sgn > 0.0)) {
                        const double a = (x0 * sgn > 0.0) ? x0 / (x0 - xs) : 0.0;
                        blocking = fmax(a, 0.0) <= alpha * (1.0 + 1e-12);
                    }
                    const double nx = x0 + alpha * (xs - x0);
                    if (blocking || (x0 != 0.0 && !(nx * sgn > 0.0))) { x[m] = 0.0; sg[m] = 0; }
                    else x[m] = nx * sgn > 0.0 ? nx : 0.0;
                }
                __syncthreads();
                continue;
            }
            for (int pp = tid; pp < scnt; pp += blockDim.x) x[idx[pp]] = rhs[pp];
            __syncthreads();
        }
        // gradient b - G_{:,S} x_S over every centre (G symmetric: coalesced rows of the support)
        for (int j = tid; j < M; j += blockDim.x) {
            double acc = 0.0;
            for (int pp = 0; pp < scnt; ++pp) acc += G[(size_t)idx[pp] * mc + j] * x[idx[pp]];
            gr[j] = bv[j] - acc;
        }
        if (tid == 0) { sh.bad = 0; sh.viol = 0; sh.worst = -1; sh.worst_v = 0.0; }
        __syncthreads();
        int my_bad = 0, my_viol = 0;
        for (int j = tid; j < M; j += blockDim.x) {
            if (sg[j] != 0) my_bad += !(x[j] * (double)sg[j] > 0.0);
            else my_viol += fabs(gr[j]) > viol_tol;
        }
        if (my_bad) atomicAdd(&sh.bad, my_bad);
        if (my_viol) atomicAdd(&sh.viol, my_viol);
        __syncthreads();
        if (sh.bad == 0 && sh.viol == 0) { certified = 1; break; }
        if (!primal) {
            if (it + 1 < kPdasFull) {
                for (int j = tid; j < M; j += blockDim.x) {
                    if (sg[j] != 0) {
                        if (!(x[j] * (double)sg[j] > 0.0)) sg[j] = 0;
                    } else if (fabs(gr[j]) > viol_tol) {
                        sg[j] = gr[j] > 0.0 ? 1 : -1;
                    }
                }
            } else {
                for (int j = tid; j < M; j += blockDim.x)
                    if (!(x[j] * (double)sg[j] > 0.0)) { sg[j] = 0; x[j] = 0.0; }
                primal = true;
            }
            __syncthreads();
            continue;
        }
        // primal phase, sign-consistent minimiser: the violators join the support
        for (int j = tid; j < M; j += blockDim.x)
            if (sg[j] == 0 && fabs(gr[j]) > viol_tol) { sg[j] = gr[j] > 0.0 ? 1 : -1; x[j] = 0.0; }
        __syncthreads();
    }
    for (int j = tid; j < M; j += blockDim.x) beta[(size_t)s * mc + j] = x[j];
    if (tid == 0) {
        int flags = inf[PAM_INFO_FLAGS] & ~(PAM_FLAG_NOT_CERTIFIED | PAM_FLAG_CHOLESKY);
        if (!certified) {
            flags |= PAM_FLAG_NOT_CERTIFIED;
            atomicAdd(&w.status[kStUncertified], 1);
        }
        if (sh.flag) flags |= PAM_FLAG_CHOLESKY;
        inf[PAM_INFO_FLAGS] = flags;
        inf[PAM_INFO_SUPPORT] = scnt;
        inf[PAM_INFO_ITERS] = it + (certified ? 1 : 0);
    }
}

__global__ void __launch_bounds__(kSolveThreads) k_solve_f64(Geo g, Par p, double *beta,
                                                             int32_t *info, Ws w, const double *lam_tab,
                                                             int all, const int32_t *fb) {
    for_each_slot(fb, w.fb_slots, blockIdx.x, gridDim.x,
                  [&](int slot, int s) { solve_item(g, p, beta, info, w, lam_tab, all, slot, s); });
}

static size_t solve_smem_bytes(int mc) {
    return (size_t)mc * (4 * sizeof(double) + 2 * sizeof(int)) + kFactorSmemBytes;
}

void launch_bgram_f64(const Geo &g, const int32_t *info, const Ws &w, cudaStream_t st, int all, int folds,
                      int fold) {
    {
        PhaseScope ps(kPhAssemble, st);
        dim3 gb((g.m_cap + 7) / 8, g.S);
        k_bvec_f64<<<gb, 256, 0, st>>>(g, info, w, all, folds, fold, nullptr);
        count_launches(1);
    }
    PhaseScope ps(kPhGram, st);
    int T = g.m_cap / kGT;
    dim3 gg(T * (T + 1) / 2, g.S);
    k_gram_f64<<<gg, 256, 0, st>>>(g, info, w, all, folds, fold, nullptr);
    count_launches(1);
}

void launch_assemble_gram_f64(const Geo &g, const int32_t *boxes, const double *centres,
                              const int32_t *info, const Ws &w, cudaStream_t st, int all) {
    size_t asm_smem = (size_t)g.m_cap * sizeof(dvec4);
    cudaFuncSetAttribute(k_assemble_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)asm_smem);
    {
        PhaseScope ps(kPhAssemble, st);
        dim3 ga((g.n_max + 127) / 128, g.S);
        k_assemble_f64<<<ga, 128, asm_smem, st>>>(g, boxes, centres, info, w, all, nullptr);
        count_launches(1);
    }
    launch_bgram_f64(g, info, w, st, all, 0, 0);
}

void launch_solve_f64(const Geo &g, const Par &p, double *beta, int32_t *info, const Ws &w,
                      const double *lam_tab, int all, cudaStream_t st) {
    size_t ss = solve_smem_bytes(g.m_cap);
    cudaFuncSetAttribute(k_solve_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss);
    PhaseScope ps(kPhSolve, st);
    k_solve_f64<<<g.S, kSolveThreads, ss, st>>>(g, p, beta, info, w, lam_tab, all, nullptr);
    count_launches(1);
}

__global__ void __launch_bounds__(128) k_residual_f64(Geo g, const double *beta, const int32_t *info, Ws w,
                                                      const int32_t *fb);

constexpr int kFbRows = 4;

// Binary64 fallback of the mixed form: every subdomain on the fallback list
// (written by the mixed solve: its fp32 iterate did not pass the optimality
// check) is solved again by the binary64 path -- assembly of E and 1/Shepard
// sum, b = W^T y, G = W^T W, the active-set solve -- on its slot of the
// fallback regions, so that it reaches the unique minimiser of Eq. (2) to
// the binary64 form's certificate; then its indicators are recomputed from
// the new coefficients (midpoint rule; the Gauss-Legendre indicators are
// recomputed for every subdomain by the refinement round anyway). The
// launches are sized for all slots; blocks past the list return at once.
void launch_fallback_f64(const Geo &g, const Par &p, const int32_t *boxes, const double *centres,
                         double *beta, int32_t *info, const Ws &w, const double *lam_tab, cudaStream_t st) {
    if (w.fb_slots <= 0) return;
    PhaseScope ps(kPhSolve, st);
    Ws wf = w;
    wf.E = w.fbE;
    wf.G = w.fbG;
    wf.L = w.fbL;
    // a few rows of blocks per kernel, each taking every rows-th listed
    // subdomain: next to nothing to launch when the list is empty (the usual
    // case), and up to kFbRows subdomains at a time otherwise
    const unsigned F = (unsigned)(w.fb_slots < kFbRows ? w.fb_slots : kFbRows);
    // the fallback kernels run between the mixed solve and the next level's
    // tensor-core Gram, both near the shared-memory maximum: the same
    // carveout keeps the SMs from reconfiguring around each (empty) launch
    static bool carveout = [] {
        cudaFuncSetAttribute(k_assemble_f64, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(k_bvec_f64, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(k_gram_f64, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(k_solve_f64, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(k_residual_f64, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        return true;
    }();
    (void)carveout;
    const size_t asm_smem = (size_t)g.m_cap * sizeof(dvec4);
    cudaFuncSetAttribute(k_assemble_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)asm_smem);
    k_assemble_f64<<<dim3((g.n_max + 127) / 128, F), 128, asm_smem, st>>>(g, boxes, centres, info, wf, 1, w.fb);
    k_bvec_f64<<<dim3((g.m_cap + 7) / 8, F), 256, 0, st>>>(g, info, wf, 1, 0, 0, w.fb);
    const int T = g.m_cap / kGT;
    k_gram_f64<<<dim3(T * (T + 1) / 2, F), 256, 0, st>>>(g, info, wf, 1, 0, 0, w.fb);
    const size_t ss = solve_smem_bytes(g.m_cap);
    cudaFuncSetAttribute(k_solve_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss);
    k_solve_f64<<<F, kSolveThreads, ss, st>>>(g, p, beta, info, wf, lam_tab, 1, w.fb);
    count_launches(4);
    if (!p.quad) {
        k_residual_f64<<<dim3((g.n_max + 127) / 128, F), 128, (size_t)g.m_cap * sizeof(double), st>>>(
            g, beta, info, wf, w.fb);
        count_launches(1);
    }
}

void launch_solve_level_f64(const Geo &g, const Par &p, const int32_t *boxes,
                            const double *centres, double *beta, int32_t *info, const Ws &w,
                            cudaStream_t st, cudaEvent_t before_solve) {
    launch_assemble_gram_f64(g, boxes, centres, info, w, st, 0);
    if (before_solve) cudaStreamWaitEvent(st, before_solve, 0);  // an error surfaces in cudaGetLastError
    launch_solve_f64(g, p, beta, info, w, nullptr, 0, st);
}

__global__ void k_copy_gram_f64(Geo g, const int32_t *info, const double *G, const double *b,
                                double *G_out, double *b_out) {
    const int s = blockIdx.y;
    const int M = info[s * kInfoN + PAM_INFO_M];
    const size_t mc = g.m_cap;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < mc * mc;
         e += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(e / mc), c = (int)(e % mc);
        G_out[s * mc * mc + e] = (r < M && c < M) ? G[s * mc * mc + e] : 0.0;
    }
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < mc;
         e += (size_t)gridDim.x * blockDim.x)
        b_out[s * mc + e] = (int)e < M ? b[s * mc + e] : 0.0;
}

void launch_copy_gram_f64(const Geo &g, const int32_t *info, const Ws &w, double *G_out,
                          double *b_out, cudaStream_t st) {
    dim3 grid(64, g.S);
    k_copy_gram_f64<<<grid, 256, 0, st>>>(g, info, w.G, w.b, G_out, b_out);
    count_launches(1);
}

// --------------------------------------------------------------------------
// Step 3: residual indicators (Eq. (4), midpoint rule, K space),
// R_T = |T| (exp(sum_m W_Tm beta_m) - K_T)^2.
// --------------------------------------------------------------------------
__device__ __forceinline__ void residual_item(const Geo &g, const double *beta, const int32_t *info, const Ws &w,
                                              int slot, int s) {
    const int32_t *inf = info + s * kInfoN;
    if (inf[PAM_INFO_STOPPED]) return;
    int M = inf[PAM_INFO_M], N = inf[PAM_INFO_N_CELLS];
    extern __shared__ double sb[];
    for (int m = threadIdx.x; m < M; m += blockDim.x) sb[m] = beta[(size_t)s * g.m_cap + m];
    __syncthreads();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    const double *E = w.E + (size_t)slot * g.m_cap * g.n_max + t;
    double acc = 0.0;
    for (int m = 0; m < M; ++m) acc += E[(size_t)m * g.n_max] * sb[m];
    size_t o = (size_t)s * g.n_max + t;
    double e = exp(acc * w.inv_s[o]) - w.kv[o];
    w.R[o] = cell_measure(g, s, t) * (e * e);
}

__global__ void __launch_bounds__(128) k_residual_f64(Geo g, const double *beta,
                                                      const int32_t *info, Ws w, const int32_t *fb) {
    for_each_slot(fb, w.fb_slots, blockIdx.y, gridDim.y,
                  [&](int slot, int s) { residual_item(g, beta, info, w, slot, s); });
}

// --------------------------------------------------------------------------
// Algorithm 1 (3)-(5): mark the k_top cells with the largest R_T >= eps_tol
// (ranked by R_T rounded to binary32, ties to the lower cell index), then
// add d+1 centres per marked cell: at x_T + eta sigma_p u_q on the vertices
// u_q of a regular simplex, p the current centre nearest to x_T (ties to the
// lower index), clipped to the patch, width eta sigma_p; beta is extended by
// zeros. The geometric decisions use unfused binary64 operations.
// --------------------------------------------------------------------------
__device__ __forceinline__ void simplex_dir(int dim, int q, double u[3]) {
    u[0] = u[1] = u[2] = 0.0;
    if (dim == 1) {
        u[0] = q == 0 ? 1.0 : -1.0;
    } else if (dim == 2) {
        const double c30 = 0.86602540378443864676;  // sqrt(3)/2
        if (q == 0) { u[0] = -c30; u[1] = -0.5; }
        else if (q == 1) { u[0] = c30; u[1] = -0.5; }
        else { u[1] = 1.0; }
    } else {
        // (1,1,1), (1,-1,-1), (-1,1,-1), (-1,-1,1), each / sqrt(3)
        const double r3 = 0.57735026918962576451;
        u[0] = (q == 0 || q == 1) ? r3 : -r3;
        u[1] = (q == 0 || q == 2) ? r3 : -r3;
        u[2] = (q == 0 || q == 3) ? r3 : -r3;
    }
}

constexpr int kMarkThreads = 256;

#ifdef PAM_SOLVE_PROFILE
// Profiling builds only: clock64 totals of the marking kernel's phases.
__device__ unsigned long long g_mark_prof[8];
#define MK_T(v) const long long v = clock64()
#define MK_ADD(k, a, b) do { if (threadIdx.x == 0) atomicAdd(&g_mark_prof[k], (unsigned long long)((b) - (a))); } while (0)
extern "C" void pam_debug_mark_profile(unsigned long long *out, int reset) {
    cudaMemcpyFromSymbol(out, g_mark_prof, sizeof(g_mark_prof));
    if (reset) {
        unsigned long long z[8] = {};
        cudaMemcpyToSymbol(g_mark_prof, z, sizeof(z));
    }
}
#else
#define MK_T(v)
#define MK_ADD(k, a, b)
#endif
constexpr int kMaxKTop = 1024;

// Power of two >= n: the length of the marking kernel's key buffer.
__host__ __device__ __forceinline__ int mark_sort_len(int n) {
    int P = 1;
    while (P < n) P <<= 1;
    return P;
}

// six blocks per SM (40 registers): the kernel is latency-bound (a sort and
// short per-cell searches between block barriers), so resident blocks pay
__global__ void __launch_bounds__(kMarkThreads, 6) k_mark_enrich(Geo g, Par p, const int32_t *boxes,
                                                              double *centres, double *beta,
                                                              int32_t *info, Ws w) {
    const int s = group_sub(g, blockIdx.x);
    int32_t *inf = info + s * kInfoN;
    if (inf[PAM_INFO_STOPPED]) return;
    const int M = inf[PAM_INFO_M], N = inf[PAM_INFO_N_CELLS], L = inf[PAM_INFO_LEVELS];
    int64_t lim = (int64_t)g.m0 + p.m_max;
    const int m_limit = (int)(lim < g.m_cap ? lim : g.m_cap);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    __shared__ int marked[kMaxKTop];
    __shared__ int n_marked;
    // the top-k selection: a digit histogram, counts, the selected keys
    __shared__ int hist[256];
    __shared__ int s_nz, s_nsel, s_digit, s_krem;
    __shared__ unsigned long long sel[kMaxKTop];
    extern __shared__ __align__(16) unsigned long long keys[];  // [P], later the enrichment tables
    if (L >= p.levels || M >= m_limit) {
        if (tid == 0) inf[PAM_INFO_STOPPED] = 1;
        return;
    }
    // the block's binary64 scalars once, by thread 0 (the binary64 pipe is
    // narrow on this part: per-thread copies of these showed as half of its
    // time in the kernel)
    __shared__ double s_atol, s_lo[3], s_hi[3];
    __shared__ float s_ek, s_eloc;
    if (tid == 0) {
        const double kmax = __longlong_as_double((long long)w.kmax_bits[s]);
        const double a_tol0 = p.eps_tol_rel * kmax;
        s_atol = a_tol0;
        s_ek = p.eps_tol_rel < 0.0 ? -INFINITY : (float)(g.vol * (a_tol0 * a_tol0));
        const int32_t *bx = boxes + s * 12;
        float ext0 = 0.f;
        for (int a = 0; a < 3; ++a) {
            s_lo[a] = 0.0;
            s_hi[a] = 0.0;
            if (a < g.dim) {
                s_lo[a] = __dmul_rn((double)bx[6 + a], g.h);
                s_hi[a] = __dmul_rn((double)bx[9 + a], g.h);
                ext0 = fmaxf(ext0, (float)(s_hi[a] - s_lo[a]));
            }
        }
        s_eloc = 2e-7f * ext0;
    }
    __syncthreads();
    const double a_tol = s_atol;
    const float ek = s_ek;
    const double *R = w.R + (size_t)s * g.n_max;
    MK_T(mk0);
    // key = (fp32 R_T + 1 ulp step, ~index): strictly ordered, ties to the
    // lower index; 0 for cells below the tolerance and for the padding
    const int P = mark_sort_len(N);
    for (int t = tid; t < P; t += blockDim.x) {
        unsigned long long k = 0ull;
        if (t < N) {
            const float key = (float)R[t];
            // elements of unequal measure: eps_T = |T| (eps_tol_rel max K)^2
            const float ekt = (g.cells && p.eps_tol_rel >= 0.0)
                                  ? (float)__dmul_rn(__dmul_rn(cell_measure(g, s, t), a_tol), a_tol)
                                  : ek;
            if (key >= ekt)
                k = ((unsigned long long)(__float_as_uint(key) + 1u) << 32) |
                    (unsigned long long)(0xffffffffu - (unsigned)t);
        }
        keys[t] = k;
    }
    if (tid == 0) { n_marked = 0; s_nz = 0; s_nsel = 0; }
    __syncthreads();
    const int k_top = p.k_top < kMaxKTop ? p.k_top : kMaxKTop;
    MK_T(mk1);
    MK_ADD(0, mk0, mk1);
    // The k_top largest nonzero keys in descending order (the keys are
    // distinct, so the set and its order are unique): the kk-th largest by a
    // radix selection over eight 8-bit digits from the top, the keys at or
    // above it gathered, then each ranked against the others.
    {
        int nz = 0;
        for (int t = tid; t < P; t += blockDim.x) nz += keys[t] != 0ull;
        for (int o = 16; o > 0; o >>= 1) nz += __shfl_xor_sync(0xffffffffu, nz, o);
        if (lane == 0 && nz) atomicAdd(&s_nz, nz);
    }
    __syncthreads();
    const int kk = k_top < s_nz ? k_top : s_nz;
    unsigned long long thr = 1ull;  // every nonzero key when kk takes them all
    if (kk > 0 && kk < s_nz) {
        unsigned long long prefix = 0ull, mask = 0ull;
        int krem = kk;
        for (int shift = 56; shift >= 0; shift -= 8) {
            for (int i = tid; i < 256; i += blockDim.x) hist[i] = 0;
            __syncthreads();
            for (int t = tid; t < P; t += blockDim.x) {
                const unsigned long long k = keys[t];
                if (k != 0ull && (k & mask) == prefix) atomicAdd(&hist[(int)((k >> shift) & 255ull)], 1);
            }
            __syncthreads();
            if (warp == 0) {
                // lane l sums the bins 255 - 8 l down to 248 - 8 l; the lane
                // whose bins hold the krem-th key (counted from the top) finds
                // its digit
                int tot = 0;
#pragma unroll
                for (int q = 0; q < 8; ++q) tot += hist[255 - 8 * lane - q];
                int inc = tot;
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += v;
                }
                int above = inc - tot;
                if (above < krem && krem <= inc) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int c = hist[255 - 8 * lane - q];
                        if (above + c >= krem) {
                            s_digit = 255 - 8 * lane - q;
                            s_krem = krem - above;
                            break;
                        }
                        above += c;
                    }
                }
            }
            __syncthreads();
            prefix |= (unsigned long long)s_digit << shift;
            mask |= 255ull << shift;
            krem = s_krem;
        }
        thr = prefix;  // all 64 bits fixed: the kk-th largest key itself
    }
    if (kk > 0) {
        for (int t = tid; t < P; t += blockDim.x) {
            const unsigned long long k = keys[t];
            if (k != 0ull && k >= thr) sel[atomicAdd(&s_nsel, 1)] = k;
        }
    }
    __syncthreads();
    for (int i = tid; i < kk; i += blockDim.x) {
        const unsigned long long k = sel[i];
        int rank = 0;
        for (int j = 0; j < kk; ++j) rank += sel[j] > k;
        marked[rank] = (int)(0xffffffffu - (unsigned)(k & 0xffffffffull));
    }
    if (tid == 0) n_marked = kk;
    __syncthreads();
    const int nm = n_marked;
    MK_T(mk2);
    MK_ADD(1, mk1, mk2);
    if (nm == 0) {
        if (tid == 0) { inf[PAM_INFO_STOPPED] = 1; inf[PAM_INFO_MARKED] = 0; }
        return;
    }
    const int per = g.dim + 1;
    int add = nm * per;
    if (add > m_limit - M) add = m_limit - M;
    const int nmu = (add + per - 1) / per;  // marked cells that receive centres
    double *cs = centres + (size_t)s * g.m_cap * 4;
    const int32_t *box = boxes + s * 12;
    const double lo[3] = {s_lo[0], s_lo[1], s_lo[2]}, hi[3] = {s_hi[0], s_hi[1], s_hi[2]};
    const float e_loc = s_eloc;
    // tables in the (now free) key space: local fp32 centres, marked-cell
    // centroids (binary64) and their local fp32 coordinates, chosen parents
    float4 *scl = reinterpret_cast<float4 *>(keys);          // [M]
    float4 *cxl = scl + M;                                    // [nmu]
    double *cxt = reinterpret_cast<double *>(cxl + nmu);      // [nmu][4]
    int *cbest = reinterpret_cast<int *>(cxt + 4 * nmu);      // [nmu]
    __syncthreads();  // every thread has read its keys
    for (int m = tid; m < M; m += blockDim.x)
        scl[m] = make_float4((float)(cs[(size_t)m * 4 + 0] - lo[0]), (float)(cs[(size_t)m * 4 + 1] - lo[1]),
                             (float)(cs[(size_t)m * 4 + 2] - lo[2]), 0.f);
    for (int r = tid; r < nmu; r += blockDim.x) {
        double xt[3];
        cell_point(g, s, box, marked[r], xt);
        for (int a = 0; a < 3; ++a) cxt[4 * r + a] = xt[a];
        cxl[r] = make_float4((float)(xt[0] - lo[0]), (float)(xt[1] - lo[1]), (float)(xt[2] - lo[2]), 0.f);
    }
    __syncthreads();
    MK_T(mk3);
    MK_ADD(2, mk2, mk3);
    // nearest current centre, one warp per marked cell: an fp32 pass in
    // patch-local coordinates bounds the minimum. Every local coordinate lies
    // in [0, ext], so each fp32 difference is off by at most e = 3 * 2^-24 ext
    // and a squared distance D by at most 3.47 e sqrt(D) + 3 e^2 + 1.8e-7 D;
    // the cut exceeds the minimum by more than twice that, so the nearest
    // centre is among the candidates below it. A single candidate is the
    // answer; several are decided by exact unfused binary64 distances, ties
    // to the lower index.
    for (int r = warp; r < nmu; r += nwarp) {
        const double xt[3] = {cxt[4 * r], cxt[4 * r + 1], cxt[4 * r + 2]};
        const float4 xl4 = cxl[r];
        const float xl[3] = {xl4.x, xl4.y, xl4.z};
        float bf = INFINITY;
        for (int m = lane; m < M; m += 32) {
            const float4 c = scl[m];
            const float d0 = c.x - xl[0], d1 = c.y - xl[1], d2 = c.z - xl[2];
            bf = fminf(bf, fmaf(d2, d2, fmaf(d1, d1, d0 * d0)));
        }
        for (int o = 16; o > 0; o >>= 1) bf = fminf(bf, __shfl_xor_sync(0xffffffffu, bf, o));
        const float cut = bf * 1.001f + 8.f * e_loc * sqrtf(bf) + 24.f * e_loc * e_loc + 1e-30f;
        int ncand = 0, first = 0x7fffffff;
        for (int m = lane; m < M; m += 32) {
            const float4 c = scl[m];
            const float d0 = c.x - xl[0], d1 = c.y - xl[1], d2 = c.z - xl[2];
            if (fmaf(d2, d2, fmaf(d1, d1, d0 * d0)) <= cut) {
                ++ncand;
                first = min(first, m);
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            ncand += __shfl_xor_sync(0xffffffffu, ncand, o);
            first = min(first, __shfl_xor_sync(0xffffffffu, first, o));
        }
        int bestm = first;
        if (ncand > 1) {
            double bd = INFINITY;
            bestm = 0x7fffffff;
            for (int m = lane; m < M; m += 32) {
                const float4 c = scl[m];
                const float d0 = c.x - xl[0], d1 = c.y - xl[1], dd2 = c.z - xl[2];
                if (fmaf(dd2, dd2, fmaf(d1, d1, d0 * d0)) > cut) continue;
                double d2 = 0.0;
                for (int a = 0; a < g.dim; ++a) {
                    double d = __dsub_rn(xt[a], cs[(size_t)m * 4 + a]);
                    d2 = __dadd_rn(d2, __dmul_rn(d, d));
                }
                if (d2 < bd) { bd = d2; bestm = m; }  // m ascends per lane: ties keep the lower
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double od = __shfl_xor_sync(0xffffffffu, bd, o);
                const int om = __shfl_xor_sync(0xffffffffu, bestm, o);
                if (od < bd || (od == bd && om < bestm)) { bd = od; bestm = om; }
            }
        }
        if (lane == 0) cbest[r] = bestm;
    }
    __syncthreads();
    // the new centres, one thread each: x_T + eta sigma_p u_q, clipped
    for (int f = tid; f < add; f += blockDim.x) {
        const int r = f / per, q = f % per;
        const double xt[3] = {cxt[4 * r], cxt[4 * r + 1], cxt[4 * r + 2]};
        const double sn = __dmul_rn(p.eta, cs[(size_t)cbest[r] * 4 + 3]);
        double u[3];
        simplex_dir(g.dim, q, u);
        double *c = cs + (size_t)(M + f) * 4;
        for (int a = 0; a < 3; ++a) {
            double v = 0.0;
            if (a < g.dim) {
                v = __dadd_rn(xt[a], __dmul_rn(sn, u[a]));
                if (v < lo[a]) v = lo[a];
                if (v > hi[a]) v = hi[a];
            }
            c[a] = v;
        }
        c[3] = sn;
        beta[(size_t)s * g.m_cap + M + f] = 0.0;
    }
    MK_T(mk4);
    MK_ADD(3, mk3, mk4);
    if (tid == 0) MK_ADD(4, 0, 1);
    if (tid == 0) {
        inf[PAM_INFO_M] = M + add;
        inf[PAM_INFO_LEVELS] = L + 1;
        inf[PAM_INFO_MARKED] = nm;
        if (add == 0) inf[PAM_INFO_STOPPED] = 1;
    }
}

void launch_mark_enrich(const Geo &g, const Par &p, const int32_t *boxes, double *centres,
                        double *beta, int32_t *info, const Ws &w, cudaStream_t st) {
    // the sort's keys, later the centre table, marked centroids and parents
    size_t sm = (size_t)mark_sort_len(g.n_max) * sizeof(unsigned long long);
    const int kt = p.k_top < kMaxKTop ? p.k_top : kMaxKTop;
    const size_t tables = (size_t)g.m_cap * sizeof(float4) +
                          (size_t)kt * (sizeof(float4) + 4 * sizeof(double) + sizeof(int));
    if (sm < tables) sm = tables;
    cudaFuncSetAttribute(k_mark_enrich, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    PhaseScope ps(kPhMark, st);
    k_mark_enrich<<<group_count(g), kMarkThreads, sm, st>>>(g, p, boxes, centres, beta, info, w);
    count_launches(1);
}

void launch_residual_f64(const Geo &g, const double *beta, const int32_t *info, const Ws &w,
                         cudaStream_t st) {
    size_t sm = (size_t)g.m_cap * sizeof(double);
    dim3 grid((g.n_max + 127) / 128, g.S);
    PhaseScope ps(kPhResidual, st);
    k_residual_f64<<<grid, 128, sm, st>>>(g, beta, info, w, nullptr);
    count_launches(1);
}

// --------------------------------------------------------------------------
// One refinement round: residuals of the current fit, then mark + enrich.
// --------------------------------------------------------------------------
void launch_residual_mixed(const Geo &g, const int32_t *boxes, const double *centres,
                           const double *beta, const int32_t *info, const Ws &w, cudaStream_t st);

void launch_refine_round(const Geo &g, const Par &p, int precision, const int32_t *boxes,
                         double *centres, double *beta, int32_t *info, const Ws &w,
                         cudaStream_t st) {
    if (p.quad)
        launch_residual_quad(g, precision, boxes, centres, beta, info, w, st);
    else if (precision == PAM_PREC_MIXED)
        launch_residual_mixed(g, boxes, centres, beta, info, w, st);
    else
        launch_residual_f64(g, beta, info, w, st);
    launch_mark_enrich(g, p, boxes, centres, beta, info, w, st);
}

}  // namespace pam
