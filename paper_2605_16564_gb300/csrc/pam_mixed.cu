// pam_mixed.cu -- the mixed-precision form of the fitting path:
//   * Shepard row statistics in fp32 (k_stats_f32),
//   * the Gram products G = W^T W, b = W^T y on the tcgen05 tensor cores
//     (k_gram_tc): W is generated in registers, split into bf16 hi + lo
//     parts, staged in shared memory, and multiplied hi*hi + hi*lo + lo*hi
//     with fp32 accumulation in TMEM (relative error ~2^-16 per entry),
//   * the Elastic Net solve in fp32 with iterative refinement against the
//     exactly recomputed gradient W^T (y - W beta) (k_solve_mixed),
//   * residual indicators with fp64 accumulation of the K-space residual.
//
// All Gaussians are evaluated in local coordinates relative to the patch
// origin, from coordinate differences, in base 2:
//   l2 = alpha_m |x - c_m|^2,  alpha_m = -log2(e) / (2 sigma_m^2).
#include <cfloat>
#include <cmath>
#include <cstdlib>

#include "pam_internal.cuh"
#include "pam_tc.cuh"

namespace pam {

// Per-centre constants in local coordinates: (c - origin, alpha).
__device__ __forceinline__ float4 local_centre(const dvec4 &c, const double o[3]) {
    float4 r;
    r.x = (float)(c.x - o[0]);
    r.y = (float)(c.y - o[1]);
    r.z = (float)(c.z - o[2]);
    const float sg = (float)c.w;  // alpha in fp32: relative error ~1e-7, no fp64 divide
    r.w = -1.44269504f / (2.f * sg * sg);
    return r;
}

__device__ __forceinline__ float logit2(const float4 &c, float x, float y, float z) {
    float dx = x - c.x, dy = y - c.y, dz = z - c.z;
    return c.w * fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}

__device__ __forceinline__ void patch_origin(const Geo &g, const int32_t *box, double o[3]) {
    for (int a = 0; a < 3; ++a) o[a] = a < g.dim ? (double)box[6 + a] * g.h : 0.0;
}

// Local coordinates of patch cell t: ((i - patch_lo) + 1/2) h, exact in fp32
// up to one rounding.
__device__ __forceinline__ void local_cell(const Geo &g, const int32_t *box, int t, float x[3]) {
    int w0 = box[9] - box[6], w1 = box[10] - box[7];
    int i = t % w0, j = (t / w0) % w1, k = t / (w0 * w1);
    float hf = (float)g.h;
    x[0] = ((float)i + 0.5f) * hf;
    x[1] = g.dim > 1 ? ((float)j + 0.5f) * hf : 0.0f;
    x[2] = g.dim > 2 ? ((float)k + 0.5f) * hf : 0.0f;
}

// --------------------------------------------------------------------------
// Row statistics of the Shepard normalisation (Eq. (10)): l2* = max_m l2_jm
// and 1 / sum_m 2^(l2_jm - l2*), one thread per patch cell.
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_stats_f32(Geo g, const int32_t *boxes,
                                                   const double *centres, const int32_t *info,
                                                   Ws w, int all) {
    const int s = blockIdx.y;
    const int32_t *inf = info + s * kInfoN;
    if (!all && inf[PAM_INFO_STOPPED]) return;
    const int M = inf[PAM_INFO_M], N = inf[PAM_INFO_N_CELLS];
    const int32_t *box = boxes + s * 12;
    extern __shared__ float4 sc[];
    double o[3];
    patch_origin(g, box, o);
    const dvec4 *cg = reinterpret_cast<const dvec4 *>(centres) + (size_t)s * g.m_cap;
    for (int m = threadIdx.x; m < M; m += blockDim.x) sc[m] = local_centre(cg[m], o);
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    float x[3];
    local_cell(g, box, t, x);
    float lmax = -INFINITY;
    for (int m = 0; m < M; ++m) lmax = fmaxf(lmax, logit2(sc[m], x[0], x[1], x[2]));
    float sum = 0.0f;
    for (int m = 0; m < M; ++m) sum += tc::ex2(logit2(sc[m], x[0], x[1], x[2]) - lmax);
    w.rowmax[(size_t)s * g.n_max + t] = lmax;
    w.rowinv[(size_t)s * g.n_max + t] = 1.0f / sum;
}

// --------------------------------------------------------------------------
// Gram products on the tensor cores. One CTA per (subdomain, strip of 128
// centres I): D = W_I^T W_{I..} (128 x R, R = centres from the strip start
// to the padded end of the dictionary) accumulates in TMEM over chunks of 32
// cells. The 256 threads generate the chunk's W values (each thread one or
// two centre rows), split them into bf16 hi/lo and store them in the
// canonical K-major layout (8-row x 16-byte core matrices); the A operand
// is the first 128 rows of the same tile. Two buffers: the threads fill one
// while the tensor core consumes the other; thread 0 issues the MMAs and
// commits them to the buffer's mbarrier.
// Epilogue: warps read the strip from TMEM and write rows of G (and the
// mirrored block below the strip) in fp32; threads of the strip's rows also
// accumulate b = W^T y.
// --------------------------------------------------------------------------
constexpr int kTcThreads = 1024;         // two producer threads per centre row
constexpr int kTcKC = 32;                 // cells per chunk (2 MMA k-steps of 16)
constexpr int kTcMaxRows = 512;           // rows of the B tile (TMEM columns)
constexpr long long kWaitBudget = 4000000000LL;  // ~2 s at 2 GHz

// Cell data of the patch, staged once: local coordinates, sh = l2* -
// log2(1/sum) (the Shepard normaliser folded into the exponent, W =
// 2^(alpha d^2 - sh); +inf for padding cells) and y = ln K.
struct TcCellAll {
    float4 p;  // (x, y, z, sh)
};

__global__ void __launch_bounds__(kTcThreads, 1) k_gram_tc(Geo g, const int32_t *boxes,
                                                           const double *centres,
                                                           const int32_t *info, Ws w, int all) {
    const int s = blockIdx.y, strip = blockIdx.x;
    const int32_t *inf = info + s * kInfoN;
    if (!all && inf[PAM_INFO_STOPPED]) return;
    const int M = inf[PAM_INFO_M], N = inf[PAM_INFO_N_CELLS];
    const int row0 = strip * 128;
    if (row0 >= M) return;
    const int Mp = (M + 31) & ~31;                 // padded dictionary size
    const int R = Mp - row0;                        // B rows = TMEM columns (multiple of 32)
    const int Rt = R < 128 ? 128 : R;               // tile rows (the A operand reads 128)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int32_t *box = boxes + s * 12;

    extern __shared__ __align__(1024) uint8_t smem[];
    // [buf][hi|lo] tiles of Rt x kTcKC bf16, each Rt * 64 bytes
    const uint32_t tile_bytes = (uint32_t)Rt * kTcKC * 2;
    uint8_t *tiles = smem;
    float4 *sc = reinterpret_cast<float4 *>(smem + 4 * (size_t)kTcMaxRows * kTcKC * 2);
    float4 *cellp = sc + kTcMaxRows;                       // [nch * 32] (x, y, z, sh)
    const int nch = (N + kTcKC - 1) / kTcKC;
    float *celly = reinterpret_cast<float *>(cellp + (size_t)nch * kTcKC);  // [nch * 32] ln K
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int timed_out;

    double o[3];
    patch_origin(g, box, o);
    const dvec4 *cg = reinterpret_cast<const dvec4 *>(centres) + (size_t)s * g.m_cap;
    for (int r = tid; r < Rt; r += blockDim.x) {
        int m = row0 + r;
        sc[r] = (r < R && m < M) ? local_centre(cg[m], o) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float *rowmax = w.rowmax + (size_t)s * g.n_max;
    const float *rowinv = w.rowinv + (size_t)s * g.n_max;
    const double *yv = w.y + (size_t)s * g.n_max;
    for (int t = tid; t < nch * kTcKC; t += blockDim.x) {
        float x[3] = {0.f, 0.f, 0.f};
        float sh = INFINITY, y = 0.f;
        if (t < N) {
            local_cell(g, box, t, x);
            sh = rowmax[t] - log2f(rowinv[t]);
            y = (float)yv[t];
        }
        cellp[t] = make_float4(x[0], x[1], x[2], sh);
        celly[t] = y;
    }
    uint32_t ncols = 32;
    while (ncols < (uint32_t)R) ncols <<= 1;
    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        tc::mbar_fence_init();
        timed_out = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, ncols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;

    const uint32_t lbo = (uint32_t)Rt * 16u, sbo = 128u;
    const int r = tid & (kTcMaxRows - 1);           // the tile row this thread produces
    const int half = tid >> 9;                      // ... for k-groups 2*half, 2*half+1
    const bool live = r < R && row0 + r < M;
    const float4 cc = r < Rt ? sc[r] : make_float4(0.f, 0.f, 0.f, 0.f);
    float bacc = 0.f;

    int issued = 0;  // chunks whose MMAs thread 0 has committed
    for (int c = 0; c < nch; ++c) {
        const int buf = c & 1;
        if (c >= 2) {  // the MMAs of chunk c-2 read this buffer
            if (!tc::mbar_wait(&mbar[buf], ((c - 2) >> 1) & 1, kWaitBudget)) timed_out = 1;
        }
        const float4 *cl = cellp + c * kTcKC;
        const float *cy = celly + c * kTcKC;
        uint8_t *hi = tiles + (size_t)buf * 2 * tile_bytes;
        uint8_t *lo = hi + tile_bytes;
        if (r < Rt) {
            float bsum = 0.f;
#pragma unroll
            for (int kh = 0; kh < 2; ++kh) {
                const int kg = 2 * half + kh;
                float v[8];
                if (live) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int k = kg * 8 + q;
                        const float4 cp = cl[k];
                        const float dx = cp.x - cc.x, dy = cp.y - cc.y, dz = cp.z - cc.z;
                        const float e = tc::ex2(fmaf(cc.w, fmaf(dz, dz, fmaf(dy, dy, dx * dx)), -cp.w));
                        v[q] = e;
                        bsum = fmaf(e, cy[k], bsum);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 8; ++q) v[q] = 0.f;
                }
                uint32_t hp[4], lp[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    hp[q] = tc::pack_bf16(v[2 * q], v[2 * q + 1]);
                    const float h0 = __uint_as_float(hp[q] << 16), h1 = __uint_as_float(hp[q] & 0xffff0000u);
                    lp[q] = tc::pack_bf16(v[2 * q] - h0, v[2 * q + 1] - h1);
                }
                const uint32_t off = (uint32_t)(kg * (Rt >> 3) + (r >> 3)) * 128u + (uint32_t)(r & 7) * 16u;
                *reinterpret_cast<uint4 *>(hi + off) = make_uint4(hp[0], hp[1], hp[2], hp[3]);
                *reinterpret_cast<uint4 *>(lo + off) = make_uint4(lp[0], lp[1], lp[2], lp[3]);
            }
            bacc += bsum;
        }
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (timed_out) break;
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t hi_a = tc::smem_u32(hi), lo_a = tc::smem_u32(lo);
#pragma unroll
            for (int ks = 0; ks < kTcKC / 16; ++ks) {
                const uint32_t koff = (uint32_t)(2 * ks) * lbo;
                const uint64_t a_hi = tc::smem_desc(hi_a + koff, lbo, sbo);
                const uint64_t a_lo = tc::smem_desc(lo_a + koff, lbo, sbo);
                for (int n0 = 0; n0 < R; n0 += 256) {
                    const uint32_t n = (uint32_t)min(256, R - n0);
                    const uint32_t id = tc::idesc_bf16_f32(n);
                    const uint32_t noff = (uint32_t)(n0 >> 3) * sbo;
                    const uint64_t b_hi = tc::smem_desc(hi_a + koff + noff, lbo, sbo);
                    const uint64_t b_lo = tc::smem_desc(lo_a + koff + noff, lbo, sbo);
                    const uint32_t d = tmem + (uint32_t)n0;
                    tc::mma_bf16(d, a_hi, b_hi, id, (c > 0 || ks > 0) ? 1u : 0u);
                    tc::mma_bf16(d, a_hi, b_lo, id, 1u);
                    tc::mma_bf16(d, a_lo, b_hi, id, 1u);
                }
            }
            tc::mma_commit(&mbar[buf]);
        }
        issued = c + 1;
    }
    // wait for the last chunk's MMAs (they complete in issue order)
    if (!timed_out && nch > 0) {
        const int last = nch - 1;
        if (!tc::mbar_wait(&mbar[last & 1], (last >> 1) & 1, kWaitBudget)) timed_out = 1;
    }
    __syncthreads();
    tc::fence_after_sync();
    if (timed_out) {
        // give the MMAs still in flight a bounded time to land before TMEM is released
        if (issued > 0) tc::mbar_wait(&mbar[(issued - 1) & 1], ((issued - 1) >> 1) & 1, kWaitBudget);
        if (tid == 0) atomicAdd(&w.status[kStTimeout], 1);
    } else {
        float *G = w.Gf + (size_t)s * g.m_cap * g.m_cap;
        // warp q reads TMEM lanes 32 (q % 4) ..; the four warps of a lane
        // quarter split the 32-column chunks. Rows go out through a padded
        // shared-memory transpose so that each store is one coalesced row
        // segment; the mirrored block below the strip is already coalesced.
        float *stage = reinterpret_cast<float *>(tiles) + (size_t)(warp & 15) * 32 * 33;
        const int lane_base = (warp & 3) * 32;
        const int rl = lane_base + lane;      // D row (TMEM lane) held by this thread
        const int rg = row0 + rl;             // its G row
        const int ncol_chunks = R / 32;
        for (int ch = warp >> 2; warp < 16 && ch < ncol_chunks; ch += 4) {
            uint32_t v[32];
            tc::tmem_ld_32x32(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(ch * 32), v);
            tc::tmem_wait_ld();
            const int c0 = row0 + ch * 32;
            if (ch * 32 >= 128) {
                for (int q = 0; q < 32; ++q) {
                    const int col = c0 + q;
                    if (col < M && rg < M) G[(size_t)col * g.m_cap + rg] = __uint_as_float(v[q]);
                }
            }
#pragma unroll
            for (int q = 0; q < 32; ++q) stage[lane * 33 + q] = __uint_as_float(v[q]);
            __syncwarp();
            const int col = c0 + lane;
            for (int q = 0; q < 32; ++q) {
                const int row = row0 + lane_base + q;
                if (row < M && col < M) G[(size_t)row * g.m_cap + col] = stage[q * 33 + lane];
            }
            __syncwarp();
        }
        // b = W^T y for the strip's rows: the two halves of a row add up
        float *bh = reinterpret_cast<float *>(sc);  // the centre table is no longer needed
        __syncthreads();
        if (half == 1 && r < 128) bh[r] = bacc;
        __syncthreads();
        if (half == 0 && r < 128 && live) w.b[(size_t)s * g.m_cap + row0 + r] = (double)(bacc + bh[r]);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

static size_t gram_tc_smem(const Geo &g) {
    const size_t cells = (size_t)((g.n_max + kTcKC - 1) / kTcKC) * kTcKC;
    return 4 * (size_t)kTcMaxRows * kTcKC * 2 + kTcMaxRows * sizeof(float4) + cells * (sizeof(float4) + sizeof(float)) + 1024;
}

void launch_stats_gram_tc(const Geo &g, const int32_t *boxes, const double *centres,
                          const int32_t *info, const Ws &w, cudaStream_t st, int all) {
    {
        PhaseScope ps(kPhStats, st);
        size_t sm = (size_t)g.m_cap * sizeof(float4);
        cudaFuncSetAttribute(k_stats_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        dim3 grid((g.n_max + 127) / 128, g.S);
        k_stats_f32<<<grid, 128, sm, st>>>(g, boxes, centres, info, w, all);
        count_launches(1);
    }
    {
        PhaseScope ps(kPhGramTC, st);
        size_t sm = gram_tc_smem(g);
        cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        dim3 grid((g.m_cap + 127) / 128, g.S);
        k_gram_tc<<<grid, kTcThreads, sm, st>>>(g, boxes, centres, info, w, all);
        count_launches(1);
    }
}

// Copies the fp32 Gram of the mixed form into caller doubles (pam_gram).
__global__ void k_copy_gram_f32(Geo g, const int32_t *info, const float *Gf, const double *b,
                                double *G_out, double *b_out) {
    const int s = blockIdx.y;
    const int M = info[s * kInfoN + PAM_INFO_M];
    const size_t mc = g.m_cap;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < mc * mc;
         e += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(e / mc), c = (int)(e % mc);
        G_out[s * mc * mc + e] = (r < M && c < M) ? (double)Gf[s * mc * mc + e] : 0.0;
    }
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < mc;
         e += (size_t)gridDim.x * blockDim.x)
        b_out[s * mc + e] = (int)e < M ? b[s * mc + e] : 0.0;
}

void launch_copy_gram_f32(const Geo &g, const int32_t *info, const Ws &w, double *G_out,
                          double *b_out, cudaStream_t st) {
    dim3 grid(64, g.S);
    k_copy_gram_f32<<<grid, 256, 0, st>>>(g, info, w.Gf, w.b, G_out, b_out);
    count_launches(1);
}

// --------------------------------------------------------------------------
// Elastic Net (Eq. (2)) in the mixed form, one block per subdomain.
// Stage 1: primal-dual active-set iterations on the tensor-core Gram G~
//   (fp32): for a support guess S with signs s, solve
//   (G~_SS + lambda2 I) x_S = b_S - lambda1 s_S by fp32 Cholesky and correct
//   the guess until sign(x_S) = s and |b_j - G~_jS x_S| <= lambda1 off S.
// Stage 2: iterative refinement against the exact gradient. With W
//   regenerated from the row statistics, e = y - W x and c = W^T e are
//   recomputed (fp32 exps, fp32 sums), the stationarity residual
//   r_S = c_S - lambda2 x_S - lambda1 s_S is corrected through the same
//   factor, x_S += (G~_SS + lambda2 I)^{-1} r_S, and the support is updated
//   from the exact optimality conditions (entries whose sign flips leave S,
//   violators |c_j| > lambda1 join it). It contracts by about
//   ||(G~ + lambda2 I)^{-1} (G - G~)|| per step (~1e-2 here).
// Finally the residual indicators R_T = |T| (exp(W x)_T - K_T)^2 of the
// final coefficients are written (fp64 for the K-space residual), so the
// refinement round needs no separate residual pass.
// --------------------------------------------------------------------------

constexpr int kMxThreads = 256;
constexpr int kMxFactorBytesDefault = 64 * 1024;
constexpr int kMxMaxRefine = 12;
constexpr int kMxMaxPdas = 200;
constexpr int kMxPdasFull = 12;

struct MxShared {
    int cnt, bad, viol, flag, changed;
    float inv_piv, dmax, xmax;
};

__device__ void mx_compact(const int *sg, int M, int *idx, int *cnt) {
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

__device__ __forceinline__ int tri_i(int p, int q) { return p * (p + 1) / 2 + q; }

#ifdef PAM_SOLVE_PROFILE
// Profiling builds only: clock64 totals per phase of the mixed solve.
__device__ unsigned long long g_solve_prof[16];
__device__ unsigned long long g_solve_blk[8192];
#define PROF_T0() long long _pt = clock64()
#define PROF_MARK(k)                                                          \
    do {                                                                      \
        if (threadIdx.x == 0) atomicAdd(&g_solve_prof[k], (unsigned long long)(clock64() - _pt)); \
        _pt = clock64();                                                      \
    } while (0)
#else
#define PROF_T0()
#define PROF_MARK(k)
#endif

// Blocked right-looking Cholesky of the packed lower s x s matrix A, in
// place, with blocks of 32 columns. Warp 0 factors the 32 x 32 diagonal
// block in registers (lane i holds row i, fully unrolled so every index is
// static; rows past the end of a partial block are padded with the
// identity); every other thread solves one panel row against it, again
// from registers, reading L_kk as shared-memory broadcasts; then all
// threads update the trailing triangle. Three block barriers per 32 columns.
// dinv[k] receives 1 / L_kk for the triangular solves.
__device__ __forceinline__ void mx_diag_block(float *A, int k0, int kw, int *flag, float *dinv) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, i = k0 + lane;
    const bool live = lane < kw;
    float a[32];
#pragma unroll
    for (int j = 0; j < 32; ++j)
        a[j] = (live && j <= lane) ? A[tri_i(i, k0 + j)] : (j == lane ? 1.f : 0.f);
    float my_iv = 1.f;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        float d = __shfl_sync(full, a[k], k);
        if (!(d > 0.f)) { bad = true; d = 1.f; }
        const float iv = rsqrtf(d);
        if (lane == k) { a[k] = d * iv; my_iv = iv; }
        else a[k] *= iv;  // above the diagonal (lane < k) the value is never used
#pragma unroll
        for (int j = k + 1; j < 32; ++j) a[j] = fmaf(-a[k], __shfl_sync(full, a[k], j), a[j]);
    }
    if (live) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (j <= lane) A[tri_i(i, k0 + j)] = a[j];
        dinv[i] = my_iv;
    }
    if (__any_sync(full, bad && live)) {
        if (lane == 0) *flag = 1;
    }
}

// Panel row i: L[i, k0:k0+32] = A[i, k0:k0+32] L_kk^{-T} (kw == 32 only:
// a partial block is the last one and has no rows below it).
__device__ __forceinline__ void mx_panel_row(float *A, int k0, int i, const float *dinv) {
    float *ri = A + tri_i(i, 0) + k0;
    float r[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) r[j] = ri[j];
#pragma unroll
    for (int q = 0; q < 32; ++q) {
        const float *lq = A + tri_i(k0 + q, 0) + k0;
        float a0 = r[q], a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
        for (int rr = 0; rr < q; ++rr) {
            if ((rr & 3) == 0) a0 = fmaf(-r[rr], lq[rr], a0);
            else if ((rr & 3) == 1) a1 = fmaf(-r[rr], lq[rr], a1);
            else if ((rr & 3) == 2) a2 = fmaf(-r[rr], lq[rr], a2);
            else a3 = fmaf(-r[rr], lq[rr], a3);
        }
        r[q] = ((a0 + a1) + (a2 + a3)) * dinv[k0 + q];
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) ri[j] = r[j];
}

__device__ void mx_cholesky(float *A, int s, int *flag, float *dinv) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    PROF_T0();
    for (int k0 = 0; k0 < s; k0 += 32) {
        const int kw = min(32, s - k0);
        if (warp == 0) mx_diag_block(A, k0, kw, flag, dinv);
        __syncthreads();
        PROF_MARK(12);
        if (k0 + kw >= s) break;  // last block: nothing below it
        for (int i = k0 + kw + tid; i < s; i += blockDim.x) mx_panel_row(A, k0, i, dinv);
        __syncthreads();
        PROF_MARK(13);
        // trailing update of rows/cols >= k0 + kw
        for (int i = k0 + kw + warp; i < s; i += nw) {
            const float *li = A + tri_i(i, 0) + k0;
            float *row = A + tri_i(i, 0);
            for (int j = k0 + kw + lane; j <= i; j += 32) {
                const float *lj = A + tri_i(j, 0) + k0;
                float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
                for (int q = 0; q < 32; q += 2) {
                    acc0 = fmaf(li[q], lj[q], acc0);
                    acc1 = fmaf(li[q + 1], lj[q + 1], acc1);
                }
                row[j] -= acc0 + acc1;
            }
        }
        __syncthreads();
        PROF_MARK(14);
    }
}

// Solves L L^T z = r in place (packed L from mx_cholesky, dinv = 1/diag):
// per 32-row block, warp 0 solves the diagonal block with shuffles (fully
// unrolled; the matrix loads do not depend on the recurrence) and all
// threads apply the block's contribution to the remaining entries.
__device__ void mx_chol_solve(const float *A, const float *dinv, int s, float *r) {
    const unsigned full = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // forward: L z = r
    for (int k0 = 0; k0 < s; k0 += 32) {
        const int kw = min(32, s - k0);
        if (warp == 0) {
            const int i = k0 + lane;
            const bool live = lane < kw;
            float ri = live ? r[i] : 0.f;
            const float di = live ? dinv[i] : 1.f;
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const float lik = (live && lane > q) ? A[tri_i(i, k0 + q)] : 0.f;
                if (lane == q) ri *= di;
                const float zq = __shfl_sync(full, ri, q);
                ri = fmaf(-lik, zq, ri);
            }
            if (live) r[i] = ri;
        }
        __syncthreads();
        if (k0 + kw < s) {
            for (int i = k0 + kw + tid; i < s; i += blockDim.x) {
                const float *li = A + tri_i(i, 0) + k0;
                float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
                for (int q = 0; q < 32; q += 2) {
                    acc0 = fmaf(li[q], r[k0 + q], acc0);
                    acc1 = fmaf(li[q + 1], r[k0 + q + 1], acc1);
                }
                r[i] -= acc0 + acc1;
            }
            __syncthreads();
        }
    }
    // backward: L^T x = z
    for (int k0 = ((s - 1) / 32) * 32; k0 >= 0 && s > 0; k0 -= 32) {
        const int kw = min(32, s - k0);
        if (warp == 0) {
            const int pr = k0 + lane;
            const bool live = lane < kw;
            float rp = live ? r[pr] : 0.f;
            const float dp = live ? dinv[pr] : 1.f;
#pragma unroll
            for (int q = 31; q >= 0; --q) {
                const float lqp = (q < kw && lane < q) ? A[tri_i(k0 + q, k0 + lane)] : 0.f;
                if (lane == q) rp *= dp;
                const float xq = __shfl_sync(full, rp, q);
                rp = fmaf(-lqp, xq, rp);
            }
            if (live) r[pr] = rp;
        }
        __syncthreads();
        if (k0 > 0) {
            for (int pr = tid; pr < k0; pr += blockDim.x) {
                float acc0 = 0.f, acc1 = 0.f;
                int q = 0;
                for (; q + 1 < kw; q += 2) {
                    acc0 = fmaf(A[tri_i(k0 + q, pr)], r[k0 + q], acc0);
                    acc1 = fmaf(A[tri_i(k0 + q + 1, pr)], r[k0 + q + 1], acc1);
                }
                if (q < kw) acc0 = fmaf(A[tri_i(k0 + q, pr)], r[k0 + q], acc0);
                r[pr] -= acc0 + acc1;
            }
            __syncthreads();
        }
    }
}

// Compensated (double-float) accumulation: s + c carries the running sum of
// exact fp32 products to about 2^-44 relative, using fp32 operations only
// (TwoProduct by fma, TwoSum by Knuth).
struct DFAcc {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add_prod(float a, float b) {
        // explicitly rounded operations: contraction into fma would break the
        // error-free transformations
        const float p = __fmul_rn(a, b);
        const float pe = fmaf(a, b, -p);
        const float t = __fadd_rn(s, p);
        const float bp = __fsub_rn(t, s);
        const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
        s = t;
        c = __fadd_rn(c, __fadd_rn(err, pe));
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

__global__ void __launch_bounds__(kMxThreads, 2) k_solve_mixed(Geo g, Par p, const int32_t *boxes,
                                                            const double *centres, double *beta,
                                                            int32_t *info, Ws w, int kMxFactorBytes) {
    const int s = blockIdx.x;
    int32_t *inf = info + s * kInfoN;
    if (inf[PAM_INFO_STOPPED]) return;
    const int M = inf[PAM_INFO_M], N = inf[PAM_INFO_N_CELLS], mc = g.m_cap;
    const float lam1 = (float)((double)N * p.lam1_hat), lam2 = (float)((double)N * p.lam2_hat);
    // stage 1 only has to find a good support: G~ carries ~1e-5 relative error
    const float tol_pdas = lam1 * (1.0f + 1e-3f);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int32_t *box = boxes + s * 12;

    extern __shared__ __align__(16) uint8_t sm[];
    float *x = reinterpret_cast<float *>(sm);     // [mc]
    float *gr = x + mc;                           // [mc] b - G~ x (stage 1), exact c (stage 2)
    float *bv = gr + mc;                          // [mc]
    float *rhs = bv + mc;                         // [mc]
    int *sg = reinterpret_cast<int *>(rhs + mc);  // [mc]
    int *idx = sg + mc;                           // [mc]
    float4 *sc = reinterpret_cast<float4 *>(idx + mc);      // [mc] local centres
    float4 *cell = sc + mc;                                 // [n_max] (x, y, z, rowmax)
    float *cinv = reinterpret_cast<float *>(cell + g.n_max);// [n_max]
    float *ce = cinv + g.n_max;                             // [n_max] y, then e = y - W x
    float *dinv = ce + g.n_max;                             // [mc] 1 / diag of the factor
    float *Asm = dinv + mc;                                 // packed factor
    __shared__ MxShared sh;

    const float *G = w.Gf + (size_t)s * mc * mc;
    const float *rowmax = w.rowmax + (size_t)s * g.n_max;
    const float *rowinv = w.rowinv + (size_t)s * g.n_max;
    double o[3];
    patch_origin(g, box, o);
    const dvec4 *cg = reinterpret_cast<const dvec4 *>(centres) + (size_t)s * mc;
    for (int j = tid; j < mc; j += blockDim.x) {
        float b0 = j < M ? (float)beta[(size_t)s * mc + j] : 0.f;
        x[j] = b0;
        bv[j] = j < M ? (float)w.b[(size_t)s * mc + j] : 0.f;
        sg[j] = (j < M) ? ((b0 > 0.f) - (b0 < 0.f)) : 0;
        if (j < M) sc[j] = local_centre(cg[j], o);
    }
    for (int t = tid; t < N; t += blockDim.x) {
        float xl[3];
        local_cell(g, box, t, xl);
        cell[t] = make_float4(xl[0], xl[1], xl[2], rowmax[t]);
        cinv[t] = rowinv[t];
    }
    if (tid == 0) sh.flag = 0;
    __syncthreads();
    PROF_T0();
    PROF_MARK(0);
#ifdef PAM_SOLVE_PROFILE
    const long long t_blk0 = clock64();
#endif

    // ---------------- stage 1: active-set iterations on G~ ----------------
    // Up to kMxPdasFull full primal-dual corrections; if the support still
    // moves, a primal active-set phase takes over from the sign-consistent
    // part of the iterate: on the current support it steps towards the
    // sign-constrained minimiser as far as the signs allow (ratio test),
    // dropping the coefficient that reaches zero, and adds violators only
    // once the minimiser on the support is
    // sign-consistent (all violators; the largest only right after a step
    // that a newly added coefficient blocked at length zero) -- the
    // objective decreases monotonically, so it ends.
    int it = 0, scnt = 0;
    float *A = Asm;
    auto factor_support = [&]() {
        mx_compact(sg, M, idx, &sh.cnt);
        scnt = sh.cnt;
        A = (tri_i(scnt, 0) * 4 <= kMxFactorBytes) ? Asm
            : (w.Lf + (size_t)s * ((size_t)mc * (mc + 1) / 2));
        PROF_MARK(8);
        for (int pp = warp; pp < scnt; pp += nw) {
            const float *Gr = G + (size_t)idx[pp] * mc;
            for (int q = lane; q <= pp; q += 32) A[tri_i(pp, q)] = Gr[idx[q]] + (q == pp ? lam2 : 0.f);
            if (lane == 0) rhs[pp] = bv[idx[pp]] - lam1 * (float)sg[idx[pp]];
        }
        __syncthreads();
        PROF_MARK(9);
        mx_cholesky(A, scnt, &sh.flag, dinv);
        PROF_MARK(10);
        if (!sh.flag) mx_chol_solve(A, dinv, scnt, rhs);
        PROF_MARK(11);
    };
    auto gradient_fp = [&]() {  // gr = b - G~ x; G~ symmetric: rows of the support, coalesced over j
        for (int j = tid; j < M; j += blockDim.x) {
            float acc0 = 0.f, acc1 = 0.f;
            int pp = 0;
            for (; pp + 1 < scnt; pp += 2) {
                const int m0 = idx[pp], m1 = idx[pp + 1];
                acc0 = fmaf(G[(size_t)m0 * mc + j], x[m0], acc0);
                acc1 = fmaf(G[(size_t)m1 * mc + j], x[m1], acc1);
            }
            if (pp < scnt) acc0 = fmaf(G[(size_t)idx[pp] * mc + j], x[idx[pp]], acc0);
            gr[j] = bv[j] - (acc0 + acc1);
        }
        __syncthreads();
    };
    bool primal = false, single_add = false;
    int last_added = -1;
    const int max_pdas = p.max_iters < kMxMaxPdas ? p.max_iters : kMxMaxPdas;
    for (; it < max_pdas; ++it) {
        factor_support();
        PROF_MARK(1);
        if (sh.flag) break;
        if (!primal) {
            for (int j = tid; j < M; j += blockDim.x) x[j] = 0.f;
            __syncthreads();
            for (int pp = tid; pp < scnt; pp += blockDim.x) x[idx[pp]] = rhs[pp];
            __syncthreads();
            gradient_fp();
            PROF_MARK(2);
            if (tid == 0) { sh.bad = 0; sh.viol = 0; }
            __syncthreads();
            int mb = 0, mv = 0;
            for (int j = tid; j < M; j += blockDim.x) {
                if (sg[j] != 0) mb += !(x[j] * (float)sg[j] > 0.f);
                else mv += fabsf(gr[j]) > tol_pdas;
            }
            if (mb) atomicAdd(&sh.bad, mb);
            if (mv) atomicAdd(&sh.viol, mv);
            __syncthreads();
            if (sh.bad == 0 && sh.viol == 0) break;
            if (it + 1 < kMxPdasFull) {
                for (int j = tid; j < M; j += blockDim.x) {
                    if (sg[j] != 0) {
                        if (!(x[j] * (float)sg[j] > 0.f)) sg[j] = 0;
                    } else if (fabsf(gr[j]) > tol_pdas) {
                        sg[j] = gr[j] > 0.f ? 1 : -1;
                    }
                }
            } else {
                // switch: keep the sign-consistent part of the iterate
                for (int j = tid; j < M; j += blockDim.x)
                    if (!(x[j] * (float)sg[j] > 0.f)) { sg[j] = 0; x[j] = 0.f; }
                primal = true;
            }
            __syncthreads();
            PROF_MARK(3);
            continue;
        }
        // primal phase: x is sign-consistent on the support; rhs = minimiser
        if (tid == 0) { sh.dmax = 2.f; sh.bad = 0; }
        __syncthreads();
        for (int pp = tid; pp < scnt; pp += blockDim.x) {
            const int m = idx[pp];
            const float xs = rhs[pp], x0 = x[m], sgn = (float)sg[m];
            if (!(xs * sgn > 0.f)) {
                const float a = (x0 * sgn > 0.f) ? x0 / (x0 - xs) : 0.f;
                atomicMin(reinterpret_cast<int *>(&sh.dmax), __float_as_int(fmaxf(a, 0.f)));
                atomicAdd(&sh.bad, 1);
            }
        }
        __syncthreads();
        if (sh.bad == 0) {
            for (int pp = tid; pp < scnt; pp += blockDim.x) x[idx[pp]] = rhs[pp];
            __syncthreads();
            gradient_fp();
            if (single_add) {
                if (tid == 0) {
                    float best = tol_pdas;
                    int bj = -1;
                    for (int j = 0; j < M; ++j)
                        if (sg[j] == 0 && fabsf(gr[j]) > best) { best = fabsf(gr[j]); bj = j; }
                    sh.viol = bj;
                    if (bj >= 0 && bj != last_added) { sg[bj] = gr[bj] > 0.f ? 1 : -1; x[bj] = 0.f; }
                }
                __syncthreads();
                if (sh.viol < 0 || sh.viol == last_added) break;  // optimal (or stalled on one index)
                last_added = sh.viol;
            } else {
                if (tid == 0) sh.viol = 0;
                __syncthreads();
                int mv = 0;
                for (int j = tid; j < M; j += blockDim.x)
                    if (sg[j] == 0 && fabsf(gr[j]) > tol_pdas) { sg[j] = gr[j] > 0.f ? 1 : -1; x[j] = 0.f; ++mv; }
                if (mv) atomicAdd(&sh.viol, mv);
                __syncthreads();
                if (sh.viol == 0) break;  // optimal
            }
            single_add = false;
        } else {
            // step alpha towards the minimiser; the blocking coefficients (the
            // ones whose ratio attains alpha) reach zero and leave the support
            const float alpha = fminf(sh.dmax, 1.f);
            single_add = !(alpha > 0.f);  // blocked by a coefficient that just joined
            for (int pp = tid; pp < scnt; pp += blockDim.x) {
                const int m = idx[pp];
                const float xs = rhs[pp], x0 = x[m], sgn = (float)sg[m];
                bool blocking = false;
                if (!(xs * sgn > 0.f)) {
                    const float a = (x0 * sgn > 0.f) ? x0 / (x0 - xs) : 0.f;
                    blocking = fmaxf(a, 0.f) <= alpha * (1.f + 1e-6f);
                }
                const float nx = x0 + alpha * (xs - x0);
                if (blocking || !(nx * sgn > 0.f)) {
                    x[m] = 0.f;
                    sg[m] = 0;
                } else {
                    x[m] = nx;
                }
            }
            __syncthreads();
        }
    }
    // ---------------- stage 2: refinement with the exact gradient ---------
    // Certified when, with the exact gradient c, the stationarity residual on
    // the support is below rtol and no coefficient off it violates
    // |c_j| <= lambda1 (1 + 1e-3): the fp32 form of the optimality conditions.
    // A coefficient inside that band has |beta_j| <= 1e-3 lambda1 / (G_jj +
    // lambda2) at the exact minimiser (changes W beta by <~1e-5); admitting it
    // only makes near-degenerate coordinates cycle in and out of the support.
    const float kkt_tol = lam1 * (1.0f + 1e-3f);
    int certified = 0, refine_it = 0;
    const double *yv = w.y + (size_t)s * g.n_max;
    for (; refine_it < kMxMaxRefine && !sh.flag; ++refine_it) {
        // e = y - W x over the patch (only the support contributes); W x is
        // accumulated in double-float and subtracted in fp64: |y| ~ 10 would
        // otherwise leave ~1e-6 of cancellation noise in e, and W^T e inherits it
        for (int t = tid; t < N; t += blockDim.x) {
            const float4 cx = cell[t];
            DFAcc acc;
            for (int pp = 0; pp < scnt; ++pp) {
                const int m = idx[pp];
                acc.add_prod(tc::ex2(logit2(sc[m], cx.x, cx.y, cx.z) - cx.w), x[m]);
            }
            ce[t] = (float)(yv[t] - acc.value() * (double)cinv[t]);
        }
        __syncthreads();
        PROF_MARK(4);
        // c_j = sum_t W_tj e_t for every centre (exact gradient of the data term)
        float cmax = 0.f;
        for (int j = tid; j < M; j += blockDim.x) {
            const float4 cj = sc[j];
            float acc = 0.f;
            for (int t = 0; t < N; ++t) {
                const float4 cx = cell[t];
                acc = fmaf(tc::ex2(logit2(cj, cx.x, cx.y, cx.z) - cx.w) * cinv[t], ce[t], acc);
            }
            gr[j] = acc;
            cmax = fmaxf(cmax, fabsf(acc));
        }
        if (tid == 0) { sh.viol = 0; sh.changed = 0; sh.dmax = 0.f; sh.xmax = 0.f; }
        __syncthreads();
        PROF_MARK(5);
        // stationarity residual on the support, violations off it
        float rmax = 0.f;
        int mv = 0;
        for (int j = tid; j < M; j += blockDim.x) {
            if (sg[j] != 0) rmax = fmaxf(rmax, fabsf(gr[j] - lam2 * x[j] - lam1 * (float)sg[j]));
            else if (fabsf(gr[j]) > kkt_tol) ++mv;
        }
        for (int o2 = 16; o2 > 0; o2 >>= 1) {
            rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o2));
            cmax = fmaxf(cmax, __shfl_xor_sync(0xffffffffu, cmax, o2));
            mv += __shfl_xor_sync(0xffffffffu, mv, o2);
        }
        if (lane == 0) {
            atomicMax(reinterpret_cast<int *>(&sh.dmax), __float_as_int(rmax));
            atomicMax(reinterpret_cast<int *>(&sh.xmax), __float_as_int(cmax));
            if (mv) atomicAdd(&sh.viol, mv);
        }
        __syncthreads();
        const float rtol = 1e-4f * lam1 + 1e-6f * sh.xmax;
        if (sh.viol == 0 && sh.dmax <= rtol) { certified = 1; break; }
        // violators join the support with the sign of their gradient
        int jn = 0;
        for (int j = tid; j < M; j += blockDim.x)
            if (sg[j] == 0 && fabsf(gr[j]) > kkt_tol) { sg[j] = gr[j] > 0.f ? 1 : -1; x[j] = 0.f; ++jn; }
        if (jn) atomicOr(&sh.changed, 1);
        __syncthreads();
        if (sh.changed) {
            mx_compact(sg, M, idx, &sh.cnt);
            scnt = sh.cnt;
            A = (tri_i(scnt, 0) * 4 <= kMxFactorBytes) ? Asm
                : (w.Lf + (size_t)s * ((size_t)mc * (mc + 1) / 2));
            for (int pp = warp; pp < scnt; pp += nw) {
                const float *Gr = G + (size_t)idx[pp] * mc;
                for (int q = lane; q <= pp; q += 32) A[tri_i(pp, q)] = Gr[idx[q]] + (q == pp ? lam2 : 0.f);
            }
            __syncthreads();
            mx_cholesky(A, scnt, &sh.flag, dinv);
            if (sh.flag) break;
        }
        // Newton correction on the support
        for (int pp = tid; pp < scnt; pp += blockDim.x) {
            const int m = idx[pp];
            rhs[pp] = gr[m] - lam2 * x[m] - lam1 * (float)sg[m];
        }
        __syncthreads();
        mx_chol_solve(A, dinv, scnt, rhs);
        int dropped = 0;
        for (int pp = tid; pp < scnt; pp += blockDim.x) {
            const int m = idx[pp];
            const float nx = x[m] + rhs[pp];
            if (!(nx * (float)sg[m] > 0.f)) { sg[m] = 0; x[m] = 0.f; ++dropped; }
            else x[m] = nx;
        }
        for (int o2 = 16; o2 > 0; o2 >>= 1) dropped += __shfl_xor_sync(0xffffffffu, dropped, o2);
        if (lane == 0 && dropped) atomicOr(&sh.changed, 2);
        __syncthreads();
        if (sh.changed & 2) {  // support shrank: recompact and refactor
            mx_compact(sg, M, idx, &sh.cnt);
            scnt = sh.cnt;
            A = (tri_i(scnt, 0) * 4 <= kMxFactorBytes) ? Asm
                : (w.Lf + (size_t)s * ((size_t)mc * (mc + 1) / 2));
            for (int pp = warp; pp < scnt; pp += nw) {
                const float *Gr = G + (size_t)idx[pp] * mc;
                for (int q = lane; q <= pp; q += 32) A[tri_i(pp, q)] = Gr[idx[q]] + (q == pp ? lam2 : 0.f);
            }
            __syncthreads();
            mx_cholesky(A, scnt, &sh.flag, dinv);
        }
    }

    PROF_MARK(6);
    // final residual e = y - W x, and the indicators R_T (Eq. (4), midpoint)
    for (int t = tid; t < N; t += blockDim.x) {
        const float4 cx = cell[t];
        DFAcc acc;
        for (int pp = 0; pp < scnt; ++pp) {
            const int m = idx[pp];
            acc.add_prod(tc::ex2(logit2(sc[m], cx.x, cx.y, cx.z) - cx.w), x[m]);
        }
        const double yhat = acc.value() * (double)cinv[t];
        const double kv = w.kv[(size_t)s * g.n_max + t];
        const double e = exp(yhat) - kv;
        w.R[(size_t)s * g.n_max + t] = g.vol * (e * e);
    }
    for (int j = tid; j < M; j += blockDim.x) beta[(size_t)s * mc + j] = (double)x[j];
    __syncthreads();
    PROF_MARK(7);
#ifdef PAM_SOLVE_PROFILE
    if (tid == 0 && s < 8192) g_solve_blk[s] = (unsigned long long)(clock64() - t_blk0);
#endif
    if (tid == 0) {
        int flags = inf[PAM_INFO_FLAGS] & ~(PAM_FLAG_NOT_CERTIFIED | PAM_FLAG_CHOLESKY);
        if (!certified) {
            flags |= PAM_FLAG_NOT_CERTIFIED;
            atomicAdd(&w.status[kStUncertified], 1);
        }
        if (sh.flag) flags |= PAM_FLAG_CHOLESKY;
        inf[PAM_INFO_FLAGS] = flags;
        inf[PAM_INFO_SUPPORT] = scnt;
        inf[PAM_INFO_ITERS] = it + 100 * refine_it;  // active-set steps + 100 x refinement steps
    }
}

// Shared-memory budget of the packed factor: supports with s (s+1)/2 fp32
// beyond it keep their factor in global memory (L1/L2). A smaller budget
// lets more subdomains share an SM. PAM_FACTOR_SMEM_KB overrides the
// default for tuning.
static int factor_smem_bytes() {
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("PAM_FACTOR_SMEM_KB");
        v = e ? atoi(e) * 1024 : kMxFactorBytesDefault;
        if (v < 4096) v = 4096;
    }
    return v;
}

static size_t solve_mixed_smem(const Geo &g) {
    return (size_t)g.m_cap * (5 * sizeof(float) + 2 * sizeof(int) + sizeof(float4)) +
           (size_t)g.n_max * (sizeof(float4) + 2 * sizeof(float)) + factor_smem_bytes() + 64;
}

#ifdef PAM_SOLVE_PROFILE
extern "C" void pam_debug_solve_blocks(unsigned long long *out, int n) {
    cudaMemcpyFromSymbol(out, g_solve_blk, sizeof(unsigned long long) * (n < 8192 ? n : 8192));
}
extern "C" void pam_debug_solve_profile(unsigned long long *out, int reset) {
    cudaMemcpyFromSymbol(out, g_solve_prof, sizeof(g_solve_prof));
    if (reset) {
        unsigned long long z[16] = {};
        cudaMemcpyToSymbol(g_solve_prof, z, sizeof(z));
    }
}
#endif

bool mixed_solve_fits(const Geo &g) {
    return solve_mixed_smem(g) <= 227 * 1024 && gram_tc_smem(g) <= 227 * 1024;
}

void launch_solve_level_mixed(const Geo &g, const Par &p, const int32_t *boxes,
                              const double *centres, double *beta, int32_t *info, const Ws &w,
                              cudaStream_t st) {
    launch_stats_gram_tc(g, boxes, centres, info, w, st, 0);
    size_t sm = solve_mixed_smem(g);
    cudaFuncSetAttribute(k_solve_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    PhaseScope ps(kPhSolve, st);
    k_solve_mixed<<<g.S, kMxThreads, sm, st>>>(g, p, boxes, centres, beta, info, w, factor_smem_bytes());
    count_launches(1);
}

// The mixed solve already wrote the indicators of its final coefficients.
void launch_residual_mixed(const Geo &, const int32_t *, const double *, const double *,
                           const int32_t *, const Ws &, cudaStream_t) {}

}  // namespace pam
