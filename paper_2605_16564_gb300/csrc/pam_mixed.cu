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
#include "pam_chol.cuh"

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

// sc[0..n) = local_centre(c[0..n)): the n centres (32 bytes each) are first
// copied into the shared-memory scratch `stage` by the bulk-copy engine (when
// use_stage, the scratch holds n x 32 bytes and the copy is aligned; plain
// loads otherwise). Called by the whole block.
__device__ __noinline__ void stage_local_centres(float4 *sc, const dvec4 *c, int n, const double o[3], void *stage,
                                                 bool use_stage) {
    __shared__ uint64_t bar;
    const bool staged = use_stage && n > 0 && tc::bulk_stage_block(stage, c, (uint32_t)n * 32u, &bar);
    const double2 *cs = reinterpret_cast<const double2 *>(stage);
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        dvec4 v;
        if (staged) {
            const double2 a = cs[2 * r], b = cs[2 * r + 1];
            v.x = a.x; v.y = a.y; v.z = b.x; v.w = b.y;
        } else {
            v = c[r];
        }
        sc[r] = local_centre(v, o);
    }
}

__device__ __forceinline__ void patch_origin(const Geo &g, const int32_t *box, double o[3]) {
    for (int a = 0; a < 3; ++a) o[a] = a < g.dim ? (double)box[6 + a] * g.h : 0.0;
}

// The same, computed once per block and read from shared memory (the
// binary64 pipe is narrow on this part; a block of 1024 threads would
// otherwise repeat the products 1024 times). Called by the whole block.
__device__ __forceinline__ void patch_origin_block(const Geo &g, const int32_t *box, double o[3]) {
    __shared__ double so[3];
    __syncthreads();  // a previous call's readers are done
    if (threadIdx.x == 0) patch_origin(g, box, so);
    __syncthreads();
    for (int a = 0; a < 3; ++a) o[a] = so[a];
}

// Local coordinates of patch cell t: ((i - patch_lo) + 1/2) h, exact in fp32
// up to one rounding; for a mesh given as cells, the gathered sampling point
// minus the patch origin, rounded once to fp32.
__device__ __forceinline__ void local_cell(const Geo &g, int s, const int32_t *box, int t, float x[3]) {
    if (g.cxv) {
        const double4_32a v = g.cxv[(size_t)s * g.n_max + t];
        x[0] = (float)(v.x - (double)box[6] * g.h);
        x[1] = g.dim > 1 ? (float)(v.y - (double)box[7] * g.h) : 0.0f;
        x[2] = g.dim > 2 ? (float)(v.z - (double)box[8] * g.h) : 0.0f;
        return;
    }
    int w0 = box[9] - box[6], w1 = box[10] - box[7];
    int i = t % w0, j = (t / w0) % w1, k = t / (w0 * w1);
    float hf = (float)g.h;
    x[0] = ((float)i + 0.5f) * hf;
    x[1] = g.dim > 1 ? ((float)j + 0.5f) * hf : 0.0f;
    x[2] = g.dim > 2 ? ((float)k + 0.5f) * hf : 0.0f;
}

// --------------------------------------------------------------------------
// Row statistics of the Shepard normalisation (Eq. (10)): a shift l2* and
// 1 / sum_m 2^(l2_jm - l2*), so that W_jm = 2^(l2_jm - l2*) / sum. Every
// l2_jm <= 0 and a patch cell lies within a few widths of the initial
// lattice, so the plain sum of 2^(l2_jm) stays far above the fp32 underflow
// and l2* = 0 serves: one pass with one exp and one add per centre, two
// cells per thread (t and t + blockDim.x) sharing each centre read. A cell
// whose plain sum falls below 2^-100 takes a second pass with the running
// maximum as the shift (the sum rescaled whenever the maximum grows).
// --------------------------------------------------------------------------
// Centre m of the statistics' shared-memory table, stored for the packed
// two-cell arithmetic as (-c_x, -c_x, -c_y, -c_y), (-c_z, -c_z, alpha, alpha).
__device__ __forceinline__ float4 stats_centre(const float4 *scp, int m) {
    const float4 a = scp[2 * m], b = scp[2 * m + 1];
    return make_float4(-a.x, -a.z, -b.x, b.z);
}

__device__ __noinline__ void stats_max_shift(const float4 *scp, int M, const float x[3], float *lmax_out,
                                             float *sum_out) {
    float lmax = -INFINITY, sum = 0.0f;
    for (int m = 0; m < M; ++m) {
        const float l = logit2(stats_centre(scp, m), x[0], x[1], x[2]);
        if (l > lmax) {
            sum = fmaf(sum, tc::ex2(lmax - l), 1.0f);
            lmax = l;
        } else {
            sum += tc::ex2(l - lmax);
        }
    }
    *lmax_out = lmax;
    *sum_out = sum;
}

__device__ __forceinline__ void stats_store(const Ws &w, size_t o, const float4 *scp, int M, const float x[3],
                                            float sum) {
    float shift = 0.0f;
    if (!(sum > 0x1p-100f)) stats_max_shift(scp, M, x, &shift, &sum);
    w.rowmax[o] = shift;
    w.rowinv[o] = 1.0f / sum;
}

// The two cells of a thread go through each centre together, one per half of
// each packed fp32x2 operation: the same operations, in the same order, as
// logit2 and the scalar sum of each cell.
__global__ void __launch_bounds__(256) k_stats_f32(Geo g, const int32_t *boxes,
                                                   const double *centres, const int32_t *info,
                                                   Ws w, int all) {
    const int s = group_sub(g, blockIdx.y);
    const int32_t *inf = info + s * kInfoN;
    if (!all && inf[PAM_INFO_STOPPED]) return;
    const int M = inf[PAM_INFO_M], N = inf[PAM_INFO_N_CELLS];
    const int32_t *box = boxes + s * 12;
    extern __shared__ float4 scp[];  // [2 * m_cap]
    double o[3];
    patch_origin_block(g, box, o);
    const dvec4 *cg = reinterpret_cast<const dvec4 *>(centres) + (size_t)s * g.m_cap;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const float4 c = local_centre(cg[m], o);
        scp[2 * m] = make_float4(-c.x, -c.x, -c.y, -c.y);
        scp[2 * m + 1] = make_float4(-c.z, -c.z, c.w, c.w);
    }
    __syncthreads();
    const int t0 = blockIdx.x * 2 * blockDim.x + threadIdx.x, t1 = t0 + blockDim.x;
    if (t0 >= N) return;
    const bool two = t1 < N;
    float x0[3], x1[3];
    local_cell(g, s, box, t0, x0);
    local_cell(g, s, box, two ? t1 : t0, x1);
    const float2 X = make_float2(x0[0], x1[0]), Y = make_float2(x0[1], x1[1]), Z = make_float2(x0[2], x1[2]);
    float2 sum = make_float2(0.f, 0.f);
    for (int m = 0; m < M; ++m) {
        const float4 a = scp[2 * m], b = scp[2 * m + 1];
        const float2 dx = __fadd2_rn(X, make_float2(a.x, a.y));
        const float2 dy = __fadd2_rn(Y, make_float2(a.z, a.w));
        const float2 dz = __fadd2_rn(Z, make_float2(b.x, b.y));
        float2 d2 = __fmul2_rn(dx, dx);
        d2 = __ffma2_rn(dy, dy, d2);
        d2 = __ffma2_rn(dz, dz, d2);
        const float2 l = __fmul2_rn(make_float2(b.z, b.w), d2);
        sum = __fadd2_rn(make_float2(tc::ex2(l.x), tc::ex2(l.y)), sum);
    }
    const size_t row = (size_t)s * g.n_max;
    stats_store(w, row + t0, scp, M, x0, sum.x);
    if (two) stats_store(w, row + t1, scp, M, x1, sum.y);
}

// --------------------------------------------------------------------------
// Gram products on the tensor cores. The dictionary (padded to Mp, a
// multiple of 32) is cut into strips of 128 centres; strip i needs
// D_i = W_{I_i}^T W_{[128 i, Mp)} (128 x R_i, R_i = Mp - 128 i: the upper
// block row, by symmetry). Consecutive strips are grouped, from the last one
// backwards, while their D blocks fit the 512 TMEM columns together; one CTA
// per (subdomain, group) generates W once for the rows from the group's
// first strip to Mp and accumulates every D block of the group over chunks
// of 32 cells. Warp-specialised pipeline over nst (3, or 2 where shared
// memory is short) stages:
//   * warps 1..31 produce: each thread generates the chunk's W values of one
//     centre row for one, two or four groups of 8 cells, splits them into
//     bf16 hi/lo parts and stores them in the canonical K-major layout
//     (8-row x 16-byte core matrices), then its warp arrives on the stage's
//     `full` barrier;
//   * one thread of warp 0 waits for `full`, issues hi*hi + hi*lo + lo*hi for
//     every strip of the group (A = the strip's 128 rows of the tile, B = the
//     tile from the same row on) and commits to the stage's `empty` barrier,
//     which the producers wait for before they overwrite the stage.
// No block-wide barrier inside the loop. Epilogue: all warps read the D
// blocks from TMEM and write rows of G (and the mirrored blocks below the
// strips) in fp32; the producers' partial sums give b = W^T y.
// --------------------------------------------------------------------------
constexpr int kTcThreads = 1024;
constexpr int kTcIssuers = 4;            // warps 0..3: one MMA-issuing thread each
constexpr int kTcProdWarps = kTcThreads / 32 - kTcIssuers;
constexpr int kTcKC = 32;                 // cells per chunk (2 MMA k-steps of 16)
constexpr int kTcMaxStages = 3;            // 3 where shared memory allows, else 2
constexpr int kTcMaxRows = kMixedMaxM;    // rows of the B tile
constexpr int kTcCols = 512;              // TMEM columns
constexpr long long kWaitBudget = 4000000000LL;  // ~2 s at 2 GHz
constexpr int kTcStageFloats = 32 * 33;   // epilogue transpose buffer per warp
constexpr size_t kSmemLimit = 227 * 1024;  // dynamic shared memory per CTA

__device__ __forceinline__ void mbar_arrive(uint64_t *m) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}\n"
                 ::"r"(tc::smem_u32(m)) : "memory");
}

// Strip group q of a padded dictionary of Mp centres: strips [*i0, *i1).
// Groups are formed from the last strip backwards while sum R_i <= 512 and
// numbered from the front. Returns the number of groups (at most 4).
__host__ __device__ __forceinline__ int tc_strip_group(int Mp, int q, int *i0, int *i1) {
    const int nS = (Mp + 127) / 128;
    int start[4], n = 0;
    for (int i = nS - 1; i >= 0 && n < 4;) {
        int sum = 0, j = i;
        while (j >= 0 && sum + (Mp - 128 * j) <= kTcCols) { sum += Mp - 128 * j; --j; }
        start[n++] = j + 1;
        i = j;
    }
    const int b = n - 1 - q;  // groups were listed back to front
    if (b >= 0 && b < n) {
        *i0 = start[b];
        *i1 = b == 0 ? nS : start[b - 1];
    }
    return n;
}

// Tile rows of a group: the generated rows, padded so that every strip's
// 128 A rows lie inside the tile.
__host__ __device__ __forceinline__ int tc_tile_rows(int Mp, int i0, int i1) {
    const int R = Mp - 128 * i0;
    return R > 128 * (i1 - i0) ? R : 128 * (i1 - i0);
}

// The largest tile of any dictionary size up to m_cap: the shared-memory
// layout of every CTA of a launch.
static int tc_rows_cap(int m_cap) {
    int cap = 128;
    for (int Mp = 32; Mp <= ((m_cap + 31) & ~31); Mp += 32) {
        int i0 = 0, i1 = 0;
        const int n = tc_strip_group(Mp, 0, &i0, &i1);
        for (int q = 0; q < n; ++q) {
            tc_strip_group(Mp, q, &i0, &i1);
            const int rt = tc_tile_rows(Mp, i0, i1);
            cap = rt > cap ? rt : cap;
        }
    }
    return cap;
}

// Producer threads per generated row: 4, 2 or 1 (each covering 4 / tpr
// k-groups of 8 cells of a chunk), the most that one thread per (row, part)
// allows.
__host__ __device__ __forceinline__ int tc_threads_per_row(int Rl) {
    return (4 * Rl <= 32 * kTcProdWarps) ? 4 : (2 * Rl <= 32 * kTcProdWarps ? 2 : 1);
}

// One generated row of the producers: the centre's constants duplicated for
// the packed two-cell arithmetic, and its running sums of W y and W (one per
// half: even and odd cells).
struct ProdRow {
    float2 ncx, ncy, ncz, cw, b, w;
};
__device__ __forceinline__ ProdRow prod_row(const float4 &cc) {
    ProdRow r;
    r.ncx = make_float2(-cc.x, -cc.x);
    r.ncy = make_float2(-cc.y, -cc.y);
    r.ncz = make_float2(-cc.z, -cc.z);
    r.cw = make_float2(cc.w, cc.w);
    r.b = make_float2(0.f, 0.f);
    r.w = make_float2(0.f, 0.f);
    return r;
}

// W of one row at a cell pair (a = (x, x', y, y'), b = (z, z', -sh, -sh'),
// yy = (ln K, ln K')): one cell per half of each packed operation -- the
// same operations, in the same order, as the scalar exponent
// cc.w |x - c|^2 - sh of each cell -- split into bf16 hi and lo pairs
// (v = hi + lo to about 2^-16 relative).
__device__ __forceinline__ void prod_pair(ProdRow &r, const float4 &a, const float4 &b, const float2 &yy,
                                          uint32_t *hp, uint32_t *lp) {
    const float2 dx = __fadd2_rn(make_float2(a.x, a.y), r.ncx);
    const float2 dy = __fadd2_rn(make_float2(a.z, a.w), r.ncy);
    const float2 dz = __fadd2_rn(make_float2(b.x, b.y), r.ncz);
    float2 d2 = __fmul2_rn(dx, dx);
    d2 = __ffma2_rn(dy, dy, d2);
    d2 = __ffma2_rn(dz, dz, d2);
    const float2 l = __ffma2_rn(r.cw, d2, make_float2(b.z, b.w));
    const float2 e = make_float2(tc::ex2(l.x), tc::ex2(l.y));
    r.b = __ffma2_rn(e, yy, r.b);
    r.w = __fadd2_rn(e, r.w);
    *hp = tc::pack_bf16(e.x, e.y);
    const float2 h = make_float2(__uint_as_float(*hp << 16), __uint_as_float(*hp & 0xffff0000u));
    const float2 rl = __ffma2_rn(h, make_float2(-1.f, -1.f), e);  // e - h, exact
    *lp = tc::pack_bf16(rl.x, rl.y);
}

#ifdef PAM_SOLVE_PROFILE
// Profiling builds only: clock64 totals of the Gram pipeline (per CTA, seen
// from the MMA thread and from the first producer thread).
__device__ unsigned long long g_gram_prof[16];
#define GP_ADD(k, v) atomicAdd(&g_gram_prof[k], (unsigned long long)(v))
#else
#define GP_ADD(k, v)
#endif

// folds > 0: only the cells t with t mod folds != fold enter G and b (the
// training rows of a cross-validation fold); the others stage as padding.
__global__ void __launch_bounds__(kTcThreads, 1) k_gram_tc(Geo g, const int32_t *boxes,
                                                           const double *centres,
                                                           const int32_t *info, Ws w, int all,
                                                           int nst, int Rcap, int folds, int fold) {
    const int s = group_sub(g, blockIdx.y);
    const int32_t *inf = info + s * kInfoN;
    if (!all && inf[PAM_INFO_STOPPED]) return;
    const int M = inf[PAM_INFO_M], N = inf[PAM_INFO_N_CELLS];
    const int Mp = (M + 31) & ~31;                 // padded dictionary size
    int i0 = 0, i1 = 0;
    if ((int)blockIdx.x >= tc_strip_group(Mp, blockIdx.x, &i0, &i1)) return;
#ifdef PAM_SOLVE_PROFILE
    const long long gp_t0 = clock64();
#endif
    const int row0 = 128 * i0;                      // first generated row
    const int Rl = M - row0;                        // live rows (the rest are zero)
    const int Rt = tc_tile_rows(Mp, i0, i1);        // tile rows (<= Rcap)
    int tcols = 0;
    for (int i = i0; i < i1; ++i) tcols += Mp - 128 * i;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int32_t *box = boxes + s * 12;

    extern __shared__ __align__(1024) uint8_t smem[];
    // stage st: hi tile then lo tile, each Rt x kTcKC bf16 (Rt * 64 bytes)
    const uint32_t tile_bytes = (uint32_t)Rt * kTcKC * 2;
    uint8_t *tiles = smem;
    const size_t tiles_region = (size_t)nst * 2 * Rcap * kTcKC * 2 > (size_t)32 * kTcStageFloats * 4
                                    ? (size_t)nst * 2 * Rcap * kTcKC * 2
                                    : (size_t)32 * kTcStageFloats * 4;
    float4 *sc = reinterpret_cast<float4 *>(smem + tiles_region);   // [Rcap]
    float *bpart = reinterpret_cast<float *>(sc + Rcap);             // [4][Rcap]
    float *wpart = bpart + 4 * Rcap;                                 // [4][Rcap]
    // the cells in pairs (2p, 2p + 1): cella[p] = (x, x', y, y'), cellb[p] =
    // (z, z', -sh, -sh'), celly2[p] = (ln K, ln K') -- 20 bytes per cell
    const int nch = (N + kTcKC - 1) / kTcKC;
    float4 *cella = reinterpret_cast<float4 *>(wpart + 4 * Rcap);    // [nch * 16]
    float4 *cellb = cella + (size_t)nch * (kTcKC / 2);               // [nch * 16]
    float2 *celly2 = reinterpret_cast<float2 *>(cellb + (size_t)nch * (kTcKC / 2));  // [nch * 16]
    __shared__ uint64_t full[kTcMaxStages], empty[kTcMaxStages], drain;
    __shared__ uint32_t tmem_base;
    __shared__ int timed_out;

    double o[3];
    patch_origin_block(g, box, o);
    const dvec4 *cg = reinterpret_cast<const dvec4 *>(centres) + (size_t)s * g.m_cap;
    // plain loads: a bulk copy of the centres into the (still free) tile
    // buffers measured 1 % slower over the step (2.110 -> 2.133 ms at the
    // last level): the 1024 threads' loads are already all in flight at once
    for (int r = tid; r < Rl; r += blockDim.x) sc[r] = local_centre(cg[row0 + r], o);
    const float *rowmax = w.rowmax + (size_t)s * g.n_max;
    const float *rowinv = w.rowinv + (size_t)s * g.n_max;
    const double *yv = w.y + (size_t)s * g.n_max;
    for (int t = tid; t < nch * kTcKC; t += blockDim.x) {
        float x[3] = {0.f, 0.f, 0.f};
        float sh = INFINITY, y = 0.f;
        if (t < N && (folds == 0 || t % folds != fold)) {
            local_cell(g, s, box, t, x);
            sh = rowmax[t] - log2f(rowinv[t]);
            y = (float)yv[t];
        }
        float *fa = reinterpret_cast<float *>(cella + (t >> 1)), *fb = reinterpret_cast<float *>(cellb + (t >> 1));
        const int h = t & 1;
        fa[h] = x[0];
        fa[2 + h] = x[1];
        fb[h] = x[2];
        fb[2 + h] = -sh;  // -inf past the patch: the weight is 0
        reinterpret_cast<float *>(celly2 + (t >> 1))[h] = y;
    }
    // rows past the live ones stay zero in every stage
    {
        const int nz = Rt - Rl, per = 4 * nz;  // (row, k-group) pairs per tile
        for (int e = tid; e < nst * 2 * per; e += blockDim.x) {
            const int t2 = e / per, rem = e % per, kg = rem / nz, r = Rl + rem % nz;
            const uint32_t off = (uint32_t)(kg * (Rt >> 3) + (r >> 3)) * 128u + (uint32_t)(r & 7) * 16u;
            *reinterpret_cast<uint4 *>(tiles + (size_t)t2 * tile_bytes + off) = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    uint32_t ncols = 32;
    while (ncols < (uint32_t)tcols) ncols <<= 1;
    // D regions (strip, 256-column piece); region k goes to issuer k % kTcIssuers
    int nreg = 0;
    for (int i = i0; i < i1; ++i) nreg += (Mp - 128 * i + 255) / 256;
    const int nact = nreg < kTcIssuers ? nreg : kTcIssuers;  // active issuers
    if (tid == 0) {
        for (int st = 0; st < nst; ++st) {
            tc::mbar_init(&full[st], kTcProdWarps);
            tc::mbar_init(&empty[st], nact);
        }
        tc::mbar_init(&drain, nact);
        tc::mbar_fence_init();
        timed_out = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, ncols);
        tc::tmem_relinquish();
    }
    tc::fence_proxy_async_smem();  // the zero rows, for the tensor core
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    volatile int *vto = &timed_out;
#ifdef PAM_SOLVE_PROFILE
    const long long gp_t1 = clock64();
    if (tid == 32 * kTcIssuers) { GP_ADD(0, gp_t1 - gp_t0); GP_ADD(15, 1); }
#endif

    if (warp < kTcIssuers) {
        // ---- MMA issuers: lane 0 of warp j issues the regions k = j mod 4 ----
        if (lane == 0 && warp < nact) {
            const uint32_t lbo = (uint32_t)Rt * 16u, sbo = 128u;
            // descriptors of the stage-0 hi tile; every other operand start is
            // a multiple of 16 bytes away (address field = byte address / 16)
            const uint64_t desc0 = tc::smem_desc(tc::smem_u32(tiles), lbo, sbo);
            for (int c = 0; c < nch; ++c) {
                const int st = c % nst;
#ifdef PAM_SOLVE_PROFILE
                const long long gw = clock64();
#endif
                if (!tc::mbar_wait(&full[st], (uint32_t)(c / nst) & 1u, kWaitBudget) || *vto) {
                    *vto = 1;
                    break;
                }
#ifdef PAM_SOLVE_PROFILE
                const long long gi = clock64();
                if (warp == 0) GP_ADD(1, gi - gw);
#endif
                tc::fence_after_sync();
                const uint64_t hi_d = desc0 + (((uint64_t)st * 2 * tile_bytes) >> 4);
                const uint64_t lo_d = hi_d + (tile_bytes >> 4);
#pragma unroll
                for (int ks = 0; ks < kTcKC / 16; ++ks) {
                    const uint64_t koff = (uint64_t)(2 * ks) * (lbo >> 4);
                    uint32_t dcol = 0;
                    int k = 0;
                    for (int i = i0; i < i1; ++i) {
                        const uint64_t roff = (uint64_t)((128 * (i - i0)) >> 3) * (sbo >> 4);
                        const uint64_t a_hi = hi_d + koff + roff, a_lo = lo_d + koff + roff;
                        const int Ri = Mp - 128 * i;
                        for (int n0 = 0; n0 < Ri; n0 += 256, ++k) {
                            if (k % kTcIssuers != warp) continue;
                            const uint32_t n = (uint32_t)min(256, Ri - n0);
                            const uint32_t id = tc::idesc_bf16_f32(n);
                            const uint64_t noff = (uint64_t)(n0 >> 3) * (sbo >> 4);
                            const uint32_t d = tmem + dcol + (uint32_t)n0;
                            tc::mma_bf16(d, a_hi, hi_d + koff + roff + noff, id, (c > 0 || ks > 0) ? 1u : 0u);
                            tc::mma_bf16(d, a_hi, lo_d + koff + roff + noff, id, 1u);
                            tc::mma_bf16(d, a_lo, hi_d + koff + roff + noff, id, 1u);
                        }
                        dcol += (uint32_t)Ri;
                    }
                }
                tc::mma_commit(&empty[st]);
                if (warp == 0) GP_ADD(2, clock64() - gi);
            }
            tc::mma_commit(&drain);  // every MMA this thread issued, done or not
        }
    } else {
        // ---- producers ----
        const int pth = tid - 32 * kTcIssuers;  // 0 .. 32 * kTcProdWarps - 1
        const int tpr = tc_threads_per_row(Rl);
        const int nkg = 4 / tpr;
        // a warp covers 32 consecutive rows with one set of k-groups: its cell
        // reads are broadcasts and its stores one contiguous 512-byte run
        const int pw = pth >> 5, part = pw % tpr, r = (pw / tpr) * 32 + lane;
        const bool live = r < Rl;
        ProdRow row = prod_row(live ? sc[r] : make_float4(0.f, 0.f, 0.f, 0.f));
        for (int c = 0; c < nch; ++c) {
            const int st = c % nst;
            bool bad = false;
#ifdef PAM_SOLVE_PROFILE
            const long long pw = clock64();
#endif
            if (c >= nst)  // the MMAs of chunk c - nst read this stage
                bad = !tc::mbar_wait(&empty[st], (uint32_t)(c / nst - 1) & 1u, kWaitBudget);
#ifdef PAM_SOLVE_PROFILE
            const long long pp0 = clock64();
            if (pth == 0) GP_ADD(3, pp0 - pw);
#endif
            if (bad) *vto = 1;
            if (__any_sync(0xffffffffu, bad || *vto)) break;  // warp-uniform exit
            if (live) {
                const float4 *pa = cella + c * (kTcKC / 2), *pb = cellb + c * (kTcKC / 2);
                const float2 *py = celly2 + c * (kTcKC / 2);
                uint8_t *hi = tiles + (size_t)st * 2 * tile_bytes;
                uint8_t *lo = hi + tile_bytes;
                for (int kk = 0; kk < nkg; ++kk) {
                    const int kg = part * nkg + kk;
                    uint32_t hp[4], lp[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int pq = kg * 4 + q;
                        prod_pair(row, pa[pq], pb[pq], py[pq], &hp[q], &lp[q]);
                    }
                    const uint32_t off = (uint32_t)(kg * (Rt >> 3) + (r >> 3)) * 128u + (uint32_t)(r & 7) * 16u;
                    *reinterpret_cast<uint4 *>(hi + off) = make_uint4(hp[0], hp[1], hp[2], hp[3]);
                    *reinterpret_cast<uint4 *>(lo + off) = make_uint4(lp[0], lp[1], lp[2], lp[3]);
                }
            }
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&full[st]);
#ifdef PAM_SOLVE_PROFILE
            if (pth == 0) GP_ADD(4, clock64() - pp0);
#endif
        }
        if (live) {
            bpart[part * Rcap + r] = row.b.x + row.b.y;
            wpart[part * Rcap + r] = row.w.x + row.w.y;
        }
    }
    // wait for the last chunk's MMAs (they complete in issue order)
#ifdef PAM_SOLVE_PROFILE
    if (tid == 32 * kTcIssuers) GP_ADD(5, clock64() - gp_t1);
#endif
    // every issuer committed its MMAs to `drain` (they complete in issue order)
    __syncthreads();
    __syncwarp();
    if (!tc::mbar_wait(&drain, 0u, kWaitBudget)) *vto = 1;
    __syncthreads();
    tc::fence_after_sync();
    if (*vto) {
        if (tid == 0) atomicAdd(&w.status[kStTimeout], 1);
    } else {
        float *G = w.Gf + (size_t)s * g.m_cap * g.m_cap;
        // warp q reads TMEM lanes 32 (q % 4) ..; the eight warps of a lane
        // quarter split the 32-column chunks of the group's D blocks. Rows go
        // out through a padded shared-memory transpose so that each store is
        // one coalesced row segment; the mirrored blocks below the strips are
        // already coalesced.
        float *stage = reinterpret_cast<float *>(tiles) + (size_t)warp * kTcStageFloats;
        const int lane_base = (warp & 3) * 32;
        for (int f = warp >> 2; f < tcols / 32; f += 8) {
            int i = i0, ch = f, dcol = 0;
            while (ch >= (Mp - 128 * i) / 32) { ch -= (Mp - 128 * i) / 32; dcol += Mp - 128 * i; ++i; }
            const int srow = 128 * i;                 // the strip's first centre
            const int rg = srow + lane_base + lane;   // G row held by this thread
            uint32_t v[32];
            tc::tmem_ld_32x32(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(dcol + ch * 32), v);
            tc::tmem_wait_ld();
            const int c0 = srow + ch * 32;
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
                const int row = srow + lane_base + q;
                if (row < M && col < M) G[(size_t)row * g.m_cap + col] = stage[q * 33 + lane];
            }
            __syncwarp();
        }
        // b = W^T y for the group's rows: the parts of a row in a fixed order
        const int tpr = tc_threads_per_row(Rl);
        const int rend = min(Rl, 128 * (i1 - i0));
        for (int r = tid; r < rend; r += blockDim.x) {
            float acc = 0.f, ws = 0.f;
            for (int q = 0; q < tpr; ++q) {
                acc += bpart[q * Rcap + r];
                ws += wpart[q * Rcap + r];
            }
            w.b[(size_t)s * g.m_cap + row0 + r] = (double)acc;
            w.wsum[(size_t)s * g.m_cap + row0 + r] = ws;  // sum_t W_tj: a row sum of G
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    __syncwarp();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
#ifdef PAM_SOLVE_PROFILE
    if (tid == 32 * kTcIssuers) GP_ADD(6, clock64() - gp_t0);
#endif
}

static_assert(kTcMaxRows <= 32 * kTcProdWarps, "one producer thread per row at least");

static size_t gram_tc_smem(const Geo &g, int stages) {
    const size_t Rcap = (size_t)tc_rows_cap(g.m_cap);
    const size_t cells = (size_t)((g.n_max + kTcKC - 1) / kTcKC) * kTcKC;
    size_t tiles = (size_t)stages * 2 * Rcap * kTcKC * 2;
    if (tiles < (size_t)32 * kTcStageFloats * 4) tiles = (size_t)32 * kTcStageFloats * 4;
    return tiles + Rcap * sizeof(float4) + 8 * Rcap * sizeof(float) + cells * (sizeof(float4) + sizeof(float));
}

// --------------------------------------------------------------------------
// Gram products of a small dictionary (M <= kSmallGramM: the initial
// lattices) on the CUDA cores. At such sizes the contraction is too thin for
// the tensor cores (one 128-row strip of N <= 64 columns per k-step: the
// tcgen05 pipeline's set-up and per-instruction cost dominate), so one block
// of 256 threads per subdomain generates W in chunks of 32 cells into shared
// memory, with the same exponent as the tensor-core Gram (the Shepard
// normaliser folded in: W = 2^(l - sh)), and accumulates W^T W in fp32 over
// 4 x 4 tiles of the upper block triangle held in registers (two float4
// loads per sixteen multiply-adds), the cells of a chunk split among
// ks = 256 / tiles thread groups whose partial tiles are summed in shared
// memory at the end. The threads that generate centre m's values also sum
// b = W^T y and the weight sum of m. Products are exact fp32 (no bf16
// split), so G~ is at least as accurate as the tensor-core one.
// --------------------------------------------------------------------------
constexpr int kSmallGramM = 64;
constexpr int kSgThreads = 256;

__global__ void __launch_bounds__(kSgThreads) k_gram_small(Geo g, const int32_t *boxes, const double *centres,
                                                          const int32_t *info, Ws w, int all) {
    const int s = group_sub(g, blockIdx.x);
    const int32_t *inf = info + s * kInfoN;
    if (!all && inf[PAM_INFO_STOPPED]) return;
    const int M = inf[PAM_INFO_M], N = inf[PAM_INFO_N_CELLS];
    if (M > kSmallGramM || M < 1) return;  // never: the launch is sized by the host's bound
    const int tid = threadIdx.x;
    const int32_t *box = boxes + s * 12;
    __shared__ float4 sc[kSmallGramM];
    __shared__ __align__(16) float Wt[kTcKC][kSmallGramM];
    __shared__ float Gs[kSgThreads * 16];  // the partial tiles; then b and the weight sums
    extern __shared__ float4 cxa[];  // [nch * 32] (x, y, z, sh) of every patch cell, then ln K
    const int nch = (N + kTcKC - 1) / kTcKC;
    float *cya = reinterpret_cast<float *>(cxa + (size_t)nch * kTcKC);
    double o[3];
    patch_origin_block(g, box, o);
    const dvec4 *cg = reinterpret_cast<const dvec4 *>(centres) + (size_t)s * g.m_cap;
    for (int m = tid; m < M; m += blockDim.x) sc[m] = local_centre(cg[m], o);
    // padding columns of W (M up to the next multiple of 4) stay zero
    const int nb = (M + 3) >> 2, ntile = nb * (nb + 1) / 2;
    for (int e = tid; e < kTcKC * kSmallGramM; e += blockDim.x) (&Wt[0][0])[e] = 0.f;
    // this thread's tile (bi <= bj, row-major over the upper block triangle)
    // and cell group kg of ks
    const int ks = kSgThreads / ntile;  // >= 1: ntile <= 136
    const int tile = tid % ntile, kg = tid / ntile;
    int bi = 0, rem = tile;
    while (rem >= nb - bi) { rem -= nb - bi; ++bi; }
    const int bj = bi + rem;
    const bool tiled = kg < ks;
    // generators: R threads per centre, each its own cells of a chunk
    const int R = kSgThreads / M, gm = tid % M, gq = tid / M;
    const bool gen = gq < R;
    const float *rowmax = w.rowmax + (size_t)s * g.n_max;
    const float *rowinv = w.rowinv + (size_t)s * g.n_max;
    const double *yv = w.y + (size_t)s * g.n_max;
    // every cell's point, shift and ln K in shared memory once (the chunks
    // below touch no global memory)
    for (int t = tid; t < nch * kTcKC; t += blockDim.x) {
        float x[3] = {0.f, 0.f, 0.f};
        float sh = INFINITY, y = 0.f;
        if (t < N) {
            local_cell(g, s, box, t, x);
            sh = rowmax[t] - log2f(rowinv[t]);
            y = (float)yv[t];
        }
        cxa[t] = make_float4(x[0], x[1], x[2], sh);
        cya[t] = y;
    }
    float acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
    float bacc = 0.f, wacc = 0.f;
    const float4 cm = gen ? sc[gm] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 *W4 = reinterpret_cast<const float4 *>(&Wt[0][0]);
    for (int t0 = 0; t0 < N; t0 += kTcKC) {
        __syncthreads();  // the cells are staged; the previous chunk's readers are done
        if (gen) {
            for (int t = gq; t < kTcKC; t += R) {
                const float4 c = cxa[t0 + t];
                const float v = tc::ex2(logit2(cm, c.x, c.y, c.z) - c.w);  // 0 past the patch (sh = inf)
                Wt[t][gm] = v;
                bacc = fmaf(v, cya[t0 + t], bacc);
                wacc += v;
            }
        }
        __syncthreads();
        if (tiled) {
            for (int t = kg; t < kTcKC; t += ks) {
                const float4 a = W4[t * (kSmallGramM / 4) + bi], b = W4[t * (kSmallGramM / 4) + bj];
                const float av[4] = {a.x, a.y, a.z, a.w}, bw[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], bw[v], acc[u][v]);
            }
        }
    }
    // partial tiles out, then each entry sums its ks parts in a fixed order
    // (the result does not depend on scheduling)
    if (tiled) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) Gs[tid * 16 + u * 4 + v] = acc[u][v];
    }
    __syncthreads();
    float *G = w.Gf + (size_t)s * g.m_cap * g.m_cap;
    for (int e = tid; e < M * M; e += blockDim.x) {
        const int i = e / M, j = e - i * M;
        const int a = i <= j ? i : j, b = i <= j ? j : i;
        const int ta = a >> 2, tl = ta * nb - ta * (ta - 1) / 2 + (b >> 2) - ta;
        const int off = tl * 16 + (a & 3) * 4 + (b & 3);
        float v = 0.f;
        for (int k = 0; k < ks; ++k) v += Gs[k * ntile * 16 + off];
        G[(size_t)i * g.m_cap + j] = v;
    }
    __syncthreads();  // Gs is free again: the generators' partial sums, R per centre
    if (gen) {
        Gs[gq * M + gm] = bacc;
        Gs[kSgThreads + gq * M + gm] = wacc;
    }
    __syncthreads();
    if (tid < M) {
        float bs = 0.f, ws = 0.f;
        for (int q = 0; q < R; ++q) {
            bs += Gs[q * M + tid];
            ws += Gs[kSgThreads + q * M + tid];
        }
        w.b[(size_t)s * g.m_cap + tid] = (double)bs;
        w.wsum[(size_t)s * g.m_cap + tid] = ws;
    }
}

void launch_gram_tc(const Geo &g, const int32_t *boxes, const double *centres, const int32_t *info,
                    const Ws &w, cudaStream_t st, int all, int folds, int fold) {
    PhaseScope ps(kPhGramTC, st);
    int stages = gram_tc_smem(g, kTcMaxStages) <= kSmemLimit ? kTcMaxStages : 2;
    if (tuning().gram_stages == 2) stages = 2;  // a tuned shallower pipeline (3 only where it fits)
    size_t sm = gram_tc_smem(g, stages);
    cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    dim3 grid((g.m_cap + 127) / 128, group_count(g));
    k_gram_tc<<<grid, kTcThreads, sm, st>>>(g, boxes, centres, info, w, all, stages, tc_rows_cap(g.m_cap),
                                            folds, fold);
    count_launches(1);
}

void launch_stats_f32(const Geo &g, const int32_t *boxes, const double *centres, const int32_t *info,
                      const Ws &w, cudaStream_t st, int all) {
    PhaseScope ps(kPhStats, st);
    size_t sm = (size_t)g.m_cap * 2 * sizeof(float4);
    cudaFuncSetAttribute(k_stats_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    // two cells per thread, 512 per block: every block converts the M
    // centres once (binary64 offsets on the narrow fp64 pipe), so fewer,
    // larger blocks per subdomain spend less of their time on it
    dim3 grid((g.n_max + 511) / 512, group_count(g));
    k_stats_f32<<<grid, 256, sm, st>>>(g, boxes, centres, info, w, all);
    count_launches(1);
}

void launch_stats_gram_tc(const Geo &g, const int32_t *boxes, const double *centres,
                          const int32_t *info, const Ws &w, cudaStream_t st, int all, int m_bound) {
    launch_stats_f32(g, boxes, centres, info, w, st, all);
    const size_t sm = (size_t)((g.n_max + kTcKC - 1) / kTcKC) * kTcKC * (sizeof(float4) + sizeof(float));
    if (m_bound > 0 && m_bound <= kSmallGramM && sm + 32 * 1024 <= kSmemLimit) {
        // every dictionary is at most m_bound centres (the initial lattices)
        PhaseScope ps(kPhGramTC, st);
        cudaFuncSetAttribute(k_gram_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_gram_small<<<group_count(g), kSgThreads, sm, st>>>(g, boxes, centres, info, w, all);
        count_launches(1);
        return;
    }
    launch_gram_tc(g, boxes, centres, info, w, st, all, 0, 0);
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
// At M <= 64 the solve is a chain of short factorisations and the
// exact-gradient passes are short: more subdomains in flight pay more than
// more threads per subdomain.
constexpr int kSmallSolveM = 64;
constexpr int kSmallSolveThreads = 64;
constexpr int kMxFactorBytesDefault = 64 * 1024;
constexpr int kMxMaxRefine = 12;
constexpr int kMxMaxPdas = 200;
constexpr int kMxPdasFull = 12;

struct MxShared {
    int cnt, bad, viol, flag, changed, nneed;
    float inv_piv, dmax, xmax, dinf, yinf;
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

// Packed support matrix: A[tri(p, q)] = G~[idx[p]][idx[q]] (+ lambda2 on
// the diagonal) for q <= p < s, flat over the packed entries so that every
// thread keeps sixteen independent gathers from G~ in flight.
__device__ void mx_build(float *A, const float *G, const int *idx, int s, int mc, float lam2) {
    const int n = s * (s + 1) / 2, nt = blockDim.x;
    for (int e0 = threadIdx.x; e0 < n; e0 += 16 * nt) {
        float v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int e = e0 + u * nt;
            v[u] = 0.f;
            if (e < n) {
                int pr = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
                if (tri_i(pr + 1, 0) <= e) ++pr;
                if (tri_i(pr, 0) > e) --pr;
                const int q = e - tri_i(pr, 0);
                v[u] = G[(size_t)idx[pr] * mc + idx[q]] + (q == pr ? lam2 : 0.f);
            }
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int e = e0 + u * nt;
            if (e < n) A[e] = v[u];
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

// Two DFAcc sums in the halves of packed fp32x2 registers, each half the
// same operations in the same order as DFAcc::add_prod (a subtraction y - x
// as fma(x, -1, y), rounded once like __fsub_rn; -p as a times -b).
struct DFAcc2 {
    float2 s = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
    __device__ __forceinline__ void add_prod(float2 a, float2 b, float2 nb) {
        const float2 m1 = make_float2(-1.f, -1.f);
        const float2 p = __fmul2_rn(a, b);
        const float2 pe = __ffma2_rn(a, b, __fmul2_rn(a, nb));  // a b - p, exact
        const float2 t = __fadd2_rn(s, p);
        const float2 bp = __ffma2_rn(s, m1, t);
        const float2 err = __fadd2_rn(__ffma2_rn(__ffma2_rn(bp, m1, t), m1, s), __ffma2_rn(bp, m1, p));
        s = t;
        c = __fadd2_rn(c, __fadd2_rn(err, pe));
    }
    __device__ __forceinline__ double value() const {
        return ((double)s.x + (double)c.x) + ((double)s.y + (double)c.y);
    }
};

// Cross-validation form (cv != nullptr, p.cv_folds > 0): the system is that
// of the training rows of fold p.cv_fold (G~ and b masked by the Gram, the
// exact gradient over the training cells only), lambda_k = N_train
// lambda_k_hat, no indicators are written, and the held-out cells' squared
// residuals (y_t - (W x)_t)^2 of the final x are added to cv[s * cv_stride]
// in a fixed order. lam_tab (optional): per-subdomain (lambda1_hat,
// lambda2_hat) pairs in place of p's; all: solve also the subdomains whose
// refinement has stopped.
template <bool SMALL>
__device__ __forceinline__ void solve_mixed_item(const Geo &g, const Par &p, const int32_t *boxes,
                                                 const double *centres, double *beta, int32_t *info,
                                                 const Ws &w, int kMxFactorBytes, const double *lam_tab,
                                                 int all, double *cv, int cv_stride, int fallback, int s) {
    const long long t_start = clock64();
    int32_t *inf = info + s * kInfoN;
    if (!all && inf[PAM_INFO_STOPPED]) return;
    const int M = inf[PAM_INFO_M], N = inf[PAM_INFO_N_CELLS], mc = g.m_cap;
    // per-centre arrays in shared memory: the capacity, or (SMALL) the bound
    // kSmallSolveM of every dictionary of the launch
    const int mcs = SMALL ? kSmallSolveM : mc;
    const int folds = cv ? p.cv_folds : 0, fold = p.cv_fold;
    const int n_out = (folds > 0 && N > fold) ? (N - 1 - fold) / folds + 1 : 0;
    const double n_fit = (double)(N - n_out);
    const double l1h = lam_tab ? lam_tab[2 * s] : p.lam1_hat, l2h = lam_tab ? lam_tab[2 * s + 1] : p.lam2_hat;
    const float lam1 = (float)(n_fit * l1h), lam2 = (float)(n_fit * l2h);
    double held = 0.0;  // this thread's held-out squared residuals of the last exact pass
    // stage 1 only has to find a good support: G~ carries ~1e-5 relative error
    const float tol_pdas = lam1 * (1.0f + 1e-3f);
    const int tid = threadIdx.x, lane = tid & 31;
    const int32_t *box = boxes + s * 12;

    extern __shared__ __align__(16) uint8_t sm[];
    float *x = reinterpret_cast<float *>(sm);      // [mcs]
    float *gr = x + mcs;                           // [mcs] b - G~ x (stage 1), exact c (stage 2)
    float *bv = gr + mcs;                          // [mcs]
    float *rhs = bv + mcs;                         // [mcs]
    int *sg = reinterpret_cast<int *>(rhs + mcs);  // [mcs]
    int *idx = sg + mcs;                           // [mcs]
    // cells in pairs (2p, 2p + 1) and the support in pairs (2q, 2q + 1), for
    // the packed fp32x2 arithmetic of the exact-gradient passes
    const int np2 = (g.n_max + 1) >> 1, ns2 = (mcs >> 1) + 2;
    float4 *sc = reinterpret_cast<float4 *>(idx + mcs);     // [mcs] local centres
    float4 *cella = sc + mcs;                               // [np2] (x, x', y, y')
    float4 *cellb = cella + np2;                            // [np2] (z, z', -rowmax, -rowmax')
    float4 *supa = cellb + np2;                             // [ns2] (-c_x, -c_x', -c_y, -c_y')
    float4 *supb = supa + ns2;                              // [ns2] (-c_z, -c_z', alpha, alpha')
    float2 *supx = reinterpret_cast<float2 *>(supb + ns2);  // [ns2] (x_m, x_m')
    float2 *supn = supx + ns2;                              // [ns2] (-x_m, -x_m')
    float *cinv = reinterpret_cast<float *>(supn + ns2);    // [2 np2] 0 past the patch
    float *ce = cinv + 2 * np2;                             // [2 np2] e = y - W x (0 past the patch)
    const float2 *cinv2 = reinterpret_cast<const float2 *>(cinv), *ce2 = reinterpret_cast<const float2 *>(ce);
    // cell t as (x, y, z, rowmax)
    auto cell_at = [&](int t) {
        const float *fa = reinterpret_cast<const float *>(cella + (t >> 1));
        const float *fb = reinterpret_cast<const float *>(cellb + (t >> 1));
        const int h = t & 1;
        return make_float4(fa[h], fa[2 + h], fb[h], -fb[2 + h]);
    };
    float *dinv = ce + 2 * np2;                             // [mcs] 1 / diag of the factor
    float *ub = dinv + mcs;                                 // [mcs] bounds on |c_j| off the support
    float *Lt = ub + mcs;                                   // [32 x 32] factorisation scratch
    float *Asm = Lt + kCholLtFloats;                        // packed factor
    __shared__ MxShared sh;

    const float *G = w.Gf + (size_t)s * mc * mc;
    {
        // the active-set steps gather rows of G~ again and again: stream the
        // M used rows into L2 once, up front (bulk prefetch, 32 KiB pieces)
        const size_t bytes = (size_t)M * mc * sizeof(float);
        for (size_t off = (size_t)tid * 32768; off < bytes; off += (size_t)blockDim.x * 32768) {
            const size_t n = bytes - off < 32768 ? bytes - off : 32768;
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;"
                         ::"l"(reinterpret_cast<const char *>(G) + off), "r"((uint32_t)((n + 15) & ~(size_t)15))
                         : "memory");
        }
    }
    const float *rowmax = w.rowmax + (size_t)s * g.n_max;
    const float *rowinv = w.rowinv + (size_t)s * g.n_max;
    double o[3];
    patch_origin_block(g, box, o);
    const dvec4 *cg = reinterpret_cast<const dvec4 *>(centres) + (size_t)s * mc;
    // the dictionary (M x 32 bytes) comes into the factor's space, free until
    // the first factorisation, by one bulk copy, and is converted to local fp32
    stage_local_centres(sc, cg, M, o, Asm, M * 32 <= kMxFactorBytes);
    for (int j = tid; j < mcs; j += blockDim.x) {
        float b0 = j < M ? (float)beta[(size_t)s * mc + j] : 0.f;
        x[j] = b0;
        bv[j] = j < M ? (float)w.b[(size_t)s * mc + j] : 0.f;
        sg[j] = (j < M) ? ((b0 > 0.f) - (b0 < 0.f)) : 0;
    }
    for (int t = tid; t < 2 * np2; t += blockDim.x) {
        float xl[3] = {0.f, 0.f, 0.f};
        float nrm = -INFINITY, ci = 0.f;  // past the patch: weight 0
        if (t < N) {
            local_cell(g, s, box, t, xl);
            nrm = -rowmax[t];
            ci = rowinv[t];
        }
        float *fa = reinterpret_cast<float *>(cella + (t >> 1)), *fb = reinterpret_cast<float *>(cellb + (t >> 1));
        const int h = t & 1;
        fa[h] = xl[0];
        fa[2 + h] = xl[1];
        fb[h] = xl[2];
        fb[2 + h] = nrm;
        cinv[t] = ci;
        ce[t] = 0.f;
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
    // dropping the coefficients that reach zero, and adds all violators only
    // once the minimiser on the support is sign-consistent. A coefficient
    // that joined at zero stays (at zero) unless its own sign blocks the
    // step, so a step of length zero sheds only the wrong-signed newcomers
    // and the next step keeps the rest -- the objective never increases and
    // every zero-length step shrinks the support, so it ends.
    int it = 0, scnt = 0;
    float *A = Asm;
    // The right-hand side b_S - lambda1 s_S rides along as row scnt of the
    // packed matrix (diagonal 1e30, never a pivot problem): the factorisation
    // leaves L^-1 rhs there, and only the backward solve remains. (Not when
    // the support is the whole capacity: no room for the extra row.)
    // the rows of G~ on the support: the build gathers from them now, the
    // fp32 gradient streams them after the factorisation; one bulk L2
    // prefetch per row keeps them on chip without holding registers
    auto prefetch_rows = [&]() {
        const uint32_t bytes = (uint32_t)((M * sizeof(float) + 15) & ~(size_t)15);
        for (int pp = tid; pp < scnt; pp += blockDim.x)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;"
                         ::"l"(G + (size_t)idx[pp] * mc), "r"(bytes) : "memory");
    };
    auto factor_support = [&]() {
        mx_compact(sg, M, idx, &sh.cnt);
        scnt = sh.cnt;
        prefetch_rows();
        const bool aug = scnt < mc;
        const int nrow = scnt + (aug ? 1 : 0);
        A = (tri_i(nrow, 0) * 4 <= kMxFactorBytes) ? Asm
            : (w.Lf + (size_t)s * ((size_t)mc * (mc + 1) / 2));
        PROF_MARK(8);
        mx_build(A, G, idx, scnt, mc, lam2);
        float *arow = A + tri_i(scnt, 0);
        for (int pp = tid; pp < scnt; pp += blockDim.x) {
            const float r = bv[idx[pp]] - lam1 * (float)sg[idx[pp]];
            if (aug) arow[pp] = r;
            else rhs[pp] = r;
        }
        if (aug && tid == 0) arow[scnt] = 1e30f;
        __syncthreads();
        PROF_MARK(9);
        mx_cholesky(A, nrow, &sh.flag, dinv, Lt);
        PROF_MARK(10);
        if (!sh.flag) {
            if (aug) {
                for (int pp = tid; pp < scnt; pp += blockDim.x) rhs[pp] = arow[pp];
                __syncthreads();
                mx_chol_backward(A, dinv, scnt, rhs);
            } else {
                mx_chol_solve(A, dinv, scnt, rhs);
            }
        }
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
    bool primal = false;
    bool gfresh = false;  // gr = b~ - G~ x holds for the current x (the fp32 optimality test passed)
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
            if (sh.bad == 0 && sh.viol == 0) { gfresh = true; break; }
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
            if (tid == 0) sh.viol = 0;
            __syncthreads();
            int mv = 0;
            for (int j = tid; j < M; j += blockDim.x)
                if (sg[j] == 0 && fabsf(gr[j]) > tol_pdas) { sg[j] = gr[j] > 0.f ? 1 : -1; x[j] = 0.f; ++mv; }
            if (mv) atomicAdd(&sh.viol, mv);
            __syncthreads();
            if (sh.viol == 0) { gfresh = true; break; }  // optimal
        } else {
            // step alpha towards the minimiser; the blocking coefficients (the
            // ones whose ratio attains alpha) reach zero and leave the support;
            // a newcomer still at zero after a zero-length step stays
            const float alpha = fminf(sh.dmax, 1.f);
            for (int pp = tid; pp < scnt; pp += blockDim.x) {
                const int m = idx[pp];
                const float xs = rhs[pp], x0 = x[m], sgn = (float)sg[m];
                bool blocking = false;
                if (!(xs * sgn > 0.f)) {
                    const float a = (x0 * sgn > 0.f) ? x0 / (x0 - xs) : 0.f;
                    blocking = fmaxf(a, 0.f) <= alpha * (1.f + 1e-6f);
                }
                const float nx = x0 + alpha * (xs - x0);
                if (blocking || (x0 != 0.f && !(nx * sgn > 0.f))) {
                    x[m] = 0.f;
                    sg[m] = 0;
                } else {
                    x[m] = nx * sgn > 0.f ? nx : 0.f;
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
    //
    // The exact gradient is computed only where it can decide something: on
    // the support (the Newton step needs it) and at the centres off it whose
    // upper bound ub_j >= |c_j| does not already show |c_j| <= kkt_tol. The
    // first bound comes from the fp32 gradient of stage 1, c~ = b~ - G~ x:
    // every W_tj >= 0 and each Shepard row sums to one, so sum_k G_jk =
    // sum_t W_tj = wsum_j, and the per-entry errors of G~ (bf16 split
    // 3 x 2^-17, fp32 accumulation N 2^-23, the exponent's rounding) and of
    // b~ (fp32 accumulation) give |c_j - c~_j| <= wsum_j (eps_g ||x||_inf +
    // eps_b ||y||_inf), taken with a factor 2 of margin. After an exact pass
    // ub_j = |c_j|; a Newton step changes c by -G dx, so ub_j grows by
    // wsum_j ||dx||_inf. Centres it settles keep |c_j| <= kkt_tol and cannot
    // be violators: the certificate is the one of the full pass.
    const float kkt_tol = lam1 * (1.0f + 1e-3f);
    int certified = 0, refine_it = 0;
    const double *yv = w.y + (size_t)s * g.n_max;
    const float *wsg = w.wsum + (size_t)s * mc;
    if (!sh.flag) {
        float xin = 0.f, yin = 0.f;
        for (int pp = tid; pp < scnt; pp += blockDim.x) xin = fmaxf(xin, fabsf(x[idx[pp]]));
        for (int t = tid; t < N; t += blockDim.x) yin = fmaxf(yin, fabsf((float)yv[t]));
        for (int o2 = 16; o2 > 0; o2 >>= 1) {
            xin = fmaxf(xin, __shfl_xor_sync(0xffffffffu, xin, o2));
            yin = fmaxf(yin, __shfl_xor_sync(0xffffffffu, yin, o2));
        }
        if (tid == 0) { sh.dinf = 0.f; sh.yinf = 0.f; }
        __syncthreads();
        if (lane == 0) {
            atomicMax(reinterpret_cast<int *>(&sh.dinf), __float_as_int(xin));
            atomicMax(reinterpret_cast<int *>(&sh.yinf), __float_as_int(yin));
        }
        __syncthreads();
        const float eps_g = 2.f * (3.7e-5f + 1.2e-7f * (float)N + 6e-8f * (float)scnt);
        const float eps_b = 2.f * (1.2e-7f * (float)N + 5e-7f);
        const float bnd = eps_g * sh.dinf + eps_b * sh.yinf;
        for (int j = tid; j < M; j += blockDim.x)
            ub[j] = (gfresh && sg[j] == 0) ? fmaf(wsg[j], bnd, fabsf(gr[j])) : INFINITY;
        __syncthreads();
    }
    int *need = reinterpret_cast<int *>(rhs);  // the c pass's list (rhs is free until the Newton step)
    for (; refine_it < kMxMaxRefine && !sh.flag; ++refine_it) {
        // e = y - W x over the patch (only the support contributes); W x is
        // accumulated in double-float and subtracted in fp64: |y| ~ 10 would
        // otherwise leave ~1e-6 of cancellation noise in e, and W^T e inherits it
        held = 0.0;
        PROF_MARK(15);  // the previous iteration's Newton step and refactorisation
        // the support in pairs (an odd one out paired with alpha = 0, x = 0)
        const int nsp = (scnt + 1) >> 1;
        for (int q = tid; q < nsp; q += blockDim.x) {
            const bool two = 2 * q + 1 < scnt;
            const int m0 = idx[2 * q], m1 = two ? idx[2 * q + 1] : m0;
            const float4 c0 = sc[m0], c1 = two ? sc[m1] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float x0 = x[m0], x1 = two ? x[m1] : 0.f;
            supa[q] = make_float4(-c0.x, -c1.x, -c0.y, -c1.y);
            supb[q] = make_float4(-c0.z, -c1.z, c0.w, c1.w);
            supx[q] = make_float2(x0, x1);
            supn[q] = make_float2(-x0, -x1);
        }
        __syncthreads();
        for (int t = tid; t < N; t += blockDim.x) {
            const float4 cx = cell_at(t);
            const float2 X = make_float2(cx.x, cx.x), Y = make_float2(cx.y, cx.y), Z = make_float2(cx.z, cx.z);
            const float2 nrm = make_float2(-cx.w, -cx.w);
            DFAcc2 acc;
#pragma unroll 2
            for (int q = 0; q < nsp; ++q) {
                // per half: ex2(logit2(c_m, x) - rowmax), as in the scalar form
                const float4 a = supa[q], b = supb[q];
                const float2 dx = __fadd2_rn(X, make_float2(a.x, a.y));
                const float2 dy = __fadd2_rn(Y, make_float2(a.z, a.w));
                const float2 dz = __fadd2_rn(Z, make_float2(b.x, b.y));
                float2 d2 = __fmul2_rn(dx, dx);
                d2 = __ffma2_rn(dy, dy, d2);
                d2 = __ffma2_rn(dz, dz, d2);
                const float2 l = __fadd2_rn(__fmul2_rn(make_float2(b.z, b.w), d2), nrm);
                acc.add_prod(make_float2(tc::ex2(l.x), tc::ex2(l.y)), supx[q], supn[q]);
            }
            const float e = (float)(yv[t] - acc.value() * (double)cinv[t]);
            if (folds > 0 && t % folds == fold) {  // held out: not in the gradient
                held += (double)e * (double)e;
                ce[t] = 0.f;
            } else {
                ce[t] = e;
            }
        }
        __syncthreads();
        PROF_MARK(4);
        // c_j = sum_t W_tj e_t (exact gradient of the data term) for the
        // support and the centres whose bound leaves them undecided
        if (threadIdx.x < 32) {
            int base = 0;
            for (int j0 = 0; j0 < M; j0 += 32) {
                const int j = j0 + lane;
                const bool on = j < M && (sg[j] != 0 || !(ub[j] <= kkt_tol));
                const unsigned bal = __ballot_sync(0xffffffffu, on);
                if (on) need[base + __popc(bal & ((1u << lane) - 1u))] = j;
                base += __popc(bal);
            }
            if (lane == 0) sh.nneed = base;
        }
        __syncthreads();
        float cmax = 0.f;
        const int ncp = (N + 1) >> 1;  // cell pairs (the odd one out pairs with weight 0)
        // gq threads per centre (a power of two up to 8, as many as the list
        // leaves room for), each over every gq-th cell pair, summed in a fixed
        // butterfly order: short lists keep every thread busy
        const int nneed = sh.nneed;
        int gq = 1;
        while (gq < 8 && nneed * gq * 2 <= (int)blockDim.x) gq <<= 1;
        const int per_sweep = (int)blockDim.x / gq, sub = tid % gq;
        for (int q0 = 0; q0 < nneed; q0 += per_sweep) {
            const int q = q0 + tid / gq;
            const bool act = q < nneed;
            const int j = need[act ? q : 0];
            const float4 cj = sc[j];
            const float2 ncx = make_float2(-cj.x, -cj.x), ncy = make_float2(-cj.y, -cj.y);
            const float2 ncz = make_float2(-cj.z, -cj.z), cw = make_float2(cj.w, cj.w);
            float2 acc2 = make_float2(0.f, 0.f);  // even and odd cells
            for (int pc = sub; pc < ncp; pc += gq) {
                // per half: fma(ex2(logit2(c_j, x_t) - rowmax_t) cinv_t, e_t, acc)
                const float4 a = cella[pc], b = cellb[pc];
                const float2 dx = __fadd2_rn(make_float2(a.x, a.y), ncx);
                const float2 dy = __fadd2_rn(make_float2(a.z, a.w), ncy);
                const float2 dz = __fadd2_rn(make_float2(b.x, b.y), ncz);
                float2 d2 = __fmul2_rn(dx, dx);
                d2 = __ffma2_rn(dy, dy, d2);
                d2 = __ffma2_rn(dz, dz, d2);
                const float2 l = __fadd2_rn(__fmul2_rn(cw, d2), make_float2(b.z, b.w));
                const float2 wt = __fmul2_rn(make_float2(tc::ex2(l.x), tc::ex2(l.y)), cinv2[pc]);
                acc2 = __ffma2_rn(wt, ce2[pc], acc2);
            }
            float acc = acc2.x + acc2.y;
            for (int o = 1; o < gq; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (act && sub == 0) {
                gr[j] = acc;
                ub[j] = fabsf(acc);
                cmax = fmaxf(cmax, fabsf(acc));
            }
        }
        if (tid == 0) { sh.viol = 0; sh.changed = 0; sh.dmax = 0.f; sh.xmax = 0.f; }
        __syncthreads();
        PROF_MARK(5);
        // stationarity residual on the support, violations off it
        float rmax = 0.f;
        int mv = 0;
        for (int j = tid; j < M; j += blockDim.x) {
            if (sg[j] != 0) rmax = fmaxf(rmax, fabsf(gr[j] - lam2 * x[j] - lam1 * (float)sg[j]));
            else if (ub[j] > kkt_tol) ++mv;  // computed this pass: ub_j = |c_j|
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
            if (sg[j] == 0 && ub[j] > kkt_tol) { sg[j] = gr[j] > 0.f ? 1 : -1; x[j] = 0.f; ++jn; }
        if (jn) atomicOr(&sh.changed, 1);
        __syncthreads();
        if (sh.changed) {
            mx_compact(sg, M, idx, &sh.cnt);
            scnt = sh.cnt;
            A = (tri_i(scnt, 0) * 4 <= kMxFactorBytes) ? Asm
                : (w.Lf + (size_t)s * ((size_t)mc * (mc + 1) / 2));
            mx_build(A, G, idx, scnt, mc, lam2);
            __syncthreads();
            mx_cholesky(A, scnt, &sh.flag, dinv, Lt);
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
        float dx = 0.f;
        if (tid == 0) sh.dinf = 0.f;
        for (int pp = tid; pp < scnt; pp += blockDim.x) {
            const int m = idx[pp];
            const float nx = x[m] + rhs[pp];
            if (!(nx * (float)sg[m] > 0.f)) { dx = fmaxf(dx, fabsf(x[m])); sg[m] = 0; x[m] = 0.f; ++dropped; }
            else { dx = fmaxf(dx, fabsf(rhs[pp])); x[m] = nx; }
        }
        for (int o2 = 16; o2 > 0; o2 >>= 1) {
            dropped += __shfl_xor_sync(0xffffffffu, dropped, o2);
            dx = fmaxf(dx, __shfl_xor_sync(0xffffffffu, dx, o2));
        }
        __syncthreads();  // sh.dinf reset before any warp adds to it
        if (lane == 0) {
            if (dropped) atomicOr(&sh.changed, 2);
            atomicMax(reinterpret_cast<int *>(&sh.dinf), __float_as_int(dx));
        }
        __syncthreads();
        {   // c moves by -G dx: the bounds off the support grow by wsum_j ||dx||_inf
            const float d = sh.dinf * 1.001f;
            for (int j = tid; j < M; j += blockDim.x)
                if (sg[j] == 0) ub[j] = fmaf(wsg[j], d, ub[j]);
        }
        if (sh.changed & 2) {  // support shrank: recompact and refactor
            mx_compact(sg, M, idx, &sh.cnt);
            scnt = sh.cnt;
            A = (tri_i(scnt, 0) * 4 <= kMxFactorBytes) ? Asm
                : (w.Lf + (size_t)s * ((size_t)mc * (mc + 1) / 2));
            mx_build(A, G, idx, scnt, mc, lam2);
            __syncthreads();
            mx_cholesky(A, scnt, &sh.flag, dinv, Lt);
        }
    }

    PROF_MARK(6);
    // indicators R_T (Eq. (4), midpoint) of the final x. A certified x is the
    // one the last gradient pass saw, with e = y - W x (fp32) in ce:
    // exp(y^) - K = K (exp(-e) - 1) = K expm1(-e), free of cancellation and
    // of binary64 work (the fp64 pipe is narrow on this part).
    if (cv) {
        // held-out residuals of the final x (the last exact pass saw it when certified)
        if (!certified) {
            held = 0.0;
            for (int t = fold + folds * tid; t < N; t += folds * (int)blockDim.x) {
                const float4 cx = cell_at(t);
                DFAcc acc;
                for (int pp = 0; pp < scnt; ++pp) {
                    const int m = idx[pp];
                    acc.add_prod(tc::ex2(logit2(sc[m], cx.x, cx.y, cx.z) - cx.w), x[m]);
                }
                const double e = yv[t] - acc.value() * (double)cinv[t];
                held += e * e;
            }
        }
        __shared__ double hpart[kMxThreads / 32];
        for (int o2 = 16; o2 > 0; o2 >>= 1) held += __shfl_xor_sync(0xffffffffu, held, o2);
        if (lane == 0) hpart[tid >> 5] = held;
        __syncthreads();
        if (tid == 0) {
            double tot = 0.0;
            for (int q = 0; q < (int)blockDim.x / 32; ++q) tot += hpart[q];
            cv[(size_t)s * cv_stride] += tot;
        }
    } else if (certified) {
        for (int t = tid; t < N; t += blockDim.x) {
            const double ev = w.kv[(size_t)s * g.n_max + t] * (double)expm1f(-ce[t]);
            w.R[(size_t)s * g.n_max + t] = cell_measure(g, s, t) * (ev * ev);
        }
    }
    // otherwise x changed after the last pass: e = y - W x once more
    for (int t = tid; t < N && !certified && !cv; t += blockDim.x) {
        const float4 cx = cell_at(t);
        DFAcc acc;
        for (int pp = 0; pp < scnt; ++pp) {
            const int m = idx[pp];
            acc.add_prod(tc::ex2(logit2(sc[m], cx.x, cx.y, cx.z) - cx.w), x[m]);
        }
        const double yhat = acc.value() * (double)cinv[t];
        const double kv = w.kv[(size_t)s * g.n_max + t];
        const double e = exp(yhat) - kv;
        w.R[(size_t)s * g.n_max + t] = cell_measure(g, s, t) * (e * e);
    }
    for (int j = tid; j < M; j += blockDim.x) beta[(size_t)s * mc + j] = (double)x[j];
    __syncthreads();
    PROF_MARK(7);
#ifdef PAM_SOLVE_PROFILE
    if (tid == 0 && s < 8192) g_solve_blk[s] = (unsigned long long)(clock64() - t_blk0);
#endif
    if (tid == 0) {
        int flags = inf[PAM_INFO_FLAGS] & ~(PAM_FLAG_NOT_CERTIFIED | PAM_FLAG_CHOLESKY | PAM_FLAG_REFINE_DIVERGED);
        if (!certified) {
            flags |= PAM_FLAG_NOT_CERTIFIED;
            // an uncertified fit takes a slot of the binary64 fallback, which
            // solves it again and sets the status if that fails too
            const int slot = (fallback && !cv) ? atomicAdd(&w.fb[0], 1) : w.fb_slots;
            if (slot < w.fb_slots) {
                w.fb[2 + slot] = s;
                flags |= PAM_FLAG_REFINE_DIVERGED;
            } else {
                atomicAdd(&w.status[kStUncertified], 1);
            }
        }
        if (sh.flag) flags |= PAM_FLAG_CHOLESKY;
        inf[PAM_INFO_FLAGS] = flags;
        inf[PAM_INFO_SUPPORT] = scnt;
        inf[PAM_INFO_ITERS] = it + 100 * refine_it;  // active-set steps + 100 x refinement steps
        const long long dt = clock64() - t_start;
        w.cost[s] = dt > 0xffffffffLL ? 0xffffffffu : (uint32_t)dt;
    }
}

// The subdomains go in decreasing cost of their previous solve, so the
// longest start first and the level does not wait on a late one. persistent
// = 0: one block per subdomain, block b taking the b-th of that order;
// persistent = 1: one block per resident slot, each taking the next
// subdomain of the order from the counter w.fb[1] until none is left.
// The body of both solve kernels: one subdomain per CTA (w.order[blockIdx.x],
// longest first), or resident CTAs taking the next subdomain of the same
// order from a counter (persistent).
template <bool SMALL>
__device__ __forceinline__ void solve_mixed_blocks(const Geo &g, const Par &p, const int32_t *boxes,
                                                   const double *centres, double *beta, int32_t *info,
                                                   const Ws &w, int kMxFactorBytes, const double *lam_tab, int all,
                                                   double *cv, int cv_stride, int fallback, int persistent) {
    if (!persistent) {
        solve_mixed_item<SMALL>(g, p, boxes, centres, beta, info, w, kMxFactorBytes, lam_tab, all, cv, cv_stride,
                                fallback, w.order[blockIdx.x]);
        return;
    }
    __shared__ int next;
    for (int it = 0;; ++it) {
        if (it) __syncthreads();  // the previous subdomain's readers are done with shared memory
        if (threadIdx.x == 0) next = atomicAdd(&w.fb[1], 1);
        __syncthreads();
        const int k = next;
        if (k >= group_count(g)) break;
        solve_mixed_item<SMALL>(g, p, boxes, centres, beta, info, w, kMxFactorBytes, lam_tab, all, cv, cv_stride,
                                fallback, w.order[k]);
    }
}

__global__ void __launch_bounds__(kMxThreads, 2) k_solve_mixed(Geo g, Par p, const int32_t *boxes,
                                                            const double *centres, double *beta,
                                                            int32_t *info, Ws w, int kMxFactorBytes,
                                                            const double *lam_tab, int all, double *cv,
                                                            int cv_stride, int fallback, int persistent) {
    solve_mixed_blocks<false>(g, p, boxes, centres, beta, info, w, kMxFactorBytes, lam_tab, all, cv, cv_stride,
                              fallback, persistent);
}

// Small dictionaries (every M <= kSmallSolveM: the initial lattices): 64
// threads per subdomain and per-centre arrays of kSmallSolveM entries, so
// that five CTAs share an SM (k_solve_mixed_small below).
// (No minimum-blocks bound: with one ptxas keeps the body in 150 registers
// without spills, while a bound of 4-6 blocks spills; shared memory holds it
// to five CTAs per SM either way.)
__global__ void __launch_bounds__(kSmallSolveThreads) k_solve_mixed_small(Geo g, Par p, const int32_t *boxes,
                                                                          const double *centres, double *beta,
                                                                          int32_t *info, Ws w, int kMxFactorBytes,
                                                                          int fallback) {
    solve_mixed_blocks<true>(g, p, boxes, centres, beta, info, w, kMxFactorBytes, nullptr, 0, nullptr, 0, fallback,
                             0);
}

// Longest-first order of the subdomains by the clock cost of their previous
// solve, by buckets of 1/8 octave (the leading bit and the next three of the
// cost): one pass of shared-memory counts, a scan from the costliest bucket
// down, one scatter. Within a bucket (costs within 12.5 %) the order is the
// atomics'; the results of the solve do not depend on the order.
__device__ __forceinline__ int cost_bucket(uint32_t c) {
    if (c < 16u) return (int)c;  // 0..15
    const int e = 31 - __clz((int)c);  // >= 4
    return 8 * e + (int)((c >> (e - 3)) & 7u) - 16;  // 16..239, increasing with c
}

// The subdomains ordered are gb + i gs for 0 <= i < n (a launch's group).
__global__ void __launch_bounds__(1024) k_solve_order(const uint32_t *cost, int n, int gb, int gs, int32_t *order,
                                                     int32_t *fb) {
    // the solve that follows fills the fallback list afresh and (persistent
    // launch) counts its subdomains from zero
    if (fb && threadIdx.x == 0) { fb[0] = 0; fb[1] = 0; }
    constexpr int kB = 256;
    __shared__ int cnt[kB], base[kB];
    for (int i = threadIdx.x; i < kB; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&cnt[cost_bucket(cost[gb + i * gs])], 1);
    __syncthreads();
    if (threadIdx.x < 32) {
        // exclusive scan from the costliest bucket down: lane l takes buckets
        // kB - 1 - 8 l down to kB - 8 - 8 l, the lanes' totals by a warp scan
        const int lane = threadIdx.x;
        int tot = 0;
        for (int u = 0; u < kB / 32; ++u) tot += cnt[kB - 1 - (kB / 32) * lane - u];
        int inc = tot;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        int run = inc - tot;
        for (int u = 0; u < kB / 32; ++u) {
            const int q = kB - 1 - (kB / 32) * lane - u;
            base[q] = run;
            run += cnt[q];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int sd = gb + i * gs;
        order[atomicAdd(&base[cost_bucket(cost[sd])], 1)] = sd;
    }
}

// Shared memory of the mixed solve besides the packed factor.
static size_t solve_mixed_smem_rest(const Geo &g, int mcs = 0) {
    if (mcs <= 0) mcs = g.m_cap;
    const size_t np2 = (size_t)(g.n_max + 1) / 2, ns2 = (size_t)mcs / 2 + 2;
    return (size_t)mcs * (6 * sizeof(float) + 2 * sizeof(int) + sizeof(float4)) +
           np2 * 2 * (sizeof(float4) + 2 * sizeof(float)) + ns2 * 2 * (sizeof(float4) + sizeof(float2)) +
           kCholLtFloats * sizeof(float) + 64;
}

// Shared-memory budget of the packed support factor (larger supports keep
// their factor in global memory, L2-resident): the largest multiple of 1 KiB
// up to 64 KiB with which two CTAs still fit on an SM (228 KiB per SM, 1 KiB
// reserved per CTA, 1 KiB of static shared memory), so that the patch size
// never halves the CTAs per SM; 64 KiB when even that cannot fit two.
// PAM_FACTOR_SMEM_KB overrides it (tuning).
static int factor_smem_bytes(const Geo &g) {
    static int env = -2;
    if (env == -2) {
        const char *e = getenv("PAM_FACTOR_SMEM_KB");
        env = e ? (atoi(e) * 1024 < 4096 ? 4096 : atoi(e) * 1024) : -1;
    }
    if (env > 0) return env;
    if (tuning().factor_kb > 0) return tuning().factor_kb * 1024;
    const long long per_cta = 228 * 1024 / 2 - 1024 - 1024;
    const long long room = (per_cta - (long long)solve_mixed_smem_rest(g)) / 1024 * 1024;
    if (room < 16 * 1024) return kMxFactorBytesDefault;
    return room < kMxFactorBytesDefault ? (int)room : kMxFactorBytesDefault;
}

static size_t solve_mixed_smem(const Geo &g) { return solve_mixed_smem_rest(g) + factor_smem_bytes(g); }

#ifdef PAM_SOLVE_PROFILE
extern "C" void pam_debug_gram_profile(unsigned long long *out, int reset) {
    cudaMemcpyFromSymbol(out, g_gram_prof, sizeof(g_gram_prof));
    if (reset) {
        unsigned long long z[16] = {};
        cudaMemcpyToSymbol(g_gram_prof, z, sizeof(z));
    }
}
extern "C" void pam_debug_solve_blocks(unsigned long long *out, int n) {
    cudaMemcpyFromSymbol(out, g_solve_blk, sizeof(unsigned long long) * (n < 8192 ? n : 8192));
}
extern "C" void pam_debug_solve_profile(unsigned long long *out, int reset) {
    cudaMemcpyFromSymbol(out, g_solve_prof, sizeof(g_solve_prof));
    cudaMemcpyFromSymbol(out + 16, g_solve_cnt, sizeof(g_solve_cnt));
    if (reset) {
        unsigned long long z[16] = {};
        cudaMemcpyToSymbol(g_solve_prof, z, sizeof(z));
        cudaMemcpyToSymbol(g_solve_cnt, z, sizeof(g_solve_cnt));
    }
}
#endif

bool mixed_solve_fits(const Geo &g) {
    return solve_mixed_smem(g) <= kSmemLimit && gram_tc_smem(g, 2) <= kSmemLimit;
}

void launch_solve_mixed(const Geo &g, const Par &p, const int32_t *boxes, const double *centres,
                        double *beta, int32_t *info, const Ws &w, const double *lam_tab, int all, double *cv,
                        int cv_stride, cudaStream_t st, int fallback, int m_bound) {
    PhaseScope ps(kPhSolve, st);
    const int fb = fallback && !cv && w.fb_slots > 0;
    if (m_bound > 0 && m_bound <= kSmallSolveM && !cv && !lam_tab && !all && kSmallSolveM <= g.m_cap) {
        // every dictionary is at most kSmallSolveM centres: the small-CTA form
        const int fbytes = ((kSmallSolveM + 2) * (kSmallSolveM + 1) / 2 * 4 + 1023) / 1024 * 1024;
        const size_t sm = solve_mixed_smem_rest(g, kSmallSolveM) + (size_t)fbytes;
        if (sm <= kSmemLimit) {
            cudaFuncSetAttribute(k_solve_mixed_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            k_solve_order<<<1, 1024, 0, st>>>(w.cost, group_count(g), g.gb, g.gs, w.order, w.fb);
            k_solve_mixed_small<<<group_count(g), kSmallSolveThreads, sm, st>>>(g, p, boxes, centres, beta, info, w, fbytes,
                                                                     fb);
            count_launches(2);
            if (fb) launch_fallback_f64(g, p, boxes, centres, beta, info, w, lam_tab, st);
            return;
        }
    }
    size_t sm = solve_mixed_smem(g);
    cudaFuncSetAttribute(k_solve_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_solve_order<<<1, 1024, 0, st>>>(w.cost, group_count(g), g.gb, g.gs, w.order, w.fb);
    count_launches(1);
    // persistent CTAs would hold every resident slot until their queue is
    // empty; in a subdomain group that would shut out the other group's
    // kernels, whose overlap is the point of the groups
    const int persistent = tuning().solve_persistent == 1 && w.fb != nullptr && g.gs == 1;
    unsigned grid = (unsigned)group_count(g);
    if (persistent) {
        // as many CTAs as fit the device at once with this launch's shared memory
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_solve_mixed, kMxThreads, sm);
        const int resident = sms * (per > 0 ? per : 1);
        grid = (unsigned)(resident < (int)grid ? resident : (int)grid);
    }
    k_solve_mixed<<<grid, kMxThreads, sm, st>>>(g, p, boxes, centres, beta, info, w, factor_smem_bytes(g),
                                                lam_tab, all, cv, cv_stride, fb, persistent);
    count_launches(1);
    if (fb) launch_fallback_f64(g, p, boxes, centres, beta, info, w, lam_tab, st);
}

void launch_solve_level_mixed(const Geo &g, const Par &p, const int32_t *boxes,
                              const double *centres, double *beta, int32_t *info, const Ws &w,
                              cudaStream_t st, cudaEvent_t before_solve, int m_bound) {
    launch_stats_gram_tc(g, boxes, centres, info, w, st, 0, m_bound);
    if (before_solve) cudaStreamWaitEvent(st, before_solve, 0);  // an error surfaces in cudaGetLastError
    launch_solve_mixed(g, p, boxes, centres, beta, info, w, nullptr, 0, nullptr, 0, st, 1, m_bound);
}

// The mixed solve already wrote the indicators of its final coefficients.
void launch_residual_mixed(const Geo &, const int32_t *, const double *, const double *,
                           const int32_t *, const Ws &, cudaStream_t) {}

// Failure-detection self-test: one thread waits on an mbarrier with the
// bounded wait of the tensor-core pipeline. arrive = 0: nothing arrives, the
// wait gives up after about `budget` clocks and flag = 1; arrive = 1: the
// barrier completes at once and flag = 0. Never traps, never hangs.
__global__ void k_wait_selftest(int arrive, long long budget, int32_t *flag) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (arrive) mbar_arrive(&bar);
        const bool ok = tc::mbar_wait(&bar, 0u, budget);
        *flag = ok ? 0 : 1;
    }
}

void launch_wait_selftest(int arrive, long long budget, int32_t *flag, cudaStream_t st) {
    k_wait_selftest<<<1, 32, 0, st>>>(arrive, budget, flag);
    count_launches(1);
}

}  // namespace pam
