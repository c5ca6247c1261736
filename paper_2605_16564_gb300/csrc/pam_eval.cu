// pam_eval.cu -- Step 4 (global reconstruction): evaluation of the piecewise
// surrogate K*(x) = exp(sum_m beta_m w_m(x)) at arbitrary points, and the
// error measures over the source cells.
//
// Evaluation buckets the points by owner subdomain first (owner of each
// point, warp-aggregated counts, an exclusive scan, a scatter of point
// indices), then one block per owner stages that owner's dictionary in
// shared memory and sweeps its points. Results are written by point index,
// so the (non-deterministic) order inside a bucket does not matter.
//
// fp64 form: two passes per point (maximum logit, then the shifted sum).
// fp32 form: one pass without a shift. Every point of a core lies within
//   half a lattice spacing (per axis) of an initial lattice centre of width
//   = the largest spacing, so the largest Gaussian is at least
//   exp(-d/8) >= 0.68: the unshifted sum neither underflows nor overflows
//   (a guard recomputes with the shift if it ever falls below 2^-100).
#include <cfloat>
#include <cmath>

#include "pam_internal.cuh"
#include "pam_tc.cuh"

namespace pam {

struct EvalWs {
    int32_t *owner, *rank, *perm, *count, *start;
    size_t bytes;
};

static size_t align256(size_t v) { return (v + 255) / 256 * 256; }

EvalWs carve_eval_workspace(int S, int64_t n, void *base) {
    EvalWs e;
    size_t off = 0;
    auto take = [&](size_t bytes) -> int32_t * {
        int32_t *p = base ? (int32_t *)((char *)base + off) : nullptr;
        off = align256(off + bytes);
        return p;
    };
    e.owner = take((size_t)n * 4);
    e.rank = take((size_t)n * 4);
    e.perm = take((size_t)n * 4);
    e.count = take((size_t)S * 4);
    e.start = take((size_t)(S + 1) * 4);
    e.bytes = off;
    return e;
}

size_t eval_workspace_bytes(int S, int64_t n_pts) { return carve_eval_workspace(S, n_pts, nullptr).bytes; }

__global__ void k_eval_owner(Geo g, const double *pts, int64_t n, int32_t *owner, int32_t *rank,
                             int32_t *count, double *out) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int s = -2;  // lanes past the end take a key no real owner has
    if (p < n) {
        double x[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (a < g.dim) x[a] = pts[p * g.dim + a];
        s = owner_of_point(g, x);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, s);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader && s >= 0) base = atomicAdd(&count[s], __popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (p < n) {
        owner[p] = s;
        rank[p] = base + __popc(peers & ((1u << lane) - 1u));
        if (s < 0) out[p] = nan("");
    }
}

// Exclusive scan of count[0..S) into start[0..S] by one block of 1024.
__global__ void __launch_bounds__(1024) k_eval_scan(const int32_t *count, int32_t *start, int S) {
    __shared__ int wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (S + 1023) / 1024;
    const int b = tid * per, e = min(S, b + per);
    int local = 0;
    for (int i = b; i < e; ++i) local += count[i];
    int v = local;
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int t = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        wsum[lane] = t;
    }
    __syncthreads();
    int run = v - local + (warp > 0 ? wsum[warp - 1] : 0);
    for (int i = b; i < e; ++i) {
        start[i] = run;
        run += count[i];
    }
    if (tid == 1023) start[S] = run;
}

__global__ void k_eval_scatter(const int32_t *owner, const int32_t *rank, const int32_t *start,
                               int32_t *perm, int64_t n) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int s = owner[p];
    if (s >= 0) perm[start[s] + rank[p]] = (int32_t)p;
}

// ---------------------------------------------------------------- fp64 ------
__device__ __forceinline__ double shepard_f64_smem(const dvec4 *sc, const double *sb, int M,
                                                   const double x[3]) {
    double lmax = -INFINITY;
    for (int m = 0; m < M; ++m) {
        const dvec4 c = sc[m];
        double d0 = x[0] - c.x, d1 = x[1] - c.y, d2 = x[2] - c.z;
        lmax = fmax(lmax, (d0 * d0 + d1 * d1 + d2 * d2) * c.w);
    }
    double num = 0.0, den = 0.0;
    for (int m = 0; m < M; ++m) {
        const dvec4 c = sc[m];
        double d0 = x[0] - c.x, d1 = x[1] - c.y, d2 = x[2] - c.z;
        double e = exp((d0 * d0 + d1 * d1 + d2 * d2) * c.w - lmax);
        num += sb[m] * e;
        den += e;
    }
    return num / den;
}

// Copies subdomain s's centres (M x 32 bytes) and coefficients (M x 8
// bytes, padded to 16 with the next entry: the capacity is a multiple of 64)
// into shared memory with the bulk-copy engine, thread 0 issuing, everyone
// waiting on one mbarrier (bounded). Returns false -- and nothing may be
// read from dst_c / dst_b -- if an address is not 16-byte aligned or the
// wait gave up; the caller then loads from global memory instead.
__device__ bool stage_bulk(const Geo &g, const double *centres, const double *beta, int s, int M, dvec4 *dst_c,
                           double *dst_b) {
    __shared__ uint64_t bar;
    __shared__ int use_bulk;
    const dvec4 *src_c = reinterpret_cast<const dvec4 *>(centres) + (size_t)s * g.m_cap;
    const double *src_b = beta + (size_t)s * g.m_cap;
    const uint32_t bytes_c = (uint32_t)M * 32u, bytes_b = ((uint32_t)M * 8u + 15u) & ~15u;
    if (threadIdx.x == 0) {
        const bool aligned = ((reinterpret_cast<uintptr_t>(src_c) | reinterpret_cast<uintptr_t>(src_b) |
                               (uintptr_t)tc::smem_u32(dst_c) | (uintptr_t)tc::smem_u32(dst_b)) & 15u) == 0;
        use_bulk = aligned && M > 0;
        if (use_bulk) {
            tc::mbar_init(&bar, 1);
            tc::mbar_fence_init();
        }
    }
    __syncthreads();
    if (!use_bulk) return false;
    if (threadIdx.x == 0) {
        tc::mbar_arrive_expect_tx(&bar, bytes_c + bytes_b);
        tc::bulk_g2s(dst_c, src_c, bytes_c, &bar);
        tc::bulk_g2s(dst_b, src_b, bytes_b, &bar);
    }
    // ~1 s at 2 GHz (a bulk copy of a few KB takes microseconds); if it gives
    // up, wait once more for the copy in flight before anyone falls back
    bool ok = tc::mbar_wait(&bar, 0, 2000000000LL);
    if (!ok) ok = tc::mbar_wait(&bar, 0, 2000000000LL);
    return __syncthreads_and(ok ? 1 : 0) != 0;
}

// Dictionary of subdomain s in shared memory: (c, -1/(2 sigma^2)) and beta.
__device__ void stage_f64(const Geo &g, const double *centres, const double *beta, int s, int M,
                          dvec4 *sc, double *sb) {
    if (stage_bulk(g, centres, beta, s, M, sc, sb)) {  // copied as is; the width becomes the logit factor
        for (int m = threadIdx.x; m < M; m += blockDim.x) {
            const double sg = sc[m].w;
            sc[m].w = -1.0 / (2.0 * sg * sg);
        }
        __syncthreads();
        return;
    }
    const dvec4 *cg = reinterpret_cast<const dvec4 *>(centres) + (size_t)s * g.m_cap;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        dvec4 c = cg[m];
        c.w = -1.0 / (2.0 * c.w * c.w);
        sc[m] = c;
        sb[m] = beta[(size_t)s * g.m_cap + m];
    }
    __syncthreads();
}

__global__ void k_eval_bucket_f64(Geo g, const double *centres, const double *beta,
                                  const int32_t *info, const double *pts, const int32_t *perm,
                                  const int32_t *start, double *out, int log_space) {
    const int s = blockIdx.x;
    const int b = start[s], e = start[s + 1];
    if (b == e) return;
    const int M = info[s * kInfoN + PAM_INFO_M];
    extern __shared__ uint8_t smb[];
    dvec4 *sc = reinterpret_cast<dvec4 *>(smb);
    double *sb = reinterpret_cast<double *>(sc + g.m_cap);
    stage_f64(g, centres, beta, s, M, sc, sb);
    for (int i = b + threadIdx.x; i < e; i += blockDim.x) {
        const int p = perm[i];
        double x[3] = {0, 0, 0};
        for (int a = 0; a < g.dim; ++a) x[a] = pts[(int64_t)p * g.dim + a];
        const double v = shepard_f64_smem(sc, sb, M, x);
        out[p] = log_space ? v : exp(v);
    }
}

// ---------------------------------------------------------------- fp32 ------
__device__ __forceinline__ float4 local_centre_e(const dvec4 &c, const double o[3]) {
    float4 r;
    r.x = (float)(c.x - o[0]);
    r.y = (float)(c.y - o[1]);
    r.z = (float)(c.z - o[2]);
    const float sg = (float)c.w;  // fp32 alpha (no fp64 divide)
    r.w = -1.44269504f / (2.f * sg * sg);
    return r;
}

// exp in fp32 on the special-function unit (relative error ~1e-7)
__device__ __forceinline__ double exp_f32(float v) { return (double)tc::ex2(v * 1.44269504f); }

__device__ __forceinline__ float logit2_e(const float4 &c, float x, float y, float z) {
    float dx = x - c.x, dy = y - c.y, dz = z - c.z;
    return c.w * fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}

__device__ __forceinline__ float shepard_f32_smem(const float4 *sc, const float *sb, int M,
                                                  float x, float y, float z) {
    float num = 0.f, den = 0.f;
    for (int m = 0; m < M; ++m) {
        const float e = tc::ex2(logit2_e(sc[m], x, y, z));
        num = fmaf(sb[m], e, num);
        den += e;
    }
    if (!(den > 7.9e-31f)) {  // 2^-100: recompute with the maximum logit subtracted
        float lmax = -INFINITY;
        for (int m = 0; m < M; ++m) lmax = fmaxf(lmax, logit2_e(sc[m], x, y, z));
        num = 0.f;
        den = 0.f;
        for (int m = 0; m < M; ++m) {
            const float e = tc::ex2(logit2_e(sc[m], x, y, z) - lmax);
            num = fmaf(sb[m], e, num);
            den += e;
        }
    }
    return num / den;
}

// Two points at once: every centre read from shared memory serves both
// (halves the shared-memory traffic per Gaussian). Falls back to the single
// point form when a sum underflows.
__device__ __forceinline__ void shepard_f32_smem2(const float4 *sc, const float *sb, int M, const float p0[3],
                                                  const float p1[3], float *v0, float *v1) {
    float n0 = 0.f, d0 = 0.f, n1 = 0.f, d1 = 0.f;
    for (int m = 0; m < M; ++m) {
        const float4 c = sc[m];
        const float bm = sb[m];
        const float e0 = tc::ex2(logit2_e(c, p0[0], p0[1], p0[2]));
        const float e1 = tc::ex2(logit2_e(c, p1[0], p1[1], p1[2]));
        n0 = fmaf(bm, e0, n0);
        d0 += e0;
        n1 = fmaf(bm, e1, n1);
        d1 += e1;
    }
    *v0 = (d0 > 7.9e-31f) ? n0 / d0 : shepard_f32_smem(sc, sb, M, p0[0], p0[1], p0[2]);
    *v1 = (d1 > 7.9e-31f) ? n1 / d1 : shepard_f32_smem(sc, sb, M, p1[0], p1[1], p1[2]);
}

// Dynamic shared memory of the fp32 staging: the converted centres and
// coefficients, then (32-byte aligned) the raw copies the bulk copy lands in.
static size_t stage_f32_smem(int m_cap) {
    return ((size_t)m_cap * (sizeof(float4) + sizeof(float)) + 31) / 32 * 32 + 32 +  // + alignment slack
           (size_t)m_cap * (sizeof(dvec4) + sizeof(double));
}

__device__ void stage_f32(const Geo &g, const int32_t *boxes, const double *centres,
                          const double *beta, int s, int M, float4 *sc, float *sb, double o[3]) {
    const int32_t *box = boxes + s * 12;
    for (int a = 0; a < 3; ++a) o[a] = a < g.dim ? (double)box[6 + a] * g.h : 0.0;
    dvec4 *raw_c = reinterpret_cast<dvec4 *>((reinterpret_cast<uintptr_t>(sb + g.m_cap) + 31) & ~(uintptr_t)31);
    double *raw_b = reinterpret_cast<double *>(raw_c + g.m_cap);
    if (stage_bulk(g, centres, beta, s, M, raw_c, raw_b)) {
        for (int m = threadIdx.x; m < M; m += blockDim.x) {
            sc[m] = local_centre_e(raw_c[m], o);
            sb[m] = (float)raw_b[m];
        }
        __syncthreads();
        return;
    }
    const dvec4 *cg = reinterpret_cast<const dvec4 *>(centres) + (size_t)s * g.m_cap;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        sc[m] = local_centre_e(cg[m], o);
        sb[m] = (float)beta[(size_t)s * g.m_cap + m];
    }
    __syncthreads();
}

// Scaled form of the evaluation's logit. With a = sqrt(log2(e) / 2) / sigma
// per centre, the base-2 logit -|x - c|^2 / (2 sigma^2) log2(e) is
// -|a x - a c|^2: three multiply-adds (a x_i - a c_i) and a sum of squares,
// six operations per centre and point against seven for the difference form.
// The rounding of a c_i costs ~2 eps a^2 R |x - c| in the logit (R the
// distance from the patch centre, the origin of the local coordinates):
// proportional to |x - c|, so it stays below ~1e-5 wherever the weight is
// not negligible. Points go through the centres in pairs, one per half of
// each packed fp32x2 operation (the same operations, in the same order, as
// for a single point). Centre m is stored duplicated for that:
// su[2m] = (-a c_x, -a c_x, -a c_y, -a c_y), su[2m + 1] = (-a c_z, -a c_z, a, a),
// sb[m] = (beta_m, beta_m).
static size_t stage_f32s_smem(int m_cap) {
    return ((size_t)m_cap * (2 * sizeof(float4) + sizeof(float2)) + 31) / 32 * 32 + 32 +  // + alignment slack
           (size_t)m_cap * (sizeof(dvec4) + sizeof(double));
}

__device__ __forceinline__ void put_centre_s(const dvec4 &c, double b, const double o[3], float4 *su, float2 *sb) {
    const float sg = (float)c.w;
    const float a = 0.84932180f / sg;  // sqrt(log2(e) / 2) / sigma
    const float ax = a * (float)(c.x - o[0]), ay = a * (float)(c.y - o[1]), az = a * (float)(c.z - o[2]);
    su[0] = make_float4(-ax, -ax, -ay, -ay);
    su[1] = make_float4(-az, -az, a, a);
    *sb = make_float2((float)b, (float)b);
}

__device__ void stage_f32s(const Geo &g, const int32_t *boxes, const double *centres, const double *beta, int s,
                           int M, float4 *su, float2 *sb, double o[3]) {
    const int32_t *box = boxes + s * 12;
    for (int a = 0; a < 3; ++a) o[a] = a < g.dim ? 0.5 * (double)(box[6 + a] + box[9 + a]) * g.h : 0.0;
    dvec4 *raw_c = reinterpret_cast<dvec4 *>((reinterpret_cast<uintptr_t>(sb + g.m_cap) + 31) & ~(uintptr_t)31);
    double *raw_b = reinterpret_cast<double *>(raw_c + g.m_cap);
    if (stage_bulk(g, centres, beta, s, M, raw_c, raw_b)) {
        for (int m = threadIdx.x; m < M; m += blockDim.x) put_centre_s(raw_c[m], raw_b[m], o, su + 2 * m, sb + m);
        __syncthreads();
        return;
    }
    const dvec4 *cg = reinterpret_cast<const dvec4 *>(centres) + (size_t)s * g.m_cap;
    for (int m = threadIdx.x; m < M; m += blockDim.x)
        put_centre_s(cg[m], beta[(size_t)s * g.m_cap + m], o, su + 2 * m, sb + m);
    __syncthreads();
}

// One point with the maximum logit subtracted (the plain sums underflowed):
// minus the logit |a x - a c|^2 per centre, as the packed form computes it.
__device__ __noinline__ float shepard_f32s_shifted(const float4 *su, const float2 *sb, int M, float x, float y,
                                                   float z) {
    auto nl = [&](int m) {
        const float4 u = su[2 * m], v = su[2 * m + 1];
        const float dx = fmaf(v.z, x, u.x), dy = fmaf(v.z, y, u.z), dz = fmaf(v.z, z, v.x);
        return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    };
    float nmin = INFINITY;
    for (int m = 0; m < M; ++m) nmin = fminf(nmin, nl(m));
    float num = 0.f, den = 0.f;
    for (int m = 0; m < M; ++m) {
        const float e = tc::ex2(nmin - nl(m));
        num = fmaf(sb[m].x, e, num);
        den += e;
    }
    return num / den;
}

// P points (P even) at once, in pairs: every centre read from shared memory
// serves all of them.
template <int P>
__device__ __forceinline__ void shepard_f32s(const float4 *su, const float2 *sb, int M, const float (&p)[P][3],
                                             float (&v)[P]) {
    constexpr int H = P / 2;
    float2 X[H], Y[H], Z[H], num[H], den[H];
#pragma unroll
    for (int k = 0; k < H; ++k) {
        X[k] = make_float2(p[2 * k][0], p[2 * k + 1][0]);
        Y[k] = make_float2(p[2 * k][1], p[2 * k + 1][1]);
        Z[k] = make_float2(p[2 * k][2], p[2 * k + 1][2]);
        num[k] = make_float2(0.f, 0.f);
        den[k] = make_float2(0.f, 0.f);
    }
    for (int m = 0; m < M; ++m) {
        const float4 u = su[2 * m], w = su[2 * m + 1];
        const float2 bm = sb[m], a2 = make_float2(w.z, w.w);
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const float2 dx = __ffma2_rn(a2, X[k], make_float2(u.x, u.y));
            const float2 dy = __ffma2_rn(a2, Y[k], make_float2(u.z, u.w));
            const float2 dz = __ffma2_rn(a2, Z[k], make_float2(w.x, w.y));
            float2 q = __fmul2_rn(dx, dx);
            q = __ffma2_rn(dy, dy, q);
            q = __ffma2_rn(dz, dz, q);
            const float2 e = make_float2(tc::ex2(-q.x), tc::ex2(-q.y));
            num[k] = __ffma2_rn(bm, e, num[k]);
            den[k] = __fadd2_rn(e, den[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < H; ++k) {
        v[2 * k] = (den[k].x > 7.9e-31f) ? num[k].x / den[k].x
                                         : shepard_f32s_shifted(su, sb, M, p[2 * k][0], p[2 * k][1], p[2 * k][2]);
        v[2 * k + 1] = (den[k].y > 7.9e-31f)
                           ? num[k].y / den[k].y
                           : shepard_f32s_shifted(su, sb, M, p[2 * k + 1][0], p[2 * k + 1][1], p[2 * k + 1][2]);
    }
}

constexpr int kEvalPts = 4;  // points per thread and pass of the fp32 bucket evaluation

__global__ void k_eval_bucket_f32(Geo g, const int32_t *boxes, const double *centres,
                                  const double *beta, const int32_t *info, const double *pts,
                                  const int32_t *perm, const int32_t *start, double *out,
                                  int log_space) {
    const int s = blockIdx.x;
    const int b = start[s], e = start[s + 1];
    if (b == e) return;
    const int M = info[s * kInfoN + PAM_INFO_M];
    extern __shared__ uint8_t smb[];
    float4 *su = reinterpret_cast<float4 *>(smb);
    float2 *sb = reinterpret_cast<float2 *>(su + 2 * g.m_cap);
    double o[3];
    stage_f32s(g, boxes, centres, beta, s, M, su, sb, o);
    // kEvalPts points per thread and pass: i, i + blockDim.x, ...
    const int bd = blockDim.x;
    for (int i = b + threadIdx.x; i < e; i += kEvalPts * bd) {
        int pi[kEvalPts];
        float x[kEvalPts][3];
#pragma unroll
        for (int k = 0; k < kEvalPts; ++k) {
            pi[k] = i + k * bd < e ? perm[i + k * bd] : -1;
            const int64_t q = pi[k] >= 0 ? pi[k] : perm[i];  // idle slots repeat the first point
#pragma unroll
            for (int a = 0; a < 3; ++a) x[k][a] = a < g.dim ? (float)(pts[q * g.dim + a] - o[a]) : 0.f;
        }
        float v[kEvalPts];
        shepard_f32s<kEvalPts>(su, sb, M, x, v);
#pragma unroll
        for (int k = 0; k < kEvalPts; ++k)
            if (pi[k] >= 0) out[pi[k]] = log_space ? (double)v[k] : exp_f32(v[k]);
    }
}

// Threads per block of the bucket kernels (the tuned value, else 256).
static int eval_block() {
    const int b = tuning().eval_block;
    return (b == 128 || b == 256 || b == 512 || b == 1024) ? b : 256;
}

// The points bucketed by owner (they and the partition only, not the model:
// a caller may run it beside the fit); NaN into out for points outside the grid.
void launch_eval_bucket(const Geo &g, const double *pts, int64_t n_pts, double *out, void *ws, cudaStream_t st) {
    PhaseScope ps(kPhEval, st);
    EvalWs e = carve_eval_workspace(g.S, n_pts, ws);
    cudaMemsetAsync(e.count, 0, (size_t)g.S * sizeof(int32_t), st);
    const unsigned nb = (unsigned)((n_pts + 255) / 256);
    k_eval_owner<<<nb, 256, 0, st>>>(g, pts, n_pts, e.owner, e.rank, e.count, out);
    k_eval_scan<<<1, 1024, 0, st>>>(e.count, e.start, g.S);
    k_eval_scatter<<<nb, 256, 0, st>>>(e.owner, e.rank, e.start, e.perm, n_pts);
    count_launches(3);
}

// The surrogate at the bucketed points, one block per owner.
void launch_eval_bucketed(const Geo &g, const int32_t *boxes, const double *centres, const double *beta,
                          const int32_t *info, const double *pts, int64_t n_pts, double *out, int log_space,
                          int precision, void *ws, cudaStream_t st) {
    PhaseScope ps(kPhEval, st);
    EvalWs e = carve_eval_workspace(g.S, n_pts, ws);
    {
        PhaseScope pk(kPhEvalKernel, st);  // the per-owner kernel alone
        if (precision == PAM_PREC_MIXED) {
            size_t sm = stage_f32s_smem(g.m_cap);
            cudaFuncSetAttribute(k_eval_bucket_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            k_eval_bucket_f32<<<g.S, eval_block(), sm, st>>>(g, boxes, centres, beta, info, pts, e.perm, e.start,
                                                             out, log_space);
        } else {
            size_t sm = (size_t)g.m_cap * (sizeof(dvec4) + sizeof(double));
            cudaFuncSetAttribute(k_eval_bucket_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            k_eval_bucket_f64<<<g.S, eval_block(), sm, st>>>(g, centres, beta, info, pts, e.perm, e.start, out,
                                                             log_space);
        }
    }
    count_launches(1);
}

void launch_eval(const Geo &g, const int32_t *boxes, const double *centres, const double *beta,
                 const int32_t *info, const double *pts, int64_t n_pts, double *out, int log_space,
                 int precision, void *ws, cudaStream_t st) {
    launch_eval_bucket(g, pts, n_pts, out, ws, st);
    launch_eval_bucketed(g, boxes, centres, beta, info, pts, n_pts, out, log_space, precision, ws, st);
}

// --------------------------------------------------------------------------
// Glued evaluation across subdomain interfaces (section 2, Step 4 remark:
// the piecewise surrogate jumps at the interfaces; a gluing of neighbouring
// local surrogates makes it continuous, the procedure left open). The local
// log-surrogates u_i = sum_m beta_m w_m are blended by a tensor-product
// partition of unity that ramps across every interior core face over a band
// of half-width delta = band * h:
//   psi_i(x) = prod_a r((x_a - lo_a + delta) / (2 delta)) r((hi_a + delta - x_a) / (2 delta)),
//   r(t) = t^2 (3 - 2 t) on [0, 1], clamped (r(t) + r(1 - t) = 1), a factor
//   of 1 at the outer faces of the grid, and
//   ln K*(x) = sum_i psi_i u_i / sum_i psi_i.
// With band <= half the narrowest core, at most two cores per axis carry
// weight at a point, so a point has at most 2^dim (point, subdomain) pairs,
// slot p * 2^dim + c with bit a of c choosing the lower (0) or upper (1)
// candidate along axis a; ascending c is ascending subdomain index.
// Pairs are bucketed by subdomain like the points of pam_eval (counts,
// scan, scatter); one block per subdomain evaluates u_i at its pairs into
// val[slot]; a last pass sums psi_i u_i over each point's pairs in slot
// order (deterministic) and divides by sum psi_i.
// --------------------------------------------------------------------------
struct GlueWs {
    int32_t *rank, *perm, *count, *start, *sub;
    double *val, *psi;   // binary64 form
    float *valf, *psif;  // fp32 form (the same memory)
    uint8_t *mask;
    size_t bytes;
};

GlueWs carve_glue_workspace(int S, int dim, int64_t n, void *base) {
    GlueWs e;
    size_t off = 0;
    const size_t slots = (size_t)n << dim;
    auto take = [&](size_t bytes) -> void * {
        void *p = base ? (void *)((char *)base + off) : nullptr;
        off = align256(off + bytes);
        return p;
    };
    e.val = (double *)take(slots * 8);
    e.psi = (double *)take(slots * 8);
    e.rank = (int32_t *)take(slots * 4);
    e.perm = (int32_t *)take(slots * 4);
    e.sub = (int32_t *)take(slots * 4);
    e.mask = (uint8_t *)take((size_t)n);
    e.valf = reinterpret_cast<float *>(e.val);
    e.psif = reinterpret_cast<float *>(e.psi);
    e.count = (int32_t *)take((size_t)S * 4);
    e.start = (int32_t *)take((size_t)(S + 1) * 4);
    e.bytes = off;
    return e;
}

size_t glue_workspace_bytes(int S, int dim, int64_t n_pts) {
    return carve_glue_workspace(S, dim, n_pts, nullptr).bytes;
}

__device__ __forceinline__ double glue_ramp(double t) {
    t = fmin(fmax(t, 0.0), 1.0);
    return __dmul_rn(__dmul_rn(t, t), __dsub_rn(3.0, __dmul_rn(2.0, t)));
}

// Face factors of core c along an axis at coordinate xa: the lower face's
// ramp (1 at the outer face) and the upper face's.
__device__ __forceinline__ void glue_factors(int c, int n, int p, double h, double delta, double two_d,
                                             double xa, double *l, double *r) {
    const int64_t lo = ((int64_t)c * n) / p, hi = ((int64_t)(c + 1) * n) / p;
    *l = c > 0 ? glue_ramp(__ddiv_rn(__dadd_rn(__dsub_rn(xa, __dmul_rn((double)lo, h)), delta), two_d)) : 1.0;
    *r = c < p - 1 ? glue_ramp(__ddiv_rn(__dsub_rn(__dadd_rn(__dmul_rn((double)hi, h), delta), xa), two_d)) : 1.0;
}

__device__ __forceinline__ float glue_ramp_f(float t) {
    t = fminf(fmaxf(t, 0.f), 1.f);
    return t * t * (3.f - 2.f * t);
}

// The pairs of point x: subdomain s[c] and weight psi[c] for the valid slots
// c (bit c of the returned mask). Mask 0: x lies outside the grid. Along
// each axis the owner core j carries weight, and so does at most one of its
// neighbours (j - 1 below it or j + 1 above it; when band <= half the
// narrowest core both can carry weight only by rounding at a ramp's end,
// weight below 2^-100, and the larger is kept). Candidate 0 is the lower
// core, so ascending c is ascending subdomain index. The weight multiplies
// the face factors axis by axis, lower face first, in unfused binary64.
template <int D>
__device__ __forceinline__ unsigned glue_pairs(const Geo &g, double delta, const double x[3], int s[8],
                                               double psi[8]) {
    const double two_d = 2.0 * delta;
    int c0[3] = {0, 0, 0}, c1[3] = {0, 0, 0}, cnt[3] = {1, 1, 1};
    double l0[3] = {1.0, 1.0, 1.0}, r0[3] = {1.0, 1.0, 1.0}, l1[3] = {1.0, 1.0, 1.0}, r1[3] = {1.0, 1.0, 1.0};
    bool inside = true;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const double u = x[a] * (double)g.nmax;
        const bool in_a = (u >= 0.0) && (u <= (double)g.n[a]);
        inside = inside && in_a;
        int i = in_a ? (int)floor(u) : 0;
        if (i >= g.n[a]) i = g.n[a] - 1;
        const int j = core_of(i, g.n[a], g.p[a]);
        // at least delta from both faces of the owner core (or at an outer
        // face): the owner's factors are exactly 1 and the neighbours' 0 up
        // to rounding (below 2^-100), so the ramps are not evaluated
        const int64_t lo = ((int64_t)j * g.n[a]) / g.p[a], hi = ((int64_t)(j + 1) * g.n[a]) / g.p[a];
        const bool far_lo = j == 0 || __dsub_rn(x[a], __dmul_rn((double)lo, g.h)) >= delta;
        const bool far_hi = j == g.p[a] - 1 || __dsub_rn(__dmul_rn((double)hi, g.h), x[a]) >= delta;
        if (far_lo && far_hi) {
            c0[a] = j;
        } else {
            double lj, rj, lm = 0.0, rm = 0.0, lp = 0.0, rp = 0.0;
            glue_factors(j, g.n[a], g.p[a], g.h, delta, two_d, x[a], &lj, &rj);
            if (!far_lo) glue_factors(j - 1, g.n[a], g.p[a], g.h, delta, two_d, x[a], &lm, &rm);
            if (!far_hi) glue_factors(j + 1, g.n[a], g.p[a], g.h, delta, two_d, x[a], &lp, &rp);
            const double wm = __dmul_rn(lm, rm), wp = __dmul_rn(lp, rp);
            bool use_m = wm > 0.0, use_p = wp > 0.0;
            if (use_m && use_p) {
                use_m = wm >= wp;
                use_p = !use_m;
            }
            c0[a] = use_m ? j - 1 : j;
            l0[a] = use_m ? lm : lj;
            r0[a] = use_m ? rm : rj;
            c1[a] = use_m ? j : j + 1;
            l1[a] = use_m ? lj : lp;
            r1[a] = use_m ? rj : rp;
            cnt[a] = (use_m || use_p) ? 2 : 1;
        }
    }
    unsigned mask = 0u;
#pragma unroll
    for (int c = 0; c < (1 << D); ++c) {
        int idx = 0, mul = 1;
        double w = 1.0;
        bool ok = inside;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const bool up = (c >> a) & 1;
            ok = ok && (!up || cnt[a] == 2);
            w = __dmul_rn(w, up ? l1[a] : l0[a]);
            w = __dmul_rn(w, up ? r1[a] : r0[a]);
            idx += (up ? c1[a] : c0[a]) * mul;
            mul *= g.p[a];
        }
        ok = ok && w > 0.0;
        s[c] = ok ? idx : 0;
        psi[c] = ok ? w : 0.0;
        mask |= ok ? (1u << c) : 0u;
    }
    return mask;
}

// The fp32 form of glue_pairs (the mixed evaluation): everything in fp32
// cell units u = x / h, the ramps ((u - lo) + band) / (2 band) and
// ((hi + band) - u) / (2 band); one conversion of each coordinate is the only
// binary64 operation (GB300's FP64 pipe is narrow). Same candidates, order
// and masks as glue_pairs, weights to fp32 rounding.
template <int D>
__device__ __forceinline__ unsigned glue_pairs_f(const Geo &g, float band, const double x[3], int s[8],
                                                 float psi[8]) {
    const float inv = 1.0f / (2.0f * band), nmax = (float)g.nmax;
    int c0[3] = {0, 0, 0}, c1[3] = {0, 0, 0}, cnt[3] = {1, 1, 1};
    float l0[3] = {1.f, 1.f, 1.f}, r0[3] = {1.f, 1.f, 1.f}, l1[3] = {1.f, 1.f, 1.f}, r1[3] = {1.f, 1.f, 1.f};
    bool inside = true;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const float u = (float)x[a] * nmax;
        const bool in_a = (u >= 0.f) && (u <= (float)g.n[a]);
        inside = inside && in_a;
        int i = in_a ? (int)floorf(u) : 0;
        if (i >= g.n[a]) i = g.n[a] - 1;
        const int j = core_of(i, g.n[a], g.p[a]);
        const int p = g.p[a], n = g.n[a];
        const int64_t lo_i = ((int64_t)j * n) / p, hi_i = ((int64_t)(j + 1) * n) / p;
        // far from both faces (with half a cell to spare for the fp32 u)
        const bool far_lo = j == 0 || u - (float)lo_i >= band + 0.5f;
        const bool far_hi = j == p - 1 || (float)hi_i - u >= band + 0.5f;
        if (far_lo && far_hi) {
            c0[a] = j;
        } else {
            // the offset from the lower face in binary64 (u ~ 1e3 cells would
            // leave ~1e-4 cells of fp32 rounding), the ramps in fp32
            const float d = (float)(x[a] * (double)g.nmax - (double)lo_i);  // u - lo
            const float w = (float)(hi_i - lo_i);                           // core width
            const float lj = j > 0 ? glue_ramp_f((d + band) * inv) : 1.f;
            const float rj = j < p - 1 ? glue_ramp_f(((w + band) - d) * inv) : 1.f;
            float lm = 0.f, rm = 0.f, lp = 0.f, rp = 0.f;
            if (j > 0) {  // core j-1: its upper face is lo
                const float wm_ = (float)(lo_i - ((int64_t)(j - 1) * n) / p);
                lm = j - 1 > 0 ? glue_ramp_f(((d + wm_) + band) * inv) : 1.f;
                rm = glue_ramp_f((band - d) * inv);
            }
            if (j < p - 1) {  // core j+1: its lower face is hi
                const float wp_ = (float)(((int64_t)(j + 2) * n) / p - hi_i);
                lp = glue_ramp_f(((d - w) + band) * inv);
                rp = j + 1 < p - 1 ? glue_ramp_f(((wp_ + band) - (d - w)) * inv) : 1.f;
            }
            const float wm = lm * rm, wp = lp * rp;
            bool use_m = wm > 0.f, use_p = wp > 0.f;
            if (use_m && use_p) {
                use_m = wm >= wp;
                use_p = !use_m;
            }
            c0[a] = use_m ? j - 1 : j;
            l0[a] = use_m ? lm : lj;
            r0[a] = use_m ? rm : rj;
            c1[a] = use_m ? j : j + 1;
            l1[a] = use_m ? lj : lp;
            r1[a] = use_m ? rj : rp;
            cnt[a] = (use_m || use_p) ? 2 : 1;
        }
    }
    unsigned mask = 0u;
#pragma unroll
    for (int c = 0; c < (1 << D); ++c) {
        int idx = 0, mul = 1;
        float w = 1.f;
        bool ok = inside;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const bool up = (c >> a) & 1;
            ok = ok && (!up || cnt[a] == 2);
            w = w * (up ? l1[a] : l0[a]) * (up ? r1[a] : r0[a]);
            idx += (up ? c1[a] : c0[a]) * mul;
            mul *= g.p[a];
        }
        ok = ok && w > 0.f;
        s[c] = ok ? idx : 0;
        psi[c] = ok ? w : 0.f;
        mask |= ok ? (1u << c) : 0u;
    }
    return mask;
}

__device__ __forceinline__ void load_point(const Geo &g, const double *pts, int64_t p, double x[3]) {
    x[0] = x[1] = x[2] = 0.0;
    for (int a = 0; a < g.dim; ++a) x[a] = pts[p * g.dim + a];
}

template <int D, bool F32W>
__global__ void k_glue_count(Geo g, double delta, const double *pts, int64_t n, int32_t *rank,
                             int32_t *count, double *out, GlueWs e) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int s[8];
    double psi[8];
    float psf[8];
    unsigned mask = 0u;
    if (p < n) {
        double x[3];
        load_point(g, pts, p, x);
        if (F32W)
            mask = glue_pairs_f<D>(g, (float)(delta * (double)g.nmax), x, s, psf);
        else
            mask = glue_pairs<D>(g, delta, x, s, psi);
        if (mask == 0u) out[p] = nan("");
        e.mask[p] = (uint8_t)mask;
    }
    constexpr int nslot = 1 << D;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < nslot; ++c) {  // uniform across the warp
        const bool have = (mask >> c) & 1u;
        const int key = have ? s[c] : -2;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (lane == leader && have) base = atomicAdd(&count[key], __popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (have) {
            rank[p * nslot + c] = base + __popc(peers & ((1u << lane) - 1u));
            e.sub[p * nslot + c] = key;
            if (F32W) e.psif[p * nslot + c] = psf[c];
            else e.psi[p * nslot + c] = psi[c];
        }
    }
}

template <int D>
__global__ void k_glue_scatter(int64_t n, const int32_t *start, GlueWs e) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const unsigned mask = e.mask[p];
    constexpr int nslot = 1 << D;
#pragma unroll
    for (int c = 0; c < nslot; ++c)
        if ((mask >> c) & 1u) {
            const int64_t slot = p * nslot + c;
            e.perm[start[e.sub[slot]] + e.rank[slot]] = (int32_t)slot;
        }
}

__global__ void k_glue_bucket_f64(Geo g, const double *centres, const double *beta, const int32_t *info,
                                  const double *pts, const int32_t *perm, const int32_t *start, double *val) {
    const int s = blockIdx.x;
    const int b = start[s], e = start[s + 1];
    if (b == e) return;
    const int M = info[s * kInfoN + PAM_INFO_M];
    extern __shared__ uint8_t smb[];
    dvec4 *sc = reinterpret_cast<dvec4 *>(smb);
    double *sb = reinterpret_cast<double *>(sc + g.m_cap);
    stage_f64(g, centres, beta, s, M, sc, sb);
    for (int i = b + threadIdx.x; i < e; i += blockDim.x) {
        const int slot = perm[i];
        double x[3];
        load_point(g, pts, (int64_t)(slot >> g.dim), x);
        val[slot] = shepard_f64_smem(sc, sb, M, x);
    }
}

__global__ void k_glue_bucket_f32(Geo g, const int32_t *boxes, const double *centres, const double *beta,
                                  const int32_t *info, const double *pts, const int32_t *perm,
                                  const int32_t *start, float *val) {
    const int s = blockIdx.x;
    const int b = start[s], e = start[s + 1];
    if (b == e) return;
    const int M = info[s * kInfoN + PAM_INFO_M];
    extern __shared__ uint8_t smb[];
    float4 *su = reinterpret_cast<float4 *>(smb);
    float2 *sb = reinterpret_cast<float2 *>(su + 2 * g.m_cap);
    double o[3];
    // the local evaluation of pam_eval's fp32 form, operation for operation
    stage_f32s(g, boxes, centres, beta, s, M, su, sb, o);
    const int bd = blockDim.x;
    for (int i = b + threadIdx.x; i < e; i += kEvalPts * bd) {
        int qi[kEvalPts];
        float x[kEvalPts][3];
#pragma unroll
        for (int k = 0; k < kEvalPts; ++k) {
            qi[k] = i + k * bd < e ? perm[i + k * bd] : -1;
            const int64_t p = (int64_t)(qi[k] >= 0 ? qi[k] : perm[i]) >> g.dim;
#pragma unroll
            for (int a = 0; a < 3; ++a) x[k][a] = a < g.dim ? (float)(pts[p * g.dim + a] - o[a]) : 0.f;
        }
        float v[kEvalPts];
        shepard_f32s<kEvalPts>(su, sb, M, x, v);
#pragma unroll
        for (int k = 0; k < kEvalPts; ++k)
            if (qi[k] >= 0) val[qi[k]] = v[k];
    }
}

template <int D, bool F32>
__global__ void k_glue_combine(int64_t n, GlueWs e, double *out, int log_space) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const unsigned mask = e.mask[p];
    if (mask == 0u) return;  // NaN written by k_glue_count
    constexpr int nslot = 1 << D;
    if (F32) {  // the fp32 form blends in fp32 (its local surrogates are fp32)
        float num = 0.f, den = 0.f;
#pragma unroll
        for (int c = 0; c < nslot; ++c)
            if ((mask >> c) & 1u) {
                const float w = e.psif[p * nslot + c];
                num = fmaf(w, e.valf[p * nslot + c], num);
                den += w;
            }
        const float v = num / den;
        out[p] = log_space ? (double)v : exp_f32(v);
        return;
    }
    double num = 0.0, den = 0.0;
#pragma unroll
    for (int c = 0; c < nslot; ++c)
        if ((mask >> c) & 1u) {
            const double w = e.psi[p * nslot + c];
            num = __dadd_rn(num, __dmul_rn(w, e.val[p * nslot + c]));
            den = __dadd_rn(den, w);
        }
    const double v = num / den;
    out[p] = log_space ? v : exp(v);
}

template <int D>
static void glue_launches(const Geo &g, const int32_t *boxes, const double *centres, const double *beta,
                          const int32_t *info, const double *pts, int64_t n_pts, double delta, double *out,
                          int log_space, int precision, const GlueWs &e, cudaStream_t st) {
    const unsigned nb = (unsigned)((n_pts + 255) / 256);
    if (precision == PAM_PREC_MIXED)
        k_glue_count<D, true><<<nb, 256, 0, st>>>(g, delta, pts, n_pts, e.rank, e.count, out, e);
    else
        k_glue_count<D, false><<<nb, 256, 0, st>>>(g, delta, pts, n_pts, e.rank, e.count, out, e);
    k_eval_scan<<<1, 1024, 0, st>>>(e.count, e.start, g.S);
    k_glue_scatter<D><<<nb, 256, 0, st>>>(n_pts, e.start, e);
    if (precision == PAM_PREC_MIXED) {
        size_t sm = stage_f32s_smem(g.m_cap);
        cudaFuncSetAttribute(k_glue_bucket_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_glue_bucket_f32<<<g.S, eval_block(), sm, st>>>(g, boxes, centres, beta, info, pts, e.perm, e.start, e.valf);
        k_glue_combine<D, true><<<nb, 256, 0, st>>>(n_pts, e, out, log_space);
    } else {
        size_t sm = (size_t)g.m_cap * (sizeof(dvec4) + sizeof(double));
        cudaFuncSetAttribute(k_glue_bucket_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_glue_bucket_f64<<<g.S, eval_block(), sm, st>>>(g, centres, beta, info, pts, e.perm, e.start, e.val);
        k_glue_combine<D, false><<<nb, 256, 0, st>>>(n_pts, e, out, log_space);
    }
}

void launch_eval_glued(const Geo &g, const int32_t *boxes, const double *centres, const double *beta,
                       const int32_t *info, const double *pts, int64_t n_pts, double band, double *out,
                       int log_space, int precision, void *ws, cudaStream_t st) {
    PhaseScope ps(kPhEval, st);
    GlueWs e = carve_glue_workspace(g.S, g.dim, n_pts, ws);
    const double delta = band * g.h;
    cudaMemsetAsync(e.count, 0, (size_t)g.S * sizeof(int32_t), st);
    if (g.dim == 1)
        glue_launches<1>(g, boxes, centres, beta, info, pts, n_pts, delta, out, log_space, precision, e, st);
    else if (g.dim == 2)
        glue_launches<2>(g, boxes, centres, beta, info, pts, n_pts, delta, out, log_space, precision, e, st);
    else
        glue_launches<3>(g, boxes, centres, beta, info, pts, n_pts, delta, out, log_space, precision, e, st);
    count_launches(5);
}

// --------------------------------------------------------------------------
// Errors over the source cells: one block per owner sweeps its core cells
// (each cell measured with its owner's surrogate at the centroid) and writes
// seven fp64 partial sums; one thread combines the S rows in order.
// --------------------------------------------------------------------------
constexpr int kErrThreads = 256;

// The fp32 form's error sums: the surrogate as pam_eval evaluates it (the
// scaled logit, points in pairs through the packed arithmetic), at the
// cells' nodes taken two at a time -- two cells' centroids, or two
// Gauss-Legendre nodes of one cell -- with ln K in fp32 (the surrogate
// carries fp32 rounding already) and the sums in binary64.
__global__ void __launch_bounds__(kErrThreads) k_errors_owner_f32(Geo g, const int32_t *boxes,
                                                                  const double *centres, const double *beta,
                                                                  const int32_t *info, const double *K, int quad,
                                                                  double *part) {
    const int s = blockIdx.x;
    const int M = info[s * kInfoN + PAM_INFO_M];
    const int32_t *box = boxes + s * 12;
    extern __shared__ uint8_t smb[];
    float4 *su = reinterpret_cast<float4 *>(smb);
    float2 *sb = reinterpret_cast<float2 *>(su + 2 * g.m_cap);
    double o[3];
    stage_f32s(g, boxes, centres, beta, s, M, su, sb, o);
    const int w0 = box[3] - box[0], w1 = box[4] - box[1], w2 = box[5] - box[2];
    const int nq = quad ? (1 << g.dim) : 1;
    const int64_t items = (int64_t)w0 * w1 * w2 * nq;  // (cell, node) pairs, node fastest
    const double off = __dmul_rn(0.5, g.h) / sqrt(3.0), wq = 1.0 / (double)nq;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int64_t pr = threadIdx.x; 2 * pr < items; pr += blockDim.x) {
        float p[2][3];
        double kk[2];
        bool live[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t it = 2 * pr + h < items ? 2 * pr + h : 2 * pr;  // an idle half repeats the first
            live[h] = 2 * pr + h < items;
            const int t = (int)(it / nq), q = (int)(it % nq);
            const int i = box[0] + t % w0, j = box[1] + (t / w0) % w1, k = box[2] + t / (w0 * w1);
            const int idx[3] = {i, j, k};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                double x = 0.0;
                if (a < g.dim) {
                    x = __dmul_rn((double)idx[a] + 0.5, g.h);
                    if (quad) x = __dadd_rn(x, ((q >> a) & 1) ? off : -off);
                }
                p[h][a] = a < g.dim ? (float)(x - o[a]) : 0.f;
            }
            kk[h] = K[(int64_t)i + (int64_t)g.n[0] * ((int64_t)j + (int64_t)g.n[1] * k)];
            if (live[h] && q == 0) {  // the cell's own terms, once
                acc[1] += fabs(kk[h]);
                acc[3] += kk[h] * kk[h];
                acc[5] += fabs((double)logf((float)kk[h]));
            }
        }
        float v[2];
        shepard_f32s<2>(su, sb, M, p, v);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (!live[h]) continue;
            const double lk = (double)logf((float)kk[h]), ks = exp_f32(v[h]);
            acc[0] += wq * fabs(kk[h] - ks);
            acc[2] += wq * ((kk[h] - ks) * (kk[h] - ks));
            acc[4] += wq * fabs(lk - (double)v[h]);
            acc[6] = fmax(acc[6], fabs(lk - (double)v[h]));
        }
    }
    __shared__ double red[kErrThreads / 32][7];
    for (int q = 0; q < 7; ++q) {
        const double val = (q == 6) ? warp_max(acc[q]) : warp_sum(acc[q]);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][q] = val;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        const int q = threadIdx.x;
        double val = 0.0;
        if (q < 7)
            for (int wdx = 0; wdx < kErrThreads / 32; ++wdx)
                val = (q == 6) ? fmax(val, red[wdx][q]) : val + red[wdx][q];
        part[(size_t)s * 8 + q] = val;
    }
}

__global__ void __launch_bounds__(kErrThreads) k_errors_owner_f64(Geo g, const int32_t *boxes,
                                                              const double *centres,
                                                              const double *beta,
                                                              const int32_t *info, const double *K,
                                                              int quad, double *part) {
    const int s = blockIdx.x;
    const int M = info[s * kInfoN + PAM_INFO_M];
    const int32_t *box = boxes + s * 12;
    extern __shared__ uint8_t smb[];
    dvec4 *sc64 = reinterpret_cast<dvec4 *>(smb);
    double *sb64 = reinterpret_cast<double *>(sc64 + g.m_cap);
    stage_f64(g, centres, beta, s, M, sc64, sb64);
    const int w0 = box[3] - box[0], w1 = box[4] - box[1], w2 = box[5] - box[2];
    const int cnt = w0 * w1 * w2;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    // the cell's nodes: its centroid, or the 2^dim Gauss-Legendre nodes
    // (weight 1/nq of the cell each); all of them lie inside the cell
    const int nq = quad ? (1 << g.dim) : 1;
    const double off = __dmul_rn(0.5, g.h) / sqrt(3.0), wq = 1.0 / (double)nq;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        const int i = box[0] + t % w0, j = box[1] + (t / w0) % w1, k = box[2] + t / (w0 * w1);
        const int idx[3] = {i, j, k};
        double xc[3] = {0, 0, 0};
        for (int a = 0; a < g.dim; ++a) xc[a] = __dmul_rn((double)idx[a] + 0.5, g.h);
        const int64_t gi = (int64_t)i + (int64_t)g.n[0] * ((int64_t)j + (int64_t)g.n[1] * k);
        const double kk = K[gi], lk = log(kk);
        acc[1] += fabs(kk);
        acc[3] += kk * kk;
        acc[5] += fabs(lk);
        for (int q = 0; q < nq; ++q) {
            double x[3] = {xc[0], xc[1], xc[2]};
            if (quad)
                for (int a = 0; a < g.dim; ++a) x[a] = __dadd_rn(xc[a], ((q >> a) & 1) ? off : -off);
            const double v = shepard_f64_smem(sc64, sb64, M, x);
            const double ks = exp(v);
            acc[0] += wq * fabs(kk - ks);
            acc[2] += wq * ((kk - ks) * (kk - ks));
            acc[4] += wq * fabs(lk - v);
            acc[6] = fmax(acc[6], fabs(lk - v));
        }
    }
    __shared__ double red[kErrThreads / 32][7];
    for (int q = 0; q < 7; ++q) {
        const double v = (q == 6) ? warp_max(acc[q]) : warp_sum(acc[q]);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        const int q = threadIdx.x;
        double v = 0.0;
        if (q < 7)
            for (int wdx = 0; wdx < kErrThreads / 32; ++wdx)
                v = (q == 6) ? fmax(v, red[wdx][q]) : v + red[wdx][q];
        part[(size_t)s * 8 + q] = v;
    }
}

// Sums the per-owner rows in a fixed order: thread t adds the contiguous
// rows [t*per, (t+1)*per) in order, then a fixed tree over the threads.
// raw = 1: err[0..6] receive the seven sums themselves (err[7] = 0), for a
// caller that adds them up over several shards before forming the ratios.
__global__ void __launch_bounds__(256) k_errors_combine(const double *part, int rows, double *err, int raw) {
    __shared__ double red[7][256];
    const int t = threadIdx.x;
    const int per = (rows + 255) / 256;
    double a[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int r = t * per; r < min(rows, (t + 1) * per); ++r)
        for (int q = 0; q < 7; ++q)
            a[q] = (q == 6) ? fmax(a[q], part[(size_t)r * 8 + q]) : a[q] + part[(size_t)r * 8 + q];
    for (int q = 0; q < 7; ++q) red[q][t] = a[q];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (t < o)
            for (int q = 0; q < 7; ++q)
                red[q][t] = (q == 6) ? fmax(red[q][t], red[q][t + o]) : red[q][t] + red[q][t + o];
        __syncthreads();
    }
    if (t == 0 && raw) {
        for (int q = 0; q < 7; ++q) err[q] = red[q][0];
        err[7] = 0.0;
    } else if (t == 0) {
        err[0] = red[0][0] / red[1][0];
        err[1] = sqrt(red[2][0] / red[3][0]);
        err[2] = red[5][0] > 0.0 ? red[4][0] / red[5][0] : red[4][0];
        err[3] = red[6][0] / log(10.0);
    }
}

void launch_errors(const Geo &g, const int32_t *boxes, const double *centres, const double *beta,
                   const int32_t *info, const double *K, double *err, int precision, int quad,
                   const Ws &w, cudaStream_t st, int row0, int row1) {
    PhaseScope ps(kPhErrors, st);
    if (precision == PAM_PREC_MIXED) {
        size_t sm = stage_f32s_smem(g.m_cap);
        cudaFuncSetAttribute(k_errors_owner_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_errors_owner_f32<<<g.S, kErrThreads, sm, st>>>(g, boxes, centres, beta, info, K, quad, w.err_part);
    } else {
        size_t sm = (size_t)g.m_cap * (sizeof(dvec4) + sizeof(double));
        cudaFuncSetAttribute(k_errors_owner_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_errors_owner_f64<<<g.S, kErrThreads, sm, st>>>(g, boxes, centres, beta, info, K, quad, w.err_part);
    }
    if (row1 < 0)  // the ratios over every subdomain
        k_errors_combine<<<1, 256, 0, st>>>(w.err_part, g.S, err, 0);
    else           // the raw sums over the subdomains [row0, row1)
        k_errors_combine<<<1, 256, 0, st>>>(w.err_part + (size_t)row0 * 8, row1 - row0, err, 1);
    count_launches(2);
}

// --------------------------------------------------------------------------
// Errors over the elements of a mesh given as cells: one block per
// subdomain sweeps its patch list and measures the elements whose sampling
// point it owns (Step 4 owner rule; every element has exactly one owner and
// lies in its owner's patch), weighted by |T|; the same seven fp64 partial
// sums and combine as the grid errors.
// --------------------------------------------------------------------------
template <bool F32>
__global__ void __launch_bounds__(kErrThreads) k_errors_cells(Geo g, const int32_t *boxes,
                                                              const double *centres, const double *beta,
                                                              const int32_t *info, const double *K,
                                                              double *part) {
    const int s = blockIdx.x;
    const int M = info[s * kInfoN + PAM_INFO_M];
    extern __shared__ uint8_t smb[];
    dvec4 *sc64 = reinterpret_cast<dvec4 *>(smb);
    double *sb64 = reinterpret_cast<double *>(sc64 + g.m_cap);
    float4 *sc32 = reinterpret_cast<float4 *>(smb);
    float *sb32 = reinterpret_cast<float *>(sc32 + g.m_cap);
    double o[3];
    if (F32) stage_f32(g, boxes, centres, beta, s, M, sc32, sb32, o);
    else stage_f64(g, centres, beta, s, M, sc64, sb64);
    const int b = g.pstart[s], N = g.pstart[s + 1] - b;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
        const int64_t e = g.pcells[b + t];
        double x[3] = {0, 0, 0};
        for (int a = 0; a < g.dim; ++a) x[a] = g.cx[e * g.dim + a];
        if (owner_of_point(g, x) != s) continue;
        const double kk = K[e], vol = g.cvol[e], lk = log(kk);
        acc[1] += vol * fabs(kk);
        acc[3] += vol * (kk * kk);
        acc[5] += vol * fabs(lk);
        double v;
        if (F32)
            v = (double)shepard_f32_smem(sc32, sb32, M, (float)(x[0] - o[0]), (float)(x[1] - o[1]),
                                         (float)(x[2] - o[2]));
        else
            v = shepard_f64_smem(sc64, sb64, M, x);
        const double ks = F32 ? exp_f32((float)v) : exp(v);
        acc[0] += vol * fabs(kk - ks);
        acc[2] += vol * ((kk - ks) * (kk - ks));
        acc[4] += vol * fabs(lk - v);
        acc[6] = fmax(acc[6], fabs(lk - v));
    }
    __shared__ double red[kErrThreads / 32][7];
    for (int q = 0; q < 7; ++q) {
        const double v = (q == 6) ? warp_max(acc[q]) : warp_sum(acc[q]);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        const int q = threadIdx.x;
        double v = 0.0;
        if (q < 7)
            for (int wdx = 0; wdx < kErrThreads / 32; ++wdx)
                v = (q == 6) ? fmax(v, red[wdx][q]) : v + red[wdx][q];
        part[(size_t)s * 8 + q] = v;
    }
}

void launch_errors_cells(const Geo &g, const int32_t *boxes, const double *centres, const double *beta,
                         const int32_t *info, const double *K, double *err, int precision, const Ws &w,
                         cudaStream_t st) {
    PhaseScope ps(kPhErrors, st);
    if (precision == PAM_PREC_MIXED) {
        size_t sm = stage_f32_smem(g.m_cap);
        cudaFuncSetAttribute(k_errors_cells<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_errors_cells<true><<<g.S, kErrThreads, sm, st>>>(g, boxes, centres, beta, info, K, w.err_part);
    } else {
        size_t sm = (size_t)g.m_cap * (sizeof(dvec4) + sizeof(double));
        cudaFuncSetAttribute(k_errors_cells<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_errors_cells<false><<<g.S, kErrThreads, sm, st>>>(g, boxes, centres, beta, info, K, w.err_part);
    }
    k_errors_combine<<<1, 256, 0, st>>>(w.err_part, g.S, err, 0);
    count_launches(2);
}

// --------------------------------------------------------------------------
// Indicators R_T (Eq. (4)) with the tensor two-point Gauss-Legendre rule:
// R_T = sum_q (|T| / 2^dim) (K*(x_q) - K_T)^2 over the nodes x_T +- h/(2
// sqrt 3) per axis, K* from the subdomain's whole dictionary at each node
// (Shepard weights, max-shifted). One block per running subdomain, a thread
// per patch cell (patch order, x fastest). The fp32 form evaluates as
// pam_eval does (the scaled logit, origin at the patch centre), four nodes
// of a cell per pass through the centres in two packed pairs; the sum keeps
// the node order in both forms.
// --------------------------------------------------------------------------
template <bool F32>
__global__ void __launch_bounds__(256) k_residual_quad(Geo g, const int32_t *boxes, const double *centres,
                                                       const double *beta, const int32_t *info, Ws w) {
    const int s = group_sub(g, blockIdx.x);
    const int32_t *inf = info + s * kInfoN;
    if (inf[PAM_INFO_STOPPED]) return;
    const int M = inf[PAM_INFO_M], N = inf[PAM_INFO_N_CELLS];
    const int32_t *box = boxes + s * 12;
    extern __shared__ uint8_t smb[];
    dvec4 *sc64 = reinterpret_cast<dvec4 *>(smb);
    double *sb64 = reinterpret_cast<double *>(sc64 + g.m_cap);
    float4 *su = reinterpret_cast<float4 *>(smb);
    float2 *sb = reinterpret_cast<float2 *>(su + 2 * g.m_cap);
    double o[3];
    if (F32) stage_f32s(g, boxes, centres, beta, s, M, su, sb, o);
    else stage_f64(g, centres, beta, s, M, sc64, sb64);
    const int w0 = box[9] - box[6], w1 = box[10] - box[7];
    const int nq = 1 << g.dim;
    const double off = __dmul_rn(0.5, g.h) / sqrt(3.0), wq = g.vol / (double)nq;
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
        const int idx[3] = {box[6] + t % w0, box[7] + (t / w0) % w1, box[8] + t / (w0 * w1)};
        double xc[3] = {0, 0, 0};
        for (int a = 0; a < g.dim; ++a) xc[a] = __dmul_rn((double)idx[a] + 0.5, g.h);
        const double kv = w.kv[(size_t)s * g.n_max + t];
        double r = 0.0;
        if (F32) {
            // K*(x_q) - K_T = K_T expm1(v_q - ln K_T) in fp32 (the surrogate's
            // logit v_q carries fp32 rounding already): no binary64 exp per
            // node, whose cost on this part's narrow fp64 pipe rivals the
            // node's pass through the centres
            const double yl = w.y[(size_t)s * g.n_max + t];
            const double c = __dmul_rn(wq, __dmul_rn(kv, kv));
            // the cell centre in local coordinates, the nodes at +-off from it in fp32
            float pc[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) pc[a] = a < g.dim ? (float)(xc[a] - o[a]) : 0.f;
            const float offf = (float)off;
            for (int q0 = 0; q0 < nq; q0 += 4) {
                float p[4][3];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int q = q0 + k < nq ? q0 + k : q0;  // 1-D: two nodes, the idle pair repeats them
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        p[k][a] = a < g.dim ? pc[a] + (((q >> a) & 1) ? offf : -offf) : 0.f;
                }
                float v[4];
                shepard_f32s<4>(su, sb, M, p, v);
                for (int k = 0; k < 4 && q0 + k < nq; ++k) {
                    const float e = expm1f((float)__dsub_rn((double)v[k], yl));
                    r = __dadd_rn(r, __dmul_rn(c, (double)(e * e)));
                }
            }
        } else {
            for (int q = 0; q < nq; q += 2) {
                double x0[3] = {0, 0, 0}, x1[3] = {0, 0, 0};
                for (int a = 0; a < g.dim; ++a) {
                    x0[a] = __dadd_rn(xc[a], ((q >> a) & 1) ? off : -off);
                    x1[a] = __dadd_rn(xc[a], (((q + 1) >> a) & 1) ? off : -off);
                }
                const double v0 = shepard_f64_smem(sc64, sb64, M, x0), v1 = shepard_f64_smem(sc64, sb64, M, x1);
                const double e0 = __dsub_rn(exp(v0), kv), e1 = __dsub_rn(exp(v1), kv);
                r = __dadd_rn(r, __dmul_rn(wq, __dmul_rn(e0, e0)));
                r = __dadd_rn(r, __dmul_rn(wq, __dmul_rn(e1, e1)));
            }
        }
        w.R[(size_t)s * g.n_max + t] = r;
    }
}

void launch_residual_quad(const Geo &g, int precision, const int32_t *boxes, const double *centres,
                          const double *beta, const int32_t *info, const Ws &w, cudaStream_t st) {
    PhaseScope ps(kPhResidual, st);
    if (precision == PAM_PREC_MIXED) {
        size_t sm = stage_f32s_smem(g.m_cap);
        cudaFuncSetAttribute(k_residual_quad<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_residual_quad<true><<<group_count(g), 256, sm, st>>>(g, boxes, centres, beta, info, w);
    } else {
        size_t sm = (size_t)g.m_cap * (sizeof(dvec4) + sizeof(double));
        cudaFuncSetAttribute(k_residual_quad<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_residual_quad<false><<<group_count(g), 256, sm, st>>>(g, boxes, centres, beta, info, w);
    }
    count_launches(1);
}

}  // namespace pam
