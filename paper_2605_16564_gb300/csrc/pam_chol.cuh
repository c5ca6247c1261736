// pam_chol.cuh -- dense fp32 kernels of the mixed-form Elastic Net solve
// (Eq. (2) restricted to a support S): the blocked Cholesky factorisation
// of the packed support matrix (G~_SS + lambda2 I) and the triangular
// solves with its factor, each run by one whole thread block. Internal to
// libpam.
//
// Layout: a packed lower-triangular s x s matrix, row-major over the lower
// triangle, A[tri_i(p, q)] for q <= p (shared memory, or global memory for
// supports whose factor exceeds the shared-memory budget).
#pragma once

#include <stdint.h>

#include "pam_tc.cuh"

namespace pam {

__device__ __forceinline__ int tri_i(int p, int q) { return p * (p + 1) / 2 + q; }

#ifdef PAM_SOLVE_PROFILE
// Profiling builds only: clock64 totals per phase of the mixed solve.
__device__ unsigned long long g_solve_prof[16];
__device__ unsigned long long g_solve_blk[8192];
__device__ unsigned long long g_solve_cnt[8];  // factorisations, sum s, sum s^3
#define PROF_CNT(k, v) do { if (threadIdx.x == 0) atomicAdd(&g_solve_cnt[k], (unsigned long long)(v)); } while (0)
#define PROF_T0() long long _pt = clock64()
#define PROF_MARK(k)                                                          \
    do {                                                                      \
        if (threadIdx.x == 0) atomicAdd(&g_solve_prof[k], (unsigned long long)(clock64() - _pt)); \
        _pt = clock64();                                                      \
    } while (0)
#else
#define PROF_CNT(k, v)
#define PROF_T0()
#define PROF_MARK(k)
#endif

// Shared-memory scratch of the factorisation: the current 32 x 32 diagonal
// block's factor, transposed (Lt[q][j] = L[k0 + j][k0 + q] for j > q, zero
// for j <= q), 16-byte aligned, so that the panel rows read a column of it
// as eight float4 broadcasts.
constexpr int kCholLtFloats = 32 * 32;

// Blocked right-looking Cholesky of the packed lower s x s matrix A, in
// place, with blocks of 32 columns. Per block: warp 0 factors the 32 x 32
// diagonal block in registers (lane i holds row i, fully unrolled so every
// index is static; rows past the end of a partial block are padded with the
// identity), broadcasting each scaled column through Lt, which then holds
// the block's factor transposed; every other row of the block
// column (the panel) is solved against it by one thread, column by column
// from registers (a chain of 32 multiply-adds, its column of L read as
// float4 broadcasts from Lt); then the trailing triangle is updated in 4 x 4
// register tiles, one per thread (sixteen multiply-adds per eight loads).
// Three block barriers per 32 columns. dinv[k] receives 1 / L_kk for the
// triangular solves; *flag = 1 if a pivot is not positive.
__device__ __forceinline__ void mx_diag_block(float *A, int k0, int kw, int *flag, float *dinv, float *Lt) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, i = k0 + lane;
    const bool live = lane < kw;
    float a[32];
#pragma unroll
    for (int j = 0; j < 32; ++j)
        a[j] = (live && j <= lane) ? A[tri_i(i, k0 + j)] : (j == lane ? 1.f : 0.f);
    float my_iv = 1.f;
    bool bad = false;
    const float4 *L4 = reinterpret_cast<const float4 *>(Lt);
    // dn: lane k's pivot a_kk after the updates of columns < k, computed by
    // lane k itself one step early, so that the column chain is
    // shfl -> rsqrt -> fmul -> fma; the scaled column k goes to row k of Lt
    // (which it keeps: Lt is the block's factor transposed) and every lane
    // reads it back as float4 broadcasts for its update, off the chain
    float dn = a[0];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        float d = __shfl_sync(full, dn, k);
        if (!(d > 0.f)) { bad = true; d = 1.f; }
        const float iv = rsqrtf(d);
        if (lane == k) { a[k] = d * iv; my_iv = iv; }
        else a[k] *= iv;  // above the diagonal (lane < k) the value is never used
        Lt[k * 32 + lane] = lane > k ? a[k] : 0.f;
        if (k + 1 < 32) dn = fmaf(-a[k], a[k], a[k + 1]);  // meaningful in lane k + 1
        __syncwarp();
#pragma unroll
        for (int g = (k + 1) >> 2; g < 8; ++g) {
            const float4 l = L4[k * 8 + g];
            if (4 * g + 0 > k) a[4 * g + 0] = fmaf(-a[k], l.x, a[4 * g + 0]);
            if (4 * g + 1 > k) a[4 * g + 1] = fmaf(-a[k], l.y, a[4 * g + 1]);
            if (4 * g + 2 > k) a[4 * g + 2] = fmaf(-a[k], l.z, a[4 * g + 2]);
            if (4 * g + 3 > k) a[4 * g + 3] = fmaf(-a[k], l.w, a[4 * g + 3]);
        }
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

// Panel row i: L[i, k0:k0+32] = A[i, k0:k0+32] L_kk^{-T} (kw == 32 only: a
// partial block is the last one and has no rows below it), by columns:
// r_q <- r_q / L_qq, then r_j -= r_q L_jq for j > q.
__device__ __forceinline__ void mx_panel_row(float *A, int k0, int i, const float *dinv, const float *Lt) {
    float *ri = A + tri_i(i, 0) + k0;
    float r[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) r[j] = ri[j];
    const float4 *L4 = reinterpret_cast<const float4 *>(Lt);
#pragma unroll
    for (int q = 0; q < 32; ++q) {
        const float rq = r[q] * dinv[k0 + q];
        r[q] = rq;
#pragma unroll
        for (int g = (q + 1) >> 2; g < 8; ++g) {
            const float4 l = L4[q * 8 + g];
            if (4 * g + 0 > q) r[4 * g + 0] = fmaf(-rq, l.x, r[4 * g + 0]);
            if (4 * g + 1 > q) r[4 * g + 1] = fmaf(-rq, l.y, r[4 * g + 1]);
            if (4 * g + 2 > q) r[4 * g + 2] = fmaf(-rq, l.z, r[4 * g + 2]);
            if (4 * g + 3 > q) r[4 * g + 3] = fmaf(-rq, l.w, r[4 * g + 3]);
        }
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) ri[j] = r[j];
}

// Trailing update after block column k0: A[i][j] -= sum_q L[i][k0+q] L[j][k0+q]
// for k0 + 32 <= j <= i < s, one 4 x 4 tile of (i, j) per thread. Tile rows
// past s read row s - 1 (their sums are discarded).
__device__ __forceinline__ void mx_trailing(float *A, int k0, int s) {
    const int c0 = k0 + 32, n = s - c0;
    const int nt = (n + 3) >> 2;
    const int ntile = nt * (nt + 1) / 2;
    for (int e = threadIdx.x; e < ntile; e += blockDim.x) {
        int ti = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
        if (tri_i(ti + 1, 0) <= e) ++ti;
        if (tri_i(ti, 0) > e) --ti;
        const int tj = e - tri_i(ti, 0);
        const int i0 = c0 + 4 * ti, j0 = c0 + 4 * tj;
        int oa[4], ob[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            oa[u] = tri_i(min(i0 + u, s - 1), 0) + k0;
            ob[u] = tri_i(min(j0 + u, s - 1), 0) + k0;
        }
        float acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
#pragma unroll 8
        for (int q = 0; q < 32; ++q) {
            float a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = A[oa[u] + q];
                b[u] = A[ob[u] + q];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int ii = i0 + u;
            if (ii >= s) break;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int jj = j0 + v;
                if (jj <= ii) A[tri_i(ii, jj)] -= acc[u][v];
            }
        }
    }
}

__device__ __noinline__ void mx_cholesky(float *A, int s, int *flag, float *dinv, float *Lt) {
    const int tid = threadIdx.x, warp = tid >> 5;
    PROF_T0();
    PROF_CNT(0, 1);
    PROF_CNT(1, s);
    PROF_CNT(2, (long long)s * s * s);
    for (int k0 = 0; k0 < s; k0 += 32) {
        const int kw = min(32, s - k0);
        if (warp == 0) mx_diag_block(A, k0, kw, flag, dinv, Lt);
        __syncthreads();
        PROF_MARK(12);
        if (k0 + kw >= s) break;  // last block: nothing below it
        for (int i = k0 + kw + tid; i < s; i += blockDim.x) mx_panel_row(A, k0, i, dinv, Lt);
        __syncthreads();
        PROF_MARK(13);
        mx_trailing(A, k0, s);
        __syncthreads();
        PROF_MARK(14);
    }
}

// Solves L L^T z = r in place (packed L from mx_cholesky, dinv = 1/diag):
// per 32-row block, warp 0 solves the diagonal block with shuffles (fully
// unrolled; the matrix loads do not depend on the recurrence) and all
// threads apply the block's contribution to the remaining entries.
__device__ void mx_chol_backward(const float *A, const float *dinv, int s, float *r);

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
    mx_chol_backward(A, dinv, s, r);
}

// Backward half: L^T x = z in place.
__device__ void mx_chol_backward(const float *A, const float *dinv, int s, float *r) {
    const unsigned full = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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

}  // namespace pam
