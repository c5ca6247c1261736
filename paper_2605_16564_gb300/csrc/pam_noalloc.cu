// pam_noalloc.cu -- pam_errors_noalloc: the error reduction of pam_errors
// without any caller workspace and without allocating device memory.
//
// Who needs it: host programs that own all device memory themselves and do
// not let a library allocate -- e.g. a reservoir or flow simulator that
// reserves the GPU's memory in its own pool at start-up, or a real-time
// loop in which a cudaMalloc (its latency, or its failure half-way through a
// time step) is not acceptable. Such callers can pass inputs and outputs
// but cannot provide, or let us obtain, scratch space.
//
// How: the per-block partial sums live in a file-scope __device__ array of
// fixed size (kNaMaxBlocks rows of 8 doubles = 256 KiB), which every GPU
// that loads this library holds until the process exits. Each block reduces
// a fixed chunk of kNaCellsPerBlock grid cells, so grids of more than
// kNaMaxBlocks * kNaCellsPerBlock = 16,777,216 cells are rejected.
#include <cmath>
#include <mutex>

#include <cuda.h>  // CUcontext and CUresult only; the call is resolved through the runtime

#include "pam_internal.cuh"

namespace pam {
namespace {

constexpr int kNaCellsPerBlock = 4096;
constexpr int kNaMaxBlocks = 4096;
constexpr int kNaThreads = 256;
constexpr int kNaMaxDevices = 128;

// Partial sums, one row of 8 per block. Shared by every call on a device.
static __device__ __align__(256) double g_err_scratch[kNaMaxBlocks * 8];

std::mutex g_na_mu;
struct NaSlot {
    CUcontext ctx;
    double *addr;
};
NaSlot g_na_slot[kNaMaxDevices] = {};

// The current context of this thread (nullptr if none or unavailable):
// cuCtxGetCurrent, resolved once through the runtime so that the library
// needs no link against the driver library.
CUcontext current_context() {
    using Fn = CUresult (*)(CUcontext *);
    static Fn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<Fn>(p);
    }();
    CUcontext c = nullptr;
    if (fn && fn(&c) != CUDA_SUCCESS) c = nullptr;
    return c;
}

// Device address of g_err_scratch in the current context: host code cannot
// use the array's name as a device address. Looked up once per device, with
// that device current, and again only when the device's context is not the
// one of the lookup (after cudaDeviceReset the module is loaded anew and the
// old address is stale).
cudaError_t scratch_address(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_na_mu);
    NaSlot &sl = g_na_slot[dev];
    const CUcontext ctx = current_context();
    if (!sl.addr || !ctx || ctx != sl.ctx) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_err_scratch);  // makes the device's context current if needed
        if (e != cudaSuccess) return e;
        sl.addr = static_cast<double *>(p);
        sl.ctx = current_context();
    }
    *out = sl.addr;
    return cudaSuccess;
}

// sum_m beta_m w_m(x) over the dictionary of subdomain s (Shepard weights,
// maximum logit subtracted first), binary64. Each logit is formed exactly
// as pam_errors forms it from its staged dictionary, |x - c|^2 times the
// factor -1 / (2 sigma^2), so the two differ only in the order of the sums;
// the centres are read from global memory per cell (no shared-memory
// staging: a block's 4096 cells may span several subdomains), which makes
// this path several times slower than pam_errors on large dictionaries.
__device__ double na_shepard_value(const Geo &g, const double *centres, const double *beta, int s,
                                   int M, const double x[3]) {
    const dvec4 *cs = reinterpret_cast<const dvec4 *>(centres) + (size_t)s * g.m_cap;
    const double *bs = beta + (size_t)s * g.m_cap;
    double lmax = -INFINITY;
    for (int m = 0; m < M; ++m) {
        const dvec4 c = cs[m];
        const double f = -1.0 / (2.0 * c.w * c.w);
        const double d0 = x[0] - c.x, d1 = x[1] - c.y, d2 = x[2] - c.z;
        lmax = fmax(lmax, (d0 * d0 + d1 * d1 + d2 * d2) * f);
    }
    double num = 0.0, den = 0.0;
    for (int m = 0; m < M; ++m) {
        const dvec4 c = cs[m];
        const double f = -1.0 / (2.0 * c.w * c.w);
        const double d0 = x[0] - c.x, d1 = x[1] - c.y, d2 = x[2] - c.z;
        const double e = exp((d0 * d0 + d1 * d1 + d2 * d2) * f - lmax);
        num += bs[m] * e;
        den += e;
    }
    return num / den;
}

// Block b reduces grid cells [b * kNaCellsPerBlock, (b+1) * kNaCellsPerBlock)
// into row b of `part`: sum |K - K*|, sum |K|, sum (K - K*)^2, sum K^2,
// sum |ln K - ln K*|, sum |ln K|, max |ln K - ln K*|. Every entry of the row
// is written, so nothing has to be cleared between calls.
__global__ void __launch_bounds__(kNaThreads) k_err_chunk(Geo g, const double *centres,
                                                          const double *beta, const int32_t *info,
                                                          const double *K, int64_t total,
                                                          double *part) {
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    const int64_t base = (int64_t)blockIdx.x * kNaCellsPerBlock;
    for (int r = threadIdx.x; r < kNaCellsPerBlock; r += blockDim.x) {
        int64_t c = base + r;
        if (c >= total) break;
        int64_t i = c % g.n[0], j = (c / g.n[0]) % g.n[1], k = c / ((int64_t)g.n[0] * g.n[1]);
        int idx[3] = {(int)i, (int)j, (int)k};
        double x[3] = {0, 0, 0};
        int js[3] = {0, 0, 0};
        for (int a = 0; a < g.dim; ++a) {
            x[a] = __dmul_rn((double)idx[a] + 0.5, g.h);
            js[a] = core_of(idx[a], g.n[a], g.p[a]);
        }
        int s = js[0] + g.p[0] * (js[1] + g.p[1] * js[2]);
        int M = info[s * kInfoN + PAM_INFO_M];
        double v = na_shepard_value(g, centres, beta, s, M, x);
        double kk = K[c], ks = exp(v), lk = log(kk);
        acc[0] += fabs(kk - ks);
        acc[1] += fabs(kk);
        acc[2] += (kk - ks) * (kk - ks);
        acc[3] += kk * kk;
        acc[4] += fabs(lk - v);
        acc[5] += fabs(lk);
        acc[6] = fmax(acc[6], fabs(lk - v));
    }
    __shared__ double red[kNaThreads / 32][7];
    for (int q = 0; q < 7; ++q) {
        double v = (q == 6) ? warp_max(acc[q]) : warp_sum(acc[q]);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        int q = threadIdx.x;
        double v = 0.0;
        if (q < 7)
            for (int w = 0; w < kNaThreads / 32; ++w) v = (q == 6) ? fmax(v, red[w][q]) : v + red[w][q];
        part[(size_t)blockIdx.x * 8 + q] = v;
    }
}

__global__ void k_err_combine(const double *part, int nblocks, double *err) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int b = 0; b < nblocks; ++b)
        for (int q = 0; q < 7; ++q)
            a[q] = (q == 6) ? fmax(a[q], part[(size_t)b * 8 + q]) : a[q] + part[(size_t)b * 8 + q];
    err[0] = a[0] / a[1];
    err[1] = sqrt(a[2] / a[3]);
    err[2] = a[5] > 0.0 ? a[4] / a[5] : a[4];
    err[3] = a[6] / log(10.0);
}

}  // namespace
}  // namespace pam

using namespace pam;

extern "C" pam_status pam_errors_noalloc(const pam_problem *prob, const pam_plan *plan,
                                         const pam_model *model, const double *d_K, double *d_err,
                                         void *stream) {
    Geo g;
    pam_status st;
    if (!make_geo(prob, nullptr, &g, nullptr, &st)) return st;
    if (!plan || plan->n_subdomains != g.S || plan->m_cap > PAM_MAX_M || plan->m_cap < 1)
        return PAM_ERR_INVALID_ARG;
    g.m_cap = plan->m_cap;
    g.n_max = plan->max_patch_cells;
    if (!model || !model->boxes || !model->centres || !model->beta || !model->info || !d_K || !d_err)
        return PAM_ERR_INVALID_ARG;
    const int64_t total = (int64_t)g.n[0] * g.n[1] * g.n[2];
    if (total > (int64_t)kNaMaxBlocks * kNaCellsPerBlock) return PAM_ERR_UNSUPPORTED;
    double *scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return PAM_ERR_CUDA;
    const int nb = (int)((total + kNaCellsPerBlock - 1) / kNaCellsPerBlock);
    cudaStream_t s = (cudaStream_t)stream;
    k_err_chunk<<<nb, kNaThreads, 0, s>>>(g, model->centres, model->beta, model->info, d_K, total,
                                          scratch);
    k_err_combine<<<1, 32, 0, s>>>(scratch, nb, d_err);
    count_launches(2);
    if (cudaGetLastError() != cudaSuccess) return PAM_ERR_CUDA;
    return PAM_OK;
}
