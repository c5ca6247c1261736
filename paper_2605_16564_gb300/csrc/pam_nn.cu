// pam_nn.cu -- the learned warm start: a small convolutional network that
// maps a subdomain patch of log10 K to a predicted support (logits) and
// initial coefficients of the patch's initial dictionary. Two
// architectures share the code:
//   PAM_NN_PATCH2D   x [B,32,32,1] (a 32 x 32 patch), 256 outputs (16 x 16
//                    dictionary):
//     conv3x3 s2 (32) -> conv3x3 s2 (64) -> conv3x3 s2 (128) -> conv3x3 s1
//     (128) -> flatten 2048 -> dense 256 -> dense 512
//   PAM_NN_LAYERED3D x [B,16,16,8] (a 3-D patch up to 16 x 16 x 8 cells, its
//                    z layers as channels), 32 outputs (4 x 4 x 2 lattice):
//     conv3x3 s2 (32) -> conv3x3 s2 (64) -> conv3x3 s1 (64) -> conv3x3 s1
//     (64) -> flatten 1024 -> dense 128 -> dense 64
// with ReLU after every layer but the last; output = [n_out support logits
// | n_out beta / 4]. Forward and backward passes are hand-written: every
// contraction (the im2col convolutions and the dense layers, forward and
// backward) runs on the tcgen05 tensor cores in bf16 with fp32 accumulation
// (k_gemm_bf16); elementwise work, the loss and AdamW are small fp32
// kernels. The layer sequence is driven from host code in this file.
// Loss: mean BCE-with-logits on the support + mean squared error of the
// scaled coefficients.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>

#include "pam_internal.cuh"
#include "pam_tc.cuh"

namespace pam {
namespace nn {

using bf16 = __nv_bfloat16;

constexpr float kBetaScale = 4.f;

struct Conv {
    int hin, cin, hout, cout, stride, kpad;  // kpad = 9 cin rounded up to 32
};
struct Dense {
    int in, out;
};
constexpr int kNConv = 4;
struct Arch {
    int h0, c0;      // input: h0 x h0 pixels, c0 channels (NHWC)
    Conv conv[kNConv];
    int flat;        // the last convolution's output, flattened (NHWC)
    Dense dense[2];
    int nout;        // dictionary entries predicted; the output has 2 nout values
};
constexpr int kNArch = 2;
constexpr Arch kArch[kNArch] = {
    {32, 1, {{32, 1, 16, 32, 2, 32}, {16, 32, 8, 64, 2, 288}, {8, 64, 4, 128, 2, 576}, {4, 128, 4, 128, 1, 1152}},
     4 * 4 * 128, {{2048, 256}, {256, 512}}, 256},
    {16, 8, {{16, 8, 8, 32, 2, 96}, {8, 32, 4, 64, 2, 288}, {4, 64, 4, 64, 1, 576}, {4, 64, 4, 64, 1, 576}},
     4 * 4 * 64, {{1024, 128}, {128, 64}}, 32},
};

// Flat fp32 parameter layout: per layer W [out][k] then b [out].
struct Layout {
    int64_t w[6], b[6], total;
    int rows[6], cols[6];
};
static Layout layout(const Arch &A) {
    Layout L;
    int64_t off = 0;
    for (int l = 0; l < 6; ++l) {
        int rows = l < 4 ? A.conv[l].cout : A.dense[l - 4].out;
        int cols = l < 4 ? A.conv[l].kpad : A.dense[l - 4].in;
        L.rows[l] = rows;
        L.cols[l] = cols;
        L.w[l] = off;
        off += (int64_t)rows * cols;
        L.b[l] = off;
        off += rows;
    }
    L.total = off;
    return L;
}

// ------------------------------------------------------------------- GEMM --
// C[M x N] = A[M x K] B[N x K]^T (+ bias[N], optional ReLU), A and B bf16
// row-major with K contiguous (lda, ldb multiples of 8, K multiple of 32).
// One CTA per 128 x 128 tile of C: 256 threads stage 32-wide K chunks of A
// and B in the canonical K-major layout (two buffers), thread 0 issues the
// MMAs (M 128, N <= 128, K 16) into a 128-column TMEM accumulator, and the
// epilogue goes out through a shared-memory transpose (coalesced rows).
constexpr int kGT = 256;
constexpr long long kGemmWait = 4000000000LL;

// Implicit-convolution A operand (inference): with h > 0, A is the NHWC
// activation [B][h][h][c] of a 3x3 pad-1 convolution (c = 2^c_log2 >= 8) and
// row p, column k of the operand are those the im2col matrix would hold
// (tap = k / c, channel k mod c; zero past 9 c and outside the image), read
// 8 channels (16 bytes) at a time straight from the activation.
struct ImplicitConv {
    int h, c_log2, ho, stride;
};

__global__ void __launch_bounds__(kGT, 1) k_gemm_bf16(const bf16 *A, int lda, const bf16 *B, int ldb,
                                                      int M, int N, int K, float *C32, bf16 *C16,
                                                      int ldc, const float *bias, int relu,
                                                      int32_t *status, ImplicitConv ic) {
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * 128;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nt = min(128, ((N - n0) + 15) & ~15);  // MMA N of this tile
    extern __shared__ __align__(1024) uint8_t smem[];
    // [buf][A|B] tiles of 128 x 32 bf16 (8 KB each)
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int timed_out;
    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        tc::mbar_fence_init();
        timed_out = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, 128);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t lbo = 128u * 16u, sbo = 128u;
    const int nk = K / 32;
    int issued = 0;
    // 128 rows x 4 segments of 8 bf16 for A and for B: 1024 segments, four
    // per thread; the next chunk's segments are loaded into registers while
    // the current one is synchronised and multiplied
    constexpr int kSeg = 1024 / kGT;
    uint4 pre[kSeg];
    // implicit operand: this thread's A rows (u = 0, 1) as (image base, top-left input pixel)
    const bf16 *img[2] = {A, A};
    int iy0[2] = {0, 0}, ix0[2] = {0, 0};
    if (ic.h > 0) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int r = ((tid + u * kGT) & 511) >> 2;
            const int64_t pidx = (int64_t)m0 + r;
            const int ox = (int)(pidx % ic.ho), oy = (int)((pidx / ic.ho) % ic.ho);
            const int64_t b = pidx / ((int64_t)ic.ho * ic.ho);
            img[u] = A + (b * ic.h * ic.h << ic.c_log2);
            iy0[u] = oy * ic.stride - 1;
            ix0[u] = ox * ic.stride - 1;
        }
    }
    auto load_chunk = [&](int kc) {
#pragma unroll
        for (int u = 0; u < kSeg; ++u) {
            const int e = tid + u * kGT;
            const int isb = e >> 9, seg = e & 511, r = seg >> 2, kg = seg & 3;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (isb == 0) {
                if (m0 + r < M) {
                    if (ic.h > 0) {
                        const int k = kc * 32 + kg * 8, tap = k >> ic.c_log2;
                        if (tap < 9) {
                            const int ky = tap / 3, iy = iy0[u] + ky, ix = ix0[u] + (tap - 3 * ky);
                            if (iy >= 0 && iy < ic.h && ix >= 0 && ix < ic.h)
                                v = *reinterpret_cast<const uint4 *>(
                                    img[u] + (((int64_t)(iy * ic.h + ix) << ic.c_log2) + (k & ((1 << ic.c_log2) - 1))));
                        }
                    } else {
                        v = *reinterpret_cast<const uint4 *>(A + (size_t)(m0 + r) * lda + kc * 32 + kg * 8);
                    }
                }
            } else {
                if (n0 + r < N) v = *reinterpret_cast<const uint4 *>(B + (size_t)(n0 + r) * ldb + kc * 32 + kg * 8);
            }
            pre[u] = v;
        }
    };
    if (nk > 0) load_chunk(0);
    for (int kc = 0; kc < nk; ++kc) {
        const int buf = kc & 1;
        if (kc >= 2 && !tc::mbar_wait(&mbar[buf], ((kc - 2) >> 1) & 1, kGemmWait)) timed_out = 1;
        uint8_t *ta = smem + (size_t)buf * 16384;
        uint8_t *tb = ta + 8192;
#pragma unroll
        for (int u = 0; u < kSeg; ++u) {
            const int e = tid + u * kGT;
            const int isb = e >> 9, seg = e & 511, r = seg >> 2, kg = seg & 3;
            const uint32_t off = (uint32_t)(kg * 16 + (r >> 3)) * 128u + (uint32_t)(r & 7) * 16u;
            *reinterpret_cast<uint4 *>((isb ? tb : ta) + off) = pre[u];
        }
        if (kc + 1 < nk) load_chunk(kc + 1);
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (timed_out) break;
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t a = tc::smem_u32(ta), b = tc::smem_u32(tb);
            const uint32_t id = tc::idesc_bf16_f32((uint32_t)nt);
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                const uint32_t koff = (uint32_t)(2 * ks) * lbo;
                tc::mma_bf16(tmem, tc::smem_desc(a + koff, lbo, sbo), tc::smem_desc(b + koff, lbo, sbo), id,
                             (kc > 0 || ks > 0) ? 1u : 0u);
            }
            tc::mma_commit(&mbar[buf]);
        }
        issued = kc + 1;
    }
    if (!timed_out && nk > 0) {
        const int last = nk - 1;
        if (!tc::mbar_wait(&mbar[last & 1], (last >> 1) & 1, kGemmWait)) timed_out = 1;
    }
    __syncthreads();
    tc::fence_after_sync();
    if (timed_out) {
        if (issued > 0) tc::mbar_wait(&mbar[(issued - 1) & 1], ((issued - 1) >> 1) & 1, kGemmWait);
        if (tid == 0) atomicAdd(status, 1);
    } else {
        float *stage = reinterpret_cast<float *>(smem) + (size_t)warp * 32 * 33;
        const int lane_base = (warp & 3) * 32;
        for (int ch = warp >> 2; ch < nt / 32 + ((nt & 31) ? 1 : 0); ch += 2) {
            uint32_t v[32];
            tc::tmem_ld_32x32(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(ch * 32), v);
            tc::tmem_wait_ld();
#pragma unroll
            for (int q = 0; q < 32; ++q) stage[lane * 33 + q] = __uint_as_float(v[q]);
            __syncwarp();
            const int col = n0 + ch * 32 + lane;
            const float bv = (bias && col < N) ? bias[col] : 0.f;
            for (int q = 0; q < 32; ++q) {
                const int row = m0 + lane_base + q;
                if (row < M && col < N && ch * 32 + lane < nt) {
                    float o = stage[q * 33 + lane] + bv;
                    if (relu) o = fmaxf(o, 0.f);
                    if (C32) C32[(size_t)row * ldc + col] = o;
                    if (C16) C16[(size_t)row * ldc + col] = __float2bfloat16_rn(o);
                }
            }
            __syncwarp();
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

static void gemm(const bf16 *A, int lda, const bf16 *B, int ldb, int M, int N, int K, float *C32,
                 bf16 *C16, int ldc, const float *bias, int relu, int32_t *status, cudaStream_t st,
                 ImplicitConv ic = {0, 0, 0, 0}) {
    // M tiles on x (up to 2^31 - 1 blocks): a 65,536-row forward pass has
    // 2^17 row tiles in its first convolution
    dim3 grid((M + 127) / 128, (N + 127) / 128);
    k_gemm_bf16<<<grid, kGT, 32768 + 1024, st>>>(A, lda, B, ldb, M, N, K, C32, C16, ldc, bias, relu, status, ic);
    count_launches(1);
}

// log2 c if c is a power of two of at least 8 (the implicit operand's
// 16-byte reads stay inside one tap), else -1.
static int implicit_c_log2(int c) {
    if (c < 8 || (c & (c - 1))) return -1;
    int l = 0;
    while ((1 << l) < c) ++l;
    return l;
}

// --------------------------------------------------------------- helpers --
__global__ void k_cast_bf16(const float *x, bf16 *y, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

// out [cols][rows] = in [rows][cols]^T (bf16), 32 x 32 tiles.
__global__ void k_transpose_bf16(const bf16 *in, int rows, int cols, int ldi, bf16 *out, int ldo) {
    __shared__ bf16 t[32][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        t[k][threadIdx.x] = (r < rows && c < cols) ? in[(size_t)r * ldi + c] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (c < cols && r < rows) out[(size_t)c * ldo + r] = t[threadIdx.x][k];
    }
}

static void transpose(const bf16 *in, int rows, int cols, int ldi, bf16 *out, int ldo, cudaStream_t st) {
    dim3 grid((rows + 31) / 32, (cols + 31) / 32), block(32, 8);  // rows on x: no 65,535 limit
    k_transpose_bf16<<<grid, block, 0, st>>>(in, rows, cols, ldi, out, ldo);
    count_launches(1);
}

// im2col of a 3x3 pad-1 convolution, NHWC input [B,h,h,c] -> [B*ho*ho][kpad],
// column (ky*3 + kx)*c + ch, zero padding and zero columns past 9c. A block
// per output pixel (grid-stride), its threads over the columns: the pixel's
// coordinates are decomposed once, the columns with 32-bit arithmetic.
__global__ void k_im2col(const bf16 *x, int B, int h, int c, int ho, int stride, int kpad, bf16 *cols) {
    const int64_t nrows = (int64_t)B * ho * ho;
    for (int64_t p = blockIdx.x; p < nrows; p += gridDim.x) {
        const int ox = (int)(p % ho), oy = (int)((p / ho) % ho), b = (int)(p / ((int64_t)ho * ho));
        bf16 *dst = cols + p * kpad;
        const bf16 *xb = x + (int64_t)b * h * h * c;
        for (int k = threadIdx.x; k < kpad; k += blockDim.x) {
            bf16 v = __float2bfloat16_rn(0.f);
            if (k < 9 * c) {
                const int tap = k / c, ch = k - tap * c, ky = tap / 3, kx = tap - 3 * ky;
                const int iy = oy * stride - 1 + ky, ix = ox * stride - 1 + kx;
                if (iy >= 0 && iy < h && ix >= 0 && ix < h) v = xb[(iy * h + ix) * c + ch];
            }
            dst[k] = v;
        }
    }
}

// The same with 16-byte moves (8 channels at a time) when c is a multiple of
// 8: a tap's channels are contiguous both in the input pixel and in the row.
__global__ void k_im2col_v8(const bf16 *x, int B, int h, int c, int ho, int stride, int kpad, bf16 *cols) {
    const int64_t nrows = (int64_t)B * ho * ho;
    const int cv = c >> 3, kv = kpad >> 3;  // 16-byte units
    for (int64_t p = blockIdx.x; p < nrows; p += gridDim.x) {
        const int ox = (int)(p % ho), oy = (int)((p / ho) % ho), b = (int)(p / ((int64_t)ho * ho));
        uint4 *dst = reinterpret_cast<uint4 *>(cols + p * kpad);
        const uint4 *xb = reinterpret_cast<const uint4 *>(x + (int64_t)b * h * h * c);
        for (int k = threadIdx.x; k < kv; k += blockDim.x) {
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (k < 9 * cv) {
                const int tap = k / cv, cq = k - tap * cv, ky = tap / 3, kx = tap - 3 * ky;
                const int iy = oy * stride - 1 + ky, ix = ox * stride - 1 + kx;
                if (iy >= 0 && iy < h && ix >= 0 && ix < h) v = xb[(iy * h + ix) * cv + cq];
            }
            dst[k] = v;
        }
    }
}

// dx [B,h,h,c] = col2im(dcols): each input element gathers the column
// entries that read it (deterministic, no atomics).
__global__ void k_col2im(const float *dcols, int B, int h, int c, int ho, int stride, int kpad, float *dx) {
    const int64_t total = (int64_t)B * h * h * c;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int ch = (int)(e % c);
        const int64_t pix = e / c;
        const int ix = (int)(pix % h), iy = (int)((pix / h) % h), b = (int)(pix / ((int64_t)h * h));
        float acc = 0.f;
        for (int ky = 0; ky < 3; ++ky)
            for (int kx = 0; kx < 3; ++kx) {
                const int ty = iy + 1 - ky, tx = ix + 1 - kx;
                if (ty % stride || tx % stride) continue;
                const int oy = ty / stride, ox = tx / stride;
                if (ty < 0 || tx < 0 || oy >= ho || ox >= ho) continue;
                acc += dcols[(((int64_t)b * ho + oy) * ho + ox) * kpad + (ky * 3 + kx) * c + ch];
            }
        dx[e] = acc;
    }
}

// dz = dy * 1[y > 0] (ReLU backward on the stored bf16 activation), bf16 out.
__global__ void k_relu_back(const float *dy, const bf16 *y, int64_t n, bf16 *dz) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dz[i] = __float2bfloat16_rn(__bfloat162float(y[i]) > 0.f ? dy[i] : 0.f);
}

// db[j] = sum_i dz[i][j], in two fixed-order stages: block (cb, ch) sums the
// rows of chunk ch for 32 columns (8 row phases x 32 columns, then the 8
// phases in order) into part[ch][j]; k_colsum_final adds the chunks in order.
constexpr int kColChunks = 64;
__global__ void k_colsum_part(const bf16 *dz, int rows, int cols, int chunk_rows, float *part) {
    __shared__ float red[8][33];
    const int c = blockIdx.x * 32 + (threadIdx.x & 31), ph = threadIdx.x >> 5;
    const int r0 = blockIdx.y * chunk_rows, r1 = min(rows, r0 + chunk_rows);
    float acc = 0.f;
    if (c < cols)
        for (int i = r0 + ph; i < r1; i += 8) acc += __bfloat162float(dz[(size_t)i * cols + c]);
    red[ph][threadIdx.x & 31] = acc;
    __syncthreads();
    if (ph == 0 && c < cols) {
        float v = 0.f;
        for (int q = 0; q < 8; ++q) v += red[q][threadIdx.x];
        part[(size_t)blockIdx.y * cols + c] = v;
    }
}
__global__ void k_colsum_final(const float *part, int nchunks, int cols, float *db) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    float acc = 0.f;
    for (int q = 0; q < nchunks; ++q) acc += part[(size_t)q * cols + j];
    db[j] = acc;
}

// Loss and its gradient wrt the 2 nout outputs. out [B][2 nout] fp32 =
// [logits | scaled beta]; targets support [B][nout] in {0,1}, beta [B][nout].
// loss[0] = BCE mean, loss[1] = MSE mean (one block, fixed order).
__global__ void k_loss(const float *out, const float *support, const float *beta, int B, int nout, float *dout,
                       float *loss) {
    __shared__ float red[2][256];
    const int n = B * nout;
    float bce = 0.f, mse = 0.f;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int b = e / nout, j = e % nout;
        const float z = out[(size_t)b * 2 * nout + j], s = support[e];
        const float sp = fmaxf(z, 0.f) + log1pf(expf(-fabsf(z)));  // softplus
        bce += sp - s * z;
        const float sg = 1.f / (1.f + expf(-z));
        if (dout) dout[(size_t)b * 2 * nout + j] = (sg - s) / (float)n;
        const float d = out[(size_t)b * 2 * nout + nout + j] - beta[e] / kBetaScale;
        mse += d * d;
        if (dout) dout[(size_t)b * 2 * nout + nout + j] = 2.f * d / (float)n;
    }
    red[0][threadIdx.x] = bce;
    red[1][threadIdx.x] = mse;
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f, c = 0.f;
        for (int t = 0; t < (int)blockDim.x; ++t) { a += red[0][t]; c += red[1][t]; }
        loss[0] = a / (float)n;
        loss[1] = c / (float)n;
    }
}

// AdamW (decoupled weight decay), fp32 master weights.
__global__ void k_adamw(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                        float eps, float wd, float c1, float c2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * p[i]);
    }
}

// Network input of the layered 3-D architecture: one row per subdomain,
// x[row][iy][ix][iz] = clip(log10 K / 3, -1, 1) at patch cell (ix, iy, iz),
// zero outside the patch (and in rows past the last subdomain).
__global__ void k_layered_inputs(Geo g, const double *K, int h0, int c0, float *x) {
    const int row = blockIdx.x;
    float *xr = x + (size_t)row * h0 * h0 * c0;
    const bool live = row < g.S;
    // the subdomain's patch (core +- overlap, clipped), as the partition lays it out
    int plo[3] = {0, 0, 0}, pw[3] = {0, 0, 0};
    if (live) {
        const int jj[3] = {row % g.p[0], (row / g.p[0]) % g.p[1], row / (g.p[0] * g.p[1])};
        for (int a = 0; a < 3; ++a) {
            int64_t lo = ((int64_t)jj[a] * g.n[a]) / g.p[a] - g.overlap;
            int64_t hi = ((int64_t)(jj[a] + 1) * g.n[a]) / g.p[a] + g.overlap;
            if (lo < 0) lo = 0;
            if (hi > g.n[a]) hi = g.n[a];
            plo[a] = (int)lo;
            pw[a] = (int)(hi - lo);
        }
    }
    for (int e = threadIdx.x; e < h0 * h0 * c0; e += blockDim.x) {
        const int iz = e % c0, ix = (e / c0) % h0, iy = e / (c0 * h0);
        float v = 0.f;
        if (live && ix < pw[0] && iy < pw[1] && iz < pw[2]) {
            const int64_t gi = (int64_t)(plo[0] + ix) +
                               (int64_t)g.n[0] * ((int64_t)(plo[1] + iy) + (int64_t)g.n[1] * (plo[2] + iz));
            v = fminf(fmaxf(log10f((float)K[gi]) * (1.f / 3.f), -1.f), 1.f);  // a bf16 input: fp32 suffices
        }
        xr[e] = v;
    }
}

// Warm start from the network output: beta[s][j] = beta_hat if |beta_hat|
// > threshold else 0, beta_hat = 4 out[s][nout + j], for the nout entries
// of the initial dictionary.
__global__ void k_seed(const float *out, int S, int nout, int m_cap, float threshold, double *beta) {
    const int s = blockIdx.x;
    if (s >= S) return;
    for (int j = threadIdx.x; j < nout; j += blockDim.x) {
        const float bh = out[(size_t)s * 2 * nout + nout + j] * kBetaScale;
        beta[(size_t)s * m_cap + j] = fabsf(bh) > threshold ? (double)bh : 0.0;
    }
}

static unsigned grid_for(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 4096); }

// -------------------------------------------------------------- driver ----
struct Ws {
    bf16 *pw;             // bf16 copy of the parameters
    bf16 *x0;             // [B,h0,h0,c0]
    bf16 *cols[4];        // im2col buffers
    bf16 *act[6];         // layer outputs (bf16, post-ReLU; act[5] = out as bf16, unused)
    float *out;           // [B,2 n_out] fp32 network output
    float *dout;          // [B,2 n_out]
    float *dbuf0, *dbuf1; // fp32 gradient scratch (max activation size)
    bf16 *dz;             // bf16 pre-activation gradient
    bf16 *tA, *tB;        // transposes
    float *loss;          // [4]
    float *colpart;       // [kColChunks][512] bias-gradient partial sums
    int32_t *status;
    size_t bytes;
};

static size_t al(size_t v) { return (v + 255) / 256 * 256; }

static Ws carve(const Arch &A, int B, void *base) {
    Ws w;
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? (char *)base + off : nullptr;
        off = al(off + bytes);
        return p;
    };
    const Layout L = layout(A);
    w.pw = (bf16 *)take((size_t)L.total * 2);
    w.x0 = (bf16 *)take((size_t)B * A.h0 * A.h0 * A.c0 * 2);
    size_t maxact = 0, maxcols = 0;
    for (int l = 0; l < 4; ++l) {
        const Conv &c = A.conv[l];
        size_t cols = (size_t)B * c.hout * c.hout * c.kpad;
        size_t act = (size_t)B * c.hout * c.hout * c.cout;
        maxcols = std::max(maxcols, cols);
        maxact = std::max(maxact, act);
        w.cols[l] = (bf16 *)take(cols * 2);
        w.act[l] = (bf16 *)take(act * 2);
    }
    w.act[4] = (bf16 *)take((size_t)B * A.dense[0].out * 2);
    w.act[5] = (bf16 *)take((size_t)B * A.dense[1].out * 2);
    maxact = std::max(maxact, std::max(maxcols, (size_t)B * A.flat));
    maxact = std::max(maxact, (size_t)B * A.dense[0].out);
    w.out = (float *)take((size_t)B * A.dense[1].out * 4);
    w.dout = (float *)take((size_t)B * A.dense[1].out * 4);
    w.dbuf0 = (float *)take(maxact * 4);
    w.dbuf1 = (float *)take(maxact * 4);
    w.dz = (bf16 *)take(maxact * 2);
    w.tA = (bf16 *)take(std::max(maxact, (size_t)L.total) * 2);
    w.tB = (bf16 *)take(std::max(maxact, (size_t)L.total) * 2);
    w.loss = (float *)take(16);
    w.colpart = (float *)take((size_t)kColChunks * 512 * 4);
    w.status = (int32_t *)take(16);
    w.bytes = off;
    return w;
}

// Forward pass; activations stay in the workspace for the backward pass.
// implicit: inference only -- the convolutions read their input directly
// (no im2col matrix; the backward pass needs it, so training passes false).
// The operands, their order and the sums are the same either way.
static void forward(const Arch &A, const float *params, const float *x, int B, Ws &w, cudaStream_t st,
                    bool implicit = false, float *out = nullptr) {
    const Layout L = layout(A);
    const int64_t nx = (int64_t)B * A.h0 * A.h0 * A.c0;
    k_cast_bf16<<<grid_for(L.total), 256, 0, st>>>(params, w.pw, L.total);
    k_cast_bf16<<<grid_for(nx), 256, 0, st>>>(x, w.x0, nx);
    count_launches(2);
    const bf16 *in = w.x0;
    for (int l = 0; l < 4; ++l) {
        const Conv &c = A.conv[l];
        const int64_t rows = (int64_t)B * c.hout * c.hout;
        const unsigned blocks = (unsigned)std::min<int64_t>(rows, 16384);
        const int cl = implicit_c_log2(c.cin);
        if (implicit && cl >= 0) {
            gemm(in, 0, w.pw + L.w[l], c.kpad, (int)rows, c.cout, c.kpad, nullptr, w.act[l], c.cout,
                 params + L.b[l], 1, w.status, st, ImplicitConv{c.hin, cl, c.hout, c.stride});
            in = w.act[l];
            continue;
        }
        if (c.cin % 8 == 0) {
            const int kv = c.kpad / 8, thr = kv < 256 ? (kv + 31) / 32 * 32 : 256;
            k_im2col_v8<<<blocks, thr, 0, st>>>(in, B, c.hin, c.cin, c.hout, c.stride, c.kpad, w.cols[l]);
        } else {
            const int thr = c.kpad < 256 ? (c.kpad + 31) / 32 * 32 : 256;
            k_im2col<<<blocks, thr, 0, st>>>(in, B, c.hin, c.cin, c.hout, c.stride, c.kpad, w.cols[l]);
        }
        count_launches(1);
        gemm(w.cols[l], c.kpad, w.pw + L.w[l], c.kpad, (int)rows, c.cout, c.kpad, nullptr, w.act[l], c.cout,
             params + L.b[l], 1, w.status, st);
        in = w.act[l];
    }
    // dense layers: act[3] viewed as [B][flat] (NHWC flatten)
    const int d0 = A.dense[0].out, d1 = A.dense[1].out;
    gemm(w.act[3], A.flat, w.pw + L.w[4], A.flat, B, d0, A.flat, nullptr, w.act[4], d0, params + L.b[4], 1,
         w.status, st);
    gemm(w.act[4], d0, w.pw + L.w[5], d0, B, d1, d0, out ? out : w.out, nullptr, d1, params + L.b[5], 0, w.status,
         st);
}

// Backward of a layer y = relu(X W^T + b) (or linear for the output layer):
// dY (fp32 [rows][n]) -> dW, db (fp32 into grads), and dX (fp32 [rows][k])
// when want_dx. X is bf16 [rows][k] (k multiple of 32).
static void layer_backward(const float *dY, const bf16 *Y, bool relu, const bf16 *X, const bf16 *Wbf, int rows,
                           int n, int k, float *gW, float *gb, float *dX, Ws &w, cudaStream_t st) {
    const int64_t ny = (int64_t)rows * n;
    if (relu) {
        k_relu_back<<<grid_for(ny), 256, 0, st>>>(dY, Y, ny, w.dz);
    } else {
        k_cast_bf16<<<grid_for(ny), 256, 0, st>>>(dY, w.dz, ny);
    }
    count_launches(1);
    {
        const int chunks = std::max(1, std::min(kColChunks, (rows + 255) / 256));
        const int chunk_rows = (rows + chunks - 1) / chunks;
        k_colsum_part<<<dim3((n + 31) / 32, chunks), 256, 0, st>>>(w.dz, rows, n, chunk_rows, w.colpart);
        k_colsum_final<<<(n + 127) / 128, 128, 0, st>>>(w.colpart, chunks, n, gb);
        count_launches(2);
    }
    // dW [n][k] = dZ^T [n][rows] . X^T [k][rows]^T  (contraction over rows)
    transpose(w.dz, rows, n, n, w.tA, rows, st);
    transpose(X, rows, k, k, w.tB, rows, st);
    gemm(w.tA, rows, w.tB, rows, n, k, rows, gW, nullptr, k, nullptr, 0, w.status, st);
    if (dX) {
        // dX [rows][k] = dZ [rows][n] . (W^T) [k][n]^T (contraction over n)
        transpose(Wbf, n, k, k, w.tB, n, st);
        gemm(w.dz, n, w.tB, n, rows, k, n, dX, nullptr, k, nullptr, 0, w.status, st);
    }
}

static void backward(const Arch &A, const float *params, int B, float *grads, Ws &w, cudaStream_t st) {
    const Layout L = layout(A);
    const int d0 = A.dense[0].out, d1 = A.dense[1].out;
    // output dense (linear)
    layer_backward(w.dout, nullptr, false, w.act[4], w.pw + L.w[5], B, d1, d0, grads + L.w[5], grads + L.b[5],
                   w.dbuf0, w, st);
    layer_backward(w.dbuf0, w.act[4], true, w.act[3], w.pw + L.w[4], B, d0, A.flat, grads + L.w[4],
                   grads + L.b[4], w.dbuf1, w, st);
    float *dy = w.dbuf1, *other = w.dbuf0;
    for (int l = 3; l >= 0; --l) {
        const Conv &c = A.conv[l];
        const int rows = B * c.hout * c.hout;
        float *dcols = l > 0 ? other : nullptr;
        layer_backward(dy, w.act[l], true, w.cols[l], w.pw + L.w[l], rows, c.cout, c.kpad, grads + L.w[l],
                       grads + L.b[l], dcols, w, st);
        if (l > 0) {
            // d input = col2im(dcols) -> fp32 [B, hin, hin, cin] into dy's buffer
            const int64_t nin = (int64_t)B * c.hin * c.hin * c.cin;
            k_col2im<<<grid_for(nin), 256, 0, st>>>(dcols, B, c.hin, c.cin, c.hout, c.stride, c.kpad, dy);
            count_launches(1);
        }
    }
    (void)params;
}

}  // namespace nn
}  // namespace pam

using namespace pam::nn;

extern "C" {

static const Arch *arch_of(int arch) { return (arch >= 0 && arch < kNArch) ? &kArch[arch] : nullptr; }

pam_status pam_nn_sizes(int arch, int batch, int64_t *n_params, size_t *workspace_bytes) {
    const Arch *A = arch_of(arch);
    if (!A || batch < 1 || batch > 65536 || batch % 32 != 0) return PAM_ERR_INVALID_ARG;
    if (n_params) *n_params = layout(*A).total;
    if (workspace_bytes) *workspace_bytes = carve(*A, batch, nullptr).bytes;
    return PAM_OK;
}

pam_status pam_nn_geometry(int arch, int32_t *h_geo) {
    const Arch *A = arch_of(arch);
    if (!A || !h_geo) return PAM_ERR_INVALID_ARG;
    h_geo[0] = A->h0;
    h_geo[1] = A->c0;
    h_geo[2] = A->nout;
    return PAM_OK;
}

pam_status pam_nn_layer_offsets(int arch, int64_t *h_offsets) {
    const Arch *A = arch_of(arch);
    if (!A || !h_offsets) return PAM_ERR_INVALID_ARG;
    const Layout L = layout(*A);
    for (int l = 0; l < 6; ++l) {
        h_offsets[4 * l + 0] = L.w[l];
        h_offsets[4 * l + 1] = L.b[l];
        h_offsets[4 * l + 2] = L.rows[l];
        h_offsets[4 * l + 3] = L.cols[l];
    }
    return PAM_OK;
}

static pam_status nn_check(const Arch *A, int batch, void *ws, size_t ws_bytes) {
    if (!A || batch < 1 || batch > 65536 || batch % 32 != 0 || !ws) return PAM_ERR_INVALID_ARG;
    if (ws_bytes < carve(*A, batch, nullptr).bytes) return PAM_ERR_WORKSPACE;
    return PAM_OK;
}

pam_status pam_nn_forward(int arch, const float *d_params, const float *d_x, int batch, float *d_out,
                          void *d_workspace, size_t workspace_bytes, void *stream) {
    const Arch *A = arch_of(arch);
    pam_status st = nn_check(A, batch, d_workspace, workspace_bytes);
    if (st != PAM_OK) return st;
    if (!d_params || !d_x || !d_out) return PAM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Ws w = carve(*A, batch, d_workspace);
    PAM_CUDA_TRY(cudaMemsetAsync(w.status, 0, 16, s));
    cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, 32768 + 1024);
    forward(*A, d_params, d_x, batch, w, s, true, d_out);
    PAM_CUDA_TRY(cudaGetLastError());
    return PAM_OK;
}

pam_status pam_nn_gradients(int arch, const float *d_params, const float *d_x, const float *d_support,
                            const float *d_beta, int batch, float *d_grads, float *d_loss, void *d_workspace,
                            size_t workspace_bytes, void *stream) {
    const Arch *A = arch_of(arch);
    pam_status st = nn_check(A, batch, d_workspace, workspace_bytes);
    if (st != PAM_OK) return st;
    if (!d_params || !d_x || !d_support || !d_beta || !d_grads || !d_loss) return PAM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Ws w = carve(*A, batch, d_workspace);
    PAM_CUDA_TRY(cudaMemsetAsync(w.status, 0, 16, s));
    cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, 32768 + 1024);
    forward(*A, d_params, d_x, batch, w, s);
    k_loss<<<1, 256, 0, s>>>(w.out, d_support, d_beta, batch, A->nout, w.dout, d_loss);
    pam::count_launches(1);
    backward(*A, d_params, batch, d_grads, w, s);
    PAM_CUDA_TRY(cudaGetLastError());
    return PAM_OK;
}

pam_status pam_nn_inputs(int arch, const pam_problem *prob, const pam_plan *plan, const double *d_K, float *d_x,
                         int n_rows, void *stream) {
    const Arch *Ap = arch_of(arch);
    if (!Ap || !prob || !plan || !d_K || !d_x) return PAM_ERR_INVALID_ARG;
    pam::Geo g;
    pam_status st;
    if (!pam::make_geo(prob, nullptr, &g, nullptr, &st)) return st;
    // 2-D patches as pixels (one channel), layered 3-D patches with the z
    // layers as channels
    const int want_dim = arch == PAM_NN_LAYERED3D ? 3 : 2;
    if (g.dim != want_dim || plan->n_subdomains != g.S || n_rows < g.S) return PAM_ERR_INVALID_ARG;
    const Arch &A = *Ap;
    // every patch must fit the input grid: widest patch per axis
    const int lim[3] = {A.h0, A.h0, A.c0};
    for (int a = 0; a < 3; ++a) {
        for (int j = 0; j < g.p[a]; ++j) {
            int64_t lo = ((int64_t)j * g.n[a]) / g.p[a] - g.overlap, hi = ((int64_t)(j + 1) * g.n[a]) / g.p[a] + g.overlap;
            if (lo < 0) lo = 0;
            if (hi > g.n[a]) hi = g.n[a];
            if (hi - lo > lim[a]) return PAM_ERR_UNSUPPORTED;
        }
    }
    k_layered_inputs<<<n_rows, 256, 0, (cudaStream_t)stream>>>(g, d_K, A.h0, A.c0, d_x);
    pam::count_launches(1);
    PAM_CUDA_TRY(cudaGetLastError());
    return PAM_OK;
}

pam_status pam_nn_layered_inputs(const pam_problem *prob, const pam_plan *plan, const double *d_K, float *d_x,
                                 int n_rows, void *stream) {
    return pam_nn_inputs(PAM_NN_LAYERED3D, prob, plan, d_K, d_x, n_rows, stream);
}

pam_status pam_nn_seed(const pam_plan *plan, int arch, const float *d_out, float threshold, pam_model *model,
                       void *stream) {
    const Arch *A = arch_of(arch);
    if (!A || !plan || !d_out || !model || !model->beta || !(threshold >= 0.f)) return PAM_ERR_INVALID_ARG;
    if (plan->m0 != A->nout) return PAM_ERR_INVALID_ARG;
    k_seed<<<plan->n_subdomains, 64, 0, (cudaStream_t)stream>>>(d_out, plan->n_subdomains, A->nout, plan->m_cap,
                                                               threshold, model->beta);
    pam::count_launches(1);
    PAM_CUDA_TRY(cudaGetLastError());
    return PAM_OK;
}

pam_status pam_nn_adamw(float *d_params, const float *d_grads, float *d_m, float *d_v, int64_t n, float lr,
                        float beta1, float beta2, float eps, float weight_decay, int step, void *stream) {
    if (!d_params || !d_grads || !d_m || !d_v || n < 1 || step < 1) return PAM_ERR_INVALID_ARG;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    k_adamw<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(d_params, d_grads, d_m, d_v, n, lr, beta1, beta2, eps,
                                                           weight_decay, c1, c2);
    pam::count_launches(1);
    PAM_CUDA_TRY(cudaGetLastError());
    return PAM_OK;
}

}  // extern "C"
