// Learned candidate proposal (this library's addition; the paper has no such
// step): a small fully convolutional network that reads the L-pixel image
// and its opaque-quadrant codes and scores, per 4x4 target block, every one
// of the 1024 DFT candidates of the greedy loop (Sec. IV, Eq. 11), plus an
// iteration count.  The top-64 candidates of a block become its shortlist
// and the loop searches only those (kernels.cu, restricted loop); blocks the
// network is unsure of run the full loop.
//
// Network (weights stored FP32 for training and used rounded to bfloat16,
// activations and accumulation in FP32; in the whole-image pass conv2 and
// conv3 run on the tensor cores and read their input taps rounded to
// bfloat16, and the head reads its features rounded to bfloat16):
//   input 5 channels on the L-pixel grid: y / 3 and the one-hot code
//   conv1 5->32 3x3 s1, conv2 32->32 3x3 s2 (target-block grid),
//   conv3 32->32 3x3 s1, all zero-padded, ReLU; activations outside the
//   image are zero after every layer;
//   head: the 3x3 block-grid neighbourhood of conv3 (288 features) times a
//   1025 x 288 matrix plus bias: 1024 candidate logits and the iteration
//   output.
// Training runs on 16x16 L-pixel patches (rows/cols [2bi - 8, 2bi + 8)), whose
// centre features equal those of the whole-image pass.
#include <cublas_v2.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "rljsde_internal.h"

namespace rljsde {
namespace net {

constexpr int kC = 32;
constexpr int kOut = 1025;
constexpr int kOutPad = 1040;    // head rows padded so the BF16 GEMM sees 16-element-aligned strides
constexpr int kHeadIn = 9 * kC;
// flat parameter layout
constexpr int kW1 = 0, kB1 = kW1 + kC * 5 * 9, kW2 = kB1 + kC, kB2 = kW2 + kC * kC * 9, kW3 = kB2 + kC,
              kB3 = kW3 + kC * kC * 9, kWh = kB3 + kC, kBh = kWh + kOut * kHeadIn, kParams = kBh + kOut;

// ------------------------------------------------------------- helpers --
__global__ void to_bf16_kernel(const float *src, __nv_bfloat16 *dst, float *rounded, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const __nv_bfloat16 b = __float2bfloat16_rn(src[i]);
        dst[i] = b;
        rounded[i] = __bfloat162float(b);
    }
}

// Head weights in bfloat16, padded with zero rows to kOutPad x 288.
__global__ void head_pad_kernel(const float *wh, __nv_bfloat16 *out, int rows, int rows_pad, int cols)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows_pad * cols; i += gridDim.x * blockDim.x)
        out[i] = i < rows * cols ? __float2bfloat16_rn(wh[i]) : __float2bfloat16_rn(0.f);
}

// Input planes of one patch per sample: x[n][5][16][16], plus its origin.
__global__ void patches_kernel(const float *lr, long long lr_pitch, const uint8_t *mask, int lr_h, int lr_w,
                               const int2 *blocks, int n, float *x)
{
    const int s = blockIdx.x;
    if (s >= n) return;
    const int2 b = blocks[s];
    const int y0 = 2 * b.x - 8, x0 = 2 * b.y - 8;
    float *o = x + (size_t)s * 5 * 256;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        const int P = y0 + i / 16, Q = x0 + i % 16;
        float v = 0.f, c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
        if (P >= 0 && P < lr_h && Q >= 0 && Q < lr_w) {
            const float yv = lr[(long long)P * lr_pitch + Q];
            v = isfinite(yv) ? yv / 3.0f : 0.f;
            const int c = mask[(long long)P * lr_w + Q];
            c0 = c == 0; c1 = c == 1; c2 = c == 2; c3 = c == 3;
        }
        o[i] = v; o[256 + i] = c0; o[512 + i] = c1; o[768 + i] = c2; o[1024 + i] = c3;
    }
}

// Input planes of a whole image: x[5][lr_h][lr_w].
__global__ void image_input_kernel(const float *lr, long long lr_pitch, const uint8_t *mask, int lr_h, int lr_w,
                                   float *x)
{
    const long long plane = (long long)lr_h * lr_w;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < plane;
         i += (long long)gridDim.x * blockDim.x) {
        const int P = (int)(i / lr_w), Q = (int)(i % lr_w);
        const float yv = lr[(long long)P * lr_pitch + Q];
        const int c = mask[i];
        x[i] = isfinite(yv) ? yv / 3.0f : 0.f;
        x[plane + i] = c == 0;
        x[2 * plane + i] = c == 1;
        x[3 * plane + i] = c == 2;
        x[4 * plane + i] = c == 3;
    }
}

// Geometry of one conv layer over n samples.  A sample's output position
// (ho, wo) is inside the image iff (oy + ho, ox + wo) lies in [0, gh) x [0, gw)
// where (oy, ox) = origin / scale of that sample.
struct ConvGeom {
    int n, ci, hi, wi, ho, wo, stride;
    int scale;           // grid step of the output in L-pixels (1 or 2)
    const int2 *origin;  // per-sample L-pixel origin, nullptr = (0, 0)
    int lr_h, lr_w;      // image size in L-pixels
};

__device__ __forceinline__ bool inside(const ConvGeom &g, int s, int ho, int wo)
{
    int oy = 0, ox = 0;
    if (g.origin) { oy = g.origin[s].x / g.scale; ox = g.origin[s].y / g.scale; }
    const int gh = g.lr_h / g.scale, gw = g.lr_w / g.scale;
    const int y = oy + ho, x = ox + wo;
    return y >= 0 && y < gh && x >= 0 && x < gw;
}

// out[s][co][ho][wo] = relu(b[co] + sum_ci,dy,dx w[co][ci][dy][dx] in[s][ci][S ho + dy - 1][S wo + dx - 1]),
// zero outside the image.  One thread per output position, all 32 channels.
template <int CI>
__global__ void __launch_bounds__(128) conv_fwd_kernel(const float *in, const float *w, const float *b, float *out,
                                                       ConvGeom g)
{
    __shared__ float ws[kC * CI * 9];
    __shared__ float bs[kC];
    for (int i = threadIdx.x; i < kC * CI * 9; i += blockDim.x) ws[i] = w[i];
    for (int i = threadIdx.x; i < kC; i += blockDim.x) bs[i] = b[i];
    __syncthreads();
    const long long per = (long long)g.ho * g.wo;
    const long long total = per * g.n;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(idx / per);
        const int pos = (int)(idx % per);
        const int ho = pos / g.wo, wo = pos % g.wo;
        float *o = out + (size_t)s * kC * per + pos;
        if (!inside(g, s, ho, wo)) {
            for (int co = 0; co < kC; ++co) o[co * per] = 0.f;
            continue;
        }
        float acc[kC];
#pragma unroll
        for (int co = 0; co < kC; ++co) acc[co] = bs[co];
        const float *src = in + (size_t)s * CI * g.hi * g.wi;
        for (int ci = 0; ci < CI; ++ci) {
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const int y = g.stride * ho + t / 3 - 1, x = g.stride * wo + t % 3 - 1;
                if (y < 0 || y >= g.hi || x < 0 || x >= g.wi) continue;
                const float v = src[((size_t)ci * g.hi + y) * g.wi + x];
#pragma unroll
                for (int co = 0; co < kC; ++co) acc[co] += ws[(co * CI + ci) * 9 + t] * v;
            }
        }
#pragma unroll
        for (int co = 0; co < kC; ++co) o[co * per] = fmaxf(acc[co], 0.f);
    }
}

// gin[s][ci][y][x] = (sum_co,t w[co][ci][t] gout[s][co][ho][wo]) * (a_in > 0),
// gout already carries the ReLU derivative of its own layer.
template <int CI>
__global__ void __launch_bounds__(128) conv_bwd_data_kernel(const float *gout, const float *w, const float *a_in,
                                                            float *gin, ConvGeom g)
{
    __shared__ float ws[kC * CI * 9];
    for (int i = threadIdx.x; i < kC * CI * 9; i += blockDim.x) ws[i] = w[i];
    __syncthreads();
    const long long per_in = (long long)g.hi * g.wi, per_out = (long long)g.ho * g.wo;
    const long long total = per_in * g.n;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(idx / per_in);
        const int pos = (int)(idx % per_in);
        const int y = pos / g.wi, x = pos % g.wi;
        float acc[CI];
#pragma unroll
        for (int ci = 0; ci < CI; ++ci) acc[ci] = 0.f;
        const float *go = gout + (size_t)s * kC * per_out;
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int ny = y + 1 - t / 3, nx = x + 1 - t % 3;    // = S ho, S wo
            if (ny < 0 || nx < 0 || ny % g.stride || nx % g.stride) continue;
            const int ho = ny / g.stride, wo = nx / g.stride;
            if (ho >= g.ho || wo >= g.wo) continue;
            for (int co = 0; co < kC; ++co) {
                const float gv = go[co * per_out + ho * g.wo + wo];
#pragma unroll
                for (int ci = 0; ci < CI; ++ci) acc[ci] += ws[(co * CI + ci) * 9 + t] * gv;
            }
        }
        float *gi = gin + (size_t)s * CI * per_in + pos;
        const float *ai = a_in + (size_t)s * CI * per_in + pos;
#pragma unroll
        for (int ci = 0; ci < CI; ++ci) gi[ci * per_in] = ai[ci * per_in] > 0.f ? acc[ci] : 0.f;
    }
}

// gw[co][ci][t] += sum_s,pos gout[s][co][pos] in[s][ci][S ho + dy - 1][S wo + dx - 1],
// gb[co] += sum gout.  Each thread owns a few weights; samples are split
// across CTAs and the partial sums added atomically.
template <int CI>
__global__ void __launch_bounds__(256) conv_bwd_w_kernel(const float *gout, const float *in, float *gw, float *gb,
                                                         ConvGeom g)
{
    constexpr int NW = kC * CI * 9;
    constexpr int PER = (NW + 255) / 256;
    float acc[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) acc[j] = 0.f;
    float bacc = 0.f;
    const long long per_in = (long long)g.hi * g.wi, per_out = (long long)g.ho * g.wo;
    for (int s = blockIdx.x; s < g.n; s += gridDim.x) {
        const float *go = gout + (size_t)s * kC * per_out;
        const float *src = in + (size_t)s * CI * per_in;
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int wi = threadIdx.x + j * 256;
            if (wi >= NW) break;
            const int co = wi / (CI * 9), ci = (wi / 9) % CI, t = wi % 9;
            const int dy = t / 3 - 1, dx = t % 3 - 1;
            float a = 0.f;
            for (int ho = 0; ho < g.ho; ++ho) {
                const int y = g.stride * ho + dy;
                if (y < 0 || y >= g.hi) continue;
                for (int wo = 0; wo < g.wo; ++wo) {
                    const int x = g.stride * wo + dx;
                    if (x < 0 || x >= g.wi) continue;
                    a += go[co * per_out + ho * g.wo + wo] * src[(ci * g.hi + y) * g.wi + x];
                }
            }
            acc[j] += a;
        }
        if (threadIdx.x < kC) {
            float a = 0.f;
            for (long long p = 0; p < per_out; ++p) a += go[threadIdx.x * per_out + p];
            bacc += a;
        }
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int wi = threadIdx.x + j * 256;
        if (wi < NW) atomicAdd(&gw[wi], acc[j]);
    }
    if (threadIdx.x < kC) atomicAdd(&gb[threadIdx.x], bacc);
}

__global__ void origins_kernel(const int2 *blocks, int2 *origin, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) origin[i] = make_int2(2 * blocks[i].x - 8, 2 * blocks[i].y - 8);
}

__global__ void add_bias_kernel(const float *z, const float *b, float *out, int n, int k)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < (long long)n * k) out[i] = z[i] + b[i % k];
}

// Head features of the patch centre block: f[s][c * 9 + t] = a3[s][c][3 + t/3][3 + t%3].
__global__ void gather_centre_kernel(const float *a3, float *f, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * kHeadIn; i += gridDim.x * blockDim.x) {
        const int s = i / kHeadIn, j = i % kHeadIn, c = j / 9, t = j % 9;
        f[i] = a3[((size_t)s * kC + c) * 64 + (3 + t / 3) * 8 + 3 + t % 3];
    }
}

// g3 = scatter of the feature gradient back to the centre 3x3, times ReLU'.
__global__ void scatter_centre_kernel(const float *gf, const float *a3, float *g3, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * kC * 64; i += gridDim.x * blockDim.x) {
        const int s = i / (kC * 64), c = (i / 64) % kC, p = i % 64, y = p / 8, x = p % 8;
        float v = 0.f;
        if (y >= 3 && y < 6 && x >= 3 && x < 6 && a3[i] > 0.f) v = gf[(size_t)s * kHeadIn + c * 9 + (y - 3) * 3 + x - 3];
        g3[i] = v;
    }
}

// C[m][n] = beta C[m][n] + sum_k A(m, k) B(k, n) with A(m, k) = A[m sam + k sak],
// B(k, n) = B[k sbk + n sbn]; 64x64 tiles, 16-deep K steps, 4x4 outputs per thread.
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, const float *A, long long sam, long long sak,
                                                   const float *B, long long sbk, long long sbn, float *C, long long ldc,
                                                   float beta)
{
    __shared__ float As[16][65];
    __shared__ float Bs[16][65];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int i = threadIdx.x; i < 16 * 64; i += 256) {
            const int kk = i / 64, mm = i % 64;
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < M && k < K) ? A[m * sam + k * sak] : 0.f;
            const int n = n0 + mm;
            Bs[kk][mm] = (n < N && k < K) ? B[k * sbk + n * sbn] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) { a[i] = As[kk][ty * 4 + i]; b[i] = Bs[kk][tx * 4 + i]; }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
            if (m < M && n < N) {
                float *c = &C[(long long)m * ldc + n];
                *c = (beta == 0.f ? 0.f : beta * *c) + acc[i][j];
            }
        }
}

// Loss (mean over samples) and its gradient w.r.t. z = logits (+bias added here).
__global__ void loss_kernel(float *z, const float *bias, const uint8_t *t, const float *nu_t, int n, float pos_w,
                            float nu_w, float *gz, float *loss)
{
    const int s = blockIdx.x;
    if (s >= n) return;
    __shared__ float red[256];
    float l = 0.f;
    for (int k = threadIdx.x; k < kOut; k += blockDim.x) {
        const float zk = z[(size_t)s * kOut + k] + bias[k];
        z[(size_t)s * kOut + k] = zk;
        float g;
        if (k < 1024) {
            const float tk = t[(size_t)s * 1024 + k] ? 1.f : 0.f;
            const float w = tk > 0.5f ? pos_w : 1.f;
            const float sp = fmaxf(zk, 0.f) + log1pf(expf(-fabsf(zk)));
            l += w * (sp - tk * zk) / 1024.f;
            g = w * (1.f / (1.f + expf(-zk)) - tk) / 1024.f;
        } else {
            const float d = zk - nu_t[s];
            l += nu_w * d * d;
            g = 2.f * nu_w * d;
        }
        gz[(size_t)s * kOut + k] = g / n;
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0] / n);
}

__global__ void colsum_kernel(const float *g, int n, int cols, float *out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float a = 0.f;
    for (int s = 0; s < n; ++s) a += g[(size_t)s * cols + c];
    out[c] += a;
}

__global__ void adam_kernel(float *p, const float *g, float *m, float *v, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// ---------------------------------------------------- whole-image pass --
// im2col of the head: f[b][c * 9 + t] (bf16) for block b = by * nbw + bx of a
// chunk, from a3[c][nbh][nbw] with zero padding, for tiles of 32 consecutive
// blocks per CTA: the 32 x 288
// values are gathered with reads that run along the blocks of a tile
// (coalesced), staged as bfloat16 in shared memory, and written out as one
// contiguous 18 KB row range with 16-byte stores.
constexpr int kFeatTile = 32;
__global__ void __launch_bounds__(256) head_features_tile_kernel(const float *a3, int nbh, int nbw, long long b0,
                                                                 int nb, __nv_bfloat16 *f)
{
    // blockDim.x must be 256 (8 threads per block of the tile)
    // rows padded to 296 bfloat16 (592 bytes): bank groups of consecutive blocks differ
    constexpr int kRow = kHeadIn + 8;
    __shared__ __align__(16) __nv_bfloat16 tile[kFeatTile * kRow];
    const int n_tiles = (nb + kFeatTile - 1) / kFeatTile;
    for (int tl = blockIdx.x; tl < n_tiles; tl += gridDim.x) {
        const int first = tl * kFeatTile;
        const int n = nb - first < kFeatTile ? nb - first : kFeatTile;
        // thread: block bt of the tile, features ct = ct0 + 8 i
        const int bt = threadIdx.x % kFeatTile, ct0 = threadIdx.x / kFeatTile;
        const long long b = b0 + first + bt;
        const int by0 = (int)(b / nbw), bx0 = (int)(b - (long long)by0 * nbw);
        const long long plane = (long long)nbh * nbw;
#pragma unroll 4
        for (int ct = ct0; ct < kHeadIn; ct += 256 / kFeatTile) {
            const int c = ct / 9, t = ct - 9 * c;
            const int by = by0 + t / 3 - 1, bx = bx0 + t % 3 - 1;
            float v = 0.f;
            if (bt < n && by >= 0 && by < nbh && bx >= 0 && bx < nbw) v = a3[c * plane + (long long)by * nbw + bx];
            tile[bt * kRow + ct] = __float2bfloat16_rn(v);
        }
        __syncthreads();
        uint4 *dst = reinterpret_cast<uint4 *>(f + (long long)first * kHeadIn);
        const int n16 = n * (kHeadIn * 2 / 16);         // 36 x 16 bytes per block
        for (int i = threadIdx.x; i < n16; i += blockDim.x) {
            const int blk = i / (kHeadIn * 2 / 16), part = i - blk * (kHeadIn * 2 / 16);
            dst[i] = reinterpret_cast<const uint4 *>(tile + blk * kRow)[part];
        }
        __syncthreads();
    }
}

// Per block (one warp): logits + bias -> shortlist of the 64 largest (ties to
// the lower index), the expected number of likely candidates left out
// (sum of sigmoid over the rest), and the iteration output.
__device__ __forceinline__ uint32_t order_key(float v)
{
    // order-preserving unsigned key of a float
    const uint32_t u = __float_as_uint(v);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_value(uint32_t k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__global__ void shortlist_kernel(const float *z, int ldz, const float *bias, long long b0, int nb, Shortlist *out)
{
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    for (long long bl = (long long)blockIdx.x * wpb + wib; bl < nb; bl += (long long)gridDim.x * wpb) {
        // z rows are relative to the chunk, shortlists are indexed by block
        const float *zb = z + bl * ldz;
        uint32_t key[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) key[j] = order_key(zb[j * 32 + lane] + bias[j * 32 + lane]);
        // Bounds on the 64th largest key from the lanes' second-largest keys:
        // at least their smallest (those 64 keys all reach it), at most their
        // largest (64 keys over 32 lanes put two in some lane, so that lane's
        // second largest reaches the 64th).  Its bits above the first bit
        // where the two bounds differ are theirs, so the search starts below
        // that bit.
        uint32_t m1 = 0, m2 = 0;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const uint32_t k = key[j];
            m2 = max(m2, min(m1, k));
            m1 = max(m1, k);
        }
        const uint32_t hi = __reduce_max_sync(0xffffffffu, m2);
        const uint32_t lo = __reduce_min_sync(0xffffffffu, m2);
        const uint32_t diff = hi ^ lo;
        const int top = diff ? 31 - __clz(diff) : -1;          // highest differing bit
        // Binary search on the remaining key bits for the 64th largest key;
        // stop early once exactly 64 keys reach the candidate (then they are
        // the set).
        // top < 0: the bounds meet, and hi is the 64th largest key
        uint32_t thr = top < 0 ? hi : top >= 31 ? 0u : (hi & ~((2u << top) - 1u));
        bool exact = false;
        for (int bit = top; bit >= 0; --bit) {
            const uint32_t cand = thr | (1u << bit);
            unsigned cnt = 0;
#pragma unroll
            for (int j = 0; j < 32; ++j) cnt += key[j] >= cand;
            cnt = __reduce_add_sync(0xffffffffu, cnt);
            if (cnt >= (unsigned)kShortlist) thr = cand;
            if (cnt == (unsigned)kShortlist) { exact = true; break; }   // warp-uniform
        }
        Shortlist &sl = out[b0 + bl];
        float rest = 0.f;
        if (exact) {
            // exactly the keys >= thr, in lane-major order
            int mine = 0;
#pragma unroll
            for (int j = 0; j < 32; ++j) mine += key[j] >= thr;
            int base = mine;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, base, o);
                if (lane >= o) base += y;
            }
            int pos = base - mine;
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (key[j] >= thr) sl.idx[pos++] = (uint16_t)(j * 32 + lane);
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (key[j] < thr) rest += __frcp_rn(1.f + __expf(-key_value(key[j])));
            for (int o = 16; o; o >>= 1) rest += __shfl_xor_sync(0xffffffffu, rest, o);
            if (lane == 0) {
                sl.missing = rest;
                sl.nu_frac = zb[1024] + bias[1024];
            }
            continue;
        }
        // thr is the 64th largest key: take keys > thr, then keys == thr by increasing index
        int above = 0;
#pragma unroll
        for (int j = 0; j < 32; ++j) above += key[j] > thr;
        const int above_total = (int)__reduce_add_sync(0xffffffffu, (unsigned)above);
        int base = above;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, base, o);
            if (lane >= o) base += y;
        }
        base -= above;                           // exclusive prefix
        int pos = base;
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (key[j] > thr) sl.idx[pos++] = (uint16_t)(j * 32 + lane);
        // equal keys, in increasing candidate index k = j * 32 + lane
        int slot = above_total;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const unsigned eq = __ballot_sync(0xffffffffu, key[j] == thr);
            const int before = __popc(eq & ((1u << lane) - 1));
            if (((eq >> lane) & 1u) && slot + before < kShortlist) sl.idx[slot + before] = (uint16_t)(j * 32 + lane);
            slot += __popc(eq);
        }
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (key[j] < thr) rest += __frcp_rn(1.f + __expf(-key_value(key[j])));
        for (int o = 16; o; o >>= 1) rest += __shfl_xor_sync(0xffffffffu, rest, o);
        if (lane == 0) {
            sl.missing = rest;
            sl.nu_frac = zb[1024] + bias[1024];
        }
    }
}

// Head im2col for the no-allocation path: the same features as
// head_features_tile_kernel, rounded through bfloat16 but stored as float so the
// FP32 GEMM kernel multiplies exactly the operands the BF16 GEMM would.
__global__ void head_features_f32_kernel(const float *a3, int nbh, int nbw, long long b0, int nb, float *f)
{
    const long long total = (long long)nb * kHeadIn;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = b0 + i / kHeadIn;
        const int j = (int)(i % kHeadIn), c = j / 9, t = j % 9;
        const int by = (int)(b / nbw) + t / 3 - 1, bx = (int)(b % nbw) + t % 3 - 1;
        float v = 0.f;
        if (by >= 0 && by < nbh && bx >= 0 && bx < nbw) v = a3[((long long)c * nbh + by) * nbw + bx];
        f[i] = __bfloat162float(__float2bfloat16_rn(v));
    }
}

// ------------------------------------------- tensor-core convolution --
// conv2 / conv3 of the whole-image pass as an implicit GEMM on the 5th-gen
// tensor cores: D[128 output positions][32 channels] = A[128][288] x B[288][32]
// with K index t * 32 + ci (tap-major, so each 8-wide K group is one tap of 8
// consecutive input channels), A = the bfloat16-rounded input
// taps (zero outside the input), B = the bfloat16 weights, FP32 accumulation
// in tensor memory.  One CTA of 128 threads walks tiles of 128 positions:
// every thread gathers its position's 288 taps into shared memory, one thread
// issues the 18 K = 16 MMAs (tcgen05.mma kind::f16, cta_group::1) and
// commits them to an mbarrier, then each warp reads its 32 accumulator rows
// back (tcgen05.ld 32x32b) and applies bias and ReLU.  Every output of the
// whole-image pass lies inside the image, so no validity mask is needed.
//
// Shared-memory operands use the no-swizzle K-major layout: 8 x 16-byte core
// matrices, the 8-element K groups of one 8-row group contiguous (leading
// byte offset 128), 8-row groups 36 x 128 bytes apart (stride byte offset).
namespace tc {
constexpr int kM = 128;                              // output positions per tile (MMA M)
constexpr int kKTot = 9 * kC;                        // 288
constexpr uint32_t kLBO = 128;                       // next 8-element K group
constexpr uint32_t kSBO = (kKTot / 8) * 128;         // next 8-row group: 4608
constexpr uint32_t kABytes = (kM / 8) * kSBO;        // 73,728
constexpr uint32_t kBBytes = (kC / 8) * kSBO;        // 18,432
constexpr uint32_t kSmem = kABytes + kBBytes + 16;   // + mbarrier and tensor-memory address
static_assert(kSmem <= 227 * 1024, "tile operands must fit in shared memory");
// D FP32, A and B BF16, both K-major, N = 32, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kC >> 3) << 17) |
                            ((uint32_t)(kM >> 4) << 24);
constexpr uint32_t kTmemCols = 32;

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t desc(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(kLBO >> 4) << 16) | ((uint64_t)(kSBO >> 4) << 32) |
           (1ull << 46);                              // descriptor version 1, no swizzle
}

__device__ __forceinline__ uint64_t now_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of the mbarrier; give up after about 2 s.
__device__ __forceinline__ bool wait_phase(uint32_t bar, uint32_t parity)
{
    const uint64_t t0 = now_ns();
    for (uint32_t i = 0; i < (1u << 24); ++i) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (done) return true;
        if ((i & 255) == 255 && now_ns() - t0 > 2000000000ull) return false;
    }
    return false;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const uint32_t a = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
    const uint32_t b = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
    return a | (b << 16);
}

// in: [32][hi][wi] FP32; out: [32][ho][wo] FP32; w: [32][32][9] (bfloat16-rounded), b: [32].
__global__ void __launch_bounds__(128, 1) conv_tc_kernel(const float *in, const float *w, const float *bias,
                                                         float *out, int hi, int wi, int ho, int wo, int stride,
                                                         int *status)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *A = sm, *B = sm + kABytes;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + kABytes + kBBytes);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + kABytes + kBBytes + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // B: weights as bfloat16 in the core-matrix layout (row = output channel,
    // K group q = tap q / 4, input channels 8 (q % 4) ..)
    for (int i = tid; i < kC * (kKTot / 8); i += blockDim.x) {
        const int co = i / (kKTot / 8), q = i % (kKTot / 8);
        const int t = q >> 2, ci0 = (q & 3) * 8;
        const float *src = w + (co * kC + ci0) * 9 + t;          // w[co][ci][t]
        uint4 v;
        v.x = pack_bf16(src[0], src[9]); v.y = pack_bf16(src[18], src[27]);
        v.z = pack_bf16(src[36], src[45]); v.w = pack_bf16(src[54], src[63]);
        *reinterpret_cast<uint4 *>(B + (co >> 3) * kSBO + q * kLBO + (co & 7) * 16) = v;
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tslot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t a_addr = saddr(A), b_addr = saddr(B), bar_addr = saddr(bar);

    const long long total = (long long)ho * wo;
    const long long n_tiles = (total + kM - 1) / kM;
    uint32_t parity = 0;
    bool failed = false;
    for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        // A: this thread's position, its 288 taps as bfloat16
        const long long pos = tile * kM + tid;
        const bool valid = pos < total;
        const int oy = valid ? (int)(pos / wo) : 0, ox = valid ? (int)(pos % wo) : 0;
        unsigned char *arow = A + (tid >> 3) * kSBO + (tid & 7) * 16;
        const long long plane = (long long)hi * wi;
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int y = stride * oy + t / 3 - 1, x = stride * ox + t % 3 - 1;
            const bool inb = valid && y >= 0 && y < hi && x >= 0 && x < wi;
            const float *src = in + (inb ? (long long)y * wi + x : 0);
#pragma unroll
            for (int cg = 0; cg < 4; ++cg) {
                float v[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) v[e] = inb ? src[(cg * 8 + e) * plane] : 0.f;
                uint4 u;
                u.x = pack_bf16(v[0], v[1]); u.y = pack_bf16(v[2], v[3]);
                u.z = pack_bf16(v[4], v[5]); u.w = pack_bf16(v[6], v[7]);
                *reinterpret_cast<uint4 *>(arow + (t * 4 + cg) * kLBO) = u;
            }
        }
        // generic-proxy writes -> tensor-core (async proxy) reads
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
#pragma unroll
            for (int j = 0; j < kKTot / 16; ++j) {
                const uint64_t da = desc(a_addr + j * 2 * kLBO), db = desc(b_addr + j * 2 * kLBO);
                asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                             " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                             ::"r"(tmem), "l"(da), "l"(db), "r"(kIdesc), "r"(j)
                             : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(bar_addr)
                         : "memory");
        }
        const bool ok = wait_phase(bar_addr, parity);
        if (__syncthreads_or(!ok)) { failed = true; break; }
        parity ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // this warp's 32 accumulator rows (TMEM lanes 32 warp ..), 32 columns each
        uint32_t r[32];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                     : "r"(tmem + ((uint32_t)(warp * 32) << 16))
                     : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (valid) {
#pragma unroll
            for (int co = 0; co < kC; ++co)
                out[(long long)co * total + pos] = fmaxf(__uint_as_float(r[co]) + bias[co], 0.f);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        (void)lane;
    }
    if (failed) {
        if (tid == 0) atomicOr(status, 2);
        wait_phase(bar_addr, parity);                 // let an MMA still in flight finish
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}
}  // namespace tc

// Fixed scratch of rljsde_propose_noalloc: part of the library image, so
// every device that loads the library holds it until the process exits.
constexpr size_t kStaticScratchBytes = 32u << 20;
constexpr int kStaticChunk = 1024;       // blocks per head GEMM in that path
static __device__ __align__(256) unsigned char g_propose_scratch[kStaticScratchBytes];

}  // namespace net
}  // namespace rljsde

using namespace rljsde;
using namespace rljsde::net;

namespace {

// Device address of g_propose_scratch, looked up once per device with that
// device current (host code may not use the symbol itself as a pointer).
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void *g_scratch_addr[kMaxDevices] = {};

int static_scratch(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RLJSDE_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return RLJSDE_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_propose_scratch) != cudaSuccess || !p) return RLJSDE_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return RLJSDE_OK;
}

}  // namespace

struct rljsde_net {
    float *master = nullptr, *rounded = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *w16 = nullptr;
    __nv_bfloat16 *head16 = nullptr;     // kOutPad x 288, zero-padded head rows
    int step = 0;
    int sm_count = 1;                    // SMs of the device the network lives on
    cublasHandle_t blas = nullptr;
    // training buffers, sized for `cap` samples
    int cap = 0;
    float *x = nullptr, *a1 = nullptr, *a2 = nullptr, *a3 = nullptr, *g1 = nullptr, *g2 = nullptr, *g3 = nullptr;
    float *f = nullptr, *gf = nullptr, *z = nullptr, *gz = nullptr, *loss = nullptr;
    int2 *origin = nullptr;
};

namespace {

void free_train(rljsde_net *n)
{
    cudaFree(n->x); cudaFree(n->a1); cudaFree(n->a2); cudaFree(n->a3); cudaFree(n->g1); cudaFree(n->g2);
    cudaFree(n->g3); cudaFree(n->f); cudaFree(n->gf); cudaFree(n->z); cudaFree(n->gz); cudaFree(n->loss);
    cudaFree(n->origin);
    n->x = n->a1 = n->a2 = n->a3 = n->g1 = n->g2 = n->g3 = n->f = n->gf = n->z = n->gz = n->loss = nullptr;
    n->origin = nullptr;
    n->cap = 0;
}

int ensure_train(rljsde_net *n, int cap)
{
    if (cap <= n->cap) return RLJSDE_OK;
    free_train(n);
    size_t s = cap;
    bool ok = cudaMalloc(&n->x, s * 5 * 256 * 4) == cudaSuccess && cudaMalloc(&n->a1, s * kC * 256 * 4) == cudaSuccess &&
              cudaMalloc(&n->a2, s * kC * 64 * 4) == cudaSuccess && cudaMalloc(&n->a3, s * kC * 64 * 4) == cudaSuccess &&
              cudaMalloc(&n->g1, s * kC * 256 * 4) == cudaSuccess && cudaMalloc(&n->g2, s * kC * 64 * 4) == cudaSuccess &&
              cudaMalloc(&n->g3, s * kC * 64 * 4) == cudaSuccess && cudaMalloc(&n->f, s * kHeadIn * 4) == cudaSuccess &&
              cudaMalloc(&n->gf, s * kHeadIn * 4) == cudaSuccess && cudaMalloc(&n->z, s * kOut * 4) == cudaSuccess &&
              cudaMalloc(&n->gz, s * kOut * 4) == cudaSuccess && cudaMalloc(&n->loss, 4) == cudaSuccess &&
              cudaMalloc(&n->origin, s * sizeof(int2)) == cudaSuccess;
    if (!ok) { free_train(n); return RLJSDE_ERR_OUT_OF_MEMORY; }
    n->cap = cap;
    return RLJSDE_OK;
}

int grid_for(long long work, int threads)
{
    long long g = (work + threads - 1) / threads;
    return (int)(g < 1 ? 1 : (g > 65535 * 16 ? 65535 * 16 : g));
}

// conv2 / conv3 of a whole image on the tensor cores (tc::conv_tc_kernel).
int conv_tc(const float *in, const float *w, const float *b, float *out, int hi, int wi, int ho, int wo, int stride,
            int sm_count, int *status, cudaStream_t s)
{
    if (cudaFuncSetAttribute(tc::conv_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::kSmem) !=
        cudaSuccess)
        return RLJSDE_ERR_CUDA;
    const long long tiles = ((long long)ho * wo + tc::kM - 1) / tc::kM;
    const long long cap = 2ll * (sm_count > 0 ? sm_count : 1);      // two 92 KB CTAs per SM
    const int grid = (int)(tiles < cap ? (tiles > 0 ? tiles : 1) : cap);
    tc::conv_tc_kernel<<<grid, 128, tc::kSmem, s>>>(in, w, b, out, hi, wi, ho, wo, stride, status);
    return cudaGetLastError() == cudaSuccess ? RLJSDE_OK : RLJSDE_ERR_CUDA;
}

void refresh_bf16(rljsde_net *n, cudaStream_t s)
{
    to_bf16_kernel<<<grid_for(kParams, 256), 256, 0, s>>>(n->master, n->w16, n->rounded, kParams);
    head_pad_kernel<<<grid_for(kOutPad * kHeadIn, 256), 256, 0, s>>>(n->master + kWh, n->head16, kOut, kOutPad,
                                                                     kHeadIn);
}

// Forward over n patches already in n->x with origins in n->origin; the
// head logits (without bias) land in n->z.
void forward_patches(rljsde_net *net, int n, int lr_h, int lr_w, cudaStream_t s)
{
    const float *r = net->rounded, *b = net->master;     // weights bf16-rounded, biases FP32
    ConvGeom g1{n, 5, 16, 16, 16, 16, 1, 1, net->origin, lr_h, lr_w};
    conv_fwd_kernel<5><<<grid_for((long long)n * 256, 128), 128, 0, s>>>(net->x, r + kW1, b + kB1, net->a1, g1);
    ConvGeom g2{n, kC, 16, 16, 8, 8, 2, 2, net->origin, lr_h, lr_w};
    conv_fwd_kernel<kC><<<grid_for((long long)n * 64, 128), 128, 0, s>>>(net->a1, r + kW2, b + kB2, net->a2, g2);
    ConvGeom g3{n, kC, 8, 8, 8, 8, 1, 2, net->origin, lr_h, lr_w};
    conv_fwd_kernel<kC><<<grid_for((long long)n * 64, 128), 128, 0, s>>>(net->a2, r + kW3, b + kB3, net->a3, g3);
    gather_centre_kernel<<<grid_for((long long)n * kHeadIn, 256), 256, 0, s>>>(net->a3, net->f, n);
    // z[s][k] = sum_j f[s][j] Wh[k][j]
    dim3 gg((kOut + 63) / 64, (n + 63) / 64);
    gemm_kernel<<<gg, 256, 0, s>>>(n, kOut, kHeadIn, net->f, kHeadIn, 1, r + kWh, 1, kHeadIn, net->z, kOut, 0.f);
}

}  // namespace

extern "C" {

int rljsde_net_create(rljsde_net_t **out, uint64_t seed)
{
    if (!out) return RLJSDE_ERR_INVALID_ARG;
    *out = nullptr;
    rljsde_net *n = new (std::nothrow) rljsde_net();
    if (!n) return RLJSDE_ERR_OUT_OF_MEMORY;
    size_t b = (size_t)kParams * 4;
    bool ok = cudaMalloc(&n->master, b) == cudaSuccess && cudaMalloc(&n->rounded, b) == cudaSuccess &&
              cudaMalloc(&n->grad, b) == cudaSuccess && cudaMalloc(&n->m, b) == cudaSuccess &&
              cudaMalloc(&n->v, b) == cudaSuccess && cudaMalloc(&n->w16, (size_t)kParams * 2) == cudaSuccess &&
              cudaMalloc(&n->head16, (size_t)kOutPad * kHeadIn * 2) == cudaSuccess;
    if (!ok || cublasCreate(&n->blas) != CUBLAS_STATUS_SUCCESS) { rljsde_net_destroy(n); return RLJSDE_ERR_OUT_OF_MEMORY; }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n->sm_count < 1) {
        rljsde_net_destroy(n);
        return RLJSDE_ERR_CUDA;
    }
    // He-style uniform init from a SplitMix64 stream; biases zero
    std::vector<float> h(kParams, 0.f);
    uint64_t st = seed;
    auto next = [&]() {
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    auto fill = [&](int off, int cnt, double fan_in) {
        const double a = std::sqrt(6.0 / fan_in);
        for (int i = 0; i < cnt; ++i) h[off + i] = (float)((2.0 * next() - 1.0) * a);
    };
    fill(kW1, kB1 - kW1, 45.0);
    fill(kW2, kB2 - kW2, 288.0);
    fill(kW3, kB3 - kW3, 288.0);
    fill(kWh, kBh - kWh, 288.0 * 8.0);
    for (int k = 0; k < 1024; ++k) h[kBh + k] = -3.0f;     // start near the ~6% positive rate
    h[kBh + 1024] = 1.0f;
    if (cudaMemcpy(n->master, h.data(), b, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(n->m, 0, b) != cudaSuccess || cudaMemset(n->v, 0, b) != cudaSuccess) {
        rljsde_net_destroy(n);
        return RLJSDE_ERR_CUDA;
    }
    refresh_bf16(n, 0);
    if (cudaDeviceSynchronize() != cudaSuccess) { rljsde_net_destroy(n); return RLJSDE_ERR_CUDA; }
    *out = n;
    return RLJSDE_OK;
}

void rljsde_net_destroy(rljsde_net_t *n)
{
    if (!n) return;
    free_train(n);
    cudaFree(n->master); cudaFree(n->rounded); cudaFree(n->grad); cudaFree(n->m); cudaFree(n->v); cudaFree(n->w16);
    cudaFree(n->head16);
    if (n->blas) cublasDestroy(n->blas);
    delete n;
}

int rljsde_net_num_params(void) { return kParams; }

int rljsde_net_get_params(const rljsde_net_t *n, float *host)
{
    if (!n || !host) return RLJSDE_ERR_INVALID_ARG;
    return cudaMemcpy(host, n->master, (size_t)kParams * 4, cudaMemcpyDeviceToHost) == cudaSuccess ? RLJSDE_OK
                                                                                                  : RLJSDE_ERR_CUDA;
}

int rljsde_net_set_params(rljsde_net_t *n, const float *host)
{
    if (!n || !host) return RLJSDE_ERR_INVALID_ARG;
    if (cudaMemcpy(n->master, host, (size_t)kParams * 4, cudaMemcpyHostToDevice) != cudaSuccess) return RLJSDE_ERR_CUDA;
    refresh_bf16(n, 0);
    return cudaDeviceSynchronize() == cudaSuccess ? RLJSDE_OK : RLJSDE_ERR_CUDA;
}

int rljsde_net_patches(const float *lr, size_t lr_pitch, const uint8_t *mask, int lr_h, int lr_w,
                       const int32_t *blocks, int n, float *x, void *stream)
{
    if (!lr || !mask || !blocks || !x || n < 0 || lr_h < 4 || lr_w < 4 || (lr_h & 1) || (lr_w & 1))
        return RLJSDE_ERR_INVALID_ARG;
    if (n == 0) return RLJSDE_OK;
    patches_kernel<<<n, 256, 0, (cudaStream_t)stream>>>(lr, (long long)lr_pitch, mask, lr_h, lr_w,
                                                         reinterpret_cast<const int2 *>(blocks), n, x);
    return cudaGetLastError() == cudaSuccess ? RLJSDE_OK : RLJSDE_ERR_CUDA;
}

// Loss and gradients of n patches (x: device [n][5][16][16], blocks: device
// [n][2] (bi, bj) of the image lr_h x lr_w they come from).  grad (device,
// num_params) receives the gradient; *loss_host the mean loss.
static int loss_grad(rljsde_net *net, const float *x, const int32_t *blocks, int n, int lr_h, int lr_w,
                     const uint8_t *targets, const float *nu_t, float pos_w, float nu_w, float *loss_host,
                     cudaStream_t s)
{
    int st = ensure_train(net, n);
    if (st) return st;
    cudaMemcpyAsync(net->x, x, (size_t)n * 5 * 256 * 4, cudaMemcpyDeviceToDevice, s);
    origins_kernel<<<grid_for(n, 256), 256, 0, s>>>(reinterpret_cast<const int2 *>(blocks), net->origin, n);
    forward_patches(net, n, lr_h, lr_w, s);
    cudaMemsetAsync(net->loss, 0, 4, s);
    const float *r = net->rounded;
    loss_kernel<<<n, 256, 0, s>>>(net->z, net->master + kBh, targets, nu_t, n, pos_w, nu_w, net->gz, net->loss);
    cudaMemsetAsync(net->grad, 0, (size_t)kParams * 4, s);
    // head: gWh[k][j] = sum_s gz[s][k] f[s][j]; gbh = sum_s gz; gf[s][j] = sum_k gz[s][k] Wh[k][j]
    dim3 gw((kHeadIn + 63) / 64, (kOut + 63) / 64);
    gemm_kernel<<<gw, 256, 0, s>>>(kOut, kHeadIn, n, net->gz, 1, kOut, net->f, kHeadIn, 1, net->grad + kWh, kHeadIn, 0.f);
    colsum_kernel<<<(kOut + 255) / 256, 256, 0, s>>>(net->gz, n, kOut, net->grad + kBh);
    dim3 gf((kHeadIn + 63) / 64, (n + 63) / 64);
    gemm_kernel<<<gf, 256, 0, s>>>(n, kHeadIn, kOut, net->gz, kOut, 1, r + kWh, kHeadIn, 1, net->gf, kHeadIn, 0.f);
    scatter_centre_kernel<<<grid_for((long long)n * kC * 64, 256), 256, 0, s>>>(net->gf, net->a3, net->g3, n);
    const int wg = 2 * net->sm_count;
    ConvGeom g3{n, kC, 8, 8, 8, 8, 1, 2, net->origin, lr_h, lr_w};
    conv_bwd_w_kernel<kC><<<wg, 256, 0, s>>>(net->g3, net->a2, net->grad + kW3, net->grad + kB3, g3);
    conv_bwd_data_kernel<kC><<<grid_for((long long)n * 64, 128), 128, 0, s>>>(net->g3, r + kW3, net->a2, net->g2, g3);
    ConvGeom g2{n, kC, 16, 16, 8, 8, 2, 2, net->origin, lr_h, lr_w};
    conv_bwd_w_kernel<kC><<<wg, 256, 0, s>>>(net->g2, net->a1, net->grad + kW2, net->grad + kB2, g2);
    conv_bwd_data_kernel<kC><<<grid_for((long long)n * 256, 128), 128, 0, s>>>(net->g2, r + kW2, net->a1, net->g1, g2);
    ConvGeom g1{n, 5, 16, 16, 16, 16, 1, 1, net->origin, lr_h, lr_w};
    conv_bwd_w_kernel<5><<<wg, 256, 0, s>>>(net->g1, net->x, net->grad + kW1, net->grad + kB1, g1);
    if (cudaGetLastError() != cudaSuccess) return RLJSDE_ERR_CUDA;
    if (loss_host && cudaMemcpyAsync(loss_host, net->loss, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return RLJSDE_ERR_CUDA;
    return RLJSDE_OK;
}

int rljsde_net_gradient(rljsde_net_t *net, const float *x, const int32_t *blocks, int n, int lr_h, int lr_w,
                        const uint8_t *targets, const float *nu_t, float pos_w, float nu_w, float *grad_out,
                        float *loss_host, void *stream)
{
    if (!net || !x || !blocks || !targets || !nu_t || n < 1) return RLJSDE_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int st = loss_grad(net, x, blocks, n, lr_h, lr_w, targets, nu_t, pos_w, nu_w, loss_host, s);
    if (st) return st;
    if (grad_out && cudaMemcpyAsync(grad_out, net->grad, (size_t)kParams * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return RLJSDE_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? RLJSDE_OK : RLJSDE_ERR_CUDA;
}

int rljsde_net_train_step(rljsde_net_t *net, const float *x, const int32_t *blocks, int n, int lr_h, int lr_w,
                          const uint8_t *targets, const float *nu_t, float pos_w, float nu_w, float lr,
                          float *loss_host, void *stream)
{
    if (!net || !x || !blocks || !targets || !nu_t || n < 1 || !(lr > 0.f)) return RLJSDE_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int st = loss_grad(net, x, blocks, n, lr_h, lr_w, targets, nu_t, pos_w, nu_w, loss_host, s);
    if (st) return st;
    net->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)net->step), c2 = 1.f - std::pow(b2, (float)net->step);
    adam_kernel<<<grid_for(kParams, 256), 256, 0, s>>>(net->master, net->grad, net->m, net->v, kParams, lr, b1, b2,
                                                       1e-8f, c1, c2);
    refresh_bf16(net, s);
    if (cudaGetLastError() != cudaSuccess) return RLJSDE_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? RLJSDE_OK : RLJSDE_ERR_CUDA;
}

// Logits (+bias) of n patches: z_out device [n][1025].
int rljsde_net_logits(rljsde_net_t *net, const float *x, const int32_t *blocks, int n, int lr_h, int lr_w,
                      float *z_out, void *stream)
{
    if (!net || !x || !blocks || !z_out || n < 1) return RLJSDE_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int st = ensure_train(net, n);
    if (st) return st;
    cudaMemcpyAsync(net->x, x, (size_t)n * 5 * 256 * 4, cudaMemcpyDeviceToDevice, s);
    origins_kernel<<<grid_for(n, 256), 256, 0, s>>>(reinterpret_cast<const int2 *>(blocks), net->origin, n);
    forward_patches(net, n, lr_h, lr_w, s);
    add_bias_kernel<<<grid_for((long long)n * kOut, 256), 256, 0, s>>>(net->z, net->master + kBh, z_out, n, kOut);
    if (cudaGetLastError() != cudaSuccess) return RLJSDE_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? RLJSDE_OK : RLJSDE_ERR_CUDA;
}

size_t rljsde_propose_workspace(const rljsde_plan_t *plan)
{
    if (!plan || plan->n_images != 1) return 0;
    const size_t P = (size_t)plan->lr_h[0] * plan->lr_w[0], nb = (size_t)plan->n_blocks;
    const size_t chunk = nb < 65536 ? nb : 65536;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    return al(5 * P * 4) + al(kC * P * 4) + 2 * al(kC * nb * 4) + al(chunk * kHeadIn * 2) + al(chunk * kOutPad * 4);
}

int rljsde_propose(const rljsde_plan_t *plan, const rljsde_net_t *net, const float *lr, size_t lr_pitch,
                   void *shortlists, void *workspace, size_t ws_bytes, void *stream)
{
    if (!plan || !net || !lr || !shortlists || !workspace) return RLJSDE_ERR_INVALID_ARG;
    if (plan->n_images != 1 || lr_pitch < (size_t)plan->lr_w[0]) return RLJSDE_ERR_INVALID_ARG;
    if (plan->params.layout != RLJSDE_LAYOUT_THREE_QUARTER) return RLJSDE_ERR_UNSUPPORTED;   // opaque-code input
    if (ws_bytes < rljsde_propose_workspace(plan)) return RLJSDE_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int lr_h = plan->lr_h[0], lr_w = plan->lr_w[0], nbh = lr_h / 2, nbw = lr_w / 2;
    const size_t P = (size_t)lr_h * lr_w, nb = (size_t)plan->n_blocks;
    const size_t chunk = nb < 65536 ? nb : 65536;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    char *w = static_cast<char *>(workspace);
    float *x = reinterpret_cast<float *>(w);            w += al(5 * P * 4);
    float *a1 = reinterpret_cast<float *>(w);           w += al(kC * P * 4);
    float *a2 = reinterpret_cast<float *>(w);           w += al(kC * nb * 4);
    float *a3 = reinterpret_cast<float *>(w);           w += al(kC * nb * 4);
    __nv_bfloat16 *f16 = reinterpret_cast<__nv_bfloat16 *>(w); w += al(chunk * kHeadIn * 2);
    float *z = reinterpret_cast<float *>(w);
    const float *r = net->rounded, *b = net->master;
    const int cap = 8 * (plan->sm_count > 0 ? plan->sm_count : 1);     // 8 CTAs per SM at most
    auto gcap = [&](long long work, int threads) { int g = grid_for(work, threads); return g < cap ? g : cap; };
    image_input_kernel<<<gcap((long long)P, 256), 256, 0, s>>>(lr, (long long)lr_pitch, plan->d_masks, lr_h, lr_w, x);
    ConvGeom g1{1, 5, lr_h, lr_w, lr_h, lr_w, 1, 1, nullptr, lr_h, lr_w};
    conv_fwd_kernel<5><<<gcap((long long)P, 128), 128, 0, s>>>(x, r + kW1, b + kB1, a1, g1);
    // conv2 (stride 2, onto the block grid) and conv3 on the tensor cores
    int cst = conv_tc(a1, r + kW2, b + kB2, a2, lr_h, lr_w, nbh, nbw, 2, plan->sm_count, plan->d_status, s);
    if (cst == RLJSDE_OK)
        cst = conv_tc(a2, r + kW3, b + kB3, a3, nbh, nbw, nbh, nbw, 1, plan->sm_count, plan->d_status, s);
    if (cst != RLJSDE_OK) return cst;
    if (cublasSetStream(net->blas, s) != CUBLAS_STATUS_SUCCESS) return RLJSDE_ERR_CUDA;
    const float one = 1.f, zero = 0.f;
    for (size_t b0 = 0; b0 < nb; b0 += chunk) {
        const int m = (int)(nb - b0 < chunk ? nb - b0 : chunk);
        head_features_tile_kernel<<<gcap(((long long)m + kFeatTile - 1) / kFeatTile * 256, 256), 256, 0, s>>>(
            a3, nbh, nbw, (long long)b0, m, f16);
        // z (row-major m x 1040) = f16 (m x 288) * Wh_pad^T: column-major z^T = Wh_pad * f16^T
        if (cublasGemmEx(net->blas, CUBLAS_OP_T, CUBLAS_OP_N, kOutPad, m, kHeadIn, &one, net->head16, CUDA_R_16BF,
                         kHeadIn, f16, CUDA_R_16BF, kHeadIn, &zero, z, CUDA_R_32F, kOutPad, CUBLAS_COMPUTE_32F,
                         CUBLAS_GEMM_DEFAULT) != CUBLAS_STATUS_SUCCESS)
            return RLJSDE_ERR_CUDA;
        shortlist_kernel<<<gcap(((long long)m + 7) / 8 * 256, 256), 256, 0, s>>>(
            z, kOutPad, b + kBh, (long long)b0, m, static_cast<Shortlist *>(shortlists));
    }
    return cudaGetLastError() == cudaSuccess ? RLJSDE_OK : RLJSDE_ERR_CUDA;
}

// The proposal pass for callers that must not allocate device memory; see
// the header for who they are and for the size limit.
int rljsde_propose_noalloc(const rljsde_plan_t *plan, const rljsde_net_t *net, const float *lr, size_t lr_pitch,
                           void *shortlists, void *stream)
{
    if (!plan || !net || !lr || !shortlists) return RLJSDE_ERR_INVALID_ARG;
    if (plan->n_images != 1 || lr_pitch < (size_t)plan->lr_w[0]) return RLJSDE_ERR_INVALID_ARG;
    if (plan->params.layout != RLJSDE_LAYOUT_THREE_QUARTER) return RLJSDE_ERR_UNSUPPORTED;   // opaque-code input
    const int lr_h = plan->lr_h[0], lr_w = plan->lr_w[0], nbh = lr_h / 2, nbw = lr_w / 2;
    const size_t P = (size_t)lr_h * lr_w, nb = (size_t)plan->n_blocks;
    const size_t chunk = nb < (size_t)kStaticChunk ? nb : (size_t)kStaticChunk;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t need = al(5 * P * 4) + al(kC * P * 4) + 2 * al(kC * nb * 4) + al(chunk * kHeadIn * 4) +
                        al(chunk * kOut * 4);
    if (need > kStaticScratchBytes) return RLJSDE_ERR_BAD_SHAPE;    // image too large for the fixed scratch
    void *base = nullptr;
    int st = static_scratch(&base);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    char *w = static_cast<char *>(base);
    float *x = reinterpret_cast<float *>(w);   w += al(5 * P * 4);
    float *a1 = reinterpret_cast<float *>(w);  w += al(kC * P * 4);
    float *a2 = reinterpret_cast<float *>(w);  w += al(kC * nb * 4);
    float *a3 = reinterpret_cast<float *>(w);  w += al(kC * nb * 4);
    float *f = reinterpret_cast<float *>(w);   w += al(chunk * kHeadIn * 4);
    float *z = reinterpret_cast<float *>(w);
    const float *r = net->rounded, *b = net->master;
    const int cap = 8 * (plan->sm_count > 0 ? plan->sm_count : 1);     // 8 CTAs per SM at most
    auto gcap = [&](long long work, int threads) { int g = grid_for(work, threads); return g < cap ? g : cap; };
    image_input_kernel<<<gcap((long long)P, 256), 256, 0, s>>>(lr, (long long)lr_pitch, plan->d_masks, lr_h, lr_w, x);
    ConvGeom g1{1, 5, lr_h, lr_w, lr_h, lr_w, 1, 1, nullptr, lr_h, lr_w};
    conv_fwd_kernel<5><<<gcap((long long)P, 128), 128, 0, s>>>(x, r + kW1, b + kB1, a1, g1);
    // conv2 (stride 2, onto the block grid) and conv3 on the tensor cores
    int cst = conv_tc(a1, r + kW2, b + kB2, a2, lr_h, lr_w, nbh, nbw, 2, plan->sm_count, plan->d_status, s);
    if (cst == RLJSDE_OK)
        cst = conv_tc(a2, r + kW3, b + kB3, a3, nbh, nbw, nbh, nbw, 1, plan->sm_count, plan->d_status, s);
    if (cst != RLJSDE_OK) return cst;
    for (size_t b0 = 0; b0 < nb; b0 += chunk) {
        const int m = (int)(nb - b0 < chunk ? nb - b0 : chunk);
        head_features_f32_kernel<<<gcap((long long)m * kHeadIn, 256), 256, 0, s>>>(a3, nbh, nbw, (long long)b0, m, f);
        dim3 gg((kOut + 63) / 64, (m + 63) / 64);
        gemm_kernel<<<gg, 256, 0, s>>>(m, kOut, kHeadIn, f, kHeadIn, 1, r + kWh, 1, kHeadIn, z, kOut, 0.f);
        shortlist_kernel<<<gcap(((long long)m + 7) / 8 * 256, 256), 256, 0, s>>>(
            z, kOut, b + kBh, (long long)b0, m, static_cast<Shortlist *>(shortlists));
    }
    return cudaGetLastError() == cudaSuccess ? RLJSDE_OK : RLJSDE_ERR_CUDA;
}

}  // extern "C"
