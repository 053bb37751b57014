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
#include <cuda.h>                 // CUtensorMap (the encoder is fetched through the runtime)
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
constexpr int kOut = 1026;      // 1024 candidate logits, iteration output, gate
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

// conv1 over a whole image, straight from the measurements: out[P][Q][co]
// (bfloat16, channels innermost) = relu(b[co] + sum over the 3x3 taps of
// w[co][0][t] y/3 + w[co][1 + code][t]), the one-hot code input reduced to
// the one weight its code selects; taps outside the image contribute
// nothing.  FP32 arithmetic on the bfloat16-rounded weights; the output is
// rounded to bfloat16, the precision conv2 reads it at.  Each thread
// computes all 32 channels of one position, weights read four channels at a
// time from shared memory.
__global__ void __launch_bounds__(128, 4) conv1_image_kernel(const float *lr, long long lr_pitch, const uint8_t *mask,
                                                          int lr_h, int lr_w, const float *w, const float *b,
                                                          __nv_bfloat16 *out)
{
    __shared__ float4 wt[5][9][kC / 4];          // [input channel][tap][output channels 4j .. 4j + 3]
    __shared__ float bs[kC];
    for (int i = threadIdx.x; i < 5 * 9 * kC; i += blockDim.x) {
        const int ci = i / (9 * kC), t = (i / kC) % 9, co = i % kC;
        reinterpret_cast<float *>(&wt[ci][t][0])[co] = w[(co * 5 + ci) * 9 + t];
    }
    for (int i = threadIdx.x; i < kC; i += blockDim.x) bs[i] = b[i];
    __syncthreads();
    const long long plane = (long long)lr_h * lr_w;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < plane;
         i += (long long)gridDim.x * blockDim.x) {
        const int P = (int)(i / lr_w), Q = (int)(i % lr_w);
        float acc[kC];
#pragma unroll
        for (int co = 0; co < kC; ++co) acc[co] = bs[co];
#pragma unroll 1
        for (int t = 0; t < 9; ++t) {
            const int y = P + t / 3 - 1, x = Q + t % 3 - 1;
            if (y < 0 || y >= lr_h || x < 0 || x >= lr_w) continue;
            const float yv = lr[(long long)y * lr_pitch + x];
            const float v = isfinite(yv) ? yv / 3.0f : 0.f;
            const int code = mask[(long long)y * lr_w + x] & 3;
#pragma unroll
            for (int j = 0; j < kC / 4; ++j) {
                const float4 a = wt[0][t][j], c = wt[1 + code][t][j];
                acc[4 * j] = fmaf(a.x, v, acc[4 * j]) + c.x;
                acc[4 * j + 1] = fmaf(a.y, v, acc[4 * j + 1]) + c.y;
                acc[4 * j + 2] = fmaf(a.z, v, acc[4 * j + 2]) + c.z;
                acc[4 * j + 3] = fmaf(a.w, v, acc[4 * j + 3]) + c.w;
            }
        }
        uint4 *dst = reinterpret_cast<uint4 *>(out + i * kC);
#pragma unroll
        for (int cg = 0; cg < 4; ++cg) {
            uint4 u;
            uint32_t *pu = reinterpret_cast<uint32_t *>(&u);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(fmaxf(acc[cg * 8 + 2 * e], 0.f)));
                const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(fmaxf(acc[cg * 8 + 2 * e + 1], 0.f)));
                pu[e] = lo | (hi << 16);
            }
            dst[cg] = u;
        }
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

// Order-preserving unsigned image of a float.
__device__ __forceinline__ uint32_t order_key(float v)
{
    const uint32_t u = __float_as_uint(v);
    return u ^ ((uint32_t)((int32_t)u >> 31) | 0x80000000u);
}

// Loss (mean over samples) and its gradient w.r.t. z = logits (+bias added
// here).  Per sample (one CTA of 256 threads):
//   candidates k < 1024: logistic loss, positives weighted pos_w, / 1024;
//   row 1024 (iteration output): nu_w (z - nu_t)^2;
//   row 1025 (gate), if mass is given: gate_w (sigmoid(z) - s)^2 with s the
//   share of the sample's mass (the plain loop's |gamma delta| per candidate)
//   that falls outside the network's own 64 largest logits; s is a target,
//   not differentiated.  Candidates tied with the 64th largest count as in.
__global__ void __launch_bounds__(256) loss_kernel(float *z, const float *bias, const uint8_t *t, const float *nu_t,
                                                   const float *mass, int n, float pos_w, float nu_w, float gate_w,
                                                   float *gz, float *loss)
{
    const int s = blockIdx.x;
    if (s >= n) return;
    __shared__ float red[256];
    __shared__ float red2[256];
    float l = 0.f;
    float *zs = z + (size_t)s * kOut;
    for (int k = threadIdx.x; k < kOut; k += blockDim.x) {
        const float zk = zs[k] + bias[k];
        zs[k] = zk;
        if (k < 1024) {
            const float tk = t[(size_t)s * 1024 + k] ? 1.f : 0.f;
            const float w = tk > 0.5f ? pos_w : 1.f;
            const float sp = fmaxf(zk, 0.f) + log1pf(expf(-fabsf(zk)));
            l += w * (sp - tk * zk) / 1024.f;
            gz[(size_t)s * kOut + k] = w * (1.f / (1.f + expf(-zk)) - tk) / 1024.f / n;
        } else if (k == 1024) {
            const float d = zk - nu_t[s];
            l += nu_w * d * d;
            gz[(size_t)s * kOut + k] = 2.f * nu_w * d / n;
        }
    }
    __syncthreads();
    float gg = 0.f;
    if (mass != nullptr) {
        // 64th largest candidate logit by bisection on the order keys
        uint32_t key[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) key[j] = order_key(zs[threadIdx.x + 256 * j]);
        uint32_t thr = 0;
        for (int bit = 31; bit >= 0; --bit) {
            const uint32_t cand = thr | (1u << bit);
            int c = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) c += key[j] >= cand;
            red[threadIdx.x] = (float)c;
            __syncthreads();
            for (int o = 128; o > 0; o >>= 1) {
                if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
                __syncthreads();
            }
            if (red[0] >= (float)kShortlist) thr = cand;
            __syncthreads();
        }
        float out_m = 0.f, all_m = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float m = mass[(size_t)s * 1024 + threadIdx.x + 256 * j];
            all_m += m;
            if (key[j] < thr) out_m += m;
        }
        red[threadIdx.x] = out_m;
        red2[threadIdx.x] = all_m;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (threadIdx.x < o) {
                red[threadIdx.x] += red[threadIdx.x + o];
                red2[threadIdx.x] += red2[threadIdx.x + o];
            }
            __syncthreads();
        }
        const float share = red2[0] > 0.f ? red[0] / red2[0] : 0.f;
        __syncthreads();
        if (threadIdx.x == 0) {
            const float sg = 1.f / (1.f + expf(-zs[1025]));
            const float d = sg - share;
            gg = gate_w * d * d;
            gz[(size_t)s * kOut + 1025] = 2.f * gate_w * d * sg * (1.f - sg) / n;
        }
    } else if (threadIdx.x == 0) {
        gz[(size_t)s * kOut + 1025] = 0.f;
    }
    red[threadIdx.x] = l + gg;
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
// Implicit-GEMM 3x3 convolution (pad 1, stride 1 or 2) of 32 bfloat16
// channels on the tensor cores.  A tile is 128 consecutive output positions
// of one output row (MMA M).  The 3 input rows it reads (3 x 130 or 3 x 260
// positions x 32 channels) come into shared memory by TMA (tiled tensor
// copies; positions outside the image read as zeros), double-buffered so that
// the next tile's rows load while this tile computes; four producer warps
// lay the 288 taps x channels of every position out as K-major core matrices
// (the A operand) from shared memory, one thread issues 18 MMAs (K 16) into
// one of two 32-column accumulators, and four epilogue warps read the
// previous tile's accumulator back, add the bias, apply ReLU and store
// bfloat16 meanwhile.
constexpr int kM = 128;                              // output positions per tile (MMA M)
constexpr int kKTot = 9 * kC;                        // 288
constexpr uint32_t kLBO = 128;                       // next 8-element K group
constexpr uint32_t kSBO = (kKTot / 8) * 128;         // next 8-row group: 4608
constexpr uint32_t kABytes = (kM / 8) * kSBO;        // 73,728
constexpr uint32_t kBBytes = (kC / 8) * kSBO;        // 18,432
constexpr int kBoxCols = 130;                        // input positions per TMA box (one row)
constexpr uint32_t kBoxBytes = kBoxCols * kC * 2;    // 8,320
constexpr uint32_t kStripBytes = 3 * 2 * kBoxBytes;  // 3 rows of 2 boxes (stride 2): 49,920
constexpr uint32_t kOffStrip = kABytes + kBBytes;    // 92,160
constexpr uint32_t kOffBar = kOffStrip + 2 * kStripBytes;
constexpr uint32_t kSmem = kOffBar + 64 + 128;       // 6 mbarriers, tensor-memory address; 128 B for alignment
static_assert(kSmem <= 227 * 1024, "tile operands must fit in shared memory");
static_assert(kOffStrip % 128 == 0 && kBoxBytes % 128 == 0 && kStripBytes % 128 == 0, "TMA destinations");
// D FP32, A and B BF16, both K-major, N = 32, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kC >> 3) << 17) |
                            ((uint32_t)(kM >> 4) << 24);
constexpr uint32_t kTmemCols = 64;                   // two 32-column accumulators

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

// B of conv2 / conv3 once per weight change: w [32][32][9] (bfloat16-rounded
// FP32) as bfloat16 core matrices (row = output channel, K group q = tap
// q / 4, input channels 8 (q % 4) ..), kBBytes each.
__global__ void pack_conv_kernel(const float *w, unsigned char *dst)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kC * (kKTot / 8)) return;
    const int co = i / (kKTot / 8), q = i % (kKTot / 8);
    const int t = q >> 2, ci0 = (q & 3) * 8;
    const float *src = w + (co * kC + ci0) * 9 + t;          // w[co][ci][t]
    uint4 v;
    v.x = pack_bf16(src[0], src[9]); v.y = pack_bf16(src[18], src[27]);
    v.z = pack_bf16(src[36], src[45]); v.w = pack_bf16(src[54], src[63]);
    *reinterpret_cast<uint4 *>(dst + (co >> 3) * kSBO + q * kLBO + (co & 7) * 16) = v;
}

// The 3 input rows of tile (oy, ox0) into the strip at `dst`: per row one
// box of 130 positions (stride 1) or two (stride 2), starting one position
// left of the first tap; completes on `bar` with the boxes' bytes.
__device__ __forceinline__ void load_strip(const CUtensorMap *tm, uint32_t dst, uint32_t bar, int stride, int oy,
                                           int ox0)
{
    const uint32_t row_bytes = (uint32_t)stride * kBoxBytes;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(3u * row_bytes)
                 : "memory");
    const int iy0 = stride * oy - 1, ix0 = stride * ox0 - 1;
    for (int r = 0; r < 3; ++r)
        for (int part = 0; part < stride; ++part)
            asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                         " [%0], [%1, {%2, %3, %4}], [%5];"
                         ::"r"(dst + r * row_bytes + part * kBoxBytes), "l"(reinterpret_cast<uint64_t>(tm)),
                         "r"(0), "r"(ix0 + part * kBoxCols), "r"(iy0 + r), "r"(bar)
                         : "memory");
}

// Producer-group and epilogue-group agreement: a named barrier over the
// group's 128 threads that also ORs a failure flag, so that every thread of
// the group leaves its loop at the same tile.
__device__ __forceinline__ bool group_or(const int id, const bool v)
{
    uint32_t r;
    asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, 128, p;\n"
                 " selp.u32 %0, 1, 0, q;\n}"
                 : "=r"(r)
                 : "r"((uint32_t)v), "r"(id)
                 : "memory");
    return r != 0;
}

// in (through tmap): [hi][wi][32] bfloat16; out: [ho][wo][32] bfloat16
// (relu(acc + b) rounded); bpack: pack_conv_kernel's B; b: [32].
// Warps 0-3 build A and issue the MMAs (thread 0 also the strip loads);
// warps 4-7 read the accumulators back and store, one tile behind, from the
// other of two 32-column accumulators.
__global__ void __launch_bounds__(256, 1) conv_tc_kernel(const __grid_constant__ CUtensorMap tmap,
                                                         const unsigned char *bpack, const float *bias,
                                                         __nv_bfloat16 *out, int ho, int wo, int stride, int *status)
{
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    // TMA destinations want 128-byte alignment
    unsigned char *sm = sm_raw + ((128u - (saddr(sm_raw) & 127u)) & 127u);
    unsigned char *B = sm + kABytes;
    // mbarriers: strip full x 2, accumulator full x 2 (MMA commit), accumulator empty x 2 (128 arrivals)
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + kOffBar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + kOffBar + 48);
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t a_addr = saddr(sm), b_addr = saddr(B), strip_addr = saddr(sm + kOffStrip);
    const uint32_t full_bar0 = saddr(&bars[0]), accf_bar0 = saddr(&bars[2]), acce_bar0 = saddr(&bars[4]);
    const int tiles_per_row = (wo + kM - 1) / kM;
    const long long n_tiles = (long long)ho * tiles_per_row;

    if (tid == 0) {
        for (int i = 0; i < 4; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bars[i])) : "memory");
        for (int i = 4; i < 6; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(saddr(&bars[i])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // the first two tiles' rows
        for (int k = 0; k < 2; ++k) {
            const long long tile = blockIdx.x + (long long)k * gridDim.x;
            if (tile < n_tiles)
                load_strip(&tmap, strip_addr + k * kStripBytes, full_bar0 + 8 * k, stride,
                           (int)(tile / tiles_per_row), (int)(tile % tiles_per_row) * kM);
        }
    }
    // B: the packed weights, 18,432 bytes
    for (int i = tid; i < (int)(kBBytes / 16); i += blockDim.x)
        reinterpret_cast<uint4 *>(B)[i] = reinterpret_cast<const uint4 *>(bpack)[i];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tslot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");     // B, written by threads, read by the MMAs
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    bool failed = false;

    if (warp < 4) {
        // ---- producers: A from the strip, the MMAs, the strip loads
        uint32_t pending = (blockIdx.x < n_tiles ? 1u : 0u) |
                           (blockIdx.x + (long long)gridDim.x < n_tiles ? 2u : 0u);   // strip loads in flight
        uint32_t full_parity = 0, accf_parity = 0, acce_parity = 0;
        bool mma_in_flight = false;                   // the last tile's MMAs may still read A
        int n = 0;                                    // tiles done by this CTA
        const uint32_t row_bytes = (uint32_t)stride * kBoxBytes;
        for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++n) {
            const int k = n & 1, b = n & 1;           // strip and accumulator of this tile
            const int p = tid;
            // this tile's rows, and A free (the previous tile's MMAs done)
            bool ok = wait_phase(full_bar0 + 8 * k, (full_parity >> k) & 1u);
            if (ok && n > 0) {
                ok = wait_phase(accf_bar0 + 8 * (b ^ 1), (accf_parity >> (b ^ 1)) & 1u);
                if (ok) { accf_parity ^= 1u << (b ^ 1); mma_in_flight = false; }
            }
            if (group_or(1, !ok)) { failed = true; break; }
            full_parity ^= 1u << k;
            pending &= ~(1u << k);
            const uint32_t srow = strip_addr + k * kStripBytes + (uint32_t)(stride * p) * (kC * 2);
            const uint32_t arow = a_addr + (p >> 3) * kSBO + (p & 7) * 16;
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const uint32_t src = srow + (t / 3) * row_bytes + (t % 3) * (kC * 2);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int cg = (i + p) & 3;      // rotated: the quarter-warp's reads in distinct bank groups
                    uint4 u;
                    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                                 : "=r"(u.x), "=r"(u.y), "=r"(u.z), "=r"(u.w) : "r"(src + cg * 16));
                    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};"
                                 ::"r"(arow + (uint32_t)(t * 4 + cg) * kLBO), "r"(u.x), "r"(u.y), "r"(u.z),
                                 "r"(u.w)
                                 : "memory");
                }
            }
            // the accumulator of this tile free (its epilogue two tiles back done)
            ok = true;
            if (n >= 2) {
                ok = wait_phase(acce_bar0 + 8 * b, (acce_parity >> b) & 1u);
                if (ok) acce_parity ^= 1u << b;
            }
            // generic-proxy writes -> tensor-core (async proxy) reads
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            if (group_or(1, !ok)) { failed = true; break; }   // also: A complete, strip k consumed
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const long long nxt = tile + 2ll * gridDim.x;    // into the strip just consumed
            if (nxt < n_tiles) pending |= 1u << k;
            mma_in_flight = true;
            if (tid == 0) {
                if (nxt < n_tiles)
                    load_strip(&tmap, strip_addr + k * kStripBytes, full_bar0 + 8 * k, stride,
                               (int)(nxt / tiles_per_row), (int)(nxt % tiles_per_row) * kM);
                const uint32_t d = tmem + (uint32_t)b * 32u;
#pragma unroll
                for (int j = 0; j < kKTot / 16; ++j) {
                    const uint64_t da = desc(a_addr + j * 2 * kLBO), db = desc(b_addr + j * 2 * kLBO);
                    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                                 ::"r"(d), "l"(da), "l"(db), "r"(kIdesc), "r"(j)
                                 : "memory");
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(accf_bar0 + 8 * b)
                             : "memory");
            }
        }
        if (failed) {
            if (tid == 0) atomicOr(status, 2);
            // let copies and MMAs still in flight land before the shared memory goes away
            for (int k = 0; k < 2; ++k)
                if ((pending >> k) & 1u) wait_phase(full_bar0 + 8 * k, (full_parity >> k) & 1u);
            if (mma_in_flight) {                      // the previous tile's MMAs, into the other accumulator
                const int b = (n & 1) ^ 1;
                wait_phase(accf_bar0 + 8 * b, (accf_parity >> b) & 1u);
            }
        }
    } else {
        // ---- epilogue: accumulator rows 32 (warp - 4) .. of each tile, one tile behind
        const int q = warp - 4, row = q * 32 + (tid & 31);
        float bv[kC];
#pragma unroll
        for (int c = 0; c < kC; ++c) bv[c] = bias[c];
        uint32_t accf_parity = 0;
        int n = 0;
        for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++n) {
            const int b = n & 1;
            const bool ok = wait_phase(accf_bar0 + 8 * b, (accf_parity >> b) & 1u);
            if (group_or(2, !ok)) { failed = true; break; }
            accf_parity ^= 1u << b;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint32_t r[32];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                         : "r"(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)b * 32u)
                         : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(acce_bar0 + 8 * b) : "memory");
            const int oy = (int)(tile / tiles_per_row), ox = (int)(tile % tiles_per_row) * kM + row;
            if (ox < wo) {
                uint4 *dst = reinterpret_cast<uint4 *>(out + ((long long)oy * wo + ox) * kC);
#pragma unroll
                for (int cg = 0; cg < 4; ++cg) {
                    float v[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) v[e] = fmaxf(__uint_as_float(r[cg * 8 + e]) + bv[cg * 8 + e], 0.f);
                    uint4 u;
                    u.x = pack_bf16(v[0], v[1]); u.y = pack_bf16(v[2], v[3]);
                    u.z = pack_bf16(v[4], v[5]); u.w = pack_bf16(v[6], v[7]);
                    dst[cg] = u;
                }
            }
        }
        if (failed && (tid & 127) == 0) atomicOr(status, 2);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}
}  // namespace tc

// ------------------------------------------ fused head and shortlist --
// The head and the top-64 selection of the whole-image pass in one kernel on
// the 5th-gen tensor cores.  Per tile of 128 consecutive blocks:
//   - four gather warps copy each block's 3x3 block-grid neighbourhood of
//     conv3 (288 bfloat16 features, K index t * 32 + ci as in conv_tc_kernel)
//     into shared memory as the A operand;
//   - one issuer thread streams the head weights (bfloat16, pre-packed in the
//     core-matrix layout, 64 rows per chunk) through two shared-memory slots
//     with bulk copies and issues, per chunk, 18 tcgen05.mma (M 128, N 64,
//     K 16) into one of two 64-column accumulators in tensor memory (an
//     M 128 MMA costs about the same whatever its N up to 64, so wider chunks
//     mean fewer of them and fewer hand-overs);
//   - eight consumer warps (two per tensor-memory lane quadrant, one block
//     per lane) read each chunk's logits, add the bias, and keep only a
//     15-bit ranking key per candidate: the logit on a fixed-point grid of
//     step 2^-9 over [-32, 32).  Two keys share a 32-bit word; twelve
//     chunks' go back into tensor memory (columns 0..383), four chunks' into
//     shared memory.
// Once a tile's logits are in, each block's 64th largest key is found by a
// safeguarded interpolation search over the key range, starting from the
// bracket given by the second-largest keys of each group of 32 candidates;
// the two warps of a lane quadrant count one half of the candidates each
// (eight packed keys per popc) and add their counts through shared memory.
// The candidates above it plus, of those equal to it, the lowest indices form
// the shortlist.  The 1024 x 4-byte logits of a block never leave the SM.
// The iteration output (head row 1024) and the gate (row 1025, whose sigmoid
// is the predicted share of the plain loop's coefficient mass the shortlist
// leaves out) are kept in FP32.
//
// Waits are bounded (about 2 s each); a wait that gives up sets bit 2 of the
// status word, makes the other roles leave their loops, and the CTA drains
// its copies and tensor-core work in flight before freeing tensor memory.
namespace hd {
constexpr int kM = 128;                                   // blocks per tile (MMA M, tensor-memory lanes)
constexpr int kNC = 64;                                   // candidates per chunk (MMA N)
constexpr int kChunks = 1024 / kNC;                       // 16 candidate chunks
constexpr int kChunksPerTile = kChunks + 1;               // + head rows 1024..1039 (N = 16)
constexpr int kKeyWords = kNC / 2;                        // 32 words of two 16-bit keys per chunk
constexpr int kHalfChunks = kChunks / 2;                  // 8 chunks (512 candidates) per half
constexpr int kHalfTmemChunks = 6;                        // per half: chunks whose keys stay in tensor memory
constexpr uint32_t kHalfTmemWords = kHalfTmemChunks * kKeyWords;   // 192
constexpr uint32_t kAccCol = 2 * kHalfTmemWords;          // 384: accumulators at 384 and 448
constexpr uint32_t kTmemCols = 512;
constexpr int kHalfSmemWords = (kHalfChunks - kHalfTmemChunks) * kKeyWords;   // per half: two chunks' keys, 64 words
constexpr int kSmemKeyStride = 2 * kHalfSmemWords + 1;    // 129: rows start in distinct banks
constexpr uint32_t kGuard = 0x80008000u;                  // bit 15 of both key halves
constexpr uint32_t kLBO = 128, kSBO = (kHeadIn / 8) * 128;              // 4608
constexpr uint32_t kABytes = (kM / 8) * kSBO;                           // 73,728
constexpr uint32_t kBChunkBytes = (kNC / 8) * kSBO;                     // 36,864
constexpr uint32_t kBExtraBytes = 2 * kSBO;                             // 9,216: 16 rows
constexpr uint32_t kPackedBytes = kChunks * kBChunkBytes + kBExtraBytes; // 599,040
constexpr int kSlots = 2;                                 // weight ring: the chunk multiplied and the next
constexpr int kBias = 1040;
constexpr uint32_t kOffB = kABytes;
constexpr uint32_t kOffKeys = kOffB + kSlots * kBChunkBytes;
constexpr uint32_t kOffBias = kOffKeys + kM * kSmemKeyStride * 4;
constexpr uint32_t kOffX = kOffBias + kBias * 4;                        // consumer exchange: 8 x 2 x 128 ints
constexpr uint32_t kOffBar = kOffX + 8 * 2 * kM * 4;
// barriers: a_full, a_free, b_full[4], b_empty[4], acc_full[2], acc_empty[2]
constexpr int kBarAFull = 0, kBarAFree = 1, kBarBFull = 2, kBarBEmpty = 2 + kSlots, kBarAccFull = 2 + 2 * kSlots,
              kBarAccEmpty = kBarAccFull + 2, kBarPair = kBarAccEmpty + 2, kNumBars = kBarPair + 4;
constexpr uint32_t kOffMisc = kOffBar + kNumBars * 8;     // tensor-memory address, abort flag
constexpr uint32_t kSmem = kOffMisc + 16;
static_assert(kSmem <= 227 * 1024, "fused head operands must fit in shared memory");
static_assert(kOffB % 128 == 0 && kOffKeys % 16 == 0 && kOffBias % 16 == 0 && kOffX % 16 == 0 && kOffBar % 8 == 0,
              "alignment");
constexpr int kSet = 128;                                 // consumer threads per set (four warps, one per lane quadrant)
constexpr int kConsumers = 2 * kSet, kGatherers = 128;
constexpr int kThreads = kConsumers + kGatherers + 32;    // + the issuer warp: 416

// D FP32, A and B bfloat16, both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
}

__device__ __forceinline__ uint64_t sdesc(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(kLBO >> 4) << 16) | ((uint64_t)(kSBO >> 4) << 32) |
           (1ull << 46);                              // descriptor version 1, no swizzle
}

// Wait for phase `parity` of a shared-memory mbarrier; give up after about
// 2 s, or as soon as another role has raised the abort flag.
__device__ __forceinline__ bool wait(uint32_t bar, uint32_t parity, volatile int *abort)
{
    const uint64_t t0 = tc::now_ns();
    for (uint32_t i = 0; i < (1u << 26); ++i) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (done) return true;
        if ((i & 255) == 255 && (*abort || tc::now_ns() - t0 > 2000000000ull)) return false;
    }
    return false;
}

__device__ __forceinline__ void arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// the same without waiting: tensor-memory loads in flight until wait_ld()
__device__ __forceinline__ void ld32_nw(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr)
                 : "memory");
}
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void ld2(uint32_t taddr, uint32_t &r0, uint32_t &r1)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(taddr) : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void st32(uint32_t taddr, const uint32_t (&r)[32])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};"
                 ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
                 "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
                 "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
                 "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
                 : "memory");
}


// 15-bit ranking key of a logit: z on a fixed-point grid of step 2^-9 over
// [-32, 32), rounded down and clamped (NaN to 0), so keys order like the
// logits up to that step.  Stored with bit 15 set (a guard bit, see
// count_half).
__device__ __forceinline__ uint32_t key15(float z)
{
    // fmaf(z, 512, 16384) rounds 512 (z + 32) once, which equals (z + 32) * 512
    // in FP32: scaling by a power of two commutes with the rounding
    const float t = fminf(fmaxf(fmaf(z, 512.f, 16384.f), 0.f), 32767.f);
    return __float2uint_rd(t);
}


// Sum over 8 key words of the halves >= cand.  Every half holds key | 0x8000,
// so w - (cand | cand << 16) borrows in neither half (cand < 0x8000) and
// leaves bit 15 (bit 31) set iff the low (high) key is >= cand; the eight
// words' flag bits are shifted into distinct positions and counted at once.
__device__ __forceinline__ uint32_t count8(const uint32_t *w, uint32_t c2)
{
    uint32_t x = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) x |= ((w[i] - c2) >> i) & (kGuard >> i);
    return __popc(x);
}

// Keys >= cand in one half of this lane's block (all 32 lanes of the warp
// call it together: the tensor-memory loads are warp-collective).
__device__ __forceinline__ uint32_t count_half(uint32_t tcol, const uint32_t *skeys, uint32_t cand)
{
    const uint32_t c2 = cand | (cand << 16);
    uint32_t n0 = 0, n1 = 0, n2 = 0, n3 = 0;
    static_assert(kHalfTmemChunks % 2 == 0 && kHalfSmemWords == 64, "pairs of 32-column loads, 64 shared words");
#pragma unroll 1
    for (int i = 0; i < kHalfTmemChunks; i += 2) {   // two loads in flight
        uint32_t v[32], u[32];
        ld32_nw(tcol + 32 * i, v);
        ld32_nw(tcol + 32 * i + 32, u);
        wait_ld();
        n0 += count8(v, c2);
        n1 += count8(v + 8, c2);
        n2 += count8(v + 16, c2);
        n3 += count8(v + 24, c2);
        n0 += count8(u, c2);
        n1 += count8(u + 8, c2);
        n2 += count8(u + 16, c2);
        n3 += count8(u + 24, c2);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t t[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) t[j] = skeys[32 * h + j];
        n0 += count8(t, c2);
        n1 += count8(t + 8, c2);
        n2 += count8(t + 16, c2);
        n3 += count8(t + 24, c2);
    }
    return (n0 + n1) + (n2 + n3);
}

// a3: conv3 output [nbh][nbw][32] bfloat16; packed: head weights (see pack_head_kernel);
// bias: 1026 FP32; out: one Shortlist per block.
//
// Consumers: warp w (0..7) reads tensor-memory lane quadrant q = w % 4 (the
// blocks 32 q .. 32 q + 31 of a tile) and belongs to set s = w / 4.  Set s
// converts the chunks that land in accumulator s (every other chunk), and
// owns candidates 512 s .. 512 s + 511 for the selection: their keys sit in
// tensor-memory columns 192 s .. 192 s + 191 (chunks 8 s .. 8 s + 5) and
// shared-memory words 64 s .. 64 s + 63 of the block's row (the last two
// chunks of the half).  The two warps of a quadrant add their counts through
// shared memory and an mbarrier with a bounded wait, so both take the same
// search steps.
__global__ void __launch_bounds__(kThreads, 1) head_select_kernel(const __nv_bfloat16 *a3, int nbh, int nbw,
                                                                  const unsigned char *packed, const float *bias,
                                                                  Shortlist *out, int *status)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *A = sm;
    uint32_t *skeys_all = reinterpret_cast<uint32_t *>(sm + kOffKeys);
    float *bias_s = reinterpret_cast<float *>(sm + kOffBias);
    uint32_t *xch = reinterpret_cast<uint32_t *>(sm + kOffX);          // [8][2][128]
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + kOffMisc);
    volatile int *abort = reinterpret_cast<volatile int *>(sm + kOffMisc + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t bar0 = tc::saddr(sm + kOffBar);
    auto bar = [&](int i) { return bar0 + 8u * (uint32_t)i; };

    for (int i = tid; i < kBias; i += blockDim.x) bias_s[i] = i < kOut ? bias[i] : 0.f;
    if (tid == 0) {
        for (int i = 0; i < kNumBars; ++i) {
            const uint32_t count = i == kBarAFull ? kGatherers : i >= kBarPair ? 64u : i >= kBarAccEmpty ? kSet : 1u;
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(i)), "r"(count) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::saddr(tslot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const long long nb = (long long)nbh * nbw;
    const long long n_tiles = (nb + kM - 1) / kM;

    if (warp < 8) {
        // ------------------------------------------------ consumers --
        const int q = warp & 3, set = warp >> 2;
        const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16);
        const int r = 32 * q + lane;
        uint32_t *srow = skeys_all + r * kSmemKeyStride;
        auto X = [&](int slot, int s) -> uint32_t & { return xch[(slot * 2 + s) * kM + r]; };
        // The two warps of a quadrant meet on an mbarrier (64 arrivals per
        // phase) with a bounded wait, so a warp that leaves on a timeout makes
        // its partner time out too instead of blocking it.
        uint32_t pphase = 0;
        auto pair_sync = [&]() -> bool {
            arrive(bar(kBarPair + q));
            const bool got = wait(bar(kBarPair + q), pphase, abort);
            pphase ^= 1u;
            return __all_sync(0xffffffffu, got);
        };
        bool ok = true;
        long long it = 0;
        for (long long tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x, ++it) {
            const long long b = tile * kM + r;
            const bool valid = b < nb;
            uint32_t lo = 0x7FFFu, hi = 0;
            for (int c = 0; c < kChunksPerTile; ++c) {
                const long long g = it * kChunksPerTile + c;
                if ((int)(g & 1) != set) continue;                      // the other set's accumulator
                const bool got = wait(bar(kBarAccFull + set), (uint32_t)((g >> 1) & 1), abort);
                if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc = trow + kAccCol + (uint32_t)(kNC * set);
                if (c == kChunks) {
                    uint32_t v0, v1;
                    ld2(acc, v0, v1);
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    arrive(bar(kBarAccEmpty + set));
                    if (valid) {
                        out[b].nu_frac = __uint_as_float(v0) + bias_s[1024];
                        out[b].missing = 1.f / (1.f + __expf(-(__uint_as_float(v1) + bias_s[1025])));
                    }
                    continue;
                }
                uint32_t v[32], u[32];
                ld32_nw(acc, v);
                ld32_nw(acc + 32, u);
                wait_ld();
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                arrive(bar(kBarAccEmpty + set));
                // word j: the keys of candidates 64 c + j (low half) and 64 c + 32 + j
                // (high half); second-largest keys per group of 32 for the bracket
                uint32_t pk[32], a1 = 0, a2 = 0, b1 = 0, b2 = 0;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const uint32_t ka = key15(__uint_as_float(v[j]) + bias_s[kNC * c + j]);
                    const uint32_t kb = key15(__uint_as_float(u[j]) + bias_s[kNC * c + 32 + j]);
                    a2 = max(a2, min(a1, ka));
                    a1 = max(a1, ka);
                    b2 = max(b2, min(b1, kb));
                    b1 = max(b1, kb);
                    pk[j] = ka | (kb << 16) | kGuard;
                }
                lo = min(lo, min(a2, b2));
                hi = max(hi, max(a2, b2));
                const int h = c / kHalfChunks, cq = c % kHalfChunks;
                if (cq < kHalfTmemChunks) {
                    st32(trow + kHalfTmemWords * h + kKeyWords * cq, pk);
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j) srow[kHalfSmemWords * h + kKeyWords * (cq - kHalfTmemChunks) + j] = pk[j];
                }
            }
            if (!ok) break;
            // keys this set stored are read by the other set too: complete the
            // stores and order them before the barrier, the reads after it
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            // the bracket from both sets' chunks: 64 keys >= lo, the 64th largest <= hi
            X(0, set) = lo;
            X(1, set) = hi;
            if (!pair_sync()) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            lo = min(X(0, 0), X(0, 1));
            hi = max(X(1, 0), X(1, 1));
            const uint32_t tcol = trow + kHalfTmemWords * set;
            const uint32_t *shalf = srow + kHalfSmemWords * set;
            // The 64th largest key T: count(L) >= 64 > count(H) with L = lo, H = hi + 1
            // at the start.  Each step counts at x strictly inside (L, H): by
            // interpolating the two known counts when the last step at least
            // halved the interval, else at the midpoint (so at most about twice
            // the bisection's steps, usually far fewer); x becomes L or H.  It
            // ends when a count is exactly 64 (the keys >= x are the shortlist)
            // or H = L + 1 (then T = L).  Counts at L and H, total and lower
            // half, are kept for the tie rule.
            uint32_t L = lo, H = hi + 1u;
            int cL = -1, cH = -1, cL0 = 0, cH0 = 0;          // -1: not counted yet
            bool active = H > L + 1u, exact = false, halved = true;
            int step = 0;
            while (__any_sync(0xffffffffu, active)) {
                uint32_t x = 0u;
                if (active) {
                    x = (L + H) >> 1;
                    if (halved && cL >= 0 && cH >= 0 && cL > cH) {
                        const uint32_t num = (uint32_t)(cL - kShortlist) * (H - L) + (uint32_t)(cL - cH) / 2u;
                        x = L + num / (uint32_t)(cL - cH);
                        x = min(max(x, L + 1u), H - 1u);
                    }
                }
                const int slot = 2 + (step & 1);
                X(slot, set) = count_half(tcol, shalf, x);
                if (!pair_sync()) { ok = false; break; }
                const int c0 = (int)X(slot, 0), c = c0 + (int)X(slot, 1);
                ++step;
                if (active) {
                    const uint32_t width = H - L;
                    if (c >= kShortlist) { L = x; cL = c; cL0 = c0; }
                    else { H = x; cH = c; cH0 = c0; }
                    halved = 2u * (H - L) <= width;
                    if (c == kShortlist) { exact = true; active = false; }
                    else if (H == L + 1u) active = false;
                }
            }
            if (!ok) break;
            const uint32_t thr = L;
            // Exactly 64 keys >= thr: take them all, the lower half's first.
            // Otherwise thr is the 64th largest key: take the keys > thr, and of
            // those equal to it the lowest indices (the lower half's first).
            if (!__all_sync(0xffffffffu, exact || (cL >= 0 && cH >= 0))) {
                // an end of the bracket that was never counted: count both per half
                const uint32_t g1 = count_half(tcol, shalf, thr + 1u);
                const uint32_t g0 = count_half(tcol, shalf, thr);
                X(4, set) = g1;
                X(5, set) = g0;
                if (!pair_sync()) { ok = false; break; }
                if (!exact && (cL < 0 || cH < 0)) {
                    cH0 = (int)X(4, 0); cH = cH0 + (int)X(4, 1);
                    cL0 = (int)X(5, 0); cL = cL0 + (int)X(5, 1);
                }
            }
            int eq_left, pos;
            if (exact) {
                eq_left = kShortlist;
                pos = set == 0 ? 0 : cL0;
            } else {
                const int quota = kShortlist - cH;                  // keys > thr are cH
                const int take0 = min(cL0 - cH0, quota);            // the lower half's keys == thr first
                eq_left = set == 0 ? take0 : quota - take0;
                pos = set == 0 ? 0 : cH0 + take0;
            }
            Shortlist *sl = out + b;
            auto take = [&](uint32_t k, int idx) {
                const bool t = k > thr || (k == thr && eq_left > 0);
                if (t) {
                    if (k == thr) --eq_left;
                    if (valid && pos < kShortlist) sl->idx[pos] = (uint16_t)idx;
                    ++pos;
                }
            };
            const int base = 512 * set;
#pragma unroll 1
            for (int i = 0; i < kHalfTmemChunks; ++i) {
                uint32_t v[32];
                ld32(tcol + 32 * i, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) take(v[j] & 0x7FFFu, base + kNC * i + j);
#pragma unroll
                for (int j = 0; j < 32; ++j) take((v[j] >> 16) & 0x7FFFu, base + kNC * i + 32 + j);
            }
#pragma unroll 1
            for (int cq = kHalfTmemChunks; cq < kHalfChunks; ++cq) {
                const uint32_t *w = shalf + kKeyWords * (cq - kHalfTmemChunks);
                for (int j = 0; j < 32; ++j) take(w[j] & 0x7FFFu, base + kNC * cq + j);
                for (int j = 0; j < 32; ++j) take((w[j] >> 16) & 0x7FFFu, base + kNC * cq + 32 + j);
            }
            // every key of the tile is read before either set converts the next tile's chunks
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            if (!pair_sync()) { ok = false; break; }
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        if (!ok) *abort = 1;
    } else if (warp < 12) {
        // -------------------------------------------------- gatherers --
        const int p = tid - kConsumers;
        unsigned char *arow = A + (p >> 3) * kSBO + (p & 7) * 16;
        long long it = 0;
        for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++it) {
            if (it > 0 && !wait(bar(kBarAFree), (uint32_t)((it - 1) & 1), abort)) { *abort = 1; break; }
            const long long b = tile * kM + p;
            const bool valid = b < nb;
            const int by = valid ? (int)(b / nbw) : 0, bx = valid ? (int)(b - (long long)by * nbw) : 0;
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const int y = by + t / 3 - 1, x = bx + t % 3 - 1;
                const bool inb = valid && y >= 0 && y < nbh && x >= 0 && x < nbw;
                const uint4 *src = reinterpret_cast<const uint4 *>(a3 + (inb ? ((long long)y * nbw + x) * kC : 0));
#pragma unroll
                for (int cg = 0; cg < 4; ++cg) {
                    const uint4 u = inb ? src[cg] : make_uint4(0u, 0u, 0u, 0u);
                    *reinterpret_cast<uint4 *>(arow + (t * 4 + cg) * kLBO) = u;
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            arrive(bar(kBarAFull));
        }
    } else if (lane == 0) {
        // ----------------------------------------------------- issuer --
        const uint32_t a_addr = tc::saddr(A), b_addr = tc::saddr(sm + kOffB);
        auto chunk_src = [&](long long h) { return packed + (size_t)(h % kChunksPerTile) * kBChunkBytes; };
        auto chunk_bytes = [&](long long h) { return h % kChunksPerTile == kChunks ? kBExtraBytes : kBChunkBytes; };
        long long loaded = 0, waited = 0, g = 0, it = 0;
        bool ok = true;
        if (n_tiles > blockIdx.x) {
            bulk_load(b_addr, chunk_src(0), chunk_bytes(0), bar(kBarBFull));
            loaded = 1;
        }
        for (long long tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x, ++it) {
            if (!wait(bar(kBarAFull), (uint32_t)(it & 1), abort)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int c = 0; c < kChunksPerTile; ++c, ++g) {
                const int slot = (int)(g % kSlots), ab = (int)(g & 1);
                if (!wait(bar(kBarBFull + slot), (uint32_t)((g / kSlots) & 1), abort)) { ok = false; break; }
                waited = g + 1;
                if (g >= 2 && !wait(bar(kBarAccEmpty + ab), (uint32_t)(((g - 2) >> 1) & 1), abort)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + kAccCol + (uint32_t)(kNC * ab);
                const uint32_t id = idesc(c == kChunks ? 16 : kNC);
                // K step j starts 2 core matrices (256 bytes) further: +16 in the
                // descriptors' address field (addr >> 4, 14 bits: no carry out)
                const uint64_t da0 = sdesc(a_addr), db0 = sdesc(b_addr + (uint32_t)slot * kBChunkBytes);
#pragma unroll
                for (int j = 0; j < kHeadIn / 16; ++j)
                    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                                 ::"r"(d), "l"(da0 + (uint64_t)(16 * j)), "l"(db0 + (uint64_t)(16 * j)), "r"(id),
                                 "r"(j)
                                 : "memory");
                commit(bar(kBarAccFull + ab));
                commit(bar(kBarBEmpty + slot));
                if (c == kChunks) commit(bar(kBarAFree));
                // the next chunk goes into the other slot once the previous chunk's
                // multiply is done with it; it lands while this chunk multiplies
                const long long h = g + 1;
                if (h >= kSlots &&
                    !wait(bar(kBarBEmpty + (int)(h % kSlots)), (uint32_t)(((h - kSlots) / kSlots) & 1), abort)) {
                    ok = false;
                    ++g;
                    break;
                }
                bulk_load(b_addr + (uint32_t)(h % kSlots) * kBChunkBytes, chunk_src(h), chunk_bytes(h),
                          bar(kBarBFull + (int)(h % kSlots)));
                loaded = h + 1;
            }
        }
        if (!ok) *abort = 1;
        // drain: copies still in flight, then the last tensor-core work
        for (long long h = waited; h < loaded; ++h) {
            volatile int no_abort = 0;
            wait(bar(kBarBFull + (int)(h % kSlots)), (uint32_t)((h / kSlots) & 1), &no_abort);
        }
        if (g > 0) {
            volatile int no_abort = 0;
            wait(bar(kBarBEmpty + (int)((g - 1) % kSlots)), (uint32_t)(((g - 1) / kSlots) & 1), &no_abort);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0 && *abort) atomicOr(status, 2);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// Head weights (FP32 [1026][288], feature index ci * 9 + t) -> bfloat16 in
// the core-matrix layout of head_select_kernel: chunk c of 32 rows (the
// last one 16 rows: 1024..1039, zero beyond 1025), K index t * 32 + ci.
__global__ void pack_head_kernel(const float *wh, unsigned char *packed)
{
    const int total = (kChunks * kNC + 16) * kHeadIn;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int n = i / kHeadIn, k = i % kHeadIn;
        const int c = n / kNC, rl = n % kNC;
        const int t = k / kC, ci = k % kC;
        const float v = n < kOut ? wh[n * kHeadIn + ci * 9 + t] : 0.f;
        const size_t off = (size_t)c * kBChunkBytes + (rl >> 3) * kSBO + (k >> 3) * kLBO + (rl & 7) * 16 + (k & 7) * 2;
        *reinterpret_cast<__nv_bfloat16 *>(packed + off) = __float2bfloat16_rn(v);
    }
}
}  // namespace hd

// Fixed scratch of rljsde_propose_noalloc: part of the library image, so
// every device that loads the library holds it until the process exits.
constexpr size_t kStaticScratchBytes = 32u << 20;
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
    unsigned char *head_packed = nullptr;   // head weights for head_select_kernel (bfloat16, 599,040 B)
    unsigned char *conv_packed = nullptr;   // conv2 and conv3 weights for conv_tc_kernel (2 x 18,432 B)
    int step = 0;
    int sm_count = 1;                    // SMs of the device the network lives on
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

// cuTensorMapEncodeTiled, looked up once through the runtime (no link
// against the driver library).
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encode_tiled()
{
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    return fn;
}

// conv2 / conv3 of a whole image on the tensor cores (tc::conv_tc_kernel):
// in [hi][wi][32] bfloat16 (256-byte aligned), bpack the packed weights.
int conv_tc(const __nv_bfloat16 *in, const unsigned char *bpack, const float *b, __nv_bfloat16 *out, int hi, int wi,
            int ho, int wo, int stride, int sm_count, int *status, cudaStream_t s)
{
    const EncodeTiled enc = encode_tiled();
    if (!enc) return RLJSDE_ERR_CUDA;
    // the input as a 3-D tensor (channel, column, row), boxes of 130 positions of one row
    CUtensorMap tm;
    const cuuint64_t dims[3] = {(cuuint64_t)kC, (cuuint64_t)wi, (cuuint64_t)hi};
    const cuuint64_t strides[2] = {(cuuint64_t)kC * 2, (cuuint64_t)wi * kC * 2};
    const cuuint32_t box[3] = {(cuuint32_t)kC, (cuuint32_t)tc::kBoxCols, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16 *>(in), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return RLJSDE_ERR_CUDA;
    if (cudaFuncSetAttribute(tc::conv_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::kSmem) !=
        cudaSuccess)
        return RLJSDE_ERR_CUDA;
    const long long tiles = (long long)ho * ((wo + tc::kM - 1) / tc::kM);
    const long long cap = sm_count > 0 ? sm_count : 1;               // one 188 KB CTA per SM
    const int grid = (int)(tiles < cap ? (tiles > 0 ? tiles : 1) : cap);
    tc::conv_tc_kernel<<<grid, 256, tc::kSmem, s>>>(tm, bpack, b, out, ho, wo, stride, status);
    return cudaGetLastError() == cudaSuccess ? RLJSDE_OK : RLJSDE_ERR_CUDA;
}

void refresh_bf16(rljsde_net *n, cudaStream_t s)
{
    to_bf16_kernel<<<grid_for(kParams, 256), 256, 0, s>>>(n->master, n->w16, n->rounded, kParams);
    hd::pack_head_kernel<<<grid_for(1040 * kHeadIn, 256), 256, 0, s>>>(n->master + kWh, n->head_packed);
    tc::pack_conv_kernel<<<grid_for(kC * (tc::kKTot / 8), 128), 128, 0, s>>>(n->rounded + kW2, n->conv_packed);
    tc::pack_conv_kernel<<<grid_for(kC * (tc::kKTot / 8), 128), 128, 0, s>>>(n->rounded + kW3,
                                                                             n->conv_packed + tc::kBBytes);
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

// Device bytes of the whole-image pass: conv1 output on the L-pixel grid,
// conv2 and conv3 outputs on the block grid, each 32 bfloat16 channels per
// position (64 bytes), 256-byte aligned.
size_t propose_bytes(size_t P, size_t nb)
{
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    return al(P * kC * 2) + 2 * al(nb * kC * 2);
}

// The whole-image pass over `ws` (propose_bytes of it): conv1 on the CUDA
// cores straight from the measurements, conv2 and conv3 on the tensor cores,
// then the fused head and top-64 selection (hd::head_select_kernel), which
// writes the shortlists.  Activations are bfloat16 with channels innermost.
int propose_pass(const rljsde_plan_t *plan, const rljsde_net_t *net, const float *lr, size_t lr_pitch,
                 void *shortlists, void *ws, cudaStream_t s)
{
    const int lr_h = plan->lr_h[0], lr_w = plan->lr_w[0], nbh = lr_h / 2, nbw = lr_w / 2;
    const size_t P = (size_t)lr_h * lr_w, nb = (size_t)plan->n_blocks;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    char *w = static_cast<char *>(ws);
    __nv_bfloat16 *a1 = reinterpret_cast<__nv_bfloat16 *>(w);  w += al(P * kC * 2);
    __nv_bfloat16 *a2 = reinterpret_cast<__nv_bfloat16 *>(w);  w += al(nb * kC * 2);
    __nv_bfloat16 *a3 = reinterpret_cast<__nv_bfloat16 *>(w);
    const float *r = net->rounded, *b = net->master;
    const int sms = plan->sm_count > 0 ? plan->sm_count : 1;
    const int cap = 8 * sms;                                   // 8 CTAs per SM at most
    auto gcap = [&](long long work, int threads) { int g = grid_for(work, threads); return g < cap ? g : cap; };
    conv1_image_kernel<<<gcap((long long)P, 128), 128, 0, s>>>(lr, (long long)lr_pitch, plan->d_masks, lr_h, lr_w,
                                                               r + kW1, b + kB1, a1);
    // conv2 (stride 2, onto the block grid) and conv3 on the tensor cores
    int cst = conv_tc(a1, net->conv_packed, b + kB2, a2, lr_h, lr_w, nbh, nbw, 2, sms, plan->d_status, s);
    if (cst == RLJSDE_OK)
        cst = conv_tc(a2, net->conv_packed + tc::kBBytes, b + kB3, a3, nbh, nbw, nbh, nbw, 1, sms, plan->d_status, s);
    if (cst != RLJSDE_OK) return cst;
    if (cudaFuncSetAttribute(hd::head_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hd::kSmem) !=
        cudaSuccess)
        return RLJSDE_ERR_CUDA;
    const long long tiles = ((long long)nb + hd::kM - 1) / hd::kM;
    const int grid = (int)(tiles < sms ? tiles : sms);             // one CTA per SM (all of tensor memory)
    hd::head_select_kernel<<<grid, hd::kThreads, hd::kSmem, s>>>(a3, nbh, nbw, net->head_packed, b + kBh,
                                                                 static_cast<Shortlist *>(shortlists), plan->d_status);
    return cudaGetLastError() == cudaSuccess ? RLJSDE_OK : RLJSDE_ERR_CUDA;
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
              cudaMalloc(&n->head_packed, hd::kPackedBytes) == cudaSuccess &&
              cudaMalloc(&n->conv_packed, 2 * tc::kBBytes) == cudaSuccess;
    if (!ok) { rljsde_net_destroy(n); return RLJSDE_ERR_OUT_OF_MEMORY; }
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
    h[kBh + 1025] = -2.0f;                                   // gate: sigmoid(-2) = 0.12 of the mass left out
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
    cudaFree(n->head_packed);
    cudaFree(n->conv_packed);
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
                     const uint8_t *targets, const float *nu_t, const float *mass, float pos_w, float nu_w,
                     float gate_w, float *loss_host, cudaStream_t s)
{
    int st = ensure_train(net, n);
    if (st) return st;
    cudaMemcpyAsync(net->x, x, (size_t)n * 5 * 256 * 4, cudaMemcpyDeviceToDevice, s);
    origins_kernel<<<grid_for(n, 256), 256, 0, s>>>(reinterpret_cast<const int2 *>(blocks), net->origin, n);
    forward_patches(net, n, lr_h, lr_w, s);
    cudaMemsetAsync(net->loss, 0, 4, s);
    const float *r = net->rounded;
    loss_kernel<<<n, 256, 0, s>>>(net->z, net->master + kBh, targets, nu_t, mass, n, pos_w, nu_w, gate_w, net->gz,
                                  net->loss);
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
                        const uint8_t *targets, const float *nu_t, const float *mass, float pos_w, float nu_w,
                        float gate_w, float *grad_out, float *loss_host, void *stream)
{
    if (!net || !x || !blocks || !targets || !nu_t || n < 1) return RLJSDE_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int st = loss_grad(net, x, blocks, n, lr_h, lr_w, targets, nu_t, mass, pos_w, nu_w, gate_w, loss_host, s);
    if (st) return st;
    if (grad_out && cudaMemcpyAsync(grad_out, net->grad, (size_t)kParams * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return RLJSDE_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? RLJSDE_OK : RLJSDE_ERR_CUDA;
}

int rljsde_net_train_step(rljsde_net_t *net, const float *x, const int32_t *blocks, int n, int lr_h, int lr_w,
                          const uint8_t *targets, const float *nu_t, const float *mass, float pos_w, float nu_w,
                          float gate_w, float lr, float *loss_host, void *stream)
{
    if (!net || !x || !blocks || !targets || !nu_t || n < 1 || !(lr > 0.f)) return RLJSDE_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int st = loss_grad(net, x, blocks, n, lr_h, lr_w, targets, nu_t, mass, pos_w, nu_w, gate_w, loss_host, s);
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

// Logits (+bias) of n patches: z_out device [n][1026].
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
    return propose_bytes((size_t)plan->lr_h[0] * plan->lr_w[0], (size_t)plan->n_blocks);
}

int rljsde_propose(const rljsde_plan_t *plan, const rljsde_net_t *net, const float *lr, size_t lr_pitch,
                   void *shortlists, void *workspace, size_t ws_bytes, void *stream)
{
    if (!plan || !net || !lr || !shortlists || !workspace) return RLJSDE_ERR_INVALID_ARG;
    if (plan->n_images != 1 || lr_pitch < (size_t)plan->lr_w[0]) return RLJSDE_ERR_INVALID_ARG;
    if (plan->params.layout != RLJSDE_LAYOUT_THREE_QUARTER) return RLJSDE_ERR_UNSUPPORTED;   // opaque-code input
    if (ws_bytes < rljsde_propose_workspace(plan)) return RLJSDE_ERR_INVALID_ARG;
    return propose_pass(plan, net, lr, lr_pitch, shortlists, workspace, (cudaStream_t)stream);
}

// The proposal pass for callers that must not allocate device memory; see
// the header for who they are and for the size limit.
int rljsde_propose_noalloc(const rljsde_plan_t *plan, const rljsde_net_t *net, const float *lr, size_t lr_pitch,
                           void *shortlists, void *stream)
{
    if (!plan || !net || !lr || !shortlists) return RLJSDE_ERR_INVALID_ARG;
    if (plan->n_images != 1 || lr_pitch < (size_t)plan->lr_w[0]) return RLJSDE_ERR_INVALID_ARG;
    if (plan->params.layout != RLJSDE_LAYOUT_THREE_QUARTER) return RLJSDE_ERR_UNSUPPORTED;   // opaque-code input
    if (rljsde_propose_workspace(plan) > kStaticScratchBytes) return RLJSDE_ERR_BAD_SHAPE;   // too large for the fixed scratch
    void *base = nullptr;
    int st = static_scratch(&base);
    if (st) return st;
    return propose_pass(plan, net, lr, lr_pitch, shortlists, base, (cudaStream_t)stream);
}

}  // extern "C"
