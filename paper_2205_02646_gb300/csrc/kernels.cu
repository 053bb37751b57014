// CUDA (sm_103a) kernels of the RL-JSDE library and the C-ABI entry points
// that launch them.
//
// Recurrent path (Sec. IV, Eqs. 11-18), one warp per 4x4 target block:
//   1. gather the block's 16x16 L-pixel window, weight it by w_m (Eq. 8);
//   2. initial projected residual (Eq. 12 with r = y) in the factored form:
//      per opaque-quadrant type t, a 16x16 DFT
//          Y_t(kap) = sum_{m: t(m) = t} w_m y_m w16^-(p kap1 + q kap2),
//      from which R_k = sum_t conj(h_t(k)) Y_t(k mod 16);
//   3. nu_max iterations of: scores q_k |R_k|^2 / D_k and their argmax
//      (Eq. 11), delta = R_uv / D_uv (Eq. 16), c_uv += gamma delta (Eq. 15),
//      and the projected-residual update of Eq. 17, carried out on Y:
//          Y_t(kap) -= gamma delta h_t(uv) G_t((uv - kap) mod 16),
//      which is Eq. 17 with C factored as C_{k,l} = sum_t conj(h_t(k)) h_t(l)
//      G_t(l - k);
//   4. Eq. 18 on the central block, accumulated as each coefficient changes.
// A persistent CTA walks chunks of 8 blocks that share one table set; the
// table set of the next chunk of the same slot parity is brought into shared
// memory with a bulk asynchronous copy (cp.async.bulk + mbarrier) while the
// current chunk runs.
//
// Direct path (Sec. IV, Eqs. 4-10): one warp per block keeps the residual r
// and recomputes the O(W^4) projection of Eq. 10 every iteration.
#include <cuda_runtime.h>

#include <cstdint>

#include "rljsde_internal.h"

namespace rljsde {

namespace {

constexpr int kStatusNonfinite = 1;
constexpr int kStatusTimeout = 2;

// ---------------------------------------------------------------- complex --
template <typename T> struct C2 { T re, im; };

template <typename T> __device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b)
{
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T> __device__ __forceinline__ C2<T> cadd(C2<T> a, C2<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T> __device__ __forceinline__ C2<T> csub(C2<T> a, C2<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T> __device__ __forceinline__ C2<T> cconj(C2<T> a) { return {a.re, -a.im}; }

template <typename T> __device__ __forceinline__ Vec4<T> ld4(const Vec4<T> *p);
template <> __device__ __forceinline__ Vec4<float> ld4(const Vec4<float> *p)
{
    float4 v = *reinterpret_cast<const float4 *>(p);
    return {v.x, v.y, v.z, v.w};
}
template <> __device__ __forceinline__ Vec4<double> ld4(const Vec4<double> *p)
{
    double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    return {a.x, a.y, b.x, b.y};
}
template <typename T> __device__ __forceinline__ void st4(Vec4<T> *p, Vec4<T> v);
template <> __device__ __forceinline__ void st4(Vec4<float> *p, Vec4<float> v)
{
    *reinterpret_cast<float4 *>(p) = make_float4(v.x, v.y, v.z, v.w);
}
template <> __device__ __forceinline__ void st4(Vec4<double> *p, Vec4<double> v)
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(v.x, v.y);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v.z, v.w);
}

// ------------------------------------------------------- mbarrier / bulk --
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from
// global memory into shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for phase `parity` of `bar` to complete; give up after ~2 s.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t a = smem_addr(bar);
    const uint64_t t0 = global_ns();
    for (uint32_t i = 0; i < (1u << 24); ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if ((i & 255) == 255 && global_ns() - t0 > 2000000000ull) return false;
    }
    return false;
}

// ------------------------------------------------------------- arguments --
struct Args {
    const WorkEntry *entries;
    const uint32_t *chunk_table;
    int n_chunks;
    const unsigned char *records;
    uint32_t record_bytes;
    const Consts *consts;
    ImageDesc single;          // used when descs == nullptr
    const ImageDesc *descs;
    int nu_max;
    double gamma;
    uint16_t *trace_sel;       // [ordinal][nu_max], optional
    float *trace_dc;           // [ordinal][nu_max][2], optional
    int *status;
    // direct path only
    const uint8_t *masks;
    const long long *mask_offset;
    const float *q;
};

// Shared memory of the recurrent kernel.
template <typename T, int WARPS>
struct SmemLayout {
    static constexpr size_t rec = sizeof(Record<T>);
    static constexpr size_t scratch = 256 * 4 * sizeof(C2<T>);   // per warp
    static constexpr size_t off_slots = 0;
    static constexpr size_t off_scratch = 2 * rec;
    static constexpr size_t off_om = off_scratch + WARPS * scratch;       // 32 x C2<T>
    static constexpr size_t off_omc = off_om + 32 * sizeof(C2<T>);        // 32 x C2<T>
    static constexpr size_t off_w = off_omc + 32 * sizeof(C2<T>);         // 256 x T
    static constexpr size_t off_bar = off_w + 256 * sizeof(T);            // 2 x u64
    static constexpr size_t bytes = off_bar + 2 * sizeof(uint64_t);
};

// ------------------------------------------------------ one target block --
// Runs steps 1-4 for `we` with the tables in `rec`.  Whole warp.
template <typename T>
__device__ __forceinline__ void recurrent_block(const Args &a, const Record<T> &rec, C2<T> *scratch,
                                                const C2<T> *om, const C2<T> *omc, const T *wt,
                                                const WorkEntry we, const int lane)
{
    const ImageDesc img = a.descs ? a.descs[we.img] : a.single;
    const int p0 = 2 * we.bi - kOff / 2, q0 = 2 * we.bj - kOff / 2;
    __syncwarp();    // the previous block of this warp is done with the scratch

    // 1. gather: x(p, q) = w(p, q) y(p, q) into the plane of its type.
    Vec4<T> *x4 = reinterpret_cast<Vec4<T> *>(scratch);
    {
        const int p = lane >> 1, P = p0 + p;
        bool bad = false;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int q = (lane & 1) * 8 + j, Q = q0 + q;
            const int code = rec.types[p * 16 + q];
            T v = 0;
            if (code < 4 && P >= 0 && P < img.lr_h && Q >= 0 && Q < img.lr_w) {
                const float y = img.lr[(long long)P * img.lr_pitch + Q];
                if (isfinite(y)) v = wt[p * 16 + q] * (T)y;
                else bad = true;
            }
            Vec4<T> o = {code == 0 ? v : T(0), code == 1 ? v : T(0), code == 2 ? v : T(0), code == 3 ? v : T(0)};
            st4(&x4[p * 16 + q], o);
        }
        if (bad) atomicOr(a.status, kStatusNonfinite);
    }
    __syncwarp();

    const int k2 = lane & 15, h = lane >> 4;

    // 2a. row DFTs: T_t(p, k2) = sum_q x_t(p, q) w16^-(q k2), p in this half.
    C2<T> acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int t = 0; t < 4; ++t) acc[i][t] = {0, 0};
#pragma unroll 4
    for (int q = 0; q < 16; ++q) {
        const C2<T> tw = omc[(2 * q * k2) & 31];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const Vec4<T> x = ld4(&x4[(8 * h + i) * 16 + q]);
            acc[i][0].re += x.x * tw.re; acc[i][0].im += x.x * tw.im;
            acc[i][1].re += x.y * tw.re; acc[i][1].im += x.y * tw.im;
            acc[i][2].re += x.z * tw.re; acc[i][2].im += x.z * tw.im;
            acc[i][3].re += x.w * tw.re; acc[i][3].im += x.w * tw.im;
        }
    }
    __syncwarp();
    // Tbuf[p][k2] = 4 complex (t = 0..3), stored as two Vec4.
    Vec4<T> *tb = reinterpret_cast<Vec4<T> *>(scratch);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int p = 8 * h + i;
        st4(&tb[(p * 16 + k2) * 2 + 0], Vec4<T>{acc[i][0].re, acc[i][0].im, acc[i][1].re, acc[i][1].im});
        st4(&tb[(p * 16 + k2) * 2 + 1], Vec4<T>{acc[i][2].re, acc[i][2].im, acc[i][3].re, acc[i][3].im});
    }
    __syncwarp();

    // 2b. column DFTs, split by parity of p: half h sums p = 2j + h for
    // kap1' in [0, 8); then Y(kap1') = E + O and Y(kap1' + 8) = E - O.
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int t = 0; t < 4; ++t) acc[i][t] = {0, 0};
#pragma unroll 2
    for (int j = 0; j < 8; ++j) {
        const int p = 2 * j + h;
        const Vec4<T> t01 = ld4(&tb[(p * 16 + k2) * 2 + 0]);
        const Vec4<T> t23 = ld4(&tb[(p * 16 + k2) * 2 + 1]);
        const C2<T> tv[4] = {{t01.x, t01.y}, {t01.z, t01.w}, {t23.x, t23.y}, {t23.z, t23.w}};
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const C2<T> tw = omc[(2 * p * i) & 31];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                acc[i][t].re += tv[t].re * tw.re - tv[t].im * tw.im;
                acc[i][t].im += tv[t].re * tw.im + tv[t].im * tw.re;
            }
        }
    }
    C2<T> Y[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const T ore = __shfl_xor_sync(0xffffffffu, acc[i][t].re, 16);
            const T oim = __shfl_xor_sync(0xffffffffu, acc[i][t].im, 16);
            // h = 0 holds E and receives O: Y = E + O; h = 1 holds O: Y = E - O
            Y[i][t] = h == 0 ? C2<T>{acc[i][t].re + ore, acc[i][t].im + oim}
                             : C2<T>{ore - acc[i][t].re, oim - acc[i][t].im};
        }

    // 3. greedy loop on the factored projected residual.
    const C2<T> e1 = omc[k2];                       // exp(-2 pi i kap2 / 32)
    const T gamma = (T)a.gamma;
    const int eta = kOff + ((lane >> 2) & 3), gam = kOff + (lane & 3);
    T fpix = 0;                                     // Eq. 18 accumulator
    int u = 0, v = 0;
    C2<T> g[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    const bool tracing = a.trace_sel != nullptr;
    const long long trow = (long long)we.ord * a.nu_max;

    for (int it = 0; it < a.nu_max; ++it) {
        T bs0 = -1, bs1 = -1;
        int bk0 = 0, bk1 = 0;
        C2<T> bR0 = {0, 0}, bR1 = {0, 0};
        const int d2 = (v - k2) & 15;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int k1 = 8 * h + i;
            if (it > 0) {
                const int d = (((u - k1) & 15) << 4) | d2;
                const Vec4<T> G01 = ld4(&rec.G01[d]), G23 = ld4(&rec.G23[d]);
                Y[i][0] = csub(Y[i][0], cmul(g[0], C2<T>{G01.x, G01.y}));
                Y[i][1] = csub(Y[i][1], cmul(g[1], C2<T>{G01.z, G01.w}));
                Y[i][2] = csub(Y[i][2], cmul(g[2], C2<T>{G23.x, G23.y}));
                Y[i][3] = csub(Y[i][3], cmul(g[3], C2<T>{G23.z, G23.w}));
            }
            // R_k = sum_s conj(e_s(k)) Z_s, Z_s = S - Y_s, e = (1, w^k2, w^k1, w^(k1+k2))
            const C2<T> S = cadd(cadd(cadd(Y[i][0], Y[i][1]), Y[i][2]), Y[i][3]);
            const C2<T> Z0 = csub(S, Y[i][0]);
            const C2<T> U = cmul(e1, csub(S, Y[i][1]));
            const C2<T> V = cmul(omc[k1], csub(S, Y[i][2]));
            const C2<T> X = cmul(omc[(k1 + k2) & 31], csub(S, Y[i][3]));
            const C2<T> pp = cadd(Z0, U), mm = csub(Z0, U), ss = cadd(V, X), dd = csub(V, X);
            const C2<T> R00 = cadd(pp, ss), R01 = cadd(mm, dd), R10 = csub(pp, ss), R11 = csub(mm, dd);
            const Vec4<T> qd = ld4(&rec.qD[k1 * 16 + k2]);
            const T s00 = qd.x * (R00.re * R00.re + R00.im * R00.im);
            const T s01 = qd.y * (R01.re * R01.re + R01.im * R01.im);
            const T s10 = qd.z * (R10.re * R10.re + R10.im * R10.im);
            const T s11 = qd.w * (R11.re * R11.re + R11.im * R11.im);
            const int k = k1 * kW + k2;
            // visited in increasing k within each half a: strict > keeps the lowest index
            if (s00 > bs0) { bs0 = s00; bk0 = k; bR0 = R00; }
            if (s01 > bs0) { bs0 = s01; bk0 = k + 16; bR0 = R01; }
            if (s10 > bs1) { bs1 = s10; bk1 = k + 512; bR1 = R10; }
            if (s11 > bs1) { bs1 = s11; bk1 = k + 528; bR1 = R11; }
        }
        if (bs1 > bs0) { bs0 = bs1; bk0 = bk1; bR0 = bR1; }
        // warp argmax, ties to the lowest index
        T bs = bs0;
        int bk = bk0;
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) {
            const T os = __shfl_xor_sync(0xffffffffu, bs, m);
            const int ok = __shfl_xor_sync(0xffffffffu, bk, m);
            if (os > bs || (os == bs && ok < bk)) { bs = os; bk = ok; }
        }
        const int wl = (bk & 15) + ((bk >> 5) & 8) * 2;    // lane owning kap = (k1 & 15, k2 & 15)
        const T Rre = __shfl_sync(0xffffffffu, bR0.re, wl);
        const T Rim = __shfl_sync(0xffffffffu, bR0.im, wl);
        const T invD = rec.invD[bk];
        const C2<T> gd = {gamma * (Rre * invD), gamma * (Rim * invD)};   // gamma * delta
        u = bk >> 5;
        v = bk & 31;
        // h_t(uv) = P - e_t with P = 1 + w^v + w^u + w^(u+v)
        const C2<T> ev = om[v], eu = om[u], euv = om[(u + v) & 31];
        const C2<T> P = cadd(cadd(cadd(C2<T>{1, 0}, ev), eu), euv);
        g[0] = cmul(gd, csub(P, C2<T>{1, 0}));
        g[1] = cmul(gd, csub(P, ev));
        g[2] = cmul(gd, csub(P, eu));
        g[3] = cmul(gd, csub(P, euv));
        const C2<T> ph = om[(eta * u + gam * v) & 31];
        fpix += gd.re * ph.re - gd.im * ph.im;
        if (tracing && lane == 0) {
            a.trace_sel[trow + it] = (uint16_t)bk;
            a.trace_dc[2 * (trow + it)] = (float)gd.re;
            a.trace_dc[2 * (trow + it) + 1] = (float)gd.im;
        }
    }

    // 4. central block -> HR image
    if (lane < 16) {
        const int yy = 4 * we.bi + (lane >> 2), xx = 4 * we.bj + (lane & 3);
        img.hr[(long long)yy * img.hr_pitch + xx] = (float)fpix;
    }
}

// --------------------------------------------------- persistent kernel --
template <typename T, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, (sizeof(T) == 4 ? 16 / WARPS : 1)) recurrent_kernel(const Args a)
{
    using L = SmemLayout<T, WARPS>;
    extern __shared__ __align__(128) unsigned char smem[];
    auto slot = [&](int s) { return reinterpret_cast<Record<T> *>(smem + L::off_slots + s * L::rec); };
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    C2<T> *scratch = reinterpret_cast<C2<T> *>(smem + L::off_scratch + warp * L::scratch);
    C2<T> *om = reinterpret_cast<C2<T> *>(smem + L::off_om);
    C2<T> *omc = reinterpret_cast<C2<T> *>(smem + L::off_omc);
    T *wt = reinterpret_cast<T *>(smem + L::off_w);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L::off_bar);

    for (int i = threadIdx.x; i < 256; i += WARPS * 32)
        wt[i] = sizeof(T) == 8 ? (T)a.consts->w64[i] : (T)a.consts->w32[i];
    for (int i = threadIdx.x; i < 32; i += WARPS * 32) {
        const T re = sizeof(T) == 8 ? (T)a.consts->om64[2 * i] : (T)a.consts->om32[2 * i];
        const T im = sizeof(T) == 8 ? (T)a.consts->om64[2 * i + 1] : (T)a.consts->om32[2 * i + 1];
        om[i] = {re, im};
        omc[i] = {re, -im};
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    const uint32_t rb = a.record_bytes;
    // Per slot s: table held (held0/held1), a load in flight (bit s of
    // pending) and the mbarrier parity to wait for (bit s of parity).
    int held0 = -1, held1 = -1;
    uint32_t pending = 0, parity = 0;
    for (int s = 0; s < 2; ++s) {
        const int c = blockIdx.x + s * gridDim.x;
        if (c < a.n_chunks) {
            const int t = a.chunk_table[c];
            if (threadIdx.x == 0) bulk_load(slot(s), a.records + (size_t)t * rb, rb, &bar[s]);
            if (s == 0) held0 = t; else held1 = t;
            pending |= 1u << s;
        }
    }
    bool failed = false;
    for (int r = 0;; ++r) {
        const int c = blockIdx.x + r * gridDim.x;
        if (c >= a.n_chunks) break;
        const int s = r & 1;
        if (pending & (1u << s)) {
            const bool ok = mbar_wait(&bar[s], (parity >> s) & 1u);
            if (!__syncthreads_and(ok)) { failed = true; break; }
            parity ^= 1u << s;
            pending &= ~(1u << s);
        }
        for (int e = warp; e < kChunk; e += WARPS) {
            const WorkEntry we = a.entries[(size_t)c * kChunk + e];
            if (we.img >= 0) recurrent_block<T>(a, *slot(s), scratch, om, omc, wt, we, lane);
        }
        __syncthreads();                       // every warp is done with slot s
        const int c2 = blockIdx.x + (r + 2) * gridDim.x;
        if (c2 < a.n_chunks) {
            const int t2 = a.chunk_table[c2];
            if (t2 != (s == 0 ? held0 : held1)) {
                if (threadIdx.x == 0) {
                    fence_proxy_async();
                    bulk_load(slot(s), a.records + (size_t)t2 * rb, rb, &bar[s]);
                }
                if (s == 0) held0 = t2; else held1 = t2;
                pending |= 1u << s;
            }
        }
    }
    if (failed) {
        if (threadIdx.x == 0) atomicOr(a.status, kStatusTimeout);
        // let copies still in flight land before the CTA's shared memory goes away
        for (int s = 0; s < 2; ++s)
            if (pending & (1u << s)) mbar_wait(&bar[s], (parity >> s) & 1u);
    }
}

// ---------------------------------------------------------- direct path --
// Direct L-JSDE (Eqs. 4-10): per block the residual r (256 complex, in the
// warp's scratch) and, every iteration, N_k = sum_m conj(a_m(k)) w_m r_m for
// all 1024 k with a_m(k) evaluated from the roots-of-unity table (O(W^4)).
constexpr int kDirectWarps = 4;
struct DirectSmem {
    float2 r[kDirectWarps][256];
    float wr[kDirectWarps][256][2];
    uint8_t type[kDirectWarps][256];
    float2 om[32];
    float w[256];
};

__global__ void __launch_bounds__(kDirectWarps * 32) direct_kernel(const Args a, int n_entries)
{
    __shared__ DirectSmem sm;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) sm.w[i] = a.consts->w32[i];
    for (int i = threadIdx.x; i < 32; i += blockDim.x) sm.om[i] = make_float2(a.consts->om32[2 * i], a.consts->om32[2 * i + 1]);
    __syncthreads();
    const float gamma = (float)a.gamma;
    for (int e = blockIdx.x * kDirectWarps + warp; e < n_entries; e += gridDim.x * kDirectWarps) {
        const WorkEntry we = a.entries[e];
        if (we.img < 0) continue;
        const ImageDesc img = a.descs ? a.descs[we.img] : a.single;
        const uint8_t *mask = a.masks + a.mask_offset[we.img];
        const int p0 = 2 * we.bi - kOff / 2, q0 = 2 * we.bj - kOff / 2;
        bool bad = false;
        for (int m = lane; m < 256; m += 32) {
            const int p = m >> 4, q = m & 15, P = p0 + p, Q = q0 + q;
            uint8_t t = 255;
            float y = 0.f;
            if (P >= 0 && P < img.lr_h && Q >= 0 && Q < img.lr_w) {
                t = mask[(long long)P * img.lr_w + Q];
                y = img.lr[(long long)P * img.lr_pitch + Q];
                if (!isfinite(y)) { bad = true; y = 0.f; }
            }
            sm.type[warp][m] = t;
            sm.r[warp][m] = make_float2(t < 4 ? y : 0.f, 0.f);
        }
        if (bad) atomicOr(a.status, kStatusNonfinite);
        __syncwarp();
        // D_k = sum_m w_m |a_m(k)|^2 for this lane's 32 candidates k = lane + 32 j
        float D[32];
        for (int j = 0; j < 32; ++j) D[j] = 0.f;
        for (int m = 0; m < 256; ++m) {
            const int t = sm.type[warp][m];
            if (t > 3) continue;
            const int p = m >> 4, q = m & 15;
            const float wm = sm.w[m];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int k1 = j, k2 = lane;
                float are = 0.f, aim = 0.f;
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    if (s == t) continue;
                    const float2 z = sm.om[((2 * p + (s >> 1)) * k1 + (2 * q + (s & 1)) * k2) & 31];
                    are += z.x;
                    aim += z.y;
                }
                D[j] += wm * (are * are + aim * aim);
            }
        }
        float fpix = 0.f;
        const int eta = kOff + ((lane >> 2) & 3), gam = kOff + (lane & 3);
        const long long trow = (long long)we.ord * a.nu_max;
        for (int it = 0; it < a.nu_max; ++it) {
            for (int m = lane; m < 256; m += 32) {
                const float wm = sm.type[warp][m] < 4 ? sm.w[m] : 0.f;
                sm.wr[warp][m][0] = wm * sm.r[warp][m].x;
                sm.wr[warp][m][1] = wm * sm.r[warp][m].y;
            }
            __syncwarp();
            float Nre[32], Nim[32];
            for (int j = 0; j < 32; ++j) Nre[j] = Nim[j] = 0.f;
            for (int m = 0; m < 256; ++m) {
                const int t = sm.type[warp][m];
                if (t > 3) continue;
                const int p = m >> 4, q = m & 15;
                const float xr = sm.wr[warp][m][0], xi = sm.wr[warp][m][1];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    float are = 0.f, aim = 0.f;
#pragma unroll
                    for (int s = 0; s < 4; ++s) {
                        if (s == t) continue;
                        const float2 z = sm.om[((2 * p + (s >> 1)) * j + (2 * q + (s & 1)) * lane) & 31];
                        are += z.x;
                        aim += z.y;
                    }
                    // conj(a) * (w r)
                    Nre[j] += are * xr + aim * xi;
                    Nim[j] += are * xi - aim * xr;
                }
            }
            float bs = -1.f;
            int bk = 0;
            float bre = 0.f, bim = 0.f;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int k = j * kW + lane;
                const float s = D[j] > 0.f ? a.q[k] * (Nre[j] * Nre[j] + Nim[j] * Nim[j]) / D[j] : 0.f;
                if (s > bs) { bs = s; bk = k; bre = Nre[j] / D[j]; bim = Nim[j] / D[j]; }
            }
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) {
                const float os = __shfl_xor_sync(0xffffffffu, bs, m);
                const int ok = __shfl_xor_sync(0xffffffffu, bk, m);
                if (os > bs || (os == bs && ok < bk)) { bs = os; bk = ok; }
            }
            const int wl = bk & 31;
            const float dre = __shfl_sync(0xffffffffu, bre, wl), dim = __shfl_sync(0xffffffffu, bim, wl);
            const float gre = gamma * dre, gim = gamma * dim;
            const int u = bk >> 5, v = bk & 31;
            // r_m -= gamma delta a_m(uv)   (Eq. 7)
            for (int m = lane; m < 256; m += 32) {
                const int t = sm.type[warp][m];
                if (t > 3) continue;
                const int p = m >> 4, q = m & 15;
                float are = 0.f, aim = 0.f;
                for (int s = 0; s < 4; ++s) {
                    if (s == t) continue;
                    const float2 z = sm.om[((2 * p + (s >> 1)) * u + (2 * q + (s & 1)) * v) & 31];
                    are += z.x;
                    aim += z.y;
                }
                float2 r = sm.r[warp][m];
                r.x -= gre * are - gim * aim;
                r.y -= gre * aim + gim * are;
                sm.r[warp][m] = r;
            }
            const float2 ph = sm.om[(eta * u + gam * v) & 31];
            fpix += gre * ph.x - gim * ph.y;
            if (a.trace_sel && lane == 0) {
                a.trace_sel[trow + it] = (uint16_t)bk;
                a.trace_dc[2 * (trow + it)] = gre;
                a.trace_dc[2 * (trow + it) + 1] = gim;
            }
            __syncwarp();
        }
        if (lane < 16) {
            const int yy = 4 * we.bi + (lane >> 2), xx = 4 * we.bj + (lane & 3);
            img.hr[(long long)yy * img.hr_pitch + xx] = fpix;
        }
        __syncwarp();
    }
}

// -------------------------------------------------------------- launch --
template <typename T, int WARPS>
cudaError_t set_smem_attr()
{
    return cudaFuncSetAttribute(recurrent_kernel<T, WARPS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)SmemLayout<T, WARPS>::bytes);
}

template <typename T, int WARPS>
int occupancy()
{
    int n = 0;
    if (set_smem_attr<T, WARPS>() != cudaSuccess) return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, recurrent_kernel<T, WARPS>, WARPS * 32,
                                                      SmemLayout<T, WARPS>::bytes) != cudaSuccess)
        return -1;
    return n;
}

Args make_args(const rljsde_plan *p)
{
    Args a{};
    a.entries = p->d_entries;
    a.chunk_table = p->d_chunk_table;
    a.n_chunks = p->n_chunks;
    a.records = static_cast<const unsigned char *>(p->d_records);
    a.record_bytes = (uint32_t)p->record_bytes;
    a.consts = p->d_consts;
    a.descs = nullptr;
    a.nu_max = p->params.nu_max;
    a.gamma = p->params.gamma_odc;
    a.status = p->d_status;
    a.masks = p->d_masks;
    a.mask_offset = p->d_mask_offset;
    a.q = p->d_qD;
    return a;
}

int launch(const rljsde_plan *p, const Args &a, cudaStream_t s)
{
    if (p->direct) {
        direct_kernel<<<p->grid, kDirectWarps * 32, 0, s>>>(a, p->n_entries);
    } else if (p->params.precision == 1) {
        if (p->warps == 4)
            recurrent_kernel<double, 4><<<p->grid, 128, SmemLayout<double, 4>::bytes, s>>>(a);
        else
            recurrent_kernel<double, 8><<<p->grid, 256, SmemLayout<double, 8>::bytes, s>>>(a);
    } else {
        if (p->warps == 4)
            recurrent_kernel<float, 4><<<p->grid, 128, SmemLayout<float, 4>::bytes, s>>>(a);
        else
            recurrent_kernel<float, 8><<<p->grid, 256, SmemLayout<float, 8>::bytes, s>>>(a);
    }
    return cudaGetLastError() == cudaSuccess ? RLJSDE_OK : RLJSDE_ERR_CUDA;
}

}  // namespace

int choose_launch(rljsde_plan *p, int warps, int ctas_per_sm)
{
    if (p->direct) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, direct_kernel, kDirectWarps * 32, 0) != cudaSuccess)
            return RLJSDE_ERR_CUDA;
        p->warps = kDirectWarps;
        p->ctas_per_sm = ctas_per_sm > 0 ? (ctas_per_sm < n ? ctas_per_sm : n) : n;
        if (p->ctas_per_sm < 1) p->ctas_per_sm = 1;
        long long want = ((long long)p->n_entries + kDirectWarps - 1) / kDirectWarps;
        long long g = (long long)p->sm_count * p->ctas_per_sm;
        p->grid = (int)(want < g ? (want > 0 ? want : 1) : g);
        return RLJSDE_OK;
    }
    if (warps == 0) warps = 8;
    int occ = p->params.precision ? (warps == 4 ? occupancy<double, 4>() : occupancy<double, 8>())
                                  : (warps == 4 ? occupancy<float, 4>() : occupancy<float, 8>());
    if (occ < 0) return RLJSDE_ERR_CUDA;
    if (occ == 0) return RLJSDE_ERR_UNSUPPORTED;
    p->warps = warps;
    p->ctas_per_sm = ctas_per_sm > 0 ? (ctas_per_sm < occ ? ctas_per_sm : occ) : occ;
    long long g = (long long)p->sm_count * p->ctas_per_sm;
    p->grid = (int)(p->n_chunks < g ? (p->n_chunks > 0 ? p->n_chunks : 1) : g);
    return RLJSDE_OK;
}

}  // namespace rljsde

using namespace rljsde;

extern "C" {

int rljsde_reconstruct_trace(const rljsde_plan_t *plan, const float *lr, size_t lr_pitch, float *hr,
                             size_t hr_pitch, uint16_t *sel, float *dc, void *stream)
{
    if (!plan || !lr || !hr) return RLJSDE_ERR_INVALID_ARG;
    if (plan->n_images != 1) return RLJSDE_ERR_INVALID_ARG;
    if (lr_pitch < (size_t)plan->lr_w[0] || hr_pitch < (size_t)(2 * plan->lr_w[0])) return RLJSDE_ERR_INVALID_ARG;
    if ((sel == nullptr) != (dc == nullptr)) return RLJSDE_ERR_INVALID_ARG;
    Args a = make_args(plan);
    a.single = {lr, hr, plan->lr_h[0], plan->lr_w[0], (long long)lr_pitch, (long long)hr_pitch};
    a.trace_sel = sel;
    a.trace_dc = dc;
    return launch(plan, a, (cudaStream_t)stream);
}

int rljsde_reconstruct(const rljsde_plan_t *plan, const float *lr, size_t lr_pitch, float *hr, size_t hr_pitch,
                       void *stream)
{
    return rljsde_reconstruct_trace(plan, lr, lr_pitch, hr, hr_pitch, nullptr, nullptr, stream);
}

int rljsde_reconstruct_batch(const rljsde_plan_t *plan, void *stream)
{
    if (!plan) return RLJSDE_ERR_INVALID_ARG;
    Args a = make_args(plan);
    a.descs = plan->d_images;
    return launch(plan, a, (cudaStream_t)stream);
}

}  // extern "C"
