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
//      and the projected-residual update of Eq. 17, R -= gamma delta C_{., uv},
//      with the column of C (Eq. 14) either
//        - read from the Gram matrix the plan stores for the block's local
//          mask (the paper's recurrent form, Table I; the default), the state
//          kept as sqrt(q_k / D_k) R_k so that the score is its squared
//          modulus (greedy_loop_stored), or
//        - rebuilt from the factored tables, the update carried out on Y:
//            Y_t(kap) -= gamma delta h_t(uv) G_t((uv - kap) mod 16),
//          which is Eq. 17 with C factored as C_{k,l} = sum_t conj(h_t(k))
//          h_t(l) G_t(l - k) (greedy_loop_f32, and the FP64 loop);
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
    const unsigned char *records_short;    // RecordShortF32 per table (shortlist loop)
    const float4 *cstore;                  // stored Gram matrices (c_supply), kStoredTableBytes each
    const int *cslot;                      // per table set: its stored matrix, or -1 (factored)
    int cfilter;                           // chunks this launch takes: 0 all, 1 those whose table set
                                           // has a stored matrix, 2 the others
    const Consts *consts;
    ImageDesc single;          // used when descs == nullptr
    const ImageDesc *descs;
    int nu_max;
    double gamma;
    uint16_t *trace_sel;       // [ordinal][nu_max], optional
    float *trace_dc;           // [ordinal][nu_max][2], optional
    int *status;
    // learned proposal (FP32 loop only)
    const Shortlist *shortlists;   // per block ordinal, or nullptr
    float max_missing;             // restrict a block iff its left-out mass <= this
    int use_nu_hat;                // iterations from the network's output
    int *n_restricted;             // optional count of restricted blocks
    // sensor layout: aperture code of slot t in bits 4t..4t+3 (MODE 3 loops)
    // and the meaning of the mask codes (direct path)
    uint32_t slot_ap;
    int layout;
    int pairs;                 // conjugate-pair update (direct path; the loops take it as a template flag)
    // direct path only
    const uint8_t *masks;
    const long long *mask_offset;
    const float *q;
};

template <typename T, int MODE = 0> struct RecOf;
template <int MODE> struct RecOf<float, MODE> { using type = RecordF32; };
template <> struct RecOf<float, 1> { using type = RecordShortF32; };
template <> struct RecOf<float, 17> { using type = RecordShortF32; };   // mode 1 with stored C
template <int MODE> struct RecOf<double, MODE> { using type = Record<double>; };

// Pair tables of the FP32 loop: for kap1 pair j, (cos, cos, sin, sin) of
// 2 pi kap1 / 32 for kap1 = 2j, 2j+1, and (-sin, -sin); the same for the
// angle index n, n+1 of exp(-2 pi i (kap1 + kap2) / 32).
struct PairTables {
    float4 e2[8];
    float2 e2n[8];
    float4 e12[32];
    float2 e12n[32];
};

// Shared memory of the recurrent kernel.
template <typename T, int WARPS, int MODE = 0>
struct SmemLayout {
    static constexpr size_t rec = sizeof(typename RecOf<T, MODE>::type);
    static constexpr size_t scratch = 256 * 2 * sizeof(C2<T>);   // per warp
    static constexpr size_t off_slots = 0;
    static constexpr size_t off_scratch = 2 * rec;
    static constexpr size_t off_om = off_scratch + WARPS * scratch;       // 32 x C2<T>
    static constexpr size_t off_omc = off_om + 32 * sizeof(C2<T>);        // 32 x C2<T>
    static constexpr size_t off_pair = off_omc + 32 * sizeof(C2<T>);      // PairTables
    static constexpr size_t off_w = off_pair + sizeof(PairTables);        // 256 x T
    static constexpr size_t off_bar = off_w + 256 * sizeof(T);            // 2 x u64
    static constexpr size_t bytes = off_bar + 2 * sizeof(uint64_t);
};

__device__ __forceinline__ const uint8_t *rec_types(const RecordF32 &r) { return r.types; }
__device__ __forceinline__ const uint8_t *rec_types(const RecordShortF32 &r) { return r.types; }
__device__ __forceinline__ const uint8_t *rec_types(const Record<double> &r) { return r.types; }

// X[i] = sum_j x_j w8^-(j i), i, j in [0, 8): radix-2 decimation in
// frequency (twiddles 1, (1 - i)/sqrt 2, -i, (-1 - i)/sqrt 2, then -i), 52
// real additions and multiplications instead of 64 complex products.  The same
// code on conjugated input gives the conjugated, index-mirrored output bit
// for bit, so mirror ties stay exact.
template <typename T>
__device__ __forceinline__ void dft8(const C2<T> (&x)[8], C2<T> (&X)[8])
{
    const T c = T(0.70710678118654752440);
    const C2<T> s0 = cadd(x[0], x[4]), s1 = cadd(x[1], x[5]), s2 = cadd(x[2], x[6]), s3 = cadd(x[3], x[7]);
    const C2<T> e1 = csub(x[1], x[5]), e2 = csub(x[2], x[6]), e3 = csub(x[3], x[7]);
    const C2<T> d0 = csub(x[0], x[4]);
    const C2<T> d1 = {c * (e1.re + e1.im), c * (e1.im - e1.re)};        // e1 (1 - i) / sqrt 2
    const C2<T> d2 = {e2.im, -e2.re};                                    // e2 (-i)
    const C2<T> d3 = {c * (e3.im - e3.re), -(c * (e3.re + e3.im))};      // e3 (-1 - i) / sqrt 2
    // even outputs: 4-point DFT of s; odd outputs: 4-point DFT of d
    const C2<T> a0 = cadd(s0, s2), a1 = cadd(s1, s3), b0 = csub(s0, s2), bm = csub(s1, s3);
    const C2<T> b1 = {bm.im, -bm.re};
    X[0] = cadd(a0, a1);
    X[4] = csub(a0, a1);
    X[2] = cadd(b0, b1);
    X[6] = csub(b0, b1);
    const C2<T> f0 = cadd(d0, d2), f1 = cadd(d1, d3), g0 = csub(d0, d2), gm = csub(d1, d3);
    const C2<T> g1 = {gm.im, -gm.re};
    X[1] = cadd(f0, f1);
    X[5] = csub(f0, f1);
    X[3] = cadd(g0, g1);
    X[7] = csub(g0, g1);
}

// ------------------------------------------- initial projected residual --
// Step 1 and the row half of step 2 for one block: gather the weighted
// window into the four type planes x_t(p, q) and sum the row DFTs
// T_t(p, k2) = sum_q x_t(p, q) w16^-(q k2).  x is real, so
// T_t(p, 16 - k2) = conj(T_t(p, k2)) and only k2 in [0, 8] is summed: lane
// (c, r) = (lane & 7, lane >> 3) takes rows p = 4r..4r+3 at k2 = c for c >= 1;
// lane c = 0 sums the two real columns, k2 = 0 (re slot) and k2 = 8 (im slot).
// With UNIT, y is taken as 1 for every present L-pixel: the result is then
// the DFT of the type-split spatial weights, whose conjugate is G_t.
template <typename T, bool UNIT = false, typename Rec>
__device__ __forceinline__ void window_rows(const Args &a, const Rec &rec, C2<T> *scratch, const C2<T> *omc,
                                            const T *wt, const WorkEntry we, const int lane, C2<T> (&acc)[4][4])
{
    const ImageDesc img = a.descs ? a.descs[we.img] : a.single;
    const int p0 = 2 * we.bi - kOff / 2, q0 = 2 * we.bj - kOff / 2;
    const uint8_t *types = rec_types(rec);
    __syncwarp();    // the previous block of this warp is done with the scratch

    // 1. gather: x(p, q) = w(p, q) y(p, q) into the plane of its type.
    Vec4<T> *x4 = reinterpret_cast<Vec4<T> *>(scratch);
    {
        const int p = lane >> 1, P = p0 + p;
        bool bad = false;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int q = (lane & 1) * 8 + j, Q = q0 + q;
            const int code = types[p * 16 + q];
            T v = 0;
            if (code < 4 && P >= 0 && P < img.lr_h && Q >= 0 && Q < img.lr_w) {
                if (UNIT) {
                    v = wt[p * 16 + q];
                } else {
                    const float y = img.lr[(long long)P * img.lr_pitch + Q];
                    if (isfinite(y)) v = wt[p * 16 + q] * (T)y;
                    else bad = true;
                }
            }
            Vec4<T> o = {code == 0 ? v : T(0), code == 1 ? v : T(0), code == 2 ? v : T(0), code == 3 ? v : T(0)};
            st4(&x4[p * 16 + q], o);
        }
        if (bad) atomicOr(a.status, kStatusNonfinite);
    }
    __syncwarp();

    // 2a. row DFTs, k2 in [0, 8] (see above)
    const int c = lane & 7, r = lane >> 3;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int t = 0; t < 4; ++t) acc[i][t] = {0, 0};
#pragma unroll 4
    for (int q = 0; q < 16; ++q) {
        const C2<T> tq = omc[(2 * q * c) & 31];
        const T twre = c == 0 ? T(1) : tq.re;
        const T twim = c == 0 ? ((q & 1) ? T(-1) : T(1)) : tq.im;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const Vec4<T> x = ld4(&x4[(4 * r + i) * 16 + q]);
            acc[i][0].re += x.x * twre; acc[i][0].im += x.x * twim;
            acc[i][1].re += x.y * twre; acc[i][1].im += x.y * twim;
            acc[i][2].re += x.z * twre; acc[i][2].im += x.z * twim;
            acc[i][3].re += x.w * twre; acc[i][3].im += x.w * twim;
        }
    }
}

// Write rows 4r..4r+3 of the type pair (2 pass, 2 pass + 1) into the scratch
// as tb[p][k2] (two complex values), all 16 columns: (p, c) and its conjugate
// (p, 16 - c), or for c = 0 the real columns (p, 0) and (p, 8).
template <typename T>
__device__ __forceinline__ void rows_to_scratch(const C2<T> (&acc)[4][4], Vec4<T> *tb, const int pass, const int lane)
{
    const int c = lane & 7, r = lane >> 3, t0 = 2 * pass;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int p = 4 * r + i;
        const C2<T> a0 = acc[i][t0], a1 = acc[i][t0 + 1];
        st4(&tb[p * 16 + c], c == 0 ? Vec4<T>{a0.re, T(0), a1.re, T(0)} : Vec4<T>{a0.re, a0.im, a1.re, a1.im});
        st4(&tb[p * 16 + (c == 0 ? 8 : 16 - c)],
            c == 0 ? Vec4<T>{a0.im, T(0), a1.im, T(0)} : Vec4<T>{a0.re, -a0.im, a1.re, -a1.im});
    }
}

// Steps 1-2 for one block: the window's row DFTs, then the column DFTs
//     Y_t(kap) = sum_{m: t(m) = t} w_m y_m w16^-(p kap1 + q kap2);
// returns Y[i][t] for kap = (8h + i, lane & 15), h = lane >> 4.
template <typename T, bool UNIT = false, typename Rec>
__device__ __forceinline__ void initial_projection(const Args &a, const Rec &rec, C2<T> *scratch,
                                                   const C2<T> *omc, const T *wt, const WorkEntry we,
                                                   const int lane, C2<T> (&Y)[8][4])
{
    C2<T> acc[4][4];
    window_rows<T, UNIT>(a, rec, scratch, omc, wt, we, lane, acc);
    const int k2 = lane & 15, h = lane >> 4;
    // 2b. column DFTs, two types at a time through the scratch, split by the
    // parity of p: half h sums p = 2j + h for kap1' in [0, 8); then
    // Y(kap1') = E + O and Y(kap1' + 8) = E - O.
    Vec4<T> *tb = reinterpret_cast<Vec4<T> *>(scratch);     // [p][k2]: 2 complex
#pragma unroll
    for (int pass = 0; pass < 2; ++pass) {
        const int t0 = 2 * pass;
        __syncwarp();
        rows_to_scratch<T>(acc, tb, pass, lane);
        __syncwarp();
        // half h: cc(i) = sum_j T(2j + h, k2) w16^-((2j + h) i) = w16^-(h i) DFT8_j(T(2j + h, k2))(i)
        C2<T> cc[8][2];
        {
            C2<T> x[2][8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const Vec4<T> tv = ld4(&tb[(2 * j + h) * 16 + k2]);
                x[0][j] = {tv.x, tv.y};
                x[1][j] = {tv.z, tv.w};
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                C2<T> X[8];
                dft8<T>(x[u], X);
                cc[0][u] = X[0];
#pragma unroll
                for (int i = 1; i < 8; ++i) cc[i][u] = cmul(X[i], omc[(2 * h * i) & 31]);
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const T ore = __shfl_xor_sync(0xffffffffu, cc[i][u].re, 16);
                const T oim = __shfl_xor_sync(0xffffffffu, cc[i][u].im, 16);
                // h = 0 holds E and receives O: Y = E + O; h = 1 holds O: Y = E - O
                Y[i][t0 + u] = h == 0 ? C2<T>{cc[i][u].re + ore, cc[i][u].im + oim}
                                      : C2<T>{ore - cc[i][u].re, oim - cc[i][u].im};
            }
    }
}

// Keep the best (score, index, R) of one candidate; candidates arrive in
// increasing index order, so a strict > keeps the lowest index on ties.
template <typename T>
__device__ __forceinline__ void keep_best(T s, int k, T re, T im, T &bs, int &bk, T &bre, T &bim)
{
    if (s > bs) { bs = s; bk = k; bre = re; bim = im; }
}

// The argmax of Eqs. 10-11 compares scores rounded to binary32 (the precision
// of the paper's complex64 tables), so the FP64 loop rounds its scores too:
// candidates whose FP64 scores differ only by rounding tie, and the lowest
// index wins, as in the FP32 loop.
template <typename T> __device__ __forceinline__ T key32(T s) { return (T)(float)s; }

// Warp argmax over (score, index), ties to the lowest index, with two warp
// reductions: the largest score (a non-negative binary32 value, so its bit
// pattern orders like the value), then the smallest index among the lanes
// holding it.  Every lane's score is a binary32 key (scores of the FP64
// loop are rounded to binary32 first), so the conversion below is exact.
__device__ __forceinline__ void warp_argmax_bits(const float s, int &bk, float &best)
{
    const unsigned bits = __float_as_uint(s);
    const unsigned smax = __reduce_max_sync(0xffffffffu, bits);
    bk = (int)__reduce_min_sync(0xffffffffu, bits == smax ? (unsigned)bk : 0xffffffffu);
    best = __uint_as_float(smax);
}
template <typename T>
__device__ __forceinline__ void warp_argmax(T &bs, int &bk)
{
    float best;
    warp_argmax_bits((float)bs, bk, best);
    bs = (T)best;
}

// Aperture structure of the table slots, fixed per plan:
//   kLayThreeQuarter: slot t holds every sub-pixel but t (three-quarter sampling);
//   kLaySingle:       slot t holds sub-pixel t only (quarter sampling);
//   kLayGeneral:      slot t holds the sub-pixels in bits 4t..4t+3 of a.slot_ap.
constexpr int kLayThreeQuarter = 0, kLayGeneral = 1, kLaySingle = 2;

// Per-iteration bookkeeping shared by both loops: delta, the update
// coefficients g_t = gamma delta h_t(uv) and the synthesis of Eq. 18.
// With PAIRS (conjugate-pair update) the selection also updates c_-uv by
// conj(gamma delta); its coefficients are conj(g_t), since h_t(-k) =
// conj h_t(k), and pw = 1 (0 when uv is its own mirror) scales them.
template <typename T, int LAY = kLayThreeQuarter, bool PAIRS = false>
__device__ __forceinline__ void select_step(const Args &a, const C2<T> *om, const T invD, const T gamma,
                                            const int bk, const T Rre, const T Rim, const int eta, const int gam,
                                            const int lane, const long long trow, const int it, int &u, int &v,
                                            C2<T> (&g)[4], T &fpix, T &pw)
{
    const C2<T> gd = {gamma * (Rre * invD), gamma * (Rim * invD)};   // gamma * delta (Eqs. 15, 16)
    u = bk >> 5;
    v = bk & 31;
    const C2<T> ev = om[v], eu = om[u], euv = om[(u + v) & 31];
    if constexpr (LAY == kLaySingle) {
        // h_t(uv) = e_t, e = (1, w^v, w^u, w^(u+v))
        g[0] = gd;
        g[1] = cmul(gd, ev);
        g[2] = cmul(gd, eu);
        g[3] = cmul(gd, euv);
    } else if constexpr (LAY == kLayGeneral) {
        // h_t(uv) = sum over slot t's sub-pixels s of e_s, e = (1, w^v, w^u, w^(u+v))
        const C2<T> e[4] = {C2<T>{1, 0}, ev, eu, euv};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            C2<T> h = {0, 0};
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
                if ((a.slot_ap >> (4 * t + sp)) & 1u) h = cadd(h, e[sp]);
            g[t] = cmul(gd, h);
        }
    } else {
        // h_t(uv) = P - e_t with P = 1 + w^v + w^u + w^(u+v)
        const C2<T> P = cadd(cadd(cadd(C2<T>{1, 0}, ev), eu), euv);
        g[0] = cmul(gd, csub(P, C2<T>{1, 0}));
        g[1] = cmul(gd, csub(P, ev));
        g[2] = cmul(gd, csub(P, eu));
        g[3] = cmul(gd, csub(P, euv));
    }
    const C2<T> ph = om[(eta * u + gam * v) & 31];
    if constexpr (PAIRS) {
        // Re(x Phi_uv) + Re(conj(x) Phi_-uv) = 2 Re(x Phi_uv) unless uv = -uv
        pw = ((u & 15) == 0 && (v & 15) == 0) ? T(0) : T(1);
        fpix += (T(1) + pw) * (gd.re * ph.re - gd.im * ph.im);
    } else {
        fpix += gd.re * ph.re - gd.im * ph.im;
    }
    if (a.trace_sel != nullptr && lane == 0) {
        a.trace_sel[trow + it] = (uint16_t)bk;
        a.trace_dc[2 * (trow + it)] = (float)gd.re;
        a.trace_dc[2 * (trow + it) + 1] = (float)gd.im;
    }
}

// ------------------------------------------------------ FP64 (scalar) loop --
template <typename T, int LAY = kLayThreeQuarter, bool PAIRS = false>
__device__ __forceinline__ void greedy_loop(const Args &a, const Record<T> &rec, const C2<T> *om,
                                            const C2<T> *omc, const WorkEntry we, const int lane,
                                            C2<T> (&Y)[8][4])
{
    const int k2 = lane & 15, h = lane >> 4;
    const C2<T> e1 = omc[k2];                       // exp(-2 pi i kap2 / 32)
    const T gamma = (T)a.gamma;
    const int eta = kOff + ((lane >> 2) & 3), gam = kOff + (lane & 3);
    T fpix = 0;                                     // Eq. 18 accumulator
    int u = 0, v = 0;
    T pw = 0;
    C2<T> g[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    const long long trow = (long long)we.ord * a.nu_max;

    for (int it = 0; it < a.nu_max; ++it) {
        T bs0 = -1, bs1 = -1, b0re = 0, b0im = 0, b1re = 0, b1im = 0;
        int bk0 = 0, bk1 = 0;
        const int d2 = (v - k2) & 15, d2c = (-v - k2) & 15;
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
                if constexpr (PAIRS) {
                    // the partner -uv: Y_t -= pw conj(g_t) G_t((-uv - kap) mod 16)
                    const int dc = (((-u - k1) & 15) << 4) | d2c;
                    const Vec4<T> H01 = ld4(&rec.G01[dc]), H23 = ld4(&rec.G23[dc]);
                    Y[i][0] = csub(Y[i][0], cmul(C2<T>{pw * g[0].re, -pw * g[0].im}, C2<T>{H01.x, H01.y}));
                    Y[i][1] = csub(Y[i][1], cmul(C2<T>{pw * g[1].re, -pw * g[1].im}, C2<T>{H01.z, H01.w}));
                    Y[i][2] = csub(Y[i][2], cmul(C2<T>{pw * g[2].re, -pw * g[2].im}, C2<T>{H23.x, H23.y}));
                    Y[i][3] = csub(Y[i][3], cmul(C2<T>{pw * g[3].re, -pw * g[3].im}, C2<T>{H23.z, H23.w}));
                }
            }
            // R_k = sum_s conj(e_s(k)) Z_s, e = (1, w^k2, w^k1, w^(k1+k2)), with Z_s the
            // sum of Y_t over the slots t whose aperture holds sub-pixel s
            // (three-quarter: Z_s = S - Y_s, S = sum_t Y_t; single: Z_s = Y_s)
            C2<T> Z[4];
            if constexpr (LAY == kLaySingle) {
#pragma unroll
                for (int sp = 0; sp < 4; ++sp) Z[sp] = Y[i][sp];
            } else if constexpr (LAY == kLayGeneral) {
#pragma unroll
                for (int sp = 0; sp < 4; ++sp) {
                    Z[sp] = {0, 0};
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        if ((a.slot_ap >> (4 * t + sp)) & 1u) Z[sp] = cadd(Z[sp], Y[i][t]);
                }
            } else {
                // Z_s = S - Y_s as the sum of the other three: 6 additions, no cancellation
                const C2<T> P01 = cadd(Y[i][0], Y[i][1]), P23 = cadd(Y[i][2], Y[i][3]);
                Z[0] = cadd(Y[i][1], P23);
                Z[1] = cadd(Y[i][0], P23);
                Z[2] = cadd(P01, Y[i][3]);
                Z[3] = cadd(P01, Y[i][2]);
            }
            const C2<T> Z0 = Z[0];
            const C2<T> U = cmul(e1, Z[1]);
            const C2<T> V = cmul(omc[k1], Z[2]);
            const C2<T> X = cmul(omc[(k1 + k2) & 31], Z[3]);
            const C2<T> pp = cadd(Z0, U), mm = csub(Z0, U), ss = cadd(V, X), dd = csub(V, X);
            const C2<T> R00 = cadd(pp, ss), R01 = cadd(mm, dd), R10 = csub(pp, ss), R11 = csub(mm, dd);
            const Vec4<T> qd = ld4(&rec.qD[k1 * 16 + k2]);
            const int k = k1 * kW + k2;
            keep_best(key32(qd.x * (R00.re * R00.re + R00.im * R00.im)), k, R00.re, R00.im, bs0, bk0, b0re, b0im);
            keep_best(key32(qd.y * (R01.re * R01.re + R01.im * R01.im)), k + 16, R01.re, R01.im, bs0, bk0, b0re, b0im);
            keep_best(key32(qd.z * (R10.re * R10.re + R10.im * R10.im)), k + 512, R10.re, R10.im, bs1, bk1, b1re, b1im);
            keep_best(key32(qd.w * (R11.re * R11.re + R11.im * R11.im)), k + 528, R11.re, R11.im, bs1, bk1, b1re, b1im);
        }
        if (bs1 > bs0) { bs0 = bs1; bk0 = bk1; b0re = b1re; b0im = b1im; }
        T bs = bs0;
        int bk = bk0;
        warp_argmax(bs, bk);
        const int wl = (bk & 15) + ((bk >> 5) & 8) * 2;    // lane owning kap = (k1 & 15, k2 & 15)
        const T Rre = __shfl_sync(0xffffffffu, b0re, wl);
        const T Rim = __shfl_sync(0xffffffffu, b0im, wl);
        select_step<T, LAY, PAIRS>(a, om, rec.invD[bk], gamma, bk, Rre, Rim, eta, gam, lane, trow, it, u, v, g, fpix,
                                   pw);
    }
    if (lane < 16) {
        const ImageDesc img = a.descs ? a.descs[we.img] : a.single;
        const int yy = 4 * we.bi + (lane >> 2), xx = 4 * we.bj + (lane & 3);
        img.hr[(long long)yy * img.hr_pitch + xx] = (float)fpix;
    }
}

// ------------------------------------------------- FP32 (f32x2) loop --
// The same iteration with two frequencies kap1 = 8h + 2jj, 8h + 2jj + 1 in
// the two halves of each packed register (Blackwell FFMA2 / FADD2 / FMUL2):
// every element still sees exactly the scalar loop's IEEE operations.
struct CP { float2 re, im; };     // two complex numbers, split re / im

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
// Shared-memory loads the compiler may not hoist out of the iteration loop:
// the tables are loop-invariant, but keeping them in registers across
// iterations would cost more registers (occupancy) than the loads cost.
__device__ __forceinline__ float4 lds4(const void *p)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(smem_addr(p)));
    return v;
}
__device__ __forceinline__ float2 lds2(const void *p)
{
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(smem_addr(p)));
    return v;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ CP addc(CP a, CP b) { return {add2(a.re, b.re), add2(a.im, b.im)}; }
__device__ __forceinline__ CP subc(CP a, CP b) { return {sub2(a.re, b.re), sub2(a.im, b.im)}; }
// exp(-i theta) * z with c = cos theta, s = sin theta, ns = -s
__device__ __forceinline__ CP rot(float2 c, float2 s, float2 ns, CP z)
{
    return {fma2(s, z.im, mul2(c, z.re)), fma2(ns, z.re, mul2(c, z.im))};
}
__device__ __forceinline__ float2 energy(float2 q, CP r) { return mul2(q, fma2(r.im, r.im, mul2(r.re, r.re))); }

// R_k at the lane's 16 candidates of frequency pair jj from the factored
// state Yj (R_k = sum_t conj(h_t(k)) Y_t(k mod 16)): per sub-pixel s the sum
// Z_s of Y_t over the slots holding it (three-quarter: S - Y_s), then a 2x2
// butterfly over the sub-pixel phases.  R[2a + b] holds k = (kap1 + 16a,
// kap2 + 16b) for kap1 = 8h + 2jj (low half of each f32x2) and kap1 + 1
// (high half).
template <int LAY>
__device__ __forceinline__ void state_to_R(const Args &a, const CP (&Yj)[4], const int h, const int jj,
                                           const int k2, const float2 e1c, const float2 e1s, const float2 e1n,
                                           const PairTables &pt, CP (&R)[4])
{
    const int k1 = 8 * h + 2 * jj;
    CP Z[4];
    if constexpr (LAY == kLaySingle) {
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) Z[sp] = Yj[sp];
    } else if constexpr (LAY == kLayGeneral) {
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) {
            Z[sp] = {f2(0.f, 0.f), f2(0.f, 0.f)};
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if ((a.slot_ap >> (4 * t + sp)) & 1u) Z[sp] = addc(Z[sp], Yj[t]);
        }
    } else {
        // Z_s = S - Y_s as the sum of the other three: 6 additions, no cancellation
        const CP P01 = addc(Yj[0], Yj[1]), P23 = addc(Yj[2], Yj[3]);
        Z[0] = addc(Yj[1], P23);
        Z[1] = addc(Yj[0], P23);
        Z[2] = addc(P01, Yj[3]);
        Z[3] = addc(P01, Yj[2]);
    }
    const CP Z0 = Z[0];
    const CP U = rot(e1c, e1s, e1n, Z[1]);
    const float4 e2 = lds4(&pt.e2[4 * h + jj]);
    const CP V = rot(f2(e2.x, e2.y), f2(e2.z, e2.w), lds2(&pt.e2n[4 * h + jj]), Z[2]);
    const float4 e12 = lds4(&pt.e12[k1 + k2]);
    const CP X = rot(f2(e12.x, e12.y), f2(e12.z, e12.w), lds2(&pt.e12n[k1 + k2]), Z[3]);
    const CP pp = addc(Z0, U), mm = subc(Z0, U), ss = addc(V, X), dd = subc(V, X);
    R[0] = addc(pp, ss);
    R[1] = addc(mm, dd);
    R[2] = subc(pp, ss);
    R[3] = subc(mm, dd);
}

// Scores q_k |R_k|^2 / D_k (Eq. 11) of the 16 candidates of pair jj, kept
// in two running maxima (rows kap1 < 16 and kap1 >= 16), each fed in
// increasing index order.
__device__ __forceinline__ void score_pair(const RecordF32 &rec, const CP (&R)[4], const int h, const int jj,
                                           const int k2, float &bs0, int &bk0, float &b0re, float &b0im,
                                           float &bs1, int &bk1, float &b1re, float &b1im)
{
    const int k1 = 8 * h + 2 * jj;
    const float4 q0 = lds4(rec.qDP[4 * h + jj][0][k2]);
    const float4 q1 = lds4(rec.qDP[4 * h + jj][1][k2]);
    const float2 s00 = energy(f2(q0.x, q0.y), R[0]), s01 = energy(f2(q0.z, q0.w), R[1]);
    const float2 s10 = energy(f2(q1.x, q1.y), R[2]), s11 = energy(f2(q1.z, q1.w), R[3]);
    const int ka = k1 * kW + k2, kb = ka + kW;
    keep_best(s00.x, ka, R[0].re.x, R[0].im.x, bs0, bk0, b0re, b0im);
    keep_best(s01.x, ka + 16, R[1].re.x, R[1].im.x, bs0, bk0, b0re, b0im);
    keep_best(s00.y, kb, R[0].re.y, R[0].im.y, bs0, bk0, b0re, b0im);
    keep_best(s01.y, kb + 16, R[1].re.y, R[1].im.y, bs0, bk0, b0re, b0im);
    keep_best(s10.x, ka + 512, R[2].re.x, R[2].im.x, bs1, bk1, b1re, b1im);
    keep_best(s11.x, ka + 528, R[3].re.x, R[3].im.x, bs1, bk1, b1re, b1im);
    keep_best(s10.y, kb + 512, R[2].re.y, R[2].im.y, bs1, bk1, b1re, b1im);
    keep_best(s11.y, kb + 528, R[3].re.y, R[3].im.y, bs1, bk1, b1re, b1im);
}

template <int LAY = kLayThreeQuarter, bool PAIRS = false>
__device__ __forceinline__ void greedy_loop_f32(const Args &a, const RecordF32 &rec, const C2<float> *om,
                                                const C2<float> *omc, const PairTables &pt, const WorkEntry we,
                                                const int lane, C2<float> (&Y0)[8][4])
{
    const int k2 = lane & 15, h = lane >> 4;
    CP Y[4][4];
#pragma unroll
    for (int jj = 0; jj < 4; ++jj)
#pragma unroll
        for (int t = 0; t < 4; ++t)
            Y[jj][t] = {f2(Y0[2 * jj][t].re, Y0[2 * jj + 1][t].re), f2(Y0[2 * jj][t].im, Y0[2 * jj + 1][t].im)};
    const float c1 = om[k2].re, s1 = om[k2].im;     // exp(-2 pi i kap2 / 32) = c1 - i s1
    const float2 e1c = f2(c1, c1), e1s = f2(s1, s1), e1n = f2(-s1, -s1);
    const float gamma = (float)a.gamma;
    const int eta = kOff + ((lane >> 2) & 3), gam = kOff + (lane & 3);
    float fpix = 0.f, pw = 0.f;
    int u = 0, v = 0;
    C2<float> g[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    const long long trow = (long long)we.ord * a.nu_max;

    for (int it = 0; it < a.nu_max; ++it) {
        float bs0 = -1.f, bs1 = -1.f, b0re = 0.f, b0im = 0.f, b1re = 0.f, b1im = 0.f;
        int bk0 = 0, bk1 = 0;
        const int d2 = (v - k2) & 15, d2c = (-v - k2) & 15;
        float2 ngre[4], gim[4], ngim[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            ngre[t] = f2(-g[t].re, -g[t].re);
            gim[t] = f2(g[t].im, g[t].im);
            ngim[t] = f2(-g[t].im, -g[t].im);
        }
        // partner coefficients pw conj(g_t) = (pr, pi), packed as -pr, pi, -pi
        float2 npre[4], ppim[4], nppim[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const float pr = pw * g[t].re, pi = -pw * g[t].im;
            npre[t] = f2(-pr, -pr);
            ppim[t] = f2(pi, pi);
            nppim[t] = f2(-pi, -pi);
        }
        // Eq. 17 for all four group pairs first, then the scores: the two
        // phases give the scheduler independent packed FP32 work (measured
        // 2.7 % faster than interleaving them per pair, same results).
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int k1 = 8 * h + 2 * jj;               // first of the pair
            if (it > 0) {
                // Eq. 17 on the factored state: Y_t -= g_t G_t((uv - kap) mod 16)
                const int d1 = (u - k1) & 15;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const float4 G = *reinterpret_cast<const float4 *>(rec.GP[t][d1][d2]);
                    const float2 Gre = f2(G.x, G.y), Gim = f2(G.z, G.w);
                    Y[jj][t].re = fma2(Gim, gim[t], fma2(Gre, ngre[t], Y[jj][t].re));
                    Y[jj][t].im = fma2(Gre, ngim[t], fma2(Gim, ngre[t], Y[jj][t].im));
                }
                if constexpr (PAIRS) {
                    // the partner -uv: Y_t -= pw conj(g_t) G_t((-uv - kap) mod 16)
                    const int d1c = (-u - k1) & 15;
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const float4 G = *reinterpret_cast<const float4 *>(rec.GP[t][d1c][d2c]);
                        const float2 Gre = f2(G.x, G.y), Gim = f2(G.z, G.w);
                        Y[jj][t].re = fma2(Gim, ppim[t], fma2(Gre, npre[t], Y[jj][t].re));
                        Y[jj][t].im = fma2(Gre, nppim[t], fma2(Gim, npre[t], Y[jj][t].im));
                    }
                }
            }
        }
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            CP R[4];
            state_to_R<LAY>(a, Y[jj], h, jj, k2, e1c, e1s, e1n, pt, R);
            score_pair(rec, R, h, jj, k2, bs0, bk0, b0re, b0im, bs1, bk1, b1re, b1im);
        }
        if (bs1 > bs0) { bs0 = bs1; bk0 = bk1; b0re = b1re; b0im = b1im; }
        float bs = bs0;
        int bk = bk0;
        warp_argmax(bs, bk);
        const int wl = (bk & 15) + ((bk >> 5) & 8) * 2;
        const float Rre = __shfl_sync(0xffffffffu, b0re, wl);
        const float Rim = __shfl_sync(0xffffffffu, b0im, wl);
        select_step<float, LAY, PAIRS>(a, om, rec.invD[bk], gamma, bk, Rre, Rim, eta, gam, lane, trow, it, u, v, g,
                                       fpix, pw);
    }
    if (lane < 16) {
        const ImageDesc img = a.descs ? a.descs[we.img] : a.single;
        const int yy = 4 * we.bi + (lane >> 2), xx = 4 * we.bj + (lane & 3);
        img.hr[(long long)yy * img.hr_pitch + xx] = fpix;
    }
}

// ----------------------------------------------- stored-C (paper) loop --
// The iteration of Eqs. 11-17 in the paper's recurrent form (Table I): the
// projected residual is the loop state, scaled per candidate as R'_k = s_k
// R_k with s_k = sqrt(q_k / D_k) so that the score of Eq. 11 is |R'_k|^2,
// and Eq. 17 subtracts gamma delta times the column of the stored Gram
// matrix (Eq. 14, rows scaled the same way) of the block's local
// measurement matrix: 8 KiB read per iteration, one float4 per lane and
// register pair, 512 contiguous bytes per warp load; delta = R'_uv / (s_uv
// D_uv) (Eq. 16) with the stored 1 / (s_uv D_uv).  R^0 comes from the same
// factored initial projection as the other loops, and the argmax and the
// bookkeeping are the factored loop's.
__device__ __forceinline__ float4 ldg_stream4(const float4 *p)
{
    float4 v;
    asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
}
__device__ __forceinline__ float ldg_stream1(const float *p)
{
    float v;
    asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

// R -= c C_{., l} over the lane's 32 candidates, column col (already loaded).
__device__ __forceinline__ void sub_column(CP (&R)[4][4], const float4 (&col)[16], const C2<float> c)
{
    const float2 ncre = f2(-c.re, -c.re), cim = f2(c.im, c.im), ncim = f2(-c.im, -c.im);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        CP &r = R[i >> 2][i & 3];
        const float2 Cre = f2(col[i].x, col[i].y), Cim = f2(col[i].z, col[i].w);
        r.re = fma2(Cim, cim, fma2(Cre, ncre, r.re));
        r.im = fma2(Cre, ncim, fma2(Cim, ncre, r.im));
    }
}

__device__ __forceinline__ void load_column(const float4 *cs, const int l, const int lane, float4 (&col)[16])
{
    const float4 *p = cs + (size_t)l * 512 + lane;
#pragma unroll
    for (int i = 0; i < 16; ++i) col[i] = ldg_stream4(p + 32 * i);
}

// The state is R'_k = s_k R_k with s_k = sqrt(q_k / D_k), so the score of
// Eq. 11 is |R'_k|^2.
__device__ __forceinline__ float2 norm2(const CP r) { return fma2(r.im, r.im, mul2(r.re, r.re)); }

// Argmax of the stored-C loop.  Slots 4 g .. 4 g + 3 (g = 4 a + jj) are
// four consecutive candidates of the lane in index order, held in R[jj][2a]
// (.x, .y: e = 0, 1 with b = 0) and R[jj][2a + 1] (b = 1).  The scan visits
// the groups in increasing g and keeps the largest score (two three-input
// max operations per group, sm_100 and later), the first group reaching it
// and three of that group's scores; the slot inside the group is the first
// whose score equals the maximum (the fourth if none of the three does).
// The same choice as comparing every candidate in index order, with 7
// operations per group instead of 12 and a dependency chain through the
// running maximum of two operations per group instead of eight.
__device__ __forceinline__ float max3f(const float a, const float b, const float c)
{
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

__device__ __forceinline__ void scan_group(const CP (&Rj)[4], const int a, const int g, float &bs, int &bg,
                                           float &t0, float &t1, float &t2)
{
    const float2 s0 = norm2(Rj[2 * a]), s1 = norm2(Rj[2 * a + 1]);
    const float m = max3f(max3f(bs, s0.x, s1.x), s0.y, s1.y);
    const bool p = m > bs;
    bg = p ? g : bg;
    t0 = p ? s0.x : t0;
    t1 = p ? s1.x : t1;
    t2 = p ? s0.y : t2;
    bs = m;
}

// R of this lane's candidate in a slot (the same slot in every lane).
template <int I>
__device__ __forceinline__ void r_slot(const CP (&R)[4][4], float &re, float &im)
{
    const CP &r = R[(I >> 2) & 3][2 * (I >> 4) + (I & 1)];
    re = ((I >> 1) & 1) ? r.re.y : r.re.x;
    im = ((I >> 1) & 1) ? r.im.y : r.im.x;
}

__device__ __forceinline__ void r_at_slot(const CP (&R)[4][4], const int slot, float &re, float &im)
{
    switch (slot) {
    case 0: r_slot<0>(R, re, im); break;
    case 1: r_slot<1>(R, re, im); break;
    case 2: r_slot<2>(R, re, im); break;
    case 3: r_slot<3>(R, re, im); break;
    case 4: r_slot<4>(R, re, im); break;
    case 5: r_slot<5>(R, re, im); break;
    case 6: r_slot<6>(R, re, im); break;
    case 7: r_slot<7>(R, re, im); break;
    case 8: r_slot<8>(R, re, im); break;
    case 9: r_slot<9>(R, re, im); break;
    case 10: r_slot<10>(R, re, im); break;
    case 11: r_slot<11>(R, re, im); break;
    case 12: r_slot<12>(R, re, im); break;
    case 13: r_slot<13>(R, re, im); break;
    case 14: r_slot<14>(R, re, im); break;
    case 15: r_slot<15>(R, re, im); break;
    case 16: r_slot<16>(R, re, im); break;
    case 17: r_slot<17>(R, re, im); break;
    case 18: r_slot<18>(R, re, im); break;
    case 19: r_slot<19>(R, re, im); break;
    case 20: r_slot<20>(R, re, im); break;
    case 21: r_slot<21>(R, re, im); break;
    case 22: r_slot<22>(R, re, im); break;
    case 23: r_slot<23>(R, re, im); break;
    case 24: r_slot<24>(R, re, im); break;
    case 25: r_slot<25>(R, re, im); break;
    case 26: r_slot<26>(R, re, im); break;
    case 27: r_slot<27>(R, re, im); break;
    case 28: r_slot<28>(R, re, im); break;
    case 29: r_slot<29>(R, re, im); break;
    case 30: r_slot<30>(R, re, im); break;
    default: r_slot<31>(R, re, im); break;
    }
}

template <int LAY = kLayThreeQuarter, bool PAIRS = false>
__device__ __forceinline__ void greedy_loop_stored(const Args &a, const RecordF32 &rec, const float4 *cs,
                                                   const C2<float> *om, const PairTables &pt, const WorkEntry we,
                                                   const int lane, C2<float> (&Y0)[8][4])
{
    const int k2 = lane & 15, h = lane >> 4;
    const float c1 = om[k2].re, s1 = om[k2].im;
    const float2 e1c = f2(c1, c1), e1s = f2(s1, s1), e1n = f2(-s1, -s1);
    CP R[4][4];
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
        CP Yj[4];
#pragma unroll
        for (int t = 0; t < 4; ++t)
            Yj[t] = {f2(Y0[2 * jj][t].re, Y0[2 * jj + 1][t].re), f2(Y0[2 * jj][t].im, Y0[2 * jj + 1][t].im)};
        state_to_R<LAY>(a, Yj, h, jj, k2, e1c, e1s, e1n, pt, R[jj]);
    }
    {
        // R' = s R, the row scales stored after the columns in the same lane order
        const float4 *sc = cs + kStoredScaleOff + lane;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float4 w = ldg_stream4(sc + 32 * i);
            CP &r = R[i >> 2][i & 3];
            r.re = mul2(r.re, f2(w.x, w.y));
            r.im = mul2(r.im, f2(w.z, w.w));
        }
    }
    const float *invd = reinterpret_cast<const float *>(cs + kStoredInvDOff);   // 1 / (s_l D_l)
    const float gamma = (float)a.gamma;
    const int eta = kOff + ((lane >> 2) & 3), gam = kOff + (lane & 3);
    float fpix = 0.f, pw = 0.f;
    int u = 0, v = 0;
    C2<float> g[4];
    const long long trow = (long long)we.ord * a.nu_max;

    for (int it = 0; it < a.nu_max; ++it) {
        // scores are >= 0: starting from 0, a lane whose scores are all 0
        // keeps group 0, slot 0, as a scan from -1 would
        float bs = 0.f, t0 = 0.f, t1 = 0.f, t2 = 0.f;
        int bg = 0;
#pragma unroll
        for (int aa = 0; aa < 2; ++aa)
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) scan_group(R[jj], aa, 4 * aa + jj, bs, bg, t0, t1, t2);
        const int el = t0 == bs ? 0 : t1 == bs ? 1 : t2 == bs ? 2 : 3;
        // slot 4 bg + el = 16 a + 4 jj + 2 e + b -> k
        int bk = (8 * h + 2 * (bg & 3) + (el >> 1) + 16 * (bg >> 2)) * kW + k2 + 16 * (el & 1);
        warp_argmax(bs, bk);
        const bool more = it + 1 < a.nu_max;
        float4 col[16];
        if (more) load_column(cs, bk, lane, col);      // in flight during the bookkeeping
        const float invD = ldg_stream1(invd + bk);
        const int wl = (bk & 15) + ((bk >> 5) & 8) * 2;
        const int slot = ((bk >> 9) << 4) | (((bk >> 6) & 3) << 2) | (((bk >> 5) & 1) << 1) | ((bk >> 4) & 1);
        float mre, mim;
        r_at_slot(R, slot, mre, mim);
        const float Rre = __shfl_sync(0xffffffffu, mre, wl);
        const float Rim = __shfl_sync(0xffffffffu, mim, wl);
        select_step<float, LAY, PAIRS>(a, om, invD, gamma, bk, Rre, Rim, eta, gam, lane, trow, it, u, v, g, fpix,
                                       pw);
        if (more) {
            const C2<float> gd = {gamma * (Rre * invD), gamma * (Rim * invD)};   // as in select_step
            sub_column(R, col, gd);
            if constexpr (PAIRS) {
                // the partner -uv gets conj(gamma delta) (none when uv = -uv)
                load_column(cs, ((-u) & 31) * kW + ((-v) & 31), lane, col);
                sub_column(R, col, C2<float>{pw * gd.re, -pw * gd.im});
            }
        }
    }
    if (lane < 16) {
        const ImageDesc img = a.descs ? a.descs[we.img] : a.single;
        const int yy = 4 * we.bi + (lane >> 2), xx = 4 * we.bj + (lane & 3);
        img.hr[(long long)yy * img.hr_pitch + xx] = fpix;
    }
}

// ------------------------------------------ restricted (shortlist) loop --
// The greedy loop of Eqs. 11-17 over the 64 shortlisted candidates only, in
// the projected-residual form, two blocks per warp: half-warp hb works on
// block hb, its lane l holding R for the candidates at positions l + 16 s,
// s = 0..3, and the column C_{k,uv} of Eq. 14 is rebuilt from the factored
// tables, C_{k,uv} = sum_t conj(h_t(k)) h_t(uv) G_t((uv - k) mod 16).  The
// per-iteration bookkeeping (delta, g_t, Eq. 18) then runs once for both
// blocks, each half-warp for its own.
__device__ __forceinline__ C2<float> h_of(const C2<float> *om, int k, int t)
{
    const int k1 = k >> 5, k2 = k & 31;
    const C2<float> ev = om[k2], eu = om[k1], euv = om[(k1 + k2) & 31];
    const C2<float> P = cadd(cadd(cadd(C2<float>{1, 0}, ev), eu), euv);
    return csub(P, t == 0 ? C2<float>{1, 0} : t == 1 ? ev : t == 2 ? eu : euv);
}

// State of one half-warp lane: its four candidates, their R, q_k / D_k, and
// h_t(k) packed by type pairs (t = 0, 1 and t = 2, 3 in the two halves of
// an f32x2 register): re, im and -im.
struct HalfState {
    int kc[4];
    int coff[4], ce;                 // stored C: each candidate's float4 in a column, and which half of it
    float2 Rre[2], Rim[2], qd[2];    // slots (0, 1) and (2, 3) packed
    float2 hre[4][2], him[4][2], nhim[4][2];
};

// Setup of one block for half-warp hb, with the whole warp working on it:
// the candidates reordered, R^0_k = sum_t conj(h_t(k)) Y_t(k mod 16) with
// the column DFTs evaluated at the candidates only, then handed to the lanes
// of half hb, which add h_t(k) and q_k / D_k.
__device__ __forceinline__ void shortlist_setup(const Args &a, const RecordShortF32 &rec, C2<float> *scratch,
                                                const C2<float> *om, const C2<float> *omc, const float *wt,
                                                const WorkEntry we, const Shortlist &sl, const int lane, const int hb,
                                                HalfState &st)
{
    // Reorder the 64 candidates so that the 8 lanes of a quarter warp hold,
    // in each slot, candidates with distinct (k2 mod 8) where possible: the
    // per-iteration table reads at ((u - k1) mod 16, (v - k2) mod 16) then
    // fall in distinct shared-memory bank groups.  Sorted position r (by k2
    // mod 8, then by list position) goes to group g = r mod 8, member r / 8; group g
    // is slot g / 2 of quarter g mod 2 of the half, i.e. position
    // 16 (g / 2) + 8 (g mod 2) + r / 8.  The order does not change any
    // result (ties are broken on the candidate index).
    int kw[2];
    {
        const int c0 = sl.idx[lane] & (kK - 1), c1 = sl.idx[lane + 32] & (kK - 1);   // in range for any input
        // rank in (k2 mod 8, list position) order: bucket sizes and the
        // position inside a bucket from ballots
        const int q0 = c0 & 7, q1 = c1 & 7;
        const unsigned lt = (1u << lane) - 1u;
        int r0 = 0, r1 = 0, below = 0;
#pragma unroll
        for (int bv = 0; bv < 8; ++bv) {
            const unsigned e0 = __ballot_sync(0xffffffffu, q0 == bv), e1 = __ballot_sync(0xffffffffu, q1 == bv);
            if (q0 == bv) r0 = below + __popc(e0 & lt);
            if (q1 == bv) r1 = below + __popc(e0) + __popc(e1 & lt);
            below += __popc(e0) + __popc(e1);
        }
        int *pos = reinterpret_cast<int *>(scratch);
        __syncwarp();    // the previous block of this warp is done with the scratch
        const int g0 = r0 & 7, g1 = r1 & 7;
        pos[(g0 >> 1) * 16 + (g0 & 1) * 8 + (r0 >> 3)] = c0;
        pos[(g1 >> 1) * 16 + (g1 & 1) * 8 + (r1 >> 3)] = c1;
        __syncwarp();
        kw[0] = pos[lane] & (kK - 1);                  // ranks are a permutation: every position is written
        kw[1] = pos[32 + lane] & (kK - 1);
    }
    // R0 of the candidates at positions lane and lane + 32: Y_t(kap) =
    // sum_p T_t(p, kap2) w16^-(p kap1) over the row DFTs of the window
    // (through the scratch, two types a pass).
    C2<float> hw[2][4];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int t = 0; t < 4; ++t) hw[c][t] = h_of(om, kw[c], t);
    C2<float> acc[4][4];
    window_rows<float>(a, rec, scratch, omc, wt, we, lane, acc);
    Vec4<float> *tb = reinterpret_cast<Vec4<float> *>(scratch);
    C2<float> Rw[2] = {{0, 0}, {0, 0}};
#pragma unroll
    for (int pass = 0; pass < 2; ++pass) {
        __syncwarp();
        rows_to_scratch<float>(acc, tb, pass, lane);
        __syncwarp();
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int kap1 = (kw[c] >> 5) & 15, kap2 = kw[c] & 15;
            C2<float> y0 = {0, 0}, y1 = {0, 0};
#pragma unroll 4
            for (int p = 0; p < 16; ++p) {
                const C2<float> tw = omc[(2 * p * kap1) & 31];
                const Vec4<float> tv = ld4(&tb[p * 16 + kap2]);
                y0 = cadd(y0, cmul(C2<float>{tv.x, tv.y}, tw));
                y1 = cadd(y1, cmul(C2<float>{tv.z, tv.w}, tw));
            }
            Rw[c] = cadd(Rw[c], cadd(cmul(cconj(hw[c][2 * pass]), y0), cmul(cconj(hw[c][2 * pass + 1]), y1)));
        }
    }
    // position 16 s + (lane & 15) sits at lane (16 s + (lane & 15)) mod 32, entry s / 2
    const int l16 = lane & 15;
    int kn[4];
    C2<float> Rn[4];
#pragma unroll
    for (int sl4 = 0; sl4 < 4; ++sl4) {
        const int src = l16 + 16 * (sl4 & 1);
        kn[sl4] = __shfl_sync(0xffffffffu, kw[sl4 >> 1], src);
        Rn[sl4].re = __shfl_sync(0xffffffffu, Rw[sl4 >> 1].re, src);
        Rn[sl4].im = __shfl_sync(0xffffffffu, Rw[sl4 >> 1].im, src);
    }
    if ((lane >> 4) == hb) {
#pragma unroll
        for (int sl4 = 0; sl4 < 4; ++sl4) {
            st.kc[sl4] = kn[sl4];
            {
                // where the stored-C loop's lanes keep candidate k in a column:
                // float4 (4 jj + 2 a + b) * 32 + 16 h + kap2, low or high half by e
                const int k1 = kn[sl4] >> 5, k2f = kn[sl4] & 31;
                st.coff[sl4] = (((k1 >> 1) & 3) * 4 + 2 * (k1 >> 4) + (k2f >> 4)) * 32 + 16 * ((k1 >> 3) & 1) +
                               (k2f & 15);
                st.ce |= (k1 & 1) << sl4;
            }
            if (sl4 & 1) { st.Rre[sl4 >> 1].y = Rn[sl4].re; st.Rim[sl4 >> 1].y = Rn[sl4].im; }
            else { st.Rre[sl4 >> 1].x = Rn[sl4].re; st.Rim[sl4 >> 1].x = Rn[sl4].im; }
            C2<float> hk[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) hk[t] = h_of(om, kn[sl4], t);
#pragma unroll
            for (int pr = 0; pr < 2; ++pr) {
                st.hre[sl4][pr] = f2(hk[2 * pr].re, hk[2 * pr + 1].re);
                st.him[sl4][pr] = f2(hk[2 * pr].im, hk[2 * pr + 1].im);
                st.nhim[sl4][pr] = f2(-hk[2 * pr].im, -hk[2 * pr + 1].im);
            }
            if (sl4 & 1) st.qd[sl4 >> 1].y = rec.qD[kn[sl4]];
            else st.qd[sl4 >> 1].x = rec.qD[kn[sl4]];
        }
    }
}

__device__ __forceinline__ int shortlist_iterations(const Args &a, const Shortlist &sl);

// The shortlist loop for up to two blocks (on[b]: block b is present), one
// per half-warp.  All lanes take part in every shuffle and ballot; a half
// whose block is absent or done only skips the update.
// STORED: the column of C comes from the plan's stored Gram matrix cs (one
// 16-byte load per candidate, gathered from the 8 KiB column) instead of
// being rebuilt from the factored tables.
template <bool STORED>
__device__ __forceinline__ void shortlist_pair(const Args &a, const RecordShortF32 &rec, C2<float> *scratch,
                                               const C2<float> *om, const C2<float> *omc, const float *wt,
                                               const WorkEntry (&we)[2], const bool (&on)[2], const int lane,
                                               const float4 *cs)
{
    const int hb = lane >> 4;
    HalfState st;
    st.ce = 0;
#pragma unroll
    for (int sl4 = 0; sl4 < 4; ++sl4) {
        st.kc[sl4] = 0;
        st.coff[sl4] = 0;
        if (sl4 < 2) st.Rre[sl4] = st.Rim[sl4] = st.qd[sl4] = f2(0.f, 0.f);
#pragma unroll
        for (int pr = 0; pr < 2; ++pr) st.hre[sl4][pr] = st.him[sl4][pr] = st.nhim[sl4][pr] = f2(0.f, 0.f);
    }
    int nu[2] = {0, 0};
#pragma unroll
    for (int b = 0; b < 2; ++b)
        if (on[b]) {
            const Shortlist &sl = a.shortlists[we[b].ord];
            shortlist_setup(a, rec, scratch, om, omc, wt, we[b], sl, lane, b, st);
            nu[b] = shortlist_iterations(a, sl);
        }
    if constexpr (STORED) {
        // the stored columns' scaled state R'_k = s_k R_k, s_k = sqrt(q_k / D_k)
        // from the record's q / D, whose score is |R'_k|^2
#pragma unroll
        for (int pr = 0; pr < 2; ++pr) {
            const float2 sk = f2(sqrtf(st.qd[pr].x), sqrtf(st.qd[pr].y));
            st.Rre[pr] = mul2(st.Rre[pr], sk);
            st.Rim[pr] = mul2(st.Rim[pr], sk);
            st.qd[pr] = f2(1.f, 1.f);
        }
    }
    const int nu_h = hb == 0 ? nu[0] : nu[1];
    const int numax = nu[0] > nu[1] ? nu[0] : nu[1];
    const WorkEntry me = hb == 0 ? we[0] : we[1];
    const float gamma = (float)a.gamma;
    const int eta = kOff + ((lane >> 2) & 3), gam = kOff + (lane & 3);
    float fpix = 0.f, unused_pw = 0.f;
    int u = 0, v = 0;
    C2<float> g[4];
    const long long trow = (long long)me.ord * a.nu_max;
    for (int it = 0; it < numax; ++it) {
        // scores of the four candidates (two f32x2 pairs), the half-warp's
        // largest by warp reductions over each half's inputs (non-negative,
        // so the bits order like the values), then the smallest index among
        // the candidates holding it
        float2 sc01 = fma2(st.Rim[0], st.Rim[0], mul2(st.Rre[0], st.Rre[0]));
        float2 sc23 = fma2(st.Rim[1], st.Rim[1], mul2(st.Rre[1], st.Rre[1]));
        if constexpr (!STORED) {
            sc01 = mul2(st.qd[0], sc01);
            sc23 = mul2(st.qd[1], sc23);
        }
        const unsigned sb[4] = {__float_as_uint(sc01.x), __float_as_uint(sc01.y), __float_as_uint(sc23.x),
                                __float_as_uint(sc23.y)};
        int bk;
        {
            const unsigned bits = max(max(sb[0], sb[1]), max(sb[2], sb[3]));
            const unsigned m0 = __reduce_max_sync(0xffffffffu, hb == 0 ? bits : 0u);
            const unsigned m1 = __reduce_max_sync(0xffffffffu, hb == 1 ? bits : 0u);
            const unsigned mh = hb == 0 ? m0 : m1;
            unsigned kmin = 0xffffffffu;
#pragma unroll
            for (int sl4 = 0; sl4 < 4; ++sl4) kmin = min(kmin, sb[sl4] == mh ? (unsigned)st.kc[sl4] : 0xffffffffu);
            const unsigned i0 = __reduce_min_sync(0xffffffffu, hb == 0 ? kmin : 0xffffffffu);
            const unsigned i1 = __reduce_min_sync(0xffffffffu, hb == 1 ? kmin : 0xffffffffu);
            bk = (int)(hb == 0 ? i0 : i1);
        }
        // the lane of this half holding bk, and its R
        const bool has = st.kc[0] == bk || st.kc[1] == bk || st.kc[2] == bk || st.kc[3] == bk;
        const unsigned mine = (__ballot_sync(0xffffffffu, has) >> (16 * hb)) & 0xFFFFu;
        const int wl = 16 * hb + (mine ? __ffs(mine) - 1 : 0);
        const float sre = st.kc[0] == bk ? st.Rre[0].x : st.kc[1] == bk ? st.Rre[0].y : st.kc[2] == bk ? st.Rre[1].x : st.Rre[1].y;
        const float sim = st.kc[0] == bk ? st.Rim[0].x : st.kc[1] == bk ? st.Rim[0].y : st.kc[2] == bk ? st.Rim[1].x : st.Rim[1].y;
        float4 cv[4];
        if (STORED && it < nu_h) {
            // the candidates' entries of column bk, in flight during the bookkeeping
            const float4 *col = cs + (size_t)(bk & (kK - 1)) * 512;
#pragma unroll
            for (int sl4 = 0; sl4 < 4; ++sl4) cv[sl4] = ldg_stream4(col + st.coff[sl4]);
        }
        const float Rre = __shfl_sync(0xffffffffu, sre, wl);
        const float Rim = __shfl_sync(0xffffffffu, sim, wl);
        if (STORED && it < nu_h) {
            // delta = R'_uv / (s_uv D_uv): a plan storing every table set's
            // Gram matrix keeps 1 / (s D) in the record's invD
            const float invD = rec.invD[bk & (kK - 1)];
            select_step<float>(a, om, invD, gamma, bk & (kK - 1), Rre, Rim, eta, gam, lane & 15, trow, it, u, v, g,
                               fpix, unused_pw);
            // Eq. 17 on the shortlist with the stored column, as the stored-C loop does
            const C2<float> gd = {gamma * (Rre * invD), gamma * (Rim * invD)};   // as in select_step
            const float2 ngr = f2(-gd.re, -gd.re), gi = f2(gd.im, gd.im), ngi = f2(-gd.im, -gd.im);
#pragma unroll
            for (int pr = 0; pr < 2; ++pr) {
                const float4 A = cv[2 * pr], B = cv[2 * pr + 1];
                const bool ea = (st.ce >> (2 * pr)) & 1, eb = (st.ce >> (2 * pr + 1)) & 1;
                const float2 Cre = f2(ea ? A.y : A.x, eb ? B.y : B.x), Cim = f2(ea ? A.w : A.z, eb ? B.w : B.z);
                st.Rre[pr] = fma2(Cim, gi, fma2(Cre, ngr, st.Rre[pr]));
                st.Rim[pr] = fma2(Cre, ngi, fma2(Cim, ngr, st.Rim[pr]));
            }
        } else if (!STORED && it < nu_h) {
            select_step<float>(a, om, rec.invD[bk & (kK - 1)], gamma, bk & (kK - 1), Rre, Rim, eta, gam, lane & 15,
                               trow, it, u, v, g, fpix, unused_pw);
            // Eq. 17 on the shortlist: R_k -= sum_t conj(h_t(k)) g_t G_t(uv - k), two
            // types per f32x2 register
            const float2 gre[2] = {f2(g[0].re, g[1].re), f2(g[2].re, g[3].re)};
            const float2 gim[2] = {f2(g[0].im, g[1].im), f2(g[2].im, g[3].im)};
            const float2 ngim[2] = {f2(-g[0].im, -g[1].im), f2(-g[2].im, -g[3].im)};
            float dre[4], dim[4];
#pragma unroll
            for (int sl4 = 0; sl4 < 4; ++sl4) {
                const int kc = st.kc[sl4];
                const int d1 = (u - (kc >> 5)) & 15, d2 = (v - kc) & 15;
                // two 16-byte loads at (d1, d2): bank group (v - k2) mod 8, which the
                // candidate order keeps distinct within each quarter warp
                const float4 G[2] = {lds4(rec.G01[d1 * 16 + d2]), lds4(rec.G23[d1 * 16 + d2])};
                float2 are = f2(0.f, 0.f), aim = f2(0.f, 0.f);
#pragma unroll
                for (int pr = 0; pr < 2; ++pr) {
                    const float2 Gre = f2(G[pr].x, G[pr].y), Gim = f2(G[pr].z, G[pr].w);
                    const float2 gGre = fma2(Gre, gre[pr], mul2(Gim, ngim[pr]));   // g_t G_t
                    const float2 gGim = fma2(Gim, gre[pr], mul2(Gre, gim[pr]));
                    are = fma2(st.hre[sl4][pr], gGre, fma2(st.him[sl4][pr], gGim, are));
                    aim = fma2(st.hre[sl4][pr], gGim, fma2(st.nhim[sl4][pr], gGre, aim));
                }
                dre[sl4] = are.x + are.y;
                dim[sl4] = aim.x + aim.y;
            }
#pragma unroll
            for (int pr = 0; pr < 2; ++pr) {
                st.Rre[pr] = sub2(st.Rre[pr], f2(dre[2 * pr], dre[2 * pr + 1]));
                st.Rim[pr] = sub2(st.Rim[pr], f2(dim[2 * pr], dim[2 * pr + 1]));
            }
        }
    }
    const bool mine_on = hb == 0 ? on[0] : on[1];
    if (mine_on) {
        if (a.trace_sel != nullptr && (lane & 15) == 0)
            for (int it = nu_h; it < a.nu_max; ++it) {
                a.trace_sel[trow + it] = 0xFFFF;
                a.trace_dc[2 * (trow + it)] = 0.f;
                a.trace_dc[2 * (trow + it) + 1] = 0.f;
            }
        const ImageDesc img = a.descs ? a.descs[me.img] : a.single;
        const int yy = 4 * me.bi + ((lane >> 2) & 3), xx = 4 * me.bj + (lane & 3);
        img.hr[(long long)yy * img.hr_pitch + xx] = fpix;
    }
}

__device__ __forceinline__ int shortlist_iterations(const Args &a, const Shortlist &sl)
{
    if (!a.use_nu_hat) return a.nu_max;
    const float f = sl.nu_frac;
    int nu = f >= 1.f ? a.nu_max : (int)ceilf(fmaxf(f, 0.08f) * a.nu_max);
    return nu > a.nu_max ? a.nu_max : nu;
}

// Kernel modes: 0 = full loop on every block; 1 = shortlist loop on the
// blocks whose left-out mass is <= max_missing, other blocks untouched;
// 2 = full loop on the other blocks only.  Modes 1 and 2 together cover
// every block once; each is its own instantiation, so the register budget
// of one does not constrain the other.  3 and 4 = mode 0 for other sensor
// layouts: slot apertures from a.slot_ap (3), or one sub-pixel per slot (4).
// Bit 3 (kModePairs) added to modes 0, 3, 4: the conjugate-pair update.
// Bit 4 (kModeStoredC) added to those: the column of C read from the stored
// Gram matrix instead of rebuilt from the factored tables.
constexpr int kModePairs = 8;
constexpr int kModeStoredC = 16;
__host__ __device__ constexpr int lay_of(int mode)
{
    return (mode & 7) == 3 ? kLayGeneral : (mode & 7) == 4 ? kLaySingle : kLayThreeQuarter;
}
__host__ __device__ constexpr bool pairs_of(int mode) { return (mode & kModePairs) != 0; }
__host__ __device__ constexpr bool stored_of(int mode) { return (mode & kModeStoredC) != 0; }
__host__ __device__ constexpr bool plain_of(int mode) { return (mode & 7) == 0 || (mode & 7) == 3 || (mode & 7) == 4; }
__host__ __device__ constexpr int learned_of(int mode) { return (mode & 7) == 1 || (mode & 7) == 2 ? (mode & 7) : 0; }

template <typename T, int MODE> struct Loop;
template <int MODE> struct Loop<float, MODE> {
    using Rec = typename RecOf<float, MODE>::type;
    static __device__ __forceinline__ void run(const Args &a, const Rec &rec, C2<float> *scratch,
                                               const C2<float> *om, const C2<float> *omc, const PairTables &pt,
                                               const float *wt, const WorkEntry we, const int lane,
                                               const float4 *cs)
    {
        // (a stored-C launch takes only chunks whose table set has a stored matrix)
        if constexpr (plain_of(MODE) && stored_of(MODE)) {
            C2<float> Y[8][4];
            initial_projection<float>(a, rec, scratch, omc, wt, we, lane, Y);
            greedy_loop_stored<lay_of(MODE), pairs_of(MODE)>(a, rec, cs, om, pt, we, lane, Y);
        } else if constexpr (plain_of(MODE)) {
            C2<float> Y[8][4];
            initial_projection<float>(a, rec, scratch, omc, wt, we, lane, Y);
            greedy_loop_f32<lay_of(MODE), pairs_of(MODE)>(a, rec, om, omc, pt, we, lane, Y);
        } else if constexpr (learned_of(MODE) == 1) {
            const Shortlist &sl = a.shortlists[we.ord];
            if (!(sl.missing <= a.max_missing)) return;
            if (a.n_restricted != nullptr && lane == 0) atomicAdd(a.n_restricted, 1);
            const WorkEntry w2[2] = {we, we};
            const bool on[2] = {true, false};
            shortlist_pair<stored_of(MODE)>(a, rec, scratch, om, omc, wt, w2, on, lane, cs);
        } else {
            const Shortlist &sl = a.shortlists[we.ord];
            if (sl.missing <= a.max_missing) return;
            C2<float> Y[8][4];
            initial_projection<float>(a, rec, scratch, omc, wt, we, lane, Y);
            if constexpr (stored_of(MODE)) greedy_loop_stored<kLayThreeQuarter>(a, rec, cs, om, pt, we, lane, Y);
            else greedy_loop_f32<kLayThreeQuarter>(a, rec, om, omc, pt, we, lane, Y);
        }
    }

    // Mode 1 with two entries per warp: the blocks that take the shortlist
    // loop run it together, one per half-warp.
    static __device__ __forceinline__ void run_pair(const Args &a, const Rec &rec, C2<float> *scratch,
                                                    const C2<float> *om, const C2<float> *omc,
                                                    const PairTables &pt, const float *wt, const WorkEntry e0,
                                                    const WorkEntry e1, const int lane, const float4 *cs)
    {
        const bool r0 = e0.img >= 0 && a.shortlists[e0.ord].missing <= a.max_missing;
        const bool r1 = e1.img >= 0 && a.shortlists[e1.ord].missing <= a.max_missing;
        if (!r0 && !r1) return;
        if (a.n_restricted != nullptr && lane == 0) atomicAdd(a.n_restricted, (int)r0 + (int)r1);
        const WorkEntry w2[2] = {e0, e1};
        const bool on[2] = {r0, r1};
        shortlist_pair<stored_of(MODE)>(a, rec, scratch, om, omc, wt, w2, on, lane, cs);
    }
};
template <int MODE> struct Loop<double, MODE> {
    static __device__ __forceinline__ void run(const Args &a, const Record<double> &rec, C2<double> *scratch,
                                               const C2<double> *om, const C2<double> *omc, const PairTables &,
                                               const double *wt, const WorkEntry we, const int lane,
                                               const float4 *)
    {
        C2<double> Y[8][4];
        initial_projection<double>(a, rec, scratch, omc, wt, we, lane, Y);
        greedy_loop<double, lay_of(MODE), pairs_of(MODE)>(a, rec, om, omc, we, lane, Y);
    }
    static __device__ __forceinline__ void run_pair(const Args &a, const Record<double> &rec, C2<double> *scratch,
                                                    const C2<double> *om, const C2<double> *omc,
                                                    const PairTables &pt, const double *wt, const WorkEntry e0,
                                                    const WorkEntry e1, const int lane, const float4 *)
    {
        if (e0.img >= 0) run(a, rec, scratch, om, omc, pt, wt, e0, lane, nullptr);
        if (e1.img >= 0) run(a, rec, scratch, om, omc, pt, wt, e1, lane, nullptr);
    }
};

// Modes 1 and 2 each take part of the blocks (by the shortlist's left-out
// mass); a chunk none of whose blocks this mode takes is skipped, table copy
// included.  Block-uniform (every thread of the CTA must call it).
template <int MODE>
__device__ __forceinline__ bool chunk_has_work(const Args &a, const int c)
{
    if constexpr (learned_of(MODE) == 0) {
        // a plan with stored and factored table sets runs them as two launches
        if (a.cfilter == 0) return true;
        const bool stored = a.cslot[a.chunk_table[c]] >= 0;
        return a.cfilter == 1 ? stored : !stored;
    } else {
        bool mine = false;
        if (threadIdx.x < kChunk) {
            const WorkEntry we = a.entries[(size_t)c * kChunk + threadIdx.x];
            if (we.img >= 0) {
                const bool restricted = a.shortlists[we.ord].missing <= a.max_missing;
                mine = learned_of(MODE) == 1 ? restricted : !restricted;
            }
        }
        return __syncthreads_or(mine) != 0;
    }
}

// --------------------------------------------------- persistent kernel --
template <typename T, int WARPS, int MINB, int MODE>
__global__ void __launch_bounds__(WARPS * 32, MINB) recurrent_kernel(const Args a)
{
    using L = SmemLayout<T, WARPS, MODE>;
    using Rec = typename RecOf<T, MODE>::type;
    extern __shared__ __align__(128) unsigned char smem[];
    auto slot = [&](int s) { return reinterpret_cast<Rec *>(smem + L::off_slots + s * L::rec); };
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    C2<T> *scratch = reinterpret_cast<C2<T> *>(smem + L::off_scratch + warp * L::scratch);
    C2<T> *om = reinterpret_cast<C2<T> *>(smem + L::off_om);
    C2<T> *omc = reinterpret_cast<C2<T> *>(smem + L::off_omc);
    PairTables *pt = reinterpret_cast<PairTables *>(smem + L::off_pair);
    T *wt = reinterpret_cast<T *>(smem + L::off_w);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L::off_bar);

    for (int i = threadIdx.x; i < 256; i += WARPS * 32) {
        if constexpr (sizeof(T) == 8) wt[i] = a.consts->w64[i];
        else wt[i] = a.consts->w32[i];
    }
    for (int i = threadIdx.x; i < 32; i += WARPS * 32) {
        T re, im;
        if constexpr (sizeof(T) == 8) { re = a.consts->om64[2 * i]; im = a.consts->om64[2 * i + 1]; }
        else { re = a.consts->om32[2 * i]; im = a.consts->om32[2 * i + 1]; }
        om[i] = {re, im};
        omc[i] = {re, -im};
        const float c0 = a.consts->om32[2 * i], s0 = a.consts->om32[2 * i + 1];
        const int n1 = (i + 1) & 31;
        const float c1 = a.consts->om32[2 * n1], s1 = a.consts->om32[2 * n1 + 1];
        pt->e12[i] = make_float4(c0, c1, s0, s1);
        pt->e12n[i] = make_float2(-s0, -s1);
        if (i < 8) {
            const float ca = a.consts->om32[4 * i], sa = a.consts->om32[4 * i + 1];
            const float cb = a.consts->om32[4 * i + 2], sb = a.consts->om32[4 * i + 3];
            pt->e2[i] = make_float4(ca, cb, sa, sb);
            pt->e2n[i] = make_float2(-sa, -sb);
        }
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    const uint32_t rb = (uint32_t)sizeof(Rec);
    const unsigned char *records = learned_of(MODE) == 1 ? a.records_short : a.records;
    // Per slot s: table held (held0/held1), a load in flight (bit s of
    // pending) and the mbarrier parity to wait for (bit s of parity).
    int held0 = -1, held1 = -1;
    uint32_t pending = 0, parity = 0;
    for (int s = 0; s < 2; ++s) {
        const int c = blockIdx.x + s * gridDim.x;
        if (c < a.n_chunks && chunk_has_work<MODE>(a, c)) {
            const int t = a.chunk_table[c];
            if (threadIdx.x == 0) bulk_load(slot(s), records + (size_t)t * rb, rb, &bar[s]);
            if (s == 0) held0 = t; else held1 = t;
            pending |= 1u << s;
        }
    }
    bool failed = false;
    for (int r = 0;; ++r) {
        const int c = blockIdx.x + r * gridDim.x;
        if (c >= a.n_chunks) break;
        const int s = r & 1;
        const bool work = chunk_has_work<MODE>(a, c);   // as when its table was fetched
        if (pending & (1u << s)) {
            const bool ok = mbar_wait(&bar[s], (parity >> s) & 1u);
            if (!__syncthreads_and(ok)) { failed = true; break; }
            parity ^= 1u << s;
            pending &= ~(1u << s);
        }
        const float4 *cs = nullptr;           // this chunk's stored Gram matrix, if any
        if constexpr (stored_of(MODE)) {
            const int cl = a.cslot[a.chunk_table[c]];
            if (cl >= 0) cs = a.cstore + (size_t)cl * (kStoredTableBytes / 16);
        }
        if (!work) {
            // no block of this chunk in this mode
        } else if constexpr (learned_of(MODE) == 1 && WARPS * 2 == kChunk) {
            const WorkEntry e0 = a.entries[(size_t)c * kChunk + warp];
            const WorkEntry e1 = a.entries[(size_t)c * kChunk + warp + WARPS];
            Loop<T, MODE>::run_pair(a, *slot(s), scratch, om, omc, *pt, wt, e0, e1, lane, cs);
        } else {
            for (int e = warp; e < kChunk; e += WARPS) {
                const WorkEntry we = a.entries[(size_t)c * kChunk + e];
                if (we.img >= 0) Loop<T, MODE>::run(a, *slot(s), scratch, om, omc, *pt, wt, we, lane, cs);
            }
        }
        __syncthreads();                       // every warp is done with slot s
        const int c2 = blockIdx.x + (r + 2) * gridDim.x;
        if (c2 < a.n_chunks && chunk_has_work<MODE>(a, c2)) {
            const int t2 = a.chunk_table[c2];
            if (t2 != (s == 0 ? held0 : held1)) {
                if (threadIdx.x == 0) {
                    fence_proxy_async();
                    bulk_load(slot(s), records + (size_t)t2 * rb, rb, &bar[s]);
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

// ------------------------------------------- tables built per block --
// For masks whose local measurement matrices rarely repeat (a non-recurrent
// sensor), each warp builds its block's factored tables itself, in FP32:
//   G_t(d) = conj(DFT of the type-t spatial weights)(d)     (the UNIT DFT),
//   D_k = sum_t |h_t(k)|^2 G_t(0),  q/D and 1/D per candidate,
// into a per-warp RecordF32 in shared memory, then runs the same FP32 loop.
// The DFT scratch of the warp aliases the record's invD array, which is
// written only after the last DFT.
constexpr int kFlyWarps = 4;
struct FlySmem {
    static constexpr size_t rec = sizeof(RecordF32);
    static constexpr size_t off_rec = 0;                                   // kFlyWarps records
    static constexpr size_t off_om = kFlyWarps * rec;
    static constexpr size_t off_omc = off_om + 32 * sizeof(C2<float>);
    static constexpr size_t off_pair = off_omc + 32 * sizeof(C2<float>);
    static constexpr size_t off_w = off_pair + sizeof(PairTables);
    static constexpr size_t off_q = off_w + 256 * sizeof(float);            // q per candidate
    static constexpr size_t bytes = off_q + kK * sizeof(float);
};
static_assert(offsetof(RecordF32, invD) % 16 == 0 && sizeof(RecordF32::invD) >= 256 * 2 * sizeof(C2<float>),
              "the DFT scratch must fit in invD");

template <bool PAIRS>
__global__ void __launch_bounds__(kFlyWarps * 32, 2) onthefly_kernel(const Args a, int n_entries)
{
    extern __shared__ __align__(128) unsigned char smem[];
    using L = FlySmem;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    RecordF32 &rec = *reinterpret_cast<RecordF32 *>(smem + L::off_rec + warp * L::rec);
    C2<float> *scratch = reinterpret_cast<C2<float> *>(rec.invD);
    C2<float> *om = reinterpret_cast<C2<float> *>(smem + L::off_om);
    C2<float> *omc = reinterpret_cast<C2<float> *>(smem + L::off_omc);
    PairTables *pt = reinterpret_cast<PairTables *>(smem + L::off_pair);
    float *wt = reinterpret_cast<float *>(smem + L::off_w);
    float *qv = reinterpret_cast<float *>(smem + L::off_q);
    for (int i = threadIdx.x; i < 256; i += blockDim.x) wt[i] = a.consts->w32[i];
    for (int i = threadIdx.x; i < kK; i += blockDim.x) qv[i] = a.q[i];
    for (int i = threadIdx.x; i < 32; i += blockDim.x) {
        const float re = a.consts->om32[2 * i], im = a.consts->om32[2 * i + 1];
        om[i] = {re, im};
        omc[i] = {re, -im};
        const int n1 = (i + 1) & 31;
        pt->e12[i] = make_float4(re, a.consts->om32[2 * n1], im, a.consts->om32[2 * n1 + 1]);
        pt->e12n[i] = make_float2(-im, -a.consts->om32[2 * n1 + 1]);
        if (i < 8) {
            const float ca = a.consts->om32[4 * i], sa = a.consts->om32[4 * i + 1];
            const float cb = a.consts->om32[4 * i + 2], sb = a.consts->om32[4 * i + 3];
            pt->e2[i] = make_float4(ca, cb, sa, sb);
            pt->e2n[i] = make_float2(-sa, -sb);
        }
    }
    __syncthreads();
    const int k2 = lane & 15, h = lane >> 4;
    for (int e = blockIdx.x * kFlyWarps + warp; e < n_entries; e += gridDim.x * kFlyWarps) {
        const WorkEntry we = a.entries[e];
        if (we.img < 0) continue;
        const ImageDesc img = a.descs ? a.descs[we.img] : a.single;
        const uint8_t *mask = a.masks + a.mask_offset[we.img];
        const int p0 = 2 * we.bi - kOff / 2, q0 = 2 * we.bj - kOff / 2;
        __syncwarp();                       // the previous block is done with the record
        for (int m = lane; m < 256; m += 32) {
            const int P = p0 + (m >> 4), Q = q0 + (m & 15);
            rec.types[m] = (P >= 0 && P < img.lr_h && Q >= 0 && Q < img.lr_w) ? mask[(long long)P * img.lr_w + Q] : 255;
        }
        __syncwarp();
        // G_t(d1, d2) = conj(Yw_t(d1, d2)) for d1 = 8h + i, d2 = k2
        C2<float> Yw[8][4];
        initial_projection<float, true>(a, rec, scratch, omc, wt, we, lane, Yw);
        C2<float> prev[4];                  // G_t(8h - 1, k2), owned by the other half
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            prev[t].re = __shfl_xor_sync(0xffffffffu, Yw[7][t].re, 16);
            prev[t].im = -__shfl_xor_sync(0xffffffffu, Yw[7][t].im, 16);
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int d1 = 8 * h + i;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const C2<float> ga = cconj(Yw[i][t]);
                const C2<float> gb = i > 0 ? cconj(Yw[i - 1][t]) : prev[t];
                *reinterpret_cast<float4 *>(rec.GP[t][d1][k2]) = make_float4(ga.re, gb.re, ga.im, gb.im);
            }
        }
        // G_t(0) = total weight of type t: from lane 0 (d = (0, 0))
        float W0[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) W0[t] = __shfl_sync(0xffffffffu, Yw[0][t].re, 0);
        // D, q/D for this lane's 32 candidates k = (8h + i + 16A, k2 + 16B)
        float invd[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float qd[4];
#pragma unroll
            for (int A = 0; A < 2; ++A)
#pragma unroll
                for (int B = 0; B < 2; ++B) {
                    const int k = (8 * h + i + 16 * A) * kW + k2 + 16 * B;
                    float D = 0.f;
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const C2<float> ht = h_of(om, k, t);
                        D += (ht.re * ht.re + ht.im * ht.im) * W0[t];
                    }
                    const float inv = D > 1e-30f ? 1.0f / D : 0.f;
                    invd[i][2 * A + B] = inv;
                    qd[2 * A + B] = qv[k] * inv;
                    if (PAIRS) {
                        // the argmax sees one member of each conjugate pair
                        const int k1 = k >> 5, kk2 = k & 31;
                        if (((-k1) & 31) * kW + ((-kk2) & 31) < k) qd[2 * A + B] = 0.f;
                    }
                }
            // qDP[j][A][k2] = (qD(2j, B=0), qD(2j+1, B=0), qD(2j, B=1), qD(2j+1, B=1))
            const int j = (8 * h + i) >> 1, el = i & 1;
#pragma unroll
            for (int A = 0; A < 2; ++A) {
                rec.qDP[j][A][k2][el] = qd[2 * A];
                rec.qDP[j][A][k2][2 + el] = qd[2 * A + 1];
            }
        }
        C2<float> Y[8][4];
        initial_projection<float>(a, rec, scratch, omc, wt, we, lane, Y);
        __syncwarp();                       // scratch (= invD) no longer needed
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int A = 0; A < 2; ++A)
#pragma unroll
                for (int B = 0; B < 2; ++B) rec.invD[(8 * h + i + 16 * A) * kW + k2 + 16 * B] = invd[i][2 * A + B];
        __syncwarp();
        greedy_loop_f32<kLayThreeQuarter, PAIRS>(a, rec, om, omc, *pt, we, lane, Y);
    }
}

// ---------------------------------------------------------- direct path --
// Direct L-JSDE (Eqs. 4-10): per block the residual r (256 complex, in the
// warp's scratch) and, every iteration, N_k = sum_m conj(a_m(k)) w_m r_m for
// all 1024 k with a_m(k) evaluated from the roots-of-unity table (O(W^4)).
// Any per-pixel aperture: a_m(k) sums the phases of m's transparent
// sub-pixels; a candidate whose phase sum cancels exactly for every aperture
// in the window is not observed by any measurement and scores 0.
constexpr int kDirectWarps = 4;
struct DirectSmem {
    float2 r[kDirectWarps][256];
    float wr[kDirectWarps][256][2];
    uint8_t type[kDirectWarps][256];     // aperture code, 0 = no measurement
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
        uint32_t present = 0;                // bit a: aperture a occurs in the window
        for (int m = lane; m < 256; m += 32) {
            const int p = m >> 4, q = m & 15, P = p0 + p, Q = q0 + q;
            int t = 0;
            float y = 0.f;
            if (P >= 0 && P < img.lr_h && Q >= 0 && Q < img.lr_w) {
                const int code = mask[(long long)P * img.lr_w + Q];
                t = a.layout == RLJSDE_LAYOUT_APERTURE ? code & 15 : 15 ^ (1 << (code & 3));
                if (t != 0) {
                    y = img.lr[(long long)P * img.lr_pitch + Q];
                    if (!isfinite(y)) { bad = true; y = 0.f; }
                }
            }
            present |= 1u << t;
            sm.type[warp][m] = (uint8_t)t;
            sm.r[warp][m] = make_float2(y, 0.f);
        }
        if (bad) atomicOr(a.status, kStatusNonfinite);
        present = __reduce_or_sync(0xffffffffu, present) & ~1u;
        __syncwarp();
        // D_k = sum_m w_m |a_m(k)|^2 for this lane's 32 candidates k = lane + 32 j
        float D[32];
        for (int j = 0; j < 32; ++j) D[j] = 0.f;
        for (int m = 0; m < 256; ++m) {
            const int t = sm.type[warp][m];
            if (t == 0) continue;
            const int p = m >> 4, q = m & 15;
            const float wm = sm.w[m];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int k1 = j, k2 = lane;
                float are = 0.f, aim = 0.f;
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    if (!((t >> s) & 1)) continue;
                    const float2 z = sm.om[((2 * p + (s >> 1)) * k1 + (2 * q + (s & 1)) * k2) & 31];
                    are += z.x;
                    aim += z.y;
                }
                D[j] += wm * (are * are + aim * aim);
            }
        }
        // candidates no aperture of the window observes
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if ((present & ~(uint32_t)a.consts->vanish[j * kW + lane]) == 0) D[j] = 0.f;
        float fpix = 0.f;
        const int eta = kOff + ((lane >> 2) & 3), gam = kOff + (lane & 3);
        const long long trow = (long long)we.ord * a.nu_max;
        for (int it = 0; it < a.nu_max; ++it) {
            for (int m = lane; m < 256; m += 32) {
                const float wm = sm.type[warp][m] != 0 ? sm.w[m] : 0.f;
                sm.wr[warp][m][0] = wm * sm.r[warp][m].x;
                sm.wr[warp][m][1] = wm * sm.r[warp][m].y;
            }
            __syncwarp();
            float Nre[32], Nim[32];
            for (int j = 0; j < 32; ++j) Nre[j] = Nim[j] = 0.f;
            for (int m = 0; m < 256; ++m) {
                const int t = sm.type[warp][m];
                if (t == 0) continue;
                const int p = m >> 4, q = m & 15;
                const float xr = sm.wr[warp][m][0], xi = sm.wr[warp][m][1];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    float are = 0.f, aim = 0.f;
#pragma unroll
                    for (int s = 0; s < 4; ++s) {
                        if (!((t >> s) & 1)) continue;
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
                // conjugate-pair update: the argmax sees one member of each pair
                if (a.pairs && ((-j) & 31) * kW + ((-lane) & 31) < k) continue;
                const float s = D[j] > 0.f ? a.q[k] * (Nre[j] * Nre[j] + Nim[j] * Nim[j]) / D[j] : 0.f;
                if (s > bs) {
                    bs = s;
                    bk = k;
                    bre = D[j] > 0.f ? Nre[j] / D[j] : 0.f;
                    bim = D[j] > 0.f ? Nim[j] / D[j] : 0.f;
                }
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
            // conjugate-pair update: c_-uv += conj(gamma delta) as well (not for uv = -uv),
            // so r -= x + conj(x) with x = gamma delta a_m(uv): twice its real part
            const float pf = (a.pairs && ((u & 15) != 0 || (v & 15) != 0)) ? 2.f : 1.f;
            // r_m -= gamma delta a_m(uv)   (Eq. 7)
            for (int m = lane; m < 256; m += 32) {
                const int t = sm.type[warp][m];
                if (t == 0) continue;
                const int p = m >> 4, q = m & 15;
                float are = 0.f, aim = 0.f;
                for (int s = 0; s < 4; ++s) {
                    if (!((t >> s) & 1)) continue;
                    const float2 z = sm.om[((2 * p + (s >> 1)) * u + (2 * q + (s & 1)) * v) & 31];
                    are += z.x;
                    aim += z.y;
                }
                float2 r = sm.r[warp][m];
                if (pf == 2.f) {
                    r.x -= 2.f * (gre * are - gim * aim);
                } else {
                    r.x -= gre * are - gim * aim;
                    r.y -= gre * aim + gim * are;
                }
                sm.r[warp][m] = r;
            }
            const float2 ph = sm.om[(eta * u + gam * v) & 31];
            fpix += pf * (gre * ph.x - gim * ph.y);
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
// Instantiations of the persistent kernel: loop precision, warps per CTA and
// the minimum resident CTAs per SM the register budget is sized for.
struct Variant {
    int fp64, warps, minb, mode;
    void (*fn)(Args);
    size_t smem;
};
#define RLJSDE_VARIANT(T, W, M, MODE) \
    {sizeof(T) == 8, W, M, MODE, recurrent_kernel<T, W, M, MODE>, SmemLayout<T, W, MODE>::bytes}
const Variant kVariants[] = {
    RLJSDE_VARIANT(float, 4, 3, 0), RLJSDE_VARIANT(float, 4, 4, 0), RLJSDE_VARIANT(float, 8, 2, 0),
    RLJSDE_VARIANT(float, 8, 1, 0), RLJSDE_VARIANT(double, 4, 1, 0), RLJSDE_VARIANT(double, 8, 1, 0),
    RLJSDE_VARIANT(float, 4, 3, 1), RLJSDE_VARIANT(float, 8, 2, 1), RLJSDE_VARIANT(float, 4, 3, 2),
    RLJSDE_VARIANT(float, 4, 3, 3), RLJSDE_VARIANT(float, 8, 2, 3), RLJSDE_VARIANT(double, 4, 1, 3),
    RLJSDE_VARIANT(float, 4, 3, 4), RLJSDE_VARIANT(float, 8, 2, 4), RLJSDE_VARIANT(double, 4, 1, 4),
    RLJSDE_VARIANT(float, 4, 3, 8), RLJSDE_VARIANT(float, 4, 3, 11), RLJSDE_VARIANT(float, 4, 3, 12),
    RLJSDE_VARIANT(double, 4, 1, 8), RLJSDE_VARIANT(double, 4, 1, 11), RLJSDE_VARIANT(double, 4, 1, 12),
    // the stored-C loop: one CTA of 8 warps per SM with the full register file
    // (254 registers, no spills) iterates 4 % faster than 4 warps x 3 CTAs
    // (168, spilling) and 2 % faster than 4 warps x 2 CTAs, but its initial
    // projection is 7 % slower: 4 x 3 for short loops (nu_max < 20)
    RLJSDE_VARIANT(float, 8, 1, 16), RLJSDE_VARIANT(float, 4, 3, 16), RLJSDE_VARIANT(float, 8, 1, 19),
    RLJSDE_VARIANT(float, 8, 1, 20),
    RLJSDE_VARIANT(float, 8, 1, 24), RLJSDE_VARIANT(float, 8, 1, 27), RLJSDE_VARIANT(float, 8, 1, 28),
    // the learned path's full loop on the blocks the gate sends back: few per
    // chunk, so more CTAs of fewer warps (with a tenth of the blocks sent
    // back the learned path ran at 551 MP/s with 4 x 3, 415 with 8 x 1)
    RLJSDE_VARIANT(float, 4, 3, 17), RLJSDE_VARIANT(float, 4, 3, 18),
};
#undef RLJSDE_VARIANT
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

int occupancy(const Variant &v)
{
    int n = 0;
    if (cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem) != cudaSuccess)
        return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, v.fn, v.warps * 32, v.smem) != cudaSuccess) return -1;
    return n;
}

Args make_args(const rljsde_plan *p)
{
    Args a{};
    a.entries = p->d_entries;
    a.chunk_table = p->d_chunk_table;
    a.n_chunks = p->n_chunks;
    a.records = static_cast<const unsigned char *>(p->d_records);
    a.records_short = static_cast<const unsigned char *>(p->d_records_short);
    a.cstore = static_cast<const float4 *>(p->d_cstore);
    a.cslot = p->d_cslot;
    a.record_bytes = (uint32_t)p->record_bytes;
    a.consts = p->d_consts;
    a.descs = nullptr;
    a.nu_max = p->params.nu_max;
    a.gamma = p->params.gamma_odc;
    a.status = p->d_status;
    a.masks = p->d_masks;
    a.mask_offset = p->d_mask_offset;
    a.q = p->d_qD;
    a.slot_ap = p->slot_ap;
    a.layout = p->params.layout;
    a.pairs = p->params.pairs;
    return a;
}

int launch(const rljsde_plan *p, const Args &a, cudaStream_t s)
{
    if (p->direct) {
        direct_kernel<<<p->grid, kDirectWarps * 32, 0, s>>>(a, p->n_entries);
    } else if (p->onthefly) {
        if (p->params.pairs) onthefly_kernel<true><<<p->grid, kFlyWarps * 32, FlySmem::bytes, s>>>(a, p->n_entries);
        else onthefly_kernel<false><<<p->grid, kFlyWarps * 32, FlySmem::bytes, s>>>(a, p->n_entries);
    } else {
        // the stored-C loop on the table sets with a stored Gram matrix, the
        // factored loop on the others: one launch each (one kernel holding
        // both loops spills and ran the stored loop 1.5x slower)
        const bool mixed = p->n_stored > 0 && p->n_stored < p->n_tables;
        if (p->n_stored > 0) {
            Args b = a;
            b.cfilter = mixed ? 1 : 0;
            const Variant &v = kVariants[p->variant_stored];
            v.fn<<<p->grid_stored, v.warps * 32, v.smem, s>>>(b);
        }
        if (p->n_stored < p->n_tables) {
            Args b = a;
            b.cfilter = mixed ? 2 : 0;
            const Variant &v = kVariants[p->variant];
            v.fn<<<p->grid, v.warps * 32, v.smem, s>>>(b);
        }
    }
    return cudaGetLastError() == cudaSuccess ? RLJSDE_OK : RLJSDE_ERR_CUDA;
}

// Launch of one learned-mode variant (mode 1 or 2) with its full occupancy.
int launch_mode(const rljsde_plan *p, const Args &a, int mode, int warps, int minb, cudaStream_t s)
{
    for (int i = 0; i < kNumVariants; ++i) {
        const Variant &v = kVariants[i];
        if (v.mode != mode || v.warps != warps || v.fp64 || (minb && v.minb != minb)) continue;
        const int occ = occupancy(v);
        if (occ <= 0) return RLJSDE_ERR_CUDA;
        long long g = (long long)p->sm_count * occ;
        const int grid = (int)(p->n_chunks < g ? (p->n_chunks > 0 ? p->n_chunks : 1) : g);
        v.fn<<<grid, v.warps * 32, v.smem, s>>>(a);
        return cudaGetLastError() == cudaSuccess ? RLJSDE_OK : RLJSDE_ERR_CUDA;
    }
    return RLJSDE_ERR_UNSUPPORTED;
}

// Stored Gram matrix (c_supply) of Eq. 14 in the factored form of the
// tables, C_{k,l} = sum_t conj(h_t(k)) h_t(l) G_t((l - k) mod 16), each row
// scaled by s_k = sqrt(q_k / D_k) (the stored-C loop's state is s R),
// evaluated in FP64 from the FP64 tables and rounded to FP32 once, in the
// loop's read order (float4 i * 32 + lane of column l: the candidates of
// lane's register pair i).  One CTA per (column, stored table set), one
// thread per float4.
__device__ __forceinline__ C2<double> h64(const double2 *om, const uint32_t slot_ap, const int t, const int k1,
                                          const int k2)
{
    const int ap = (int)(slot_ap >> (4 * t)) & 15;
    C2<double> z = {0.0, 0.0};
    for (int e = 0; e < 2; ++e)
        for (int g = 0; g < 2; ++g)
            if ((ap >> (2 * e + g)) & 1) {
                const double2 w = om[(e * k1 + g * k2) & 31];
                z.re += w.x;
                z.im += w.y;
            }
    return z;
}

// The candidate k of float4 i * 32 + lane of a stored column (low half; the
// high half holds k + 32).
__device__ __forceinline__ int stored_k(const int i, const int lane)
{
    const int jj = i >> 2, qa = (i >> 1) & 1, qb = i & 1;
    return (8 * (lane >> 4) + 2 * jj + 16 * qa) * kW + (lane & 15) + 16 * qb;
}

__global__ void __launch_bounds__(512) build_c_kernel(const double *g64, const Consts *consts,
                                                      const uint32_t slot_ap, float4 *out)
{
    __shared__ double2 G[4][256];
    __shared__ double2 om[32];
    const int l = blockIdx.x, tab = blockIdx.y;
    const double *src = g64 + (size_t)tab * kStoredBuildDoubles;
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) G[i >> 8][i & 255] = make_double2(src[2 * i], src[2 * i + 1]);
    if (threadIdx.x < 32) om[threadIdx.x] = make_double2(consts->om64[2 * threadIdx.x], consts->om64[2 * threadIdx.x + 1]);
    __syncthreads();
    const int i = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int l1 = l >> 5, l2 = l & 31;
    float re[2], im[2];
    for (int e = 0; e < 2; ++e) {
        const int k = stored_k(i, lane) + kW * e, k1 = k >> 5, k2 = k & 31;
        const int d = ((l1 - k1) & 15) * 16 + ((l2 - k2) & 15);
        double cre = 0.0, cim = 0.0;
        for (int t = 0; t < 4; ++t) {
            const C2<double> hk = h64(om, slot_ap, t, k1, k2), hl = h64(om, slot_ap, t, l1, l2);
            const C2<double> z = cmul(cconj(hk), hl);
            const double2 gt = G[t][d];
            cre += z.re * gt.x - z.im * gt.y;
            cim += z.re * gt.y + z.im * gt.x;
        }
        const double sk = sqrt(src[2048 + k]);
        re[e] = (float)(sk * cre);
        im[e] = (float)(sk * cim);
    }
    out[(size_t)tab * (kStoredTableBytes / 16) + (size_t)l * 512 + threadIdx.x] =
        make_float4(re[0], re[1], im[0], im[1]);
}

// The row scales s_k in the lane order and 1 / (s_l D_l) of each stored
// table set; one CTA of 512 threads per table set.
__global__ void __launch_bounds__(512) build_c_scales_kernel(const double *g64, float4 *out)
{
    const int tab = blockIdx.x;
    const double *src = g64 + (size_t)tab * kStoredBuildDoubles;
    float4 *base = out + (size_t)tab * (kStoredTableBytes / 16);
    const int i = threadIdx.x >> 5, lane = threadIdx.x & 31, k = stored_k(i, lane);
    const float s0 = (float)sqrt(src[2048 + k]), s1 = (float)sqrt(src[2048 + k + kW]);
    base[kStoredScaleOff + threadIdx.x] = make_float4(s0, s1, s0, s1);
    float *invd = reinterpret_cast<float *>(base + kStoredInvDOff);
    for (int l = threadIdx.x; l < kK; l += blockDim.x) {
        const double sl = sqrt(src[2048 + l]), invD = src[2048 + kK + l];
        invd[l] = sl > 0.0 ? (float)(invD / sl) : 0.f;
    }
}

}  // namespace

int build_stored_c(rljsde_plan *p, const double *d_g64)
{
    if (!p->d_cstore || p->n_stored < 1 || p->n_stored > 65535) return RLJSDE_ERR_INVALID_ARG;
    build_c_kernel<<<dim3(kK, p->n_stored), 512>>>(d_g64, p->d_consts, p->slot_ap,
                                                  static_cast<float4 *>(p->d_cstore));
    build_c_scales_kernel<<<p->n_stored, 512>>>(d_g64, static_cast<float4 *>(p->d_cstore));
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return RLJSDE_ERR_CUDA;
    return RLJSDE_OK;
}

int choose_launch(rljsde_plan *p, int warps, int ctas_per_sm)
{
    if (p->onthefly) {
        int n = 0;
        void (*fly)(const Args, int) = p->params.pairs ? onthefly_kernel<true> : onthefly_kernel<false>;
        if (cudaFuncSetAttribute(fly, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FlySmem::bytes) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fly, kFlyWarps * 32, FlySmem::bytes) != cudaSuccess)
            return RLJSDE_ERR_CUDA;
        if (n < 1) return RLJSDE_ERR_UNSUPPORTED;
        p->warps = kFlyWarps;
        p->ctas_per_sm = ctas_per_sm > 0 ? (ctas_per_sm < n ? ctas_per_sm : n) : n;
        long long want = ((long long)p->n_entries + kFlyWarps - 1) / kFlyWarps;
        long long g = (long long)p->sm_count * p->ctas_per_sm;
        p->grid = (int)(want < g ? (want > 0 ? want : 1) : g);
        return RLJSDE_OK;
    }
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
    // Default: 4 warps per CTA, as many CTAs as the 168-register variant fits.
    if (warps == 0) { warps = 4; if (ctas_per_sm == 0) ctas_per_sm = 3; }
    const int fp64 = p->params.precision == 1;
    const int mode = (p->kind == 1 ? 3 : p->kind == 3 ? 4 : 0) | (p->params.pairs ? kModePairs : 0);
    if (p->n_stored > 0 && !fp64) {
        // the stored-C loop: 8 warps in one CTA per SM, or 4 warps x 3 CTAs for
        // short loops where that instantiation exists
        const int want_warps = p->params.nu_max >= 20 ? 8 : 4;
        p->variant_stored = -1;
        for (int i = 0; i < kNumVariants; ++i)
            if (!kVariants[i].fp64 && kVariants[i].mode == (mode | kModeStoredC) &&
                (p->variant_stored < 0 || kVariants[i].warps == want_warps))
                p->variant_stored = i;
        if (p->variant_stored < 0) return RLJSDE_ERR_UNSUPPORTED;
        const int occ = occupancy(kVariants[p->variant_stored]);
        if (occ < 0) return RLJSDE_ERR_CUDA;
        if (occ == 0) return RLJSDE_ERR_UNSUPPORTED;
        long long g = (long long)p->sm_count * occ;
        p->grid_stored = (int)(p->n_chunks < g ? (p->n_chunks > 0 ? p->n_chunks : 1) : g);
        p->ctas_stored = occ;
        p->warps_stored = kVariants[p->variant_stored].warps;
    }
    // The variant with this precision and warp count whose register budget
    // admits the requested CTAs per SM (the largest one not above it).
    int best = -1, best_occ = 0;
    for (int pass = 0; pass < 2 && best < 0; ++pass)    // second pass: smallest budget above the request
        for (int i = 0; i < kNumVariants; ++i) {
            const Variant &v = kVariants[i];
            if (v.fp64 != fp64 || v.warps != warps || v.mode != mode) continue;
            if (pass == 0 && ctas_per_sm > 0 && v.minb > ctas_per_sm) continue;
            const int occ = occupancy(v);
            if (occ < 0) return RLJSDE_ERR_CUDA;
            if (occ == 0) continue;
            const bool better = best < 0 || (pass == 0 ? v.minb > kVariants[best].minb
                                                       : v.minb < kVariants[best].minb);
            if (better) { best = i; best_occ = occ; }
        }
    if (best < 0) return RLJSDE_ERR_UNSUPPORTED;
    p->variant = best;
    p->warps = warps;
    p->ctas_per_sm = ctas_per_sm > 0 ? (ctas_per_sm < best_occ ? ctas_per_sm : best_occ) : best_occ;
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

int rljsde_reconstruct_learned(const rljsde_plan_t *plan, const float *lr, size_t lr_pitch, float *hr,
                               size_t hr_pitch, const void *shortlists, float max_missing, int use_nu_hat,
                               uint16_t *sel, float *dc, int *n_restricted, void *stream)
{
    if (!plan || !lr || !hr || !shortlists) return RLJSDE_ERR_INVALID_ARG;
    if (plan->n_images != 1 || plan->direct || plan->onthefly || plan->params.precision != 0 || plan->kind != 0 ||
        plan->params.layout != RLJSDE_LAYOUT_THREE_QUARTER || plan->params.pairs)
        return RLJSDE_ERR_UNSUPPORTED;
    if (lr_pitch < (size_t)plan->lr_w[0] || hr_pitch < (size_t)(2 * plan->lr_w[0])) return RLJSDE_ERR_INVALID_ARG;
    if ((sel == nullptr) != (dc == nullptr)) return RLJSDE_ERR_INVALID_ARG;
    Args a = make_args(plan);
    a.single = {lr, hr, plan->lr_h[0], plan->lr_w[0], (long long)lr_pitch, (long long)hr_pitch};
    a.trace_sel = sel;
    a.trace_dc = dc;
    a.shortlists = static_cast<const Shortlist *>(shortlists);
    a.max_missing = max_missing;
    a.use_nu_hat = use_nu_hat;
    a.n_restricted = n_restricted;
    // shortlist blocks first, then the full loop on the rest
    // with every table set's Gram matrix stored, both loops read its columns
    const int sc = plan->n_stored > 0 && plan->n_stored == plan->n_tables ? kModeStoredC : 0;
    const int lw = sc ? 4 : plan->learned_warps, lm = sc ? 3 : plan->learned_minb;
    int st = launch_mode(plan, a, 1 | sc, lw, lm, (cudaStream_t)stream);
    if (st == RLJSDE_OK) st = launch_mode(plan, a, 2 | sc, 4, 0, (cudaStream_t)stream);
    return st;
}

int rljsde_reconstruct_batch(const rljsde_plan_t *plan, void *stream)
{
    if (!plan) return RLJSDE_ERR_INVALID_ARG;
    Args a = make_args(plan);
    a.descs = plan->d_images;
    return launch(plan, a, (cudaStream_t)stream);
}

int rljsde_autotune(rljsde_plan_t *plan, const float *lr, size_t lr_pitch, float *hr, size_t hr_pitch, int reps,
                    void *stream, int *warps_out, int *ctas_out, float *ms_out)
{
    if (!plan || reps < 1 || reps > 1000) return RLJSDE_ERR_INVALID_ARG;
    if ((lr == nullptr) != (hr == nullptr)) return RLJSDE_ERR_INVALID_ARG;
    if (lr && plan->n_images != 1) return RLJSDE_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Args a = make_args(plan);
    if (lr) {
        if (lr_pitch < (size_t)plan->lr_w[0] || hr_pitch < (size_t)(2 * plan->lr_w[0])) return RLJSDE_ERR_INVALID_ARG;
        a.single = {lr, hr, plan->lr_h[0], plan->lr_w[0], (long long)lr_pitch, (long long)hr_pitch};
    } else {
        a.descs = plan->d_images;
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return RLJSDE_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return RLJSDE_ERR_CUDA; }
    const int keep_w = plan->warps, keep_c = plan->ctas_per_sm;
    float best_ms = 1e30f;
    int best_w = keep_w, best_c = keep_c, st = RLJSDE_OK;
    const int shapes[][2] = {{4, 1}, {4, 2}, {4, 3}, {4, 4}, {8, 1}, {8, 2}};
    for (const auto &sh : shapes) {
        if (plan->direct || plan->onthefly) break;
        if (choose_launch(plan, sh[0], sh[1]) != RLJSDE_OK) continue;
        if (plan->ctas_per_sm != sh[1]) continue;          // did not fit
        if ((st = launch(plan, a, s)) != RLJSDE_OK) break; // warm-up
        float ms = 1e30f;
        for (int r = 0; r < reps && st == RLJSDE_OK; ++r) {
            cudaEventRecord(e0, s);
            st = launch(plan, a, s);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) { st = RLJSDE_ERR_CUDA; break; }
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (t < ms) ms = t;
        }
        if (st != RLJSDE_OK) break;
        if (ms < best_ms) { best_ms = ms; best_w = sh[0]; best_c = sh[1]; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int st2 = choose_launch(plan, best_w, best_c);
    if (st == RLJSDE_OK) st = st2;
    if (warps_out) *warps_out = plan->warps;
    if (ctas_out) *ctas_out = plan->ctas_per_sm;
    if (ms_out) *ms_out = best_ms < 1e29f ? best_ms : 0.f;
    (void)keep_w; (void)keep_c;
    return st;
}

int rljsde_graph_capture(rljsde_plan_t *plan, void *stream)
{
    if (!plan) return RLJSDE_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (s == nullptr) return RLJSDE_ERR_INVALID_ARG;      // the legacy stream cannot be captured
    if (plan->graph_exec) { cudaGraphExecDestroy((cudaGraphExec_t)plan->graph_exec); plan->graph_exec = nullptr; }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return RLJSDE_ERR_CUDA;
    int st = rljsde_reconstruct_batch(plan, stream);
    cudaError_t ce = cudaStreamEndCapture(s, &g);
    if (st != RLJSDE_OK || ce != cudaSuccess) { if (g) cudaGraphDestroy(g); return st ? st : RLJSDE_ERR_CUDA; }
    cudaGraphExec_t ex = nullptr;
    ce = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return RLJSDE_ERR_CUDA;
    plan->graph_exec = ex;
    return RLJSDE_OK;
}

int rljsde_graph_launch(const rljsde_plan_t *plan, void *stream)
{
    if (!plan || !plan->graph_exec) return RLJSDE_ERR_INVALID_ARG;
    return cudaGraphLaunch((cudaGraphExec_t)plan->graph_exec, (cudaStream_t)stream) == cudaSuccess
               ? RLJSDE_OK : RLJSDE_ERR_CUDA;
}

}  // extern "C"
