// Internal layout shared by the host plan builder (plan.cpp) and the CUDA
// kernels (kernels.cu).  Not part of the public ABI.
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "rljsde.h"

namespace rljsde {

constexpr int kW = 32;          // model window edge, HR pixels (Sec. III)
constexpr int kB = 4;           // target block edge, HR pixels (Sec. III)
constexpr int kL = kW / 2;      // window edge in L-pixels
constexpr int kK = kW * kW;     // candidate atoms
constexpr int kOff = (kW - kB) / 2;   // block offset inside the window (14)
constexpr int kChunk = 8;       // work entries per chunk; one table per chunk

// One image of the work list (device copy for batches).
struct ImageDesc {
    const float *lr;
    float *hr;
    int lr_h, lr_w;
    long long lr_pitch, hr_pitch;
};

// One target block to reconstruct; img < 0 marks padding.
struct WorkEntry {
    int img, bi, bj, ord;
};

// Plan-independent constants: spatial weights w(p, q) of the window's
// L-pixels and exp(2 pi i n / 32), each in FP32 and FP64; per candidate k,
// the apertures whose sub-pixel phase sum h(k) is exactly zero (bit a set:
// aperture code a, sub-pixel bit 2 * dy + dx).
struct Consts {
    float w32[256];
    float om32[64];     // (re, im) for n = 0..31
    double w64[256];
    double om64[64];
    uint16_t vanish[kK];
};

template <typename T>
struct alignas(16) Vec4 {
    T x, y, z, w;
};

// Tables of one local measurement matrix in the factored form.
//
// With t(m) the aperture type (slot 0..3) of L-pixel m at window LR position
// (p, q) -- for three-quarter sampling, its opaque quadrant -- the integrated
// atom of Eq. 4 factors as
//     a_m(k) = w32^(2 p k1 + 2 q k2) h_t(k),
//     h_t(k) = sum over the transparent offsets (e, g) of type t of w32^(e k1 + g k2),
// so the Gram matrix of Eq. 14 is
//     C_{k,l} = sum_t conj(h_t(k)) h_t(l) G_t((l - k) mod 16),
//     G_t(d) = sum_{m: t(m) = t} w_m w16^(p d1 + q d2),
// and D_k = C_{k,k} (Eq. 13) = sum_t |h_t(k)|^2 G_t(0).
template <typename T>
struct Record {
    Vec4<T> G01[256];     // (G_0(d), G_1(d)) as (re, im, re, im), d = d1 * 16 + d2
    Vec4<T> G23[256];     // (G_2(d), G_3(d))
    Vec4<T> qD[256];      // q_k / D_k at k = (kap1 + 16a, kap2 + 16b), entry 2a + b
    T invD[kK];           // 1 / D_k, k = k1 * 32 + k2
    uint8_t types[256];   // aperture slot per window L-pixel (p * 16 + q), 255 = absent
};
static_assert(sizeof(Record<double>) % 16 == 0, "record size must allow bulk copies");

// FP32 loop tables, the same quantities laid out for packed two-lane (f32x2)
// arithmetic over frequency pairs (kap1, kap1 + 1), kap1 even:
//   GP[t][d1][d2]   = (G_t(d1, d2).re, G_t(d1 - 1, d2).re, G_t(d1, d2).im, G_t(d1 - 1, d2).im)
//                     (d1 - 1 taken mod 16), so that the update of both members
//                     of a pair reads one 16-byte entry at d1 = (u - kap1) mod 16;
//   qDP[j][a][kap2] = (qD(2j, b=0), qD(2j+1, b=0), qD(2j, b=1), qD(2j+1, b=1)) at
//                     k = (kap1 + 16a, kap2 + 16b).
// Lanes differ in kap2, so consecutive lanes read consecutive 16-byte entries.
struct RecordF32 {
    float GP[4][16][16][4];
    float qDP[8][2][16][4];
    float invD[kK];
    uint8_t types[256];
};
static_assert(sizeof(RecordF32) % 16 == 0, "record size must allow bulk copies");

// FP32 tables of the shortlist loop, which reads the four G_t at one
// (d1, d2) per candidate: G01[d] = (G_0(d), G_1(d)), G23[d] = (G_2(d), G_3(d))
// as (re, re, im, im) so that each pair of types fills one f32x2 register
// pair, d = d1 * 16 + d2; qD and invD by linear k.  When every table set of
// the plan stores its Gram matrix, invD holds 1 / (s_k D_k), s_k =
// sqrt(q_k / D_k), the stored shortlist loop's delta factor.
struct RecordShortF32 {
    float G01[256][4];
    float G23[256][4];
    float qD[kK];
    float invD[kK];
    uint8_t types[256];
};
static_assert(sizeof(RecordShortF32) % 16 == 0, "record size must allow bulk copies");

// Learned proposal of one block: the candidates the loop may select, the
// network's expected number of likely candidates left out, and its
// iteration output (fraction of nu_max).
constexpr int kShortlist = 64;
struct Shortlist {
    uint16_t idx[kShortlist];
    float missing;
    float nu_frac;
};
static_assert(sizeof(Shortlist) == 136, "shortlist layout");

// Stored Gram matrix of one table set (c_supply), the stored-C loop's
// state being R'_k = s_k R_k with s_k = sqrt(q_k / D_k), so that the score
// of Eq. 11 is |R'_k|^2:
//   C'_{k,l} = s_k C_{k,l}: 1024 columns of 8 KiB, each as 16 x 32 float4
//     (C'_{k,l}.re, C'_{k+32,l}.re, C'_{k,l}.im, C'_{k+32,l}.im), entry
//     i * 32 + lane holding the two candidates that lane of the FP32 loop
//     updates in its register pair i;
//   then s_k in the same lane order, as float4 (s_k, s_k+32, s_k, s_k+32);
//   then 1 / (s_l D_l) by linear l (0 where s_l D_l is 0), so that
//     delta = R_uv / D_uv = R'_uv / (s_uv D_uv) (Eq. 16).
constexpr size_t kStoredColsBytes = (size_t)kK * kK * 8;
constexpr size_t kStoredTableBytes = kStoredColsBytes + 8192 + 4096;
constexpr size_t kStoredScaleOff = kStoredColsBytes / 16;          // in float4
constexpr size_t kStoredInvDOff = kStoredColsBytes / 16 + 512;     // in float4
// c_supply 3 stores the matrix of a table set that at least this many blocks
// use (border table sets of a recurrent mask are used by few blocks each);
// the others run the factored loop in a second kernel.
constexpr int kStoredMinBlocks = 256;

}  // namespace rljsde

// The opaque plan object of the C ABI.
struct rljsde_plan {
    rljsde_params params{};
    std::vector<double> q;            // W*W frequency weights (FP64)
    int n_images = 0;
    std::vector<int> lr_h, lr_w;
    int n_blocks = 0, n_tables = 0, n_interior = 0;
    int n_entries = 0, n_chunks = 0;
    int direct = 0;                   // path == 2
    int onthefly = 0;                 // tables built per block in the kernel (path 3, or auto)
    int kind = 0;                     // 0: three-quarter apertures (slot t = opaque quadrant t);
                                      // 1: up to four other apertures; 2: more (direct path only);
                                      // 3: single sub-pixels (slot t = sub-pixel t)
    uint32_t slot_ap = 0;             // aperture code of slot t in bits 4t..4t+3
    int n_apertures = 0;              // distinct non-empty apertures in the masks
    int device = 0, sm_count = 0;
    int warps = 4, ctas_per_sm = 0, grid = 0, variant = 0;   // factored loop (and FP64, learned)
    int variant_stored = 0, grid_stored = 0, ctas_stored = 0, warps_stored = 0;   // stored-C loop, if n_stored > 0
    int learned_warps = 4;            // warps per CTA of the shortlist-loop kernel (4: two blocks per warp)
    int learned_minb = 3;             // its register budget: resident CTAs per SM
    // device memory, all owned by the plan
    void *d_records = nullptr;        // n_tables records (float or double)
    size_t record_bytes = 0;
    void *d_records_short = nullptr;  // n_tables RecordShortF32 (FP32 plans)
    int n_stored = 0;                 // table sets whose Gram matrix is stored (c_supply)
    int n_stored_blocks = 0;          // blocks that use them
    std::vector<int> cslot;           // per table set: its stored matrix, or -1 (factored)
    int *d_cslot = nullptr;
    void *d_cstore = nullptr;         // n_stored x kStoredTableBytes, in the stored-C loop's read order
    size_t cstore_bytes = 0;
    rljsde::WorkEntry *d_entries = nullptr;
    uint32_t *d_chunk_table = nullptr;
    rljsde::Consts *d_consts = nullptr;
    float *d_qD = nullptr;            // direct path: W*W q values (float)
    uint8_t *d_masks = nullptr;       // direct path: all masks, concatenated
    std::vector<long long> mask_offset;
    long long *d_mask_offset = nullptr;
    int *d_status = nullptr;
    rljsde::ImageDesc *d_images = nullptr;
    std::vector<int> ord_base;        // first block ordinal of each image
    void *graph_exec = nullptr;       // cudaGraphExec_t of one batch launch
};

namespace rljsde {
// Implemented in kernels.cu.
int choose_launch(rljsde_plan *plan, int warps, int ctas_per_sm);
// Fill plan->d_cstore from FP64 tables of the stored table sets (device, in
// stored order, kStoredBuildDoubles per table: G_t as 4 x 256 x (re, im),
// t-major, then q_k / D_k and 1 / D_k by linear k); synchronous.
constexpr int kStoredBuildDoubles = 2048 + 2 * kK;
int build_stored_c(rljsde_plan *plan, const double *d_g64);
const char *last_cuda_error();
}  // namespace rljsde
