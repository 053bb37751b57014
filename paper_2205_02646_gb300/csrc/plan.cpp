// Host side of the RL-JSDE library: parameter checks, classification of every
// target block's local measurement matrix, FP64 construction of the factored
// tables (Sec. IV, Eqs. 12-14, built once per distinct local matrix), the
// plan-sorted work list, and the plan's C-ABI entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <unordered_map>

#include "rljsde_internal.h"

using namespace rljsde;

namespace {

struct Cd {
    double re, im;
};

// exp(2 pi i n / 32), n in [0, 32).  The first quadrant is evaluated with
// cos/sin; the rest follows from exact symmetries, so entry 32-n is exactly
// the conjugate of entry n and entry n+16 exactly its negative.
void unit_roots_32(Cd *r)
{
    for (int n = 0; n <= 8; ++n) {
        if (n == 0) r[n] = {1.0, 0.0};
        else if (n == 8) r[n] = {0.0, 1.0};
        else r[n] = {std::cos(2.0 * M_PI * n / 32.0), std::sin(2.0 * M_PI * n / 32.0)};
    }
    for (int n = 9; n <= 16; ++n) r[n] = {-r[16 - n].re, r[16 - n].im};
    for (int n = 17; n < 32; ++n) r[n] = {r[32 - n].re, -r[32 - n].im};
}

// Spatial weight of window L-pixel (p, q): rho^d with d the distance in HR
// pixels from the centre of its 2x2 footprint (2p + 0.5, 2q + 0.5) to the
// block centre (15.5, 15.5) in window coordinates (Eq. 8 reading).
double spatial_weight(double rho, int p, int q)
{
    double dy = 2.0 * p + 0.5 - 15.5, dx = 2.0 * q + 0.5 - 15.5;
    return std::pow(rho, std::sqrt(dy * dy + dx * dx));
}

// Frequency weight q (Eq. 11 reading): 1 at DC, falling with the signed
// frequency radius, 0 at (W/2, W/2).
void frequency_weight(const rljsde_params &p, std::vector<double> &q)
{
    q.assign(kK, 1.0);
    if (p.q_mode == 1) return;
    for (int s = 0; s < kW; ++s)
        for (int r = 0; r < kW; ++r) {
            if (p.q_mode == 2) { q[s * kW + r] = p.q_table[s * kW + r]; continue; }
            double fs = s <= kW / 2 ? s : s - kW, fr = r <= kW / 2 ? r : r - kW;
            double v = 1.0 - std::sqrt(fs * fs + fr * fr) / (kW / std::sqrt(2.0));
            q[s * kW + r] = v * v;
        }
}

// Aperture (set of transparent sub-pixels, bit 2 * dy + dx) of a mask code.
inline int aperture_of(int layout, int code) { return layout == RLJSDE_LAYOUT_APERTURE ? code : 15 ^ (1 << code); }

// Exact test that h(k) = sum over the aperture's sub-pixels (dy, dx) of
// w32^(dy k1 + dx k2) is zero: w32's minimal polynomial is x^16 + 1, so
// w32^0..w32^15 are independent over the rationals and a sum of powers with
// integer counts c_n vanishes iff c_n = c_(n+16) for every n < 16.
bool aperture_vanishes(int ap, int k1, int k2)
{
    int c[32] = {0};
    for (int s = 0; s < 4; ++s)
        if ((ap >> s) & 1) ++c[((s >> 1) * k1 + (s & 1) * k2) & 31];
    for (int n = 0; n < 16; ++n)
        if (c[n] != c[n + 16]) return false;
    return true;
}

// The window's key: aperture slot per L-pixel, 255 outside the image or
// where the aperture is empty.
void window_key(const uint8_t *mask, int lr_h, int lr_w, int bi, int bj, const uint8_t *slot_of_code,
                uint8_t *key)
{
    int p0 = 2 * bi - kOff / 2, q0 = 2 * bj - kOff / 2;
    for (int p = 0; p < kL; ++p) {
        int P = p0 + p;
        for (int q = 0; q < kL; ++q) {
            int Q = q0 + q;
            key[p * kL + q] =
                (P < 0 || P >= lr_h || Q < 0 || Q >= lr_w) ? 255 : slot_of_code[mask[(size_t)P * lr_w + Q]];
        }
    }
}

// FP64 factored tables of one local measurement matrix:
//   G_t(d) = sum_{m: t(m) = t} w_m w16^(p d1 + q d2),  w16^n = w32^(2n),
//   D_k    = sum_t |h_t(k)|^2 G_t(0)  (= C_{k,k}, Eq. 13),
//   h_t(k) = sum over the transparent offsets (e, g) of slot t's aperture
//            (bits 4t..4t+3 of slot_ap) of w32^(e k1 + g k2).
// A candidate whose h_t vanishes exactly for every slot present in the
// window has no measurement that sees it: D_k is set to 0 (score 0) rather
// than left at the rounding residue of a cancelled sum.
struct Tables {
    double Gre[4][256], Gim[4][256];
    double D[kK];
};

void build_tables(const uint8_t *key, const double *w, const Cd *r32, uint32_t slot_ap, Tables &T)
{
    for (int t = 0; t < 4; ++t)
        for (int d = 0; d < 256; ++d) T.Gre[t][d] = T.Gim[t][d] = 0.0;
    for (int p = 0; p < kL; ++p)
        for (int qq = 0; qq < kL; ++qq) {
            int t = key[p * kL + qq];
            if (t > 3) continue;
            double wm = w[p * kL + qq];
            for (int d1 = 0; d1 < 16; ++d1)
                for (int d2 = 0; d2 < 16; ++d2) {
                    const Cd &e = r32[(2 * (p * d1 + qq * d2)) & 31];
                    T.Gre[t][d1 * 16 + d2] += wm * e.re;
                    T.Gim[t][d1 * 16 + d2] += wm * e.im;
                }
        }
    for (int k1 = 0; k1 < kW; ++k1)
        for (int k2 = 0; k2 < kW; ++k2) {
            double dk = 0.0;
            bool seen = false;
            for (int t = 0; t < 4; ++t) {
                const int ap = (slot_ap >> (4 * t)) & 15;
                double hre = 0.0, him = 0.0;
                for (int e = 0; e < 2; ++e)
                    for (int g = 0; g < 2; ++g) {
                        if (!((ap >> (2 * e + g)) & 1)) continue;
                        const Cd &z = r32[(e * k1 + g * k2) & 31];
                        hre += z.re;
                        him += z.im;
                    }
                dk += (hre * hre + him * him) * T.Gre[t][0];
                if (T.Gre[t][0] > 0.0 && !aperture_vanishes(ap, k1, k2)) seen = true;
            }
            T.D[k1 * kW + k2] = seen ? dk : 0.0;
        }
}

inline double inv_or_zero(double num, double den) { return den > 1e-300 ? num / den : 0.0; }

// Conjugate-pair update: the argmax sees only k <= -k (linear order); the
// other member of each pair gets q/D = 0.
inline bool pair_hidden(bool pairs, int k) { return pairs && ((-(k / kW)) & 31) * kW + ((-(k % kW)) & 31) < k; }

void build_record64(const uint8_t *key, const double *w, const Cd *r32, uint32_t slot_ap, bool pairs,
                    const std::vector<double> &q, Record<double> *rec)
{
    static thread_local Tables T;
    build_tables(key, w, r32, slot_ap, T);
    for (int d = 0; d < 256; ++d) {
        rec->G01[d] = {T.Gre[0][d], T.Gim[0][d], T.Gre[1][d], T.Gim[1][d]};
        rec->G23[d] = {T.Gre[2][d], T.Gim[2][d], T.Gre[3][d], T.Gim[3][d]};
    }
    for (int k = 0; k < kK; ++k) rec->invD[k] = inv_or_zero(1.0, T.D[k]);
    for (int k1 = 0; k1 < 16; ++k1)
        for (int k2 = 0; k2 < 16; ++k2) {
            double v[4];
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) {
                    int k = (k1 + 16 * a) * kW + k2 + 16 * b;
                    v[2 * a + b] = pair_hidden(pairs, k) ? 0.0 : inv_or_zero(q[k], T.D[k]);
                }
            rec->qD[k1 * 16 + k2] = {v[0], v[1], v[2], v[3]};
        }
    std::memcpy(rec->types, key, 256);
}

void build_record32(const uint8_t *key, const double *w, const Cd *r32, uint32_t slot_ap, bool pairs,
                    const std::vector<double> &q, RecordF32 *rec, RecordShortF32 *sh, double *g64,
                    bool scaled_invd)
{
    static thread_local Tables T;
    build_tables(key, w, r32, slot_ap, T);
    if (g64) {   // FP64 tables for the stored Gram matrix: G_t [t][d] as (re, im), q/D, 1/D
        for (int t = 0; t < 4; ++t)
            for (int d = 0; d < 256; ++d) {
                g64[(t * 256 + d) * 2] = T.Gre[t][d];
                g64[(t * 256 + d) * 2 + 1] = T.Gim[t][d];
            }
        for (int k = 0; k < kK; ++k) {
            g64[2048 + k] = pair_hidden(pairs, k) ? 0.0 : inv_or_zero(q[k], T.D[k]);
            g64[2048 + kK + k] = inv_or_zero(1.0, T.D[k]);
        }
    }
    for (int d = 0; d < 256; ++d) {
        float *a = sh->G01[d], *b = sh->G23[d];
        a[0] = (float)T.Gre[0][d]; a[1] = (float)T.Gre[1][d]; a[2] = (float)T.Gim[0][d]; a[3] = (float)T.Gim[1][d];
        b[0] = (float)T.Gre[2][d]; b[1] = (float)T.Gre[3][d]; b[2] = (float)T.Gim[2][d]; b[3] = (float)T.Gim[3][d];
    }
    for (int k = 0; k < kK; ++k) {
        sh->qD[k] = (float)inv_or_zero(q[k], T.D[k]);
        // the stored shortlist loop keeps R'_k = sqrt(q_k / D_k) R_k and needs
        // 1 / (sqrt(q_uv / D_uv) D_uv) for delta
        const double qd = inv_or_zero(q[k], T.D[k]);
        sh->invD[k] = (float)(scaled_invd ? (qd > 0.0 ? inv_or_zero(1.0, T.D[k]) / std::sqrt(qd) : 0.0)
                                          : inv_or_zero(1.0, T.D[k]));
    }
    std::memcpy(sh->types, key, 256);
    for (int d1 = 0; d1 < 16; ++d1)
        for (int d2 = 0; d2 < 16; ++d2) {
            int da = d1 * 16 + d2, db = ((d1 + 15) & 15) * 16 + d2;
            for (int t = 0; t < 4; ++t) {
                float *g = rec->GP[t][d1][d2];
                g[0] = (float)T.Gre[t][da];
                g[1] = (float)T.Gre[t][db];
                g[2] = (float)T.Gim[t][da];
                g[3] = (float)T.Gim[t][db];
            }
        }
    for (int k = 0; k < kK; ++k) rec->invD[k] = (float)inv_or_zero(1.0, T.D[k]);
    for (int j = 0; j < 8; ++j)
        for (int k2 = 0; k2 < 16; ++k2)
            for (int a = 0; a < 2; ++a) {
                float *v = rec->qDP[j][a][k2];
                for (int b = 0; b < 2; ++b)
                    for (int e = 0; e < 2; ++e) {
                        int k = (2 * j + e + 16 * a) * kW + k2 + 16 * b;
                        v[2 * b + e] = pair_hidden(pairs, k) ? 0.f : (float)inv_or_zero(q[k], T.D[k]);
                    }
            }
    std::memcpy(rec->types, key, 256);
}

void release(rljsde_plan *p)
{
    if (!p) return;
    if (p->graph_exec) cudaGraphExecDestroy((cudaGraphExec_t)p->graph_exec);
    cudaFree(p->d_records);
    cudaFree(p->d_records_short);
    cudaFree(p->d_cstore);
    cudaFree(p->d_cslot);
    cudaFree(p->d_entries);
    cudaFree(p->d_chunk_table);
    cudaFree(p->d_consts);
    cudaFree(p->d_qD);
    cudaFree(p->d_masks);
    cudaFree(p->d_mask_offset);
    cudaFree(p->d_status);
    cudaFree(p->d_images);
    delete p;
}

int check_params(const rljsde_params *p)
{
    if (!p) return RLJSDE_ERR_INVALID_ARG;
    if (p->block != kB || p->window != kW) return RLJSDE_ERR_UNSUPPORTED;
    if (p->nu_max < 1 || p->nu_max > 4096) return RLJSDE_ERR_INVALID_ARG;
    if (!(p->gamma_odc > 0.0 && p->gamma_odc < 2.0)) return RLJSDE_ERR_INVALID_ARG;
    if (!(p->rho_decay > 0.0 && p->rho_decay <= 1.0)) return RLJSDE_ERR_INVALID_ARG;
    if (p->q_mode < 0 || p->q_mode > 2 || (p->q_mode == 2 && !p->q_table)) return RLJSDE_ERR_INVALID_ARG;
    if (p->q_mode == 2)
        for (int k = 0; k < kK; ++k)
            if (!(p->q_table[k] >= 0.0) || !std::isfinite(p->q_table[k])) return RLJSDE_ERR_INVALID_ARG;
    if (p->precision != 0 && p->precision != 1) return RLJSDE_ERR_INVALID_ARG;
    if (p->path < 0 || p->path > 3) return RLJSDE_ERR_INVALID_ARG;
    if (p->layout != RLJSDE_LAYOUT_THREE_QUARTER && p->layout != RLJSDE_LAYOUT_APERTURE)
        return RLJSDE_ERR_INVALID_ARG;
    if (p->pairs != 0 && p->pairs != 1) return RLJSDE_ERR_INVALID_ARG;
    if ((p->path == 2 || p->path == 3) && p->precision != 0) return RLJSDE_ERR_UNSUPPORTED;
    if (p->c_supply < 0 || p->c_supply > 3) return RLJSDE_ERR_INVALID_ARG;
    if ((p->c_supply == 1 || p->c_supply == 3) && (p->precision != 0 || p->path == 2 || p->path == 3))
        return RLJSDE_ERR_UNSUPPORTED;
    return RLJSDE_OK;
}

template <typename T>
int upload(T **dst, const void *src, size_t bytes)
{
    if (cudaMalloc((void **)dst, bytes ? bytes : 16) != cudaSuccess) return RLJSDE_ERR_OUT_OF_MEMORY;
    if (bytes && cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return RLJSDE_ERR_CUDA;
    return RLJSDE_OK;
}

struct KeyHash {
    size_t operator()(const std::string &s) const noexcept
    {
        // FNV-1a over the 256 codes
        uint64_t h = 1469598103934665603ull;
        for (unsigned char c : s) { h ^= c; h *= 1099511628211ull; }
        return (size_t)h;
    }
};

int create(rljsde_plan **out, int n_images, const uint8_t *const *masks, const int *lr_h,
           const int *lr_w, const rljsde_params *prm)
{
    if (!out) return RLJSDE_ERR_INVALID_ARG;
    *out = nullptr;
    int st = check_params(prm);
    if (st) return st;
    if (n_images < 1 || !masks || !lr_h || !lr_w) return RLJSDE_ERR_INVALID_ARG;
    long long total_blocks = 0;
    const int max_code = prm->layout == RLJSDE_LAYOUT_APERTURE ? 15 : 3;
    uint32_t present = 0;                       // bit a: aperture a occurs
    for (int i = 0; i < n_images; ++i) {
        if (!masks[i]) return RLJSDE_ERR_INVALID_ARG;
        if (lr_h[i] < 4 || lr_w[i] < 4 || lr_h[i] > 32768 || lr_w[i] > 32768 || (lr_h[i] & 1) || (lr_w[i] & 1))
            return RLJSDE_ERR_BAD_SHAPE;
        uint32_t seen = 0;
        for (size_t j = 0; j < (size_t)lr_h[i] * lr_w[i]; ++j) {
            if (masks[i][j] > max_code) return RLJSDE_ERR_BAD_MASK;
            seen |= 1u << masks[i][j];
        }
        for (int c = 0; c <= max_code; ++c)
            if ((seen >> c) & 1) present |= 1u << aperture_of(prm->layout, c);
        total_blocks += (long long)(lr_h[i] / 2) * (lr_w[i] / 2);
    }
    if (total_blocks > (1ll << 30)) return RLJSDE_ERR_BAD_SHAPE;

    // Aperture slots of the factored tables (Sec. I layouts).  Three-quarter
    // apertures keep slot t = opaque quadrant t, single sub-pixels (quarter
    // sampling) slot t = sub-pixel t; up to four other apertures take slots in
    // increasing code order; more need the direct path.
    present &= ~1u;                             // an empty aperture measures nothing
    int n_ap = 0;
    for (int a = 1; a < 16; ++a) n_ap += (present >> a) & 1;
    const uint32_t tq = (1u << 14) | (1u << 13) | (1u << 11) | (1u << 7);
    const uint32_t single = (1u << 1) | (1u << 2) | (1u << 4) | (1u << 8);
    int kind;
    uint32_t slot_ap = 0;
    uint8_t slot_of_ap[16];
    std::memset(slot_of_ap, 255, sizeof(slot_of_ap));
    if ((present & ~tq) == 0) {
        kind = 0;
        for (int t = 0; t < 4; ++t) { slot_of_ap[15 ^ (1 << t)] = (uint8_t)t; slot_ap |= (uint32_t)(15 ^ (1 << t)) << (4 * t); }
    } else if ((present & ~single) == 0) {
        kind = 3;
        for (int t = 0; t < 4; ++t) { slot_of_ap[1 << t] = (uint8_t)t; slot_ap |= (uint32_t)(1 << t) << (4 * t); }
    } else if (n_ap <= 4) {
        kind = 1;
        int t = 0;
        for (int a = 1; a < 16; ++a)
            if ((present >> a) & 1) { slot_of_ap[a] = (uint8_t)t; slot_ap |= (uint32_t)a << (4 * t); ++t; }
    } else {
        kind = 2;
    }
    if (kind == 2 && (prm->path == 1 || prm->path == 3)) return RLJSDE_ERR_UNSUPPORTED;
    if (kind == 2 && prm->precision != 0) return RLJSDE_ERR_UNSUPPORTED;
    if (kind != 0 && prm->path == 3) return RLJSDE_ERR_UNSUPPORTED;
    uint8_t slot_of_code[256];
    std::memset(slot_of_code, 255, sizeof(slot_of_code));
    for (int c = 0; c <= max_code; ++c) slot_of_code[c] = slot_of_ap[aperture_of(prm->layout, c)];

    rljsde_plan *p = new (std::nothrow) rljsde_plan();
    if (!p) return RLJSDE_ERR_OUT_OF_MEMORY;
    p->params = *prm;
    p->params.q_table = nullptr;
    p->n_images = n_images;
    p->lr_h.assign(lr_h, lr_h + n_images);
    p->lr_w.assign(lr_w, lr_w + n_images);
    p->direct = prm->path == 2 || kind == 2;
    p->kind = kind;
    p->slot_ap = slot_ap;
    p->n_apertures = n_ap;
    frequency_weight(*prm, p->q);
    // The stored-C loop folds q_k / D_k into its state (R'_k = sqrt(q_k / D_k)
    // R_k), which loses R_k where q_k = 0 although the argmax may still pick
    // k (every score 0): such a q keeps the factored loop.
    bool foldable = true;
    for (int k = 0; k < kK; ++k)
        if (!pair_hidden(prm->pairs != 0, k) && !(p->q[k] > 0.0)) foldable = false;
    if (!foldable && (prm->c_supply == 1 || prm->c_supply == 3)) {
        release(p);
        return RLJSDE_ERR_UNSUPPORTED;
    }
    if (cudaGetDevice(&p->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) {
        release(p);
        return RLJSDE_ERR_CUDA;
    }

    double w64[256];
    float w32[256];
    for (int a = 0; a < kL; ++a)
        for (int b = 0; b < kL; ++b) {
            w64[a * kL + b] = spatial_weight(prm->rho_decay, a, b);
            w32[a * kL + b] = (float)w64[a * kL + b];
        }
    Cd r32[32];
    unit_roots_32(r32);

    // Classify every block; group by local measurement matrix.
    std::vector<WorkEntry> blocks;
    std::vector<int> table_of;
    std::vector<std::string> keys;
    std::vector<char> interior;
    blocks.reserve((size_t)total_blocks);
    table_of.reserve((size_t)total_blocks);
    p->ord_base.resize(n_images);
    int ord = 0;
    if (!p->direct) {
        std::unordered_map<std::string, int, KeyHash> ids;
        std::string key(256, '\0');
        for (int i = 0; i < n_images; ++i) {
            p->ord_base[i] = ord;
            int nbh = lr_h[i] / 2, nbw = lr_w[i] / 2;
            for (int bi = 0; bi < nbh; ++bi)
                for (int bj = 0; bj < nbw; ++bj) {
                    window_key(masks[i], lr_h[i], lr_w[i], bi, bj, slot_of_code, (uint8_t *)&key[0]);
                    auto it = ids.find(key);
                    int id;
                    if (it == ids.end()) {
                        id = (int)keys.size();
                        ids.emplace(key, id);
                        keys.push_back(key);
                        int p0 = 2 * bi - kOff / 2, q0 = 2 * bj - kOff / 2;
                        interior.push_back(p0 >= 0 && q0 >= 0 && p0 + kL <= lr_h[i] && q0 + kL <= lr_w[i]);
                    } else {
                        id = it->second;
                    }
                    blocks.push_back({i, bi, bj, ord++});
                    table_of.push_back(id);
                }
        }
        p->n_tables = (int)keys.size();
        for (char c : interior) p->n_interior += c;
        // Mostly unique windows (a non-recurrent sensor): build each block's
        // tables in the kernel instead of one host table set per block.
        // (Small images keep host tables: their build is cheap.)
        p->onthefly = prm->path == 3 || (prm->path == 0 && prm->precision == 0 && kind == 0 &&
                                         4ll * p->n_tables > ord && p->n_tables > 4096);
        if (p->onthefly)
            for (auto &t : table_of) t = 0;
    } else {
        if (prm->c_supply == 1 || prm->c_supply == 3) {      // the direct path has no Gram matrix
            release(p);
            return RLJSDE_ERR_UNSUPPORTED;
        }
        for (int i = 0; i < n_images; ++i) {
            p->ord_base[i] = ord;
            for (int bi = 0; bi < lr_h[i] / 2; ++bi)
                for (int bj = 0; bj < lr_w[i] / 2; ++bj) {
                    blocks.push_back({i, bi, bj, ord++});
                    table_of.push_back(0);
                }
        }
    }
    p->n_blocks = ord;
    if ((prm->c_supply == 1 || prm->c_supply == 3) && p->onthefly) {
        release(p);
        return RLJSDE_ERR_UNSUPPORTED;
    }

    // Work list: blocks sorted by table, each table's run padded to whole
    // chunks so that every chunk uses exactly one table.
    int n_groups = (p->direct || p->onthefly) ? 1 : p->n_tables;
    std::vector<int> count(n_groups, 0), start(n_groups + 1, 0);
    for (int t : table_of) ++count[t];
    for (int g = 0; g < n_groups; ++g) start[g + 1] = start[g] + (count[g] + kChunk - 1) / kChunk * kChunk;
    std::vector<WorkEntry> entries(start[n_groups], WorkEntry{-1, 0, 0, -1});
    std::vector<int> fill(start.begin(), start.end() - 1);
    for (size_t b = 0; b < blocks.size(); ++b) entries[fill[table_of[b]]++] = blocks[b];
    p->n_entries = (int)entries.size();
    p->n_chunks = p->n_entries / kChunk;
    std::vector<uint32_t> chunk_table(p->n_chunks);
    for (int g = 0; g < n_groups; ++g)
        for (int e = start[g]; e < start[g + 1]; e += kChunk) chunk_table[e / kChunk] = (uint32_t)g;

    // Table sets whose Gram matrix is stored (c_supply): all of them (1),
    // those at least kStoredMinBlocks blocks use (3), or (auto) all, the most
    // used first, within an eighth of the free device memory.
    if (!p->direct && !p->onthefly && prm->precision == 0 && prm->c_supply != 2 && foldable) {
        p->cslot.assign(p->n_tables, -1);
        if (prm->c_supply != 0) {
            for (int t = 0; t < p->n_tables; ++t) {
                if (prm->c_supply == 3 && count[t] < kStoredMinBlocks) continue;
                p->cslot[t] = p->n_stored++;
                p->n_stored_blocks += count[t];
            }
        } else {
            size_t free_b = 0, total_b = 0;
            if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = 0;
            const size_t budget = free_b / 8;
            std::vector<int> order(p->n_tables);
            for (int t = 0; t < p->n_tables; ++t) order[t] = t;
            std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return count[x] > count[y]; });
            for (int t : order) {
                if ((size_t)(p->n_stored + 1) * kStoredTableBytes > budget) break;
                p->cslot[t] = p->n_stored++;
                p->n_stored_blocks += count[t];
            }
        }
    }

    st = upload(&p->d_entries, entries.data(), entries.size() * sizeof(WorkEntry));
    if (!st) st = upload(&p->d_chunk_table, chunk_table.data(), chunk_table.size() * sizeof(uint32_t));
    if (!st) {
        Consts c;
        for (int i = 0; i < 256; ++i) { c.w32[i] = w32[i]; c.w64[i] = w64[i]; }
        for (int n = 0; n < 32; ++n) {
            c.om32[2 * n] = (float)r32[n].re;
            c.om32[2 * n + 1] = (float)r32[n].im;
            c.om64[2 * n] = r32[n].re;
            c.om64[2 * n + 1] = r32[n].im;
        }
        for (int k = 0; k < kK; ++k) {
            uint16_t v = 0;
            for (int a = 1; a < 16; ++a)
                if (aperture_vanishes(a, k / kW, k % kW)) v |= (uint16_t)(1u << a);
            c.vanish[k] = v;
        }
        st = upload(&p->d_consts, &c, sizeof(c));
    }
    if (!st && (cudaMalloc((void **)&p->d_status, sizeof(int)) != cudaSuccess ||
                cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess))
        st = RLJSDE_ERR_CUDA;
    if (!st) {
        std::vector<ImageDesc> descs(n_images);
        for (int i = 0; i < n_images; ++i) descs[i] = {nullptr, nullptr, lr_h[i], lr_w[i], 0, 0};
        st = upload(&p->d_images, descs.data(), descs.size() * sizeof(ImageDesc));
    }
    if (!st && !p->direct && !p->onthefly) {
        // FP64 tables per distinct local matrix, stored in the loop's precision.
        p->record_bytes = prm->precision ? sizeof(Record<double>) : sizeof(RecordF32);
        std::vector<unsigned char> host, host_short;
        std::vector<double> g64;
        try {
            host.resize(p->record_bytes * (size_t)p->n_tables);
            if (!prm->precision) host_short.resize(sizeof(RecordShortF32) * (size_t)p->n_tables);
            if (p->n_stored) g64.resize((size_t)p->n_stored * kStoredBuildDoubles);
        } catch (...) {
            st = RLJSDE_ERR_OUT_OF_MEMORY;
        }
        if (!st) {
            #pragma omp parallel for schedule(dynamic, 4)
            for (int t = 0; t < p->n_tables; ++t) {
                const uint8_t *key = (const uint8_t *)keys[t].data();
                if (prm->precision)
                    build_record64(key, w64, r32, slot_ap, prm->pairs != 0, p->q,
                                   (Record<double> *)(host.data() + p->record_bytes * t));
                else
                    build_record32(key, w64, r32, slot_ap, prm->pairs != 0, p->q,
                                   (RecordF32 *)(host.data() + p->record_bytes * t),
                                   (RecordShortF32 *)(host_short.data() + sizeof(RecordShortF32) * t),
                                   p->n_stored && p->cslot[t] >= 0
                                       ? g64.data() + (size_t)kStoredBuildDoubles * p->cslot[t]
                                       : nullptr,
                                   p->n_stored > 0 && p->n_stored == p->n_tables);
            }
            st = upload(&p->d_records, host.data(), host.size());
            if (!st && !prm->precision) st = upload(&p->d_records_short, host_short.data(), host_short.size());
            if (!st && p->n_stored) {
                // the Gram matrices (Eq. 14) of the stored table sets, built on the device
                double *d_g64 = nullptr;
                p->cstore_bytes = kStoredTableBytes * (size_t)p->n_stored;
                if (cudaMalloc(&p->d_cstore, p->cstore_bytes) != cudaSuccess) {
                    p->d_cstore = nullptr;
                    cudaGetLastError();
                    st = RLJSDE_ERR_OUT_OF_MEMORY;
                }
                if (!st) st = upload(&d_g64, g64.data(), g64.size() * sizeof(double));
                if (!st) st = upload(&p->d_cslot, p->cslot.data(), p->cslot.size() * sizeof(int));
                if (!st) st = build_stored_c(p, d_g64);
                cudaFree(d_g64);
            }
        }
    }
    if (!st && (p->direct || p->onthefly)) {
        // Direct path and in-kernel tables: q on the device, no host tables.
        std::vector<float> qf(kK);
        for (int k = 0; k < kK; ++k) qf[k] = (float)p->q[k];
        st = upload(&p->d_qD, qf.data(), qf.size() * sizeof(float));
    }
    if (!st) {
        // The masks on the device (direct path, learned proposal).
        long long tot = 0;
        p->mask_offset.resize(n_images);
        for (int i = 0; i < n_images; ++i) { p->mask_offset[i] = tot; tot += (long long)lr_h[i] * lr_w[i]; }
        std::vector<uint8_t> all((size_t)tot);
        for (int i = 0; i < n_images; ++i)
            std::memcpy(all.data() + p->mask_offset[i], masks[i], (size_t)lr_h[i] * lr_w[i]);
        if (!st) st = upload(&p->d_masks, all.data(), all.size());
        if (!st) st = upload(&p->d_mask_offset, p->mask_offset.data(), p->mask_offset.size() * sizeof(long long));
    }
    if (!st) st = choose_launch(p, 0, 0);
    if (st) {
        release(p);
        return st;
    }
    *out = p;
    return RLJSDE_OK;
}

}  // namespace

extern "C" {

int rljsde_default_params(rljsde_params *p)
{
    if (!p) return RLJSDE_ERR_INVALID_ARG;
    p->block = kB;
    p->window = kW;
    p->nu_max = 100;
    p->gamma_odc = 0.5;
    p->rho_decay = 0.7;
    p->q_mode = 0;
    p->q_table = nullptr;
    p->precision = 0;
    p->path = 0;
    p->layout = RLJSDE_LAYOUT_THREE_QUARTER;
    p->pairs = 0;
    p->c_supply = 0;
    return RLJSDE_OK;
}

int rljsde_plan_create(rljsde_plan_t **out, const uint8_t *mask, int lr_h, int lr_w, const rljsde_params *p)
{
    const uint8_t *masks[1] = {mask};
    return create(out, 1, masks, &lr_h, &lr_w, p);
}

int rljsde_plan_create_batch(rljsde_plan_t **out, int n_images, const uint8_t *const *masks, const int *lr_h,
                             const int *lr_w, const rljsde_params *p)
{
    return create(out, n_images, masks, lr_h, lr_w, p);
}

int rljsde_set_images(rljsde_plan_t *plan, const rljsde_image *images)
{
    if (!plan || !images) return RLJSDE_ERR_INVALID_ARG;
    std::vector<ImageDesc> d(plan->n_images);
    for (int i = 0; i < plan->n_images; ++i) {
        if (!images[i].lr || !images[i].hr || images[i].lr_pitch < plan->lr_w[i] ||
            images[i].hr_pitch < 2 * plan->lr_w[i])
            return RLJSDE_ERR_INVALID_ARG;
        d[i] = {images[i].lr, images[i].hr, plan->lr_h[i], plan->lr_w[i], images[i].lr_pitch, images[i].hr_pitch};
    }
    if (cudaMemcpy(plan->d_images, d.data(), d.size() * sizeof(ImageDesc), cudaMemcpyHostToDevice) != cudaSuccess)
        return RLJSDE_ERR_CUDA;
    return RLJSDE_OK;
}

int rljsde_plan_info(const rljsde_plan_t *p, rljsde_plan_info_t *out)
{
    if (!p || !out) return RLJSDE_ERR_INVALID_ARG;
    out->n_images = p->n_images;
    out->n_blocks = p->n_blocks;
    out->n_tables = p->n_tables;
    out->n_interior_tables = p->n_interior;
    out->n_work_entries = p->n_entries;
    const bool all_stored = p->n_stored > 0 && p->n_stored == p->n_tables;
    out->warps_per_cta = all_stored ? p->warps_stored : p->warps;
    out->ctas_per_sm = all_stored ? p->ctas_stored : p->ctas_per_sm;
    out->grid = all_stored ? p->grid_stored : p->grid;
    out->device_table_bytes = (int64_t)p->record_bytes * p->n_tables;
    out->paper_B_bytes = (int64_t)p->n_tables * 256 * kK * 8;
    out->paper_C_bytes = (int64_t)p->n_tables * kK * kK * 8;
    out->paper_D_bytes = (int64_t)p->n_tables * kK * 8;
    out->path = p->direct ? 2 : p->onthefly ? 3 : 1;
    out->n_apertures = p->n_apertures;
    out->n_stored_c_tables = p->n_stored;
    out->n_stored_c_blocks = p->n_stored_blocks;
    out->device_c_bytes = (int64_t)p->cstore_bytes;
    out->n_launches = (p->n_stored > 0 && p->n_stored < p->n_tables) ? 2 : 1;
    return RLJSDE_OK;
}

int rljsde_set_launch(rljsde_plan_t *plan, int warps_per_cta, int ctas_per_sm)
{
    if (!plan) return RLJSDE_ERR_INVALID_ARG;
    if (warps_per_cta != 0 && warps_per_cta != 4 && warps_per_cta != 8) return RLJSDE_ERR_INVALID_ARG;
    if (ctas_per_sm < 0 || ctas_per_sm > 4) return RLJSDE_ERR_INVALID_ARG;
    return choose_launch(plan, warps_per_cta, ctas_per_sm);
}

int rljsde_check(const rljsde_plan_t *plan, void *stream)
{
    if (!plan) return RLJSDE_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaStreamSynchronize(s) != cudaSuccess) return RLJSDE_ERR_CUDA;
    int v = 0;
    if (cudaMemcpy(&v, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return RLJSDE_ERR_CUDA;
    if (v && cudaMemset(plan->d_status, 0, sizeof(int)) != cudaSuccess) return RLJSDE_ERR_CUDA;
    if (v & 2) return RLJSDE_ERR_TIMEOUT;
    if (v & 1) return RLJSDE_ERR_NONFINITE_INPUT;
    return RLJSDE_OK;
}

void rljsde_plan_destroy(rljsde_plan_t *plan) { release(plan); }

const char *rljsde_status_string(int s)
{
    switch (s) {
    case RLJSDE_OK: return "ok";
    case RLJSDE_ERR_INVALID_ARG: return "invalid argument";
    case RLJSDE_ERR_BAD_SHAPE: return "bad shape (LR dimensions must be even, 4..32768)";
    case RLJSDE_ERR_BAD_MASK: return "bad mask (codes must be 0..3)";
    case RLJSDE_ERR_OUT_OF_MEMORY: return "out of memory";
    case RLJSDE_ERR_CUDA: return "CUDA runtime error";
    case RLJSDE_ERR_TIMEOUT: return "a bounded device wait timed out";
    case RLJSDE_ERR_NONFINITE_INPUT: return "non-finite measurement (treated as absent)";
    case RLJSDE_ERR_UNSUPPORTED: return "unsupported parameter combination";
    default: return "unknown status";
    }
}

}  // extern "C"
