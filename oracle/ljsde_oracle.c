/*
 * FP64 CPU oracle for (recurrent) local joint sparse deconvolution and
 * extrapolation, L-JSDE / RL-JSDE (Grosche et al., "Fast Reconstruction of
 * Three-Quarter Sampling Measurements Using Recurrent Local Joint Sparse
 * Deconvolution and Extrapolation", TCAS-II 2022).
 *
 * TEST INFRASTRUCTURE.  This file is the slow, plain reference that the
 * CUDA library is checked against.  Only the test suite, the package smoke
 * check and the CPU-baseline leg of the benchmark may load it; the library
 * itself never calls it and shares no code, table or helper with it.
 *
 * What it implements, in the paper's order and notation:
 *   - the sensor model, Eq. 1 (coefficients A = 1 on the transparent
 *     sub-pixels of each L-pixel, i.e. a sum): three-quarter sampling, where
 *     one of the four sub-pixels is opaque, or any other per-pixel aperture
 *     (Sec. I: arbitrary periodically repeating layouts), given as the set
 *     of transparent sub-pixels;
 *   - the window model of Eqs. 2-3 with the Fourier basis
 *     Phi_{eta,gamma,sigma,rho} = exp(2 pi j (eta sigma + gamma rho) / W)
 *     (Sec. III prints M and N in the exponent; the sums run over the W x W
 *     window and Table I counts W^2 atoms, so W is used);
 *   - direct L-JSDE (Sec. IV, Eqs. 4-10, 15, 16, 18): every iteration
 *     recomputes the weighted projection of the residual onto every atom
 *     (the O(W^4) matrix-vector product of Eq. 10), picks the argmax,
 *     updates one coefficient and the residual r (Eq. 7);
 *   - recurrent RL-JSDE (Eqs. 11-17): the projection matrix B (Eq. 12), the
 *     four-index matrix C (Eq. 14) and its diagonal D (Eq. 13) are built once
 *     per distinct local measurement matrix, and the loop only updates the
 *     projected residual R (Eq. 17).
 *
 * Readings where the paper is silent (each is also stated in the design
 * notes of the repository):
 *   - spatial weight (Eq. 8): w_m = rho^d_m, d_m the Euclidean distance in HR
 *     pixels from the centre of the L-pixel's 2x2 footprint to the centre of
 *     the target block;
 *   - frequency weight (Eq. 11): with the signed frequency kt = k for
 *     k <= W/2 and k - W otherwise, q = (1 - |kt| / (W / sqrt 2))^2;
 *   - argmax (Eqs. 10, 11): evaluated on the score rounded to binary32, the
 *     precision of the paper's complex64 tables (Table I); ties go to the
 *     lowest linear index sigma * W + rho;
 *   - a window position outside the image holds no measurement, and neither
 *     does an L-pixel whose aperture is empty;
 *   - a candidate whose atom vanishes identically on every measurement of
 *     the window (its sub-pixel phases cancel in antipodal pairs, e.g. the
 *     Nyquist row or column under a full 2x2 aperture) cannot be observed:
 *     its score is 0 and its delta 0, instead of a ratio of two rounding
 *     residues;
 *   - the target block sits at window offset (W - B) / 2 in both axes;
 *   - the output is the real part of the back-transformed model (Eq. 18).
 *
 * Variant (pairs = 1), the conjugate-pair update of the frequency selective
 * reconstruction family, for real measurements: the argmax runs over one
 * half of the candidates (k with k <= -k mod W in linear order, the other
 * half being their conjugate mirrors), and each selection updates both
 * c_k += gamma delta and c_-k += conj(gamma delta), so the model and the
 * residual stay real.  A self-conjugate k (k = -k) is updated once.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fcx-limited-range -shared -fPIC
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

typedef struct {
    int window;          /* W: model window edge in HR pixels (multiple of 8) */
    int block;           /* B: target block edge in HR pixels (4)             */
    int nu_max;          /* iterations per block                              */
    double gamma_odc;    /* orthogonality deficiency compensation, Eq. 15     */
    double rho_decay;    /* base of the isotropic spatial weight, Eq. 8       */
    int q_mode;          /* 0: default q, 1: q = 1, 2: q_table                */
    const double *q_table; /* W*W entries, row-major over (sigma, rho)        */
    int layout;          /* mask codes: 0 = index of the opaque sub-pixel of
                            a three-quarter pixel (0..3); 1 = set of
                            transparent sub-pixels, bit 2 * dy + dx (0..15) */
    int pairs;           /* 0: one complex coefficient per iteration (Eq. 15);
                            1: conjugate-pair update (see above)            */
} orc_params;

/* Linear index of the conjugate mirror -k (mod W in both axes). */
static int mirror_of(int k, int W)
{
    int k1 = k / W, k2 = k % W;
    return ((W - k1) % W) * W + (W - k2) % W;
}

/* Sub-pixel s = 2 * dy + dx of an L-pixel with mask code `code` is
 * transparent (Eq. 1: A = 1 there). */
static int transparent(int layout, int code, int s)
{
    return layout == 1 ? (code >> s) & 1 : s != code;
}

static int code_valid(int layout, int code)
{
    return layout == 1 ? code >= 0 && code <= 15 : code >= 0 && code <= 3;
}

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2 };

/* exp(2 pi j n / W) for n in [0, W), built so that entry W-n is exactly the
 * conjugate of entry n and entry n+W/2 exactly its negative. */
static void roots_of_unity(int W, cplx *tab)
{
    int quarter = W / 4;
    for (int n = 0; n <= quarter; ++n) {
        double re, im;
        if (n == 0) { re = 1.0; im = 0.0; }
        else if (n == quarter) { re = 0.0; im = 1.0; }
        else { re = cos(2.0 * M_PI * n / W); im = sin(2.0 * M_PI * n / W); }
        tab[n] = CMPLX(re, im);
    }
    for (int n = quarter + 1; n <= W / 2; ++n)
        tab[n] = CMPLX(-creal(tab[W / 2 - n]), cimag(tab[W / 2 - n]));
    for (int n = W / 2 + 1; n < W; ++n)
        tab[n] = conj(tab[W - n]);
}

/* Frequency weight q_{sigma rho} (Eq. 11): default low-pass reading. */
static void frequency_weight(const orc_params *p, double *q)
{
    int W = p->window;
    for (int s = 0; s < W; ++s)
        for (int r = 0; r < W; ++r) {
            double v;
            if (p->q_mode == 1) v = 1.0;
            else if (p->q_mode == 2) v = p->q_table[s * W + r];
            else {
                double ks = s <= W / 2 ? s : s - W;
                double kr = r <= W / 2 ? r : r - W;
                double t = 1.0 - sqrt(ks * ks + kr * kr) / (W / sqrt(2.0));
                v = t * t;
            }
            q[s * W + r] = v;
        }
}

/* ------------------------------------------------------------------ */
/* Generic window: nm measurements, measurement m integrates npx[m]    */
/* (<= 4) HR pixels at window coordinates (eta, gamma).                */
/* ------------------------------------------------------------------ */
typedef struct {
    int W, nm;
    const int *npx;        /* nm                                   */
    const int *eta, *gam;  /* nm * 4                               */
    const double *w;       /* nm, spatial weight w_m                */
    const double *y_re, *y_im; /* nm; y_im may be NULL (real data)  */
} orc_window;

typedef struct {
    cplx *c;           /* W*W model coefficients (out)                      */
    int32_t *sel;      /* nu_max selected linear indices (out, may be NULL) */
    double *dc;        /* nu_max * 2: gamma_odc * delta per iteration        */
    double *gap;       /* nu_max: relative gap of the chosen score to the
                          best other score (FP64)                            */
    double *energy;    /* nu_max + 1: E_w before / after each iteration;
                          direct variant only                                */
    cplx *r;           /* nm: final residual; direct variant only            */
} orc_trace;

/* a_m(k) = sum over the pixels of measurement m of Phi(eta, gamma, k)
 * (Eq. 4 with A^local = 1 on the integrated pixels).  Layout [m][k]. */
static void measurement_atoms(const orc_window *win, const cplx *om, cplx *a)
{
    int W = win->W, K = W * W;
    for (int m = 0; m < win->nm; ++m) {
        cplx *am = a + (size_t)m * K;
        for (int s = 0; s < W; ++s)
            for (int r = 0; r < W; ++r) {
                cplx acc = 0.0;
                for (int i = 0; i < win->npx[m]; ++i) {
                    int e = win->eta[4 * m + i], g = win->gam[4 * m + i];
                    acc += om[(e * s + g * r) % W];
                }
                am[s * W + r] = acc;
            }
    }
}

/* Exact test that a_m(k) = sum_i w^(n_i) vanishes.  For W a power of two the
 * cyclotomic polynomial of w is x^(W/2) + 1, so 1, w, ..., w^(W/2 - 1) are
 * linearly independent over the rationals and a sum with integer counts c_n
 * of each power vanishes iff c_n = c_(n + W/2) for every n < W/2 (the terms
 * cancel in antipodal pairs).  For other W this is the pairwise part of the
 * condition only. */
static int atom_vanishes(const orc_window *win, int m, int s, int r)
{
    int W = win->W, cnt[128] = {0};
    for (int i = 0; i < win->npx[m]; ++i)
        ++cnt[(win->eta[4 * m + i] * s + win->gam[4 * m + i] * r) % W];
    for (int n = 0; n < W / 2; ++n)
        if (cnt[n] != cnt[n + W / 2]) return 0;
    return 1;
}

/* flag[k] = 1 when the atom of candidate k vanishes on every measurement. */
static void unobservable(const orc_window *win, char *flag)
{
    int W = win->W;
    for (int s = 0; s < W; ++s)
        for (int r = 0; r < W; ++r) {
            int all = 1;
            for (int m = 0; m < win->nm && all; ++m) all = atom_vanishes(win, m, s, r);
            flag[s * W + r] = (char)all;
        }
}

/* Argmax of Eq. 10 / Eq. 11 on binary32-rounded scores, lowest index on
 * ties; with `half`, over the candidates k <= mirror(k) only.  Also reports
 * the FP64 relative gap to the best other candidate. */
static int select_atom(int K, int W, int half, const double *score, double *gap_out)
{
    int best = 0;
    float bkey = (float)score[0];
    for (int k = 1; k < K; ++k) {
        if (half && mirror_of(k, W) < k) continue;
        float key = (float)score[k];
        if (key > bkey) { bkey = key; best = k; }
    }
    double other = 0.0;
    for (int k = 0; k < K; ++k)
        if (k != best && !(half && mirror_of(k, W) < k) && score[k] > other) other = score[k];
    if (gap_out)
        *gap_out = score[best] > 0.0 ? (score[best] - other) / score[best] : 0.0;
    return best;
}

static double weighted_energy(int nm, const double *w, const cplx *r)
{
    double e = 0.0;
    for (int m = 0; m < nm; ++m) e += w[m] * (creal(r[m]) * creal(r[m]) + cimag(r[m]) * cimag(r[m]));
    return e;
}

/* Direct L-JSDE on one window (Eqs. 4-10, 15, 16). */
static int window_direct(const orc_window *win, const orc_params *p, const cplx *om,
                         const double *q, orc_trace *tr)
{
    int W = win->W, K = W * W, nm = win->nm;
    cplx *a = malloc(sizeof(cplx) * (size_t)nm * K);
    cplx *r = malloc(sizeof(cplx) * (size_t)(nm > 0 ? nm : 1));
    cplx *wr = malloc(sizeof(cplx) * (size_t)(nm > 0 ? nm : 1));
    cplx *N = malloc(sizeof(cplx) * K);
    double *D = malloc(sizeof(double) * K), *score = malloc(sizeof(double) * K);
    char *zero = malloc(K);
    if (!a || !r || !wr || !N || !D || !score || !zero) {
        free(a); free(r); free(wr); free(N); free(D); free(score); free(zero);
        return ORC_ENOMEM;
    }
    measurement_atoms(win, om, a);
    unobservable(win, zero);
    /* denominator of Eq. 10: D_k = sum_m w_m |a_m(k)|^2 */
    for (int k = 0; k < K; ++k) D[k] = 0.0;
    for (int m = 0; m < nm; ++m) {
        const cplx *am = a + (size_t)m * K;
        for (int k = 0; k < K; ++k)
            D[k] += win->w[m] * (creal(am[k]) * creal(am[k]) + cimag(am[k]) * cimag(am[k]));
    }
    /* model initialised to zero, so r^(0) = y (Eq. 6) */
    for (int m = 0; m < nm; ++m)
        r[m] = CMPLX(win->y_re[m], win->y_im ? win->y_im[m] : 0.0);
    for (int k = 0; k < K; ++k) tr->c[k] = 0.0;
    if (tr->energy) tr->energy[0] = weighted_energy(nm, win->w, r);

    for (int nu = 0; nu < p->nu_max; ++nu) {
        /* numerator of Eq. 10: N_k = sum_m conj(a_m(k)) w_m r_m */
        for (int k = 0; k < K; ++k) N[k] = 0.0;
        for (int m = 0; m < nm; ++m) wr[m] = win->w[m] * r[m];
        for (int m = 0; m < nm; ++m) {
            const cplx *am = a + (size_t)m * K;
            cplx x = wr[m];
            for (int k = 0; k < K; ++k) N[k] += conj(am[k]) * x;
        }
        for (int k = 0; k < K; ++k)
            score[k] = (D[k] < 1e-300 || zero[k]) ? 0.0
                     : q[k] * (creal(N[k]) * creal(N[k]) + cimag(N[k]) * cimag(N[k])) / D[k];
        int uv = select_atom(K, W, p->pairs, score, tr->gap ? &tr->gap[nu] : NULL);
        cplx delta = (D[uv] < 1e-300 || zero[uv]) ? 0.0 : N[uv] / D[uv];      /* Eq. 16 */
        cplx step = p->gamma_odc * delta;
        int vu = mirror_of(uv, W);
        tr->c[uv] += step;                                         /* Eq. 15 */
        const cplx *au = a + (size_t)uv;
        if (p->pairs && vu != uv) {
            /* conjugate partner: c_-k += conj(step), r -= step a_k + conj(step) a_-k */
            tr->c[vu] += conj(step);
            const cplx *av = a + (size_t)vu;
            for (int m = 0; m < nm; ++m)
                r[m] -= step * au[(size_t)m * K] + conj(step) * av[(size_t)m * K];
        } else {
            for (int m = 0; m < nm; ++m) r[m] -= step * au[(size_t)m * K];   /* Eq. 7 */
        }
        if (tr->sel) tr->sel[nu] = uv;
        if (tr->dc) { tr->dc[2 * nu] = creal(step); tr->dc[2 * nu + 1] = cimag(step); }
        if (tr->energy) tr->energy[nu + 1] = weighted_energy(nm, win->w, r);
    }
    if (tr->r) memcpy(tr->r, r, sizeof(cplx) * (size_t)nm);
    free(a); free(r); free(wr); free(N); free(D); free(score); free(zero);
    return ORC_OK;
}

/* Tables of the recurrent form for one local measurement matrix:
 * B_{m,k} = w_m conj(a_m(k)) (Eq. 12), C_{k,l} = sum_m B_{m,k} a_m(l)
 * (Eq. 14, stored transposed: CT[l][k] = C_{k,l}), D_k = C_{k,k} (Eq. 13). */
typedef struct { int nm, K; cplx *B, *CT; double *D; } orc_tables;

static void tables_free(orc_tables *t) { free(t->B); free(t->CT); free(t->D); t->B = t->CT = NULL; t->D = NULL; }

static int tables_build(const orc_window *win, const cplx *om, orc_tables *t, int nthreads)
{
    int W = win->W, K = W * W, nm = win->nm;
    t->nm = nm; t->K = K;
    cplx *a = malloc(sizeof(cplx) * (size_t)(nm > 0 ? nm : 1) * K);
    t->B = malloc(sizeof(cplx) * (size_t)(nm > 0 ? nm : 1) * K);
    t->CT = malloc(sizeof(cplx) * (size_t)K * K);
    t->D = malloc(sizeof(double) * K);
    if (!a || !t->B || !t->CT || !t->D) { free(a); tables_free(t); return ORC_ENOMEM; }
    measurement_atoms(win, om, a);
    for (int m = 0; m < nm; ++m)
        for (int k = 0; k < K; ++k)
            t->B[(size_t)m * K + k] = win->w[m] * conj(a[(size_t)m * K + k]);
    #pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int l = 0; l < K; ++l) {
        cplx *row = t->CT + (size_t)l * K;
        for (int k = 0; k < K; ++k) row[k] = 0.0;
        for (int m = 0; m < nm; ++m) {
            cplx al = a[(size_t)m * K + l];
            const cplx *Bm = t->B + (size_t)m * K;
            for (int k = 0; k < K; ++k) row[k] += Bm[k] * al;
        }
    }
    for (int k = 0; k < K; ++k) t->D[k] = creal(t->CT[(size_t)k * K + k]);
    free(a);
    return ORC_OK;
}

/* RL-JSDE loop on one window given its tables (Eqs. 11-17). */
static int window_recurrent(const orc_window *win, const orc_tables *t, const orc_params *p,
                            const double *q, orc_trace *tr)
{
    int K = t->K, nm = win->nm;
    cplx *R = malloc(sizeof(cplx) * K);
    double *score = malloc(sizeof(double) * K);
    char *zero = malloc(K);
    if (!R || !score || !zero) { free(R); free(score); free(zero); return ORC_ENOMEM; }
    unobservable(win, zero);
    /* R^(0)_k = sum_m B_{m,k} y_m  (Eq. 12 with r^(0) = y) */
    for (int k = 0; k < K; ++k) R[k] = 0.0;
    for (int m = 0; m < nm; ++m) {
        cplx ym = CMPLX(win->y_re[m], win->y_im ? win->y_im[m] : 0.0);
        const cplx *Bm = t->B + (size_t)m * K;
        for (int k = 0; k < K; ++k) R[k] += Bm[k] * ym;
    }
    for (int k = 0; k < K; ++k) tr->c[k] = 0.0;
    for (int nu = 0; nu < p->nu_max; ++nu) {
        for (int k = 0; k < K; ++k)                                   /* Eq. 11 */
            score[k] = (t->D[k] < 1e-300 || zero[k]) ? 0.0
                     : q[k] * (creal(R[k]) * creal(R[k]) + cimag(R[k]) * cimag(R[k])) / t->D[k];
        int uv = select_atom(K, win->W, p->pairs, score, tr->gap ? &tr->gap[nu] : NULL);
        cplx delta = (t->D[uv] < 1e-300 || zero[uv]) ? 0.0 : R[uv] / t->D[uv];    /* Eq. 16 */
        cplx step = p->gamma_odc * delta;
        int vu = mirror_of(uv, win->W);
        tr->c[uv] += step;                                            /* Eq. 15 */
        const cplx *Cu = t->CT + (size_t)uv * K;
        if (p->pairs && vu != uv) {
            tr->c[vu] += conj(step);
            const cplx *Cv = t->CT + (size_t)vu * K;
            for (int k = 0; k < K; ++k) R[k] -= step * Cu[k] + conj(step) * Cv[k];
        } else {
            for (int k = 0; k < K; ++k) R[k] -= step * Cu[k];         /* Eq. 17 */
        }
        if (tr->sel) tr->sel[nu] = uv;
        if (tr->dc) { tr->dc[2 * nu] = creal(step); tr->dc[2 * nu + 1] = cimag(step); }
    }
    free(R); free(score); free(zero);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Public generic-window entry points (used by the pins).              */
/* ------------------------------------------------------------------ */
static int check_params(const orc_params *p)
{
    if (!p || p->window < 8 || p->window % 8 || p->window > 128 || p->nu_max < 0) return ORC_EINVAL;
    if (p->q_mode == 2 && !p->q_table) return ORC_EINVAL;
    if (p->layout != 0 && p->layout != 1) return ORC_EINVAL;
    if (p->pairs != 0 && p->pairs != 1) return ORC_EINVAL;
    return ORC_OK;
}

int orc_window_solve(int recurrent, int W, int nm, const int *npx, const int *eta, const int *gam,
                     const double *w, const double *y_re, const double *y_im,
                     const orc_params *p, double *c_out /* W*W*2 */, int32_t *sel, double *dc,
                     double *gap, double *energy, double *r_out /* nm*2 */)
{
    if (check_params(p) || W != p->window || nm < 0) return ORC_EINVAL;
    int K = W * W;
    cplx *om = malloc(sizeof(cplx) * W);
    double *q = malloc(sizeof(double) * K);
    cplx *c = malloc(sizeof(cplx) * K);
    cplx *r = malloc(sizeof(cplx) * (size_t)(nm > 0 ? nm : 1));
    if (!om || !q || !c || !r) { free(om); free(q); free(c); free(r); return ORC_ENOMEM; }
    roots_of_unity(W, om);
    frequency_weight(p, q);
    orc_window win = { W, nm, npx, eta, gam, w, y_re, y_im };
    orc_trace tr = { c, sel, dc, gap, energy, r };
    int st;
    if (recurrent) {
        orc_tables t = {0};
        st = tables_build(&win, om, &t, 1);
        if (!st) st = window_recurrent(&win, &t, p, q, &tr);
        tables_free(&t);
    } else {
        st = window_direct(&win, p, om, q, &tr);
        if (!st && r_out)
            for (int m = 0; m < nm; ++m) { r_out[2 * m] = creal(r[m]); r_out[2 * m + 1] = cimag(r[m]); }
    }
    if (!st)
        for (int k = 0; k < K; ++k) { c_out[2 * k] = creal(c[k]); c_out[2 * k + 1] = cimag(c[k]); }
    free(om); free(q); free(c); free(r);
    return st;
}

/* B (nm x K), C (K x K, row k, column l) and D (K) of Eqs. 12-14. */
int orc_window_tables(int W, int nm, const int *npx, const int *eta, const int *gam,
                      const double *w, double *B_out, double *C_out, double *D_out)
{
    if (W < 8 || W % 8 || W > 128 || nm < 0) return ORC_EINVAL;
    int K = W * W;
    cplx *om = malloc(sizeof(cplx) * W);
    if (!om) return ORC_ENOMEM;
    roots_of_unity(W, om);
    orc_window win = { W, nm, npx, eta, gam, w, NULL, NULL };
    orc_tables t = {0};
    int st = tables_build(&win, om, &t, 1);
    if (!st) {
        for (size_t i = 0; i < (size_t)nm * K; ++i) { B_out[2 * i] = creal(t.B[i]); B_out[2 * i + 1] = cimag(t.B[i]); }
        for (int k = 0; k < K; ++k)
            for (int l = 0; l < K; ++l) {
                cplx v = t.CT[(size_t)l * K + k];
                C_out[2 * ((size_t)k * K + l)] = creal(v);
                C_out[2 * ((size_t)k * K + l) + 1] = cimag(v);
            }
        memcpy(D_out, t.D, sizeof(double) * K);
    }
    tables_free(&t);
    free(om);
    return st;
}

/* ------------------------------------------------------------------ */
/* Images: three-quarter sampling and other per-pixel apertures.       */
/* ------------------------------------------------------------------ */

/* Eq. 1: y[p][q] = sum of the transparent sub-pixels of L-pixel (p, q). */
int orc_measure(const double *f, const uint8_t *mask, int lr_h, int lr_w, int layout, double *y)
{
    if (!f || !mask || !y || lr_h <= 0 || lr_w <= 0 || (layout != 0 && layout != 1)) return ORC_EINVAL;
    int N = 2 * lr_w;
    for (int p = 0; p < lr_h; ++p)
        for (int q = 0; q < lr_w; ++q) {
            int code = mask[p * lr_w + q];
            if (!code_valid(layout, code)) return ORC_EINVAL;
            double s = 0.0;
            for (int de = 0; de < 2; ++de)
                for (int dg = 0; dg < 2; ++dg)
                    if (transparent(layout, code, de * 2 + dg)) s += f[(2 * p + de) * N + 2 * q + dg];
            y[p * lr_w + q] = s;
        }
    return ORC_OK;
}

/* The measurements of the model window of block (bi, bj): every L-pixel
 * whose 2x2 footprint lies in both the window and the image and whose
 * aperture is not empty. */
typedef struct {
    int nm;
    int npx[4096];
    int eta[4 * 4096], gam[4 * 4096];
    double w[4096], y[4096];
    uint8_t key[4096];   /* mask code per window L-pixel, 255 = absent */
} block_window;

static void gather_block(const double *y, const uint8_t *mask, int lr_h, int lr_w,
                         const orc_params *p, int bi, int bj, block_window *bw)
{
    int W = p->window, Bk = p->block, off = (W - Bk) / 2, L = W / 2;
    int p0 = (bi * Bk - off) / 2, q0 = (bj * Bk - off) / 2;
    double centre = (W - 1) / 2.0;   /* block centre in window coordinates */
    bw->nm = 0;
    for (int pm = 0; pm < L; ++pm)
        for (int qm = 0; qm < L; ++qm) {
            int P = p0 + pm, Q = q0 + qm;
            if (P < 0 || P >= lr_h || Q < 0 || Q >= lr_w) { bw->key[pm * L + qm] = 255; continue; }
            int code = mask[P * lr_w + Q];
            bw->key[pm * L + qm] = (uint8_t)code;
            int m = bw->nm, n = 0;
            for (int de = 0; de < 2; ++de)
                for (int dg = 0; dg < 2; ++dg) {
                    if (!transparent(p->layout, code, de * 2 + dg)) continue;
                    bw->eta[4 * m + n] = 2 * pm + de;
                    bw->gam[4 * m + n] = 2 * qm + dg;
                    ++n;
                }
            if (n == 0) continue;          /* empty aperture: no measurement */
            bw->nm++;
            bw->npx[m] = n;
            double dy = 2 * pm + 0.5 - centre, dx = 2 * qm + 0.5 - centre;
            bw->w[m] = pow(p->rho_decay, sqrt(dy * dy + dx * dx));
            bw->y[m] = y[P * lr_w + Q];
        }
}

/* Eq. 18 on the central B x B block of the window. */
static void write_block(const orc_params *p, const cplx *om, const cplx *c, int bi, int bj,
                        double *hr, int N)
{
    int W = p->window, Bk = p->block, off = (W - Bk) / 2, K = W * W;
    for (int e = off; e < off + Bk; ++e)
        for (int g = off; g < off + Bk; ++g) {
            cplx v = 0.0;
            for (int s = 0; s < W; ++s)
                for (int r = 0; r < W; ++r) {
                    int k = s * W + r;
                    if (c[k] != 0.0) v += c[k] * om[(e * s + g * r) % W];
                }
            (void)K;
            hr[(size_t)(bi * Bk + e - off) * N + bj * Bk + g - off] = creal(v);
        }
}

static int cmp_key_len;
static const uint8_t *cmp_keys;
static int cmp_block_keys(const void *x, const void *y)
{
    int a = *(const int *)x, b = *(const int *)y;
    int c = memcmp(cmp_keys + (size_t)a * cmp_key_len, cmp_keys + (size_t)b * cmp_key_len, cmp_key_len);
    return c ? c : (a > b) - (a < b);
}

/*
 * Reconstruct the listed target blocks of an image measured by Eq. 1.
 *   y:      lr_h x lr_w measurements (row-major)
 *   mask:   lr_h x lr_w codes in p->layout (opaque sub-pixel 0..3, or the
 *           set of transparent sub-pixels 0..15)
 *   blocks: n_blocks linear block indices bi * (N/B) + bj, or NULL for all
 *   hr:     (2 lr_h) x (2 lr_w) output; only the listed blocks are written
 *   sel, dc, gap: per listed block nu_max entries (dc: 2 per entry); may be NULL
 * recurrent = 0 runs direct L-JSDE, 1 runs RL-JSDE with tables shared by all
 * blocks of equal local measurement matrix.
 */
int orc_reconstruct(int recurrent, const double *y, const uint8_t *mask, int lr_h, int lr_w,
                    const orc_params *p, const int32_t *blocks, int n_blocks, double *hr,
                    int32_t *sel, double *dc, double *gap, int n_threads)
{
    if (check_params(p) || !y || !mask || !hr || lr_h <= 0 || lr_w <= 0) return ORC_EINVAL;
    int W = p->window, Bk = p->block;
    if (Bk != 4 || (W - Bk) % 4 != 0 || (2 * lr_h) % Bk || (2 * lr_w) % Bk || W / 2 > 64) return ORC_EINVAL;
    for (size_t i = 0; i < (size_t)lr_h * lr_w; ++i) if (!code_valid(p->layout, mask[i])) return ORC_EINVAL;
    int nbh = 2 * lr_h / Bk, nbw = 2 * lr_w / Bk, N = 2 * lr_w, K = W * W, L2 = (W / 2) * (W / 2);
    int total = nbh * nbw;
    if (!blocks) n_blocks = total;
    if (n_threads <= 0) n_threads = 1;
    for (int i = 0; blocks && i < n_blocks; ++i) if (blocks[i] < 0 || blocks[i] >= total) return ORC_EINVAL;

    cplx *om = malloc(sizeof(cplx) * W);
    double *q = malloc(sizeof(double) * K);
    if (!om || !q) { free(om); free(q); return ORC_ENOMEM; }
    roots_of_unity(W, om);
    frequency_weight(p, q);
    int status = ORC_OK;

    if (!recurrent) {
        #pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
        for (int i = 0; i < n_blocks; ++i) {
            int b = blocks ? blocks[i] : i;
            block_window *bw = malloc(sizeof(block_window));
            cplx *c = malloc(sizeof(cplx) * K);
            if (!bw || !c) { free(bw); free(c); status = ORC_ENOMEM; continue; }
            gather_block(y, mask, lr_h, lr_w, p, b / nbw, b % nbw, bw);
            orc_window win = { W, bw->nm, bw->npx, bw->eta, bw->gam, bw->w, bw->y, NULL };
            orc_trace tr = { c, sel ? sel + (size_t)i * p->nu_max : NULL,
                             dc ? dc + (size_t)i * 2 * p->nu_max : NULL,
                             gap ? gap + (size_t)i * p->nu_max : NULL, NULL, NULL };
            if (window_direct(&win, p, om, q, &tr)) status = ORC_ENOMEM;
            else write_block(p, om, c, b / nbw, b % nbw, hr, N);
            free(bw); free(c);
        }
    } else {
        /* group blocks by local measurement matrix (the window's codes) */
        uint8_t *keys = malloc((size_t)n_blocks * L2);
        int *order = malloc(sizeof(int) * (n_blocks > 0 ? n_blocks : 1));
        block_window *bw0 = malloc(sizeof(block_window));
        if (!keys || !order || !bw0) { free(keys); free(order); free(bw0); free(om); free(q); return ORC_ENOMEM; }
        for (int i = 0; i < n_blocks; ++i) {
            int b = blocks ? blocks[i] : i;
            gather_block(y, mask, lr_h, lr_w, p, b / nbw, b % nbw, bw0);
            memcpy(keys + (size_t)i * L2, bw0->key, L2);
            order[i] = i;
        }
        cmp_keys = keys; cmp_key_len = L2;
        qsort(order, n_blocks, sizeof(int), cmp_block_keys);
        for (int g0 = 0; g0 < n_blocks && !status; ) {
            int g1 = g0 + 1;
            while (g1 < n_blocks && !memcmp(keys + (size_t)order[g0] * L2, keys + (size_t)order[g1] * L2, L2)) ++g1;
            int b0 = blocks ? blocks[order[g0]] : order[g0];
            gather_block(y, mask, lr_h, lr_w, p, b0 / nbw, b0 % nbw, bw0);
            orc_window win0 = { W, bw0->nm, bw0->npx, bw0->eta, bw0->gam, bw0->w, bw0->y, NULL };
            orc_tables t = {0};
            if (tables_build(&win0, om, &t, n_threads)) { status = ORC_ENOMEM; break; }
            #pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
            for (int j = g0; j < g1; ++j) {
                int i = order[j], b = blocks ? blocks[i] : i;
                block_window *bw = malloc(sizeof(block_window));
                cplx *c = malloc(sizeof(cplx) * K);
                if (!bw || !c) { free(bw); free(c); status = ORC_ENOMEM; continue; }
                gather_block(y, mask, lr_h, lr_w, p, b / nbw, b % nbw, bw);
                orc_window win = { W, bw->nm, bw->npx, bw->eta, bw->gam, bw->w, bw->y, NULL };
                orc_trace tr = { c, sel ? sel + (size_t)i * p->nu_max : NULL,
                                 dc ? dc + (size_t)i * 2 * p->nu_max : NULL,
                                 gap ? gap + (size_t)i * p->nu_max : NULL, NULL, NULL };
                if (window_recurrent(&win, &t, p, q, &tr)) status = ORC_ENOMEM;
                else write_block(p, om, c, b / nbw, b % nbw, hr, N);
                free(bw); free(c);
            }
            tables_free(&t);
            g0 = g1;
        }
        free(keys); free(order); free(bw0);
    }
    free(om); free(q);
    return status;
}

/* The frequency weight q (W*W entries) the loop uses for these parameters. */
int orc_frequency_weight(const orc_params *p, double *q)
{
    if (check_params(p) || !q) return ORC_EINVAL;
    frequency_weight(p, q);
    return ORC_OK;
}

/* Number of distinct local measurement matrices among all target blocks
 * (the tables RL-JSDE precomputes, Sec. IV and Table I); interior counts
 * only windows that lie wholly inside the image. */
int orc_count_local_masks(const uint8_t *mask, int lr_h, int lr_w, const orc_params *p,
                          int *n_all, int *n_interior)
{
    if (check_params(p) || !mask) return ORC_EINVAL;
    int W = p->window, Bk = p->block, L = W / 2, L2 = L * L, off = (W - Bk) / 2;
    int nbh = 2 * lr_h / Bk, nbw = 2 * lr_w / Bk, total = nbh * nbw;
    uint8_t *keys = malloc((size_t)total * L2);
    uint8_t *inside = malloc((size_t)total);
    int *order = malloc(sizeof(int) * (total > 0 ? total : 1));
    if (!keys || !order || !inside) { free(keys); free(order); free(inside); return ORC_ENOMEM; }
    for (int b = 0; b < total; ++b) {
        int p0 = ((b / nbw) * Bk - off) / 2, q0 = ((b % nbw) * Bk - off) / 2;
        inside[b] = p0 >= 0 && q0 >= 0 && p0 + L <= lr_h && q0 + L <= lr_w;
        for (int pm = 0; pm < L; ++pm)
            for (int qm = 0; qm < L; ++qm) {
                int P = p0 + pm, Q = q0 + qm;
                keys[(size_t)b * L2 + pm * L + qm] =
                    (P < 0 || P >= lr_h || Q < 0 || Q >= lr_w) ? 255 : mask[P * lr_w + Q];
            }
        order[b] = b;
    }
    cmp_keys = keys; cmp_key_len = L2;
    qsort(order, total, sizeof(int), cmp_block_keys);
    int all = 0, interior = 0;
    for (int j = 0; j < total; ++j) {
        if (j > 0 && !memcmp(keys + (size_t)order[j] * L2, keys + (size_t)order[j - 1] * L2, L2)) continue;
        ++all;
        if (inside[order[j]]) ++interior;
    }
    *n_all = all; *n_interior = interior;
    free(keys); free(order); free(inside);
    return ORC_OK;
}
