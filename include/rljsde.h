/*
 * rljsde.h -- C ABI of the GB300 (sm_103a) RL-JSDE library.
 *
 * Reconstructs a 2x-resolution image from three-quarter sampling
 * measurements with recurrent local joint sparse deconvolution and
 * extrapolation (RL-JSDE; Grosche, Regensky, Sinn, Seiler, Kaup, TCAS-II
 * 2022).  The calls follow the paper's statement of the problem:
 *
 *   - Sec. II, Eq. 1: each L-pixel value y is the SUM of the three
 *     transparent HR sub-pixels of its 2x2 footprint; mask[p][q] in 0..3 names
 *     the opaque one (0 top-left, 1 top-right, 2 bottom-left, 3 bottom-right).
 *     lr_h x lr_w measurements give a (2 lr_h) x (2 lr_w) HR image.
 *     Sec. I extends the method to any periodically repeating sensor layout:
 *     with params.layout = RLJSDE_LAYOUT_APERTURE, mask[p][q] in 0..15 is
 *     instead the set of transparent sub-pixels (bit 2 * dy + dx), e.g.
 *     quarter sampling (one bit), pairs, or the full 2x2 aperture.
 *   - Sec. III: every B x B = 4 x 4 HR target block is rebuilt from a
 *     W x W = 32 x 32 model window of DFT atoms centred on it; only the
 *     central block is kept.
 *   - Sec. IV, Eqs. 11-17: per block, nu_max greedy iterations over the
 *     W^2 = 1024 candidates on the projected residual R, using tables
 *     precomputed once per distinct local measurement matrix (a "plan
 *     entry"); Eq. 18: the model is transformed back.
 *
 * Pointer conventions: "host" pointers are read during the call only;
 * "device" pointers must be CUDA device (or managed) memory on the current
 * device and stay valid until the work on `stream` has finished.  A NULL
 * stream is the legacy default stream.  Pitches are in ELEMENTS.
 *
 * Errors: every function returns an rljsde_status.  Asynchronous problems a
 * kernel detects (non-finite input, a table load that did not arrive) are
 * recorded in a device status word of the plan and reported by
 * rljsde_check(); no kernel traps.
 */
#ifndef RLJSDE_H
#define RLJSDE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RLJSDE_OK = 0,
    RLJSDE_ERR_INVALID_ARG = 1,     /* NULL pointer, bad parameter value        */
    RLJSDE_ERR_BAD_SHAPE = 2,       /* lr_h / lr_w not even, or too large        */
    RLJSDE_ERR_BAD_MASK = 3,        /* a mask code outside 0..3 (0..15 apertures) */
    RLJSDE_ERR_OUT_OF_MEMORY = 4,   /* host or device allocation failed          */
    RLJSDE_ERR_CUDA = 5,            /* a CUDA runtime call failed                */
    RLJSDE_ERR_TIMEOUT = 6,         /* a bounded device wait gave up             */
    RLJSDE_ERR_NONFINITE_INPUT = 7, /* NaN/Inf measurement (treated as absent)   */
    RLJSDE_ERR_UNSUPPORTED = 8      /* valid request this build does not offer   */
} rljsde_status;

/* Meaning of the mask codes (rljsde_params.layout). */
enum {
    RLJSDE_LAYOUT_THREE_QUARTER = 0,   /* code 0..3: the one opaque sub-pixel     */
    RLJSDE_LAYOUT_APERTURE = 1         /* code 0..15: bit 2*dy+dx set = sub-pixel
                                          (dy, dx) transparent; 0 = no measurement */
};

/* Reconstruction parameters.  The paper fixes B and W (Sec. III); it names
 * nu_max, gamma_odc, the spatial weight w_m and the frequency weight q but
 * gives no values: the defaults below are this library's readings. */
typedef struct {
    int block;            /* B: must be 4 (Sec. III)                                */
    int window;           /* W: must be 32 (Sec. III)                               */
    int nu_max;           /* iterations per block, 1..4096 (Sec. IV); default 100   */
    double gamma_odc;     /* orthogonality deficiency compensation, Eq. 15; 0.5     */
    double rho_decay;     /* w_m = rho^d_m, d_m the HR-pixel distance from the
                             L-pixel's 2x2 centre to the block centre (Eq. 8); 0.7  */
    int q_mode;           /* Eq. 11 frequency weight: 0 = (1 - |kt| / (W/sqrt2))^2
                             with signed frequency kt; 1 = all ones; 2 = q_table    */
    const double *q_table;/* host, W*W entries row-major over (sigma, rho), q_mode 2 */
    int precision;        /* 0 = FP32 loop (tables built in FP64, stored FP32);
                             1 = FP64 loop                                           */
    int path;             /* 1 = recurrent with one table set per distinct local
                             measurement matrix built on the host (Eqs. 11-17);
                             2 = direct L-JSDE (Eqs. 4-10: residual r kept, O(W^4)
                             projection every iteration, no tables); 3 = recurrent
                             with each block's tables built in the kernel in FP32
                             (for non-recurrent sensors, FP32 loops only);
                             0 = auto: 3 if precision is 0 and there are more than
                             4096 distinct local matrices, more than a quarter of
                             the blocks, else 1.  Aperture layouts: path 1 holds
                             up to four distinct non-empty apertures per mask;
                             with more, auto runs path 2 and path 1 is refused
                             (RLJSDE_ERR_UNSUPPORTED); path 3 and auto's choice
                             of it need three-quarter apertures               */
    int layout;           /* RLJSDE_LAYOUT_*: meaning of the mask codes; default
                             three-quarter.  A candidate whose atom cancels on
                             every measurement of its window (e.g. the Nyquist
                             row under full 2x2 apertures) is never selected   */
    int pairs;            /* 0 (default) = one complex coefficient per iteration
                             (Eq. 15, the paper's loop); 1 = conjugate-pair
                             update of the frequency selective reconstruction
                             family: the argmax runs over k <= -k (linear order)
                             and each selection adds gamma delta to c_k and its
                             conjugate to c_-k (once if k = -k), so model and
                             residual stay real.  Not with the learned proposal */
    int c_supply;         /* where the loop's Gram column C_{k,uv} of Eq. 17 comes
                             from, per table set (distinct local matrix):
                             1 = stored, the paper's recurrent form (Table I):
                             the whole C of Eq. 14, built in FP64 on the device
                             and stored FP32 (8 MiB per table set), one 8 KiB
                             column read per block and iteration; 2 = factored,
                             rebuilt every iteration from 16 KB of tables with
                             no memory traffic; 3 = stored for the table sets
                             at least 256 blocks use, factored for the others
                             (border table sets of a recurrent mask: less
                             memory, one more kernel); 0 = auto (default):
                             stored for every table set, the most used first,
                             while the matrices fit in an eighth of the free
                             device memory, factored for the rest and for FP64
                             loops, paths 2 and 3 and frequency weights with a
                             zero (the stored loop's state is sqrt(q / D) R,
                             which cannot hold R where q is 0).  1 and 3 need
                             the FP32 loop on path 1 and q > 0 wherever it
                             counts (RLJSDE_ERR_UNSUPPORTED otherwise, also
                             when auto would choose path 2 or 3) and fail with
                             RLJSDE_ERR_OUT_OF_MEMORY when the matrices do not
                             fit.  A plan with both kinds of
                             table sets runs two kernels per reconstruction;
                             the stored-C loop runs one CTA of 8 warps per SM
                             (4 warps x 3 CTAs below nu_max 20; rljsde_set_launch
                             and rljsde_autotune shape the factored loop).  The
                             learned proposal's loops always use the factored
                             form                                              */
} rljsde_params;

/* Fill *p with the defaults above.  Returns RLJSDE_ERR_INVALID_ARG on NULL. */
int rljsde_default_params(rljsde_params *p);

typedef struct rljsde_plan rljsde_plan_t;   /* opaque; owns all its device memory */

/*
 * Build a plan for one image size and sensor mask (Sec. IV: the tables of a
 * local measurement matrix are computed once and shared by every model
 * window that has that matrix).
 *   mask: host, lr_h x lr_w codes (0..3, or 0..15 for aperture layouts),
 *         row-major, contiguous.
 *   lr_h, lr_w: even, 4 .. 32768.
 * Every target block's local measurement matrix (the window's codes, with
 * positions outside the image absent) is classified; tables are built in FP64
 * on the host per distinct one and uploaded.  Synchronous; allocates device
 * memory on the current device.  *out is NULL on failure.
 */
int rljsde_plan_create(rljsde_plan_t **out, const uint8_t *mask, int lr_h, int lr_w,
                       const rljsde_params *p);

/*
 * The same for a batch of n_images images of possibly different sizes
 * (masks[i]: host, lr_h[i] x lr_w[i]).  Blocks of all images go into one
 * work list; table sets are shared across images.
 */
int rljsde_plan_create_batch(rljsde_plan_t **out, int n_images, const uint8_t *const *masks,
                             const int *lr_h, const int *lr_w, const rljsde_params *p);

/*
 * Reconstruct one image: lr (device, lr_h x lr_w floats, pitch lr_pitch >= lr_w)
 * -> hr (device, 2lr_h x 2lr_w floats, pitch hr_pitch >= 2 lr_w).  Every HR
 * pixel is written.  Only for single-image plans.  Asynchronous on `stream`,
 * allocates nothing, one kernel launch (two when the plan stores the Gram
 * matrices of some of its table sets only: rljsde_plan_info n_launches).
 */
int rljsde_reconstruct(const rljsde_plan_t *plan, const float *lr, size_t lr_pitch,
                       float *hr, size_t hr_pitch, void *stream);

/*
 * As rljsde_reconstruct, and also records every block's greedy trace:
 *   sel: device, n_blocks * nu_max uint16 selected linear indices sigma*W+rho;
 *   dc:  device, n_blocks * nu_max * 2 floats, gamma_odc * delta (re, im);
 * block b = bi * (2 lr_w / 4) + bj (row-major over target blocks).
 */
int rljsde_reconstruct_trace(const rljsde_plan_t *plan, const float *lr, size_t lr_pitch,
                             float *hr, size_t hr_pitch, uint16_t *sel, float *dc,
                             void *stream);

/* Device-side description of one image of a batch (device pointers). */
typedef struct {
    const float *lr;      /* lr_h x lr_w, pitch lr_pitch  */
    float *hr;            /* 2lr_h x 2lr_w, pitch hr_pitch */
    int64_t lr_pitch;
    int64_t hr_pitch;
} rljsde_image;

/*
 * Copy the batch's image pointers (host array of n_images entries, in the
 * order given at plan creation) into plan-owned device memory.  Synchronous.
 * Call again whenever buffers change; not needed for single-image plans.
 */
int rljsde_set_images(rljsde_plan_t *plan, const rljsde_image *images);

/*
 * Reconstruct every image of a batch plan in ONE persistent kernel launch
 * (two as above).  Reads the pointers stored by rljsde_set_images.
 * Asynchronous, allocates nothing, launches nothing else: safe to capture in
 * a CUDA graph.
 */
int rljsde_reconstruct_batch(const rljsde_plan_t *plan, void *stream);

/* Launch shape of the persistent factored-loop kernel: warps per CTA (4 or
 * 8) and resident CTAs per SM to launch (1..4; clamped to what fits).  0
 * restores defaults.  The stored-C loop keeps its own shape. */
int rljsde_set_launch(rljsde_plan_t *plan, int warps_per_cta, int ctas_per_sm);

/*
 * Autotuner (this library's, not the paper's): times every launch shape of
 * the persistent kernel that fits (warps per CTA x resident CTAs per SM) on
 * the plan's own work, `reps` timed launches each after one warm-up, and
 * keeps the fastest on the plan.  lr/hr as for rljsde_reconstruct (single-image
 * plans), or both NULL to use the images stored by rljsde_set_images.
 * Synchronous (events on `stream`); writes hr.  Outputs may be NULL.
 */
int rljsde_autotune(rljsde_plan_t *plan, const float *lr, size_t lr_pitch, float *hr, size_t hr_pitch,
                    int reps, void *stream, int *warps_out, int *ctas_out, float *best_ms_out);

/*
 * Capture one rljsde_reconstruct_batch launch on `stream` (not the legacy
 * NULL stream) into a CUDA graph owned by the plan, replacing any earlier
 * one; rljsde_graph_launch replays it.  The graph reads the image pointers
 * from plan memory, so rljsde_set_images may change them between replays.
 */
int rljsde_graph_capture(rljsde_plan_t *plan, void *stream);
int rljsde_graph_launch(const rljsde_plan_t *plan, void *stream);

/* ------------------------------------------------------------------------
 * Learned candidate proposal.  The paper has no counterpart: this library's
 * extension, which predicts per block the 64 candidates (of Eq. 11's 1024)
 * the greedy loop is likely to select, so the loop can search those only.
 * ---------------------------------------------------------------------- */
typedef struct rljsde_net rljsde_net_t;   /* weights, Adam state, packed head weights */

/* One block's proposal (device layout, 136 bytes):
 *   idx: the 64 candidates sigma * W + rho with the largest logits z, ranked
 *        by z on a fixed-point grid of step 2^-9 over [-32, 32) (rounded
 *        down, clamped), ties to the lower index, in increasing index order;
 *   missing: the network's gate, sigmoid of head row 1025: its prediction of
 *        the share of the plain loop's coefficient mass (sum of |gamma delta|
 *        per candidate over nu_max iterations, Eq. 15) that falls on
 *        candidates outside idx;
 *   nu_frac: its iteration output (head row 1024), a fraction of nu_max. */
typedef struct {
    uint16_t idx[64];
    float missing;
    float nu_frac;
} rljsde_shortlist;

/* Create a network on the current device with seeded random weights. */
int rljsde_net_create(rljsde_net_t **out, uint64_t seed);
void rljsde_net_destroy(rljsde_net_t *net);
int rljsde_net_num_params(void);
/* Copy all parameters (FP32, fixed order: conv1.w, conv1.b, conv2.w,
 * conv2.b, conv3.w, conv3.b, head.w (1026 x 288), head.b (1026)) to / from
 * host.  Head rows: 1024 candidate logits, the iteration output, the gate. */
int rljsde_net_get_params(const rljsde_net_t *net, float *host);
int rljsde_net_set_params(rljsde_net_t *net, const float *host);
/* Training patches: x (device, n x 5 x 16 x 16) for blocks (device int32
 * pairs (bi, bj)) of an image lr (device) with mask (device codes). */
int rljsde_net_patches(const float *lr, size_t lr_pitch, const uint8_t *mask, int lr_h, int lr_w,
                       const int32_t *blocks, int n, float *x, void *stream);
/* Loss and gradient of n patches: targets (device, n x 1024 bytes, 1 = in
 * the block's reference shortlist), nu_t (device, n floats in [0, 1]), mass
 * (device, n x 1024 floats: the plain loop's |gamma delta| summed per
 * candidate; NULL = no gate term).  Loss per patch: the logistic loss of the
 * candidates (positives weigh pos_weight) averaged over the 1024, plus
 * nu_weight (z_1024 - nu_t)^2, plus gate_weight (sigmoid(z_1025) - s)^2 with
 * s the share of the mass outside the patch's own 64 largest logits (a
 * target, not differentiated).  grad_out (device, num_params floats) may be
 * NULL; loss_host receives the mean loss.  Synchronous. */
int rljsde_net_gradient(rljsde_net_t *net, const float *x, const int32_t *blocks, int n, int lr_h, int lr_w,
                        const uint8_t *targets, const float *nu_t, const float *mass, float pos_weight,
                        float nu_weight, float gate_weight, float *grad_out, float *loss_host, void *stream);
/* The same followed by one Adam step with learning rate lr.  Synchronous. */
int rljsde_net_train_step(rljsde_net_t *net, const float *x, const int32_t *blocks, int n, int lr_h, int lr_w,
                          const uint8_t *targets, const float *nu_t, const float *mass, float pos_weight,
                          float nu_weight, float gate_weight, float lr, float *loss_host, void *stream);
/* Logits including bias (device, n x 1026) of n patches.  Synchronous. */
int rljsde_net_logits(rljsde_net_t *net, const float *x, const int32_t *blocks, int n, int lr_h, int lr_w,
                      float *z_out, void *stream);
/* Device workspace bytes rljsde_propose needs for a single-image plan. */
size_t rljsde_propose_workspace(const rljsde_plan_t *plan);
/* Run the network over the whole image and write one rljsde_shortlist per
 * block (device, n_blocks entries, block order bi * (2 lr_w / 4) + bj):
 * conv1 on the CUDA cores straight from lr and the plan's mask, conv2 and
 * conv3 on the tensor cores (bfloat16 activations, FP32 accumulation), then
 * one kernel that gathers each block's head features, multiplies them by the
 * head on the tensor cores (bfloat16 operands, FP32 accumulation in tensor
 * memory) and selects the 64 largest logits on the SM, so the logits never
 * reach device memory.  A tensor-core or copy wait that gives up is reported
 * by rljsde_check.  Asynchronous; the caller owns shortlists and workspace
 * (rljsde_propose_workspace bytes: 96 bytes per L-pixel).  The network reads
 * opaque-sub-pixel codes: plans of the three-quarter layout only. */
int rljsde_propose(const rljsde_plan_t *plan, const rljsde_net_t *net, const float *lr, size_t lr_pitch,
                   void *shortlists, void *workspace, size_t workspace_bytes, void *stream);
/*
 * rljsde_propose without any device allocation.  The paper has no
 * counterpart; this is for callers that cannot call cudaMalloc or hand over
 * a workspace, for example code running in a process whose device memory is
 * owned by another allocator (a framework's caching allocator, a fixed
 * budget reserved at start-up), or a camera pipeline that must not allocate
 * once it is streaming.
 *
 * The scratch is one fixed 32 MiB array inside the library, so every GPU
 * that loads the library holds it until the process exits.  Images whose
 * working set does not fit are rejected with RLJSDE_ERR_BAD_SHAPE: about
 * 349,000 L-pixels at most (96 bytes each; for example 590 x 590 L-pixels,
 * a 1180 x 1180 HR image).  The first call on a device looks the array's
 * address up (cudaGetSymbolAddress); make that first call before any stream
 * capture.  All calls share the one array: two calls whose work overlaps on
 * the GPU (different streams, or different host threads) race and corrupt
 * each other's results, so serialise them.  Nothing in the array needs to
 * start at zero; each call overwrites what it reads.  It runs the same
 * kernels as rljsde_propose, so the shortlists are identical.  Arguments,
 * output and the remaining errors are those of rljsde_propose.
 */
int rljsde_propose_noalloc(const rljsde_plan_t *plan, const rljsde_net_t *net, const float *lr, size_t lr_pitch,
                           void *shortlists, void *stream);
/* Reconstruct using shortlists: a block whose `missing` <= max_missing runs
 * the greedy loop over its 64 candidates (nu_max iterations, or the
 * network's iteration output if use_nu_hat), every other block the full
 * loop.  sel/dc as for rljsde_reconstruct_trace (unused iterations get
 * 0xFFFF), n_restricted (device int, added to) may be NULL.  FP32 plans of
 * the three-quarter layout on the recurrent host-table path. */
int rljsde_reconstruct_learned(const rljsde_plan_t *plan, const float *lr, size_t lr_pitch, float *hr,
                               size_t hr_pitch, const void *shortlists, float max_missing, int use_nu_hat,
                               uint16_t *sel, float *dc, int *n_restricted, void *stream);

/*
 * Measurement helper (this library's; the paper has no counterpart).  The
 * greedy loop of Eqs. 11-17 is bound by FP32 arithmetic, so its roofline
 * needs the device's FP32 FMA rate.  This times a kernel of independent FMA
 * chains on every SM of the current device (packed FFMA2 and scalar FFMA
 * variants, four 256-thread CTAs per SM), reps timed launches of each after
 * one warm-up (reps 1..1000), with CUDA events on `stream`.  *tflops_out gets
 * the best rate in TFLOP/s (an FMA counts 2 flops), *ms_out (may be NULL) the
 * duration of that launch.  Synchronous; allocates nothing.  Errors:
 * RLJSDE_ERR_INVALID_ARG (reps out of range, NULL tflops_out),
 * RLJSDE_ERR_CUDA.
 */
int rljsde_fp32_peak(int reps, void *stream, double *tflops_out, float *ms_out);

/*
 * Measurement helper (this library's).  The stored-C loop (c_supply) reads
 * one 8 KiB Gram column per block and iteration (Eq. 17 with C stored, Table
 * I), mostly from the L2; this times the L2 read bandwidth: every SM reads a
 * 32 MiB buffer (resident in the L2 after a warm-up launch) 128 times with
 * 16-byte non-coherent loads, reps timed launches (reps 1..1000) with CUDA
 * events on `stream`.  *gbs_out gets the best rate in GB/s, *ms_out (may be
 * NULL) that launch's duration.  Synchronous; allocates and frees 32 MiB of
 * device memory.  Errors: RLJSDE_ERR_INVALID_ARG, RLJSDE_ERR_OUT_OF_MEMORY,
 * RLJSDE_ERR_CUDA.
 */
int rljsde_l2_read_peak(int reps, void *stream, double *gbs_out, float *ms_out);

typedef struct {
    int n_images;
    int n_blocks;           /* target blocks over all images                  */
    int n_tables;           /* distinct local measurement matrices (plans)    */
    int n_interior_tables;  /* of which windows lie wholly inside the image   */
    int n_work_entries;     /* blocks after padding each table's run          */
    int warps_per_cta, ctas_per_sm, grid;   /* launch shape in effect (of the
                                               factored loop; of the stored-C
                                               loop when every table set is
                                               stored)                        */
    int64_t device_table_bytes;   /* factored tables actually stored (device) */
    int64_t paper_B_bytes;        /* Table I equivalent: n_tables x 256 x 1024 x 8 B */
    int64_t paper_C_bytes;        /* n_tables x 1024^2 x 8 B                  */
    int64_t paper_D_bytes;        /* n_tables x 1024 x 8 B                    */
    int path;                     /* path in effect: 1, 2 or 3 (rljsde_params) */
    int n_apertures;              /* distinct non-empty apertures in the masks  */
    int n_stored_c_tables;        /* table sets whose C is stored (c_supply)     */
    int n_stored_c_blocks;        /* blocks that use them                       */
    int64_t device_c_bytes;       /* their stored C on the device               */
    int n_launches;               /* kernels one rljsde_reconstruct launches    */
} rljsde_plan_info_t;

int rljsde_plan_info(const rljsde_plan_t *plan, rljsde_plan_info_t *out);

/* Synchronise `stream`, read and clear the plan's device status word.
 * Returns RLJSDE_OK or the first asynchronous error recorded. */
int rljsde_check(const rljsde_plan_t *plan, void *stream);

void rljsde_plan_destroy(rljsde_plan_t *plan);

const char *rljsde_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* RLJSDE_H */
