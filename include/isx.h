/*
 * isx.h -- C interface of the GB300 (sm_103a) library for hierarchical iso-surface extraction on
 * MLP implicit neural representations (Li & Shen, "Improving Efficiency of Iso-Surface
 * Extraction on Implicit Neural Representations Using Uncertainty Propagation").
 *
 * Conventions for every entry point
 *  - Pointers named d_* are CUDA device pointers on the current device, owned by the caller; the
 *    library never frees them.  Host pointers (descriptors, iso-value arrays) are read during the
 *    call only.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Work is enqueued
 *    on it; entry points that must read counts back (extraction) synchronise it before returning.
 *  - Every entry point returns an isx_status; nothing throws across this interface.  On failure
 *    isx_last_error() returns a message for the calling thread.  A capacity shortfall returns
 *    ISX_ERR_CAPACITY after filling in the required sizes, without writing past any capacity.
 *  - Cells of octree level l are integer triples (i, j, k) in [0, 2^l)^3 with box
 *    lo = -1 + 2 (i, j, k) / 2^l, hi = lo + 2 / 2^l; they are passed packed as
 *    code = i | j << 10 | k << 20, so levels go up to ISX_MAX_LEVEL = 10 (1024^3 cells).
 *  - The library keeps a per-INR workspace in device memory (grown with cudaMalloc on first use
 *    of a larger problem and freed by isx_destroy_inr).  Calls on one INR handle share that
 *    workspace, so they must not overlap: issue them from one thread, on one stream (or
 *    synchronise between streams).  Different handles are independent.
 */
#ifndef ISX_H
#define ISX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ISX_MAX_ISO 32
#define ISX_MAX_LEVEL 10
#define ISX_MAX_LAYERS 16
#define ISX_MC_MAX_TRI 5

typedef struct isx_inr_s* isx_inr;
typedef struct isx_proposer_s* isx_proposer;

typedef enum {
  ISX_OK = 0,
  ISX_ERR_ARG = 1,          /* invalid argument (null pointer, bad size, unsupported shape)      */
  ISX_ERR_CUDA = 2,         /* a CUDA runtime call or kernel launch failed                       */
  ISX_ERR_CAPACITY = 3,     /* an output buffer is too small; required sizes were filled in      */
  ISX_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up; the context stays usable     */
  ISX_ERR_UNSUPPORTED = 5,  /* valid request the library does not implement (e.g. width for BF16) */
  ISX_ERR_NOMEM = 6         /* workspace allocation failed                                       */
} isx_status;

/* How a cell's output range is bounded.
 *  SOUND: affine arithmetic (Sec. III-A, Eqs. 1-4): [x0 - r, x0 + r], r = sum |x_i| (Eq. 2), with
 *         the minimax (Chebyshev) linearisation of ReLU (Eq. 4).
 *  CLT:   uncertainty propagation with probabilistic affine forms (Sec. IV-B/C, Eqs. 6-10): input
 *         symbols scaled by 1/sqrt(3), ReLU linearised by least squares under N(mu, sigma^2)
 *         (Table VII), output N(mu, sigma^2) with sigma^2 = sum x_i^2 (Eq. 7), bound mu +- k sigma
 *         (Algorithm 1).
 *  RAUA:  SOUND propagation, then sigma^2 = (1/3) sum x_i^2 at the output only (Sec. IV-A),
 *         bound x0 +- k sigma.
 *  RAFIXED: the reduced range-analysis baseline (Sec. V-A.4, App. A): sound affine arithmetic
 *         that keeps the three input symbols and condenses every other coefficient of a neuron into
 *         one private radius (linear layers carry it through |W|); bound x0 +- r, k unused.
 *         Float32 only (prec = ISX_PREC_BF16 gives ISX_ERR_UNSUPPORTED); inflate applies as for
 *         SOUND.  Hidden widths that are multiples of 16. */
typedef enum { ISX_BOUND_SOUND = 0, ISX_BOUND_CLT = 1, ISX_BOUND_RAUA = 2, ISX_BOUND_RAFIXED = 3 } isx_bound_mode;

/* Arithmetic of the coefficient propagation.  FP32: float32 storage and FMA.  BF16: coefficient
 * matrices stored in bfloat16 and multiplied on tcgen05 tensor cores with float32 accumulation;
 * centres, reductions and linearisations stay float32.  Two BF16 kernels exist:
 *  - the row-batched path (hidden widths 64, 128, 256, 512; SOUND with or without inflation, CLT,
 *    RAUA):
 *    cells of a chunk are propagated layer by layer, the symbol rows of all cells in one tensor-core
 *    GEMM per layer, symbols whose coefficient is exactly 0 never created;
 *  - the per-cell persistent kernel (hidden widths 128, 256): isx_bound_cells_noalloc.
 * The choice is fixed by that rule (no switch).  Both stay within the BF16 rounding band of the
 * float64 propagation; they are not bit-identical. */
typedef enum { ISX_PREC_FP32 = 0, ISX_PREC_BF16 = 1 } isx_precision;

/* Activation applied after every linear layer but the last: ReLU (the ReLU INRs of App. E), ELU
 * (x for x > 0, e^x - 1 otherwise; App. A, App. E) or sine (the SIREN INRs of Sec. V-A.2, with the
 * frequency factor omega_0 folded into W and b by the caller, so the activation is sin z).
 * ELU and sine networks are bounded by the uncertainty-propagation rule only (ISX_BOUND_CLT, with
 * the ELU / sine rows of Table VII); the sound modes return ISX_ERR_UNSUPPORTED for them. */
typedef enum { ISX_ACT_RELU = 0, ISX_ACT_ELU = 1, ISX_ACT_SINE = 2 } isx_activation;

/* An MLP: n_layers linear layers 3 -> w -> ... -> w -> 1 with the activation after every layer but
 * the last.  All hidden widths must be equal.  W[l] is row-major [dims[l+1]][dims[l]] float32, b[l]
 * has dims[l+1] entries; both are HOST pointers, copied by isx_create_inr (the caller keeps
 * ownership).  A zero-initialised `activation` is ReLU. */
typedef struct {
  int n_layers;             /* 2 .. ISX_MAX_LAYERS                     */
  const int* dims;          /* n_layers + 1 entries, dims[0] = 3, dims[n_layers] = 1 */
  const float* const* W;
  const float* const* b;
  int activation;           /* isx_activation                          */
} isx_inr_desc;

/* Copies the weights to the current device (float32, transposed and bfloat16 copies for the
 * kernels).  Errors: ISX_ERR_ARG for a malformed descriptor, ISX_ERR_CUDA / ISX_ERR_NOMEM. */
isx_status isx_create_inr(const isx_inr_desc* desc, isx_inr* out);
isx_status isx_destroy_inr(isx_inr inr);

/* Bounds the INR over n axis-aligned boxes (the per-node step of Algorithm 1: node set-up,
 * propagation, read-off).  d_lo, d_hi: device float32 [n][3], lo <= hi componentwise.
 * Outputs (device float32 [n]): d_center = x0 (SOUND, RAUA) or mu (CLT); d_spread = r (SOUND) or
 * sigma (CLT, RAUA).  `inflate` != 0 (SOUND only) widens r by a bound on every rounding error of
 * the chosen precision so that [x0 - r, x0 + r] encloses the exact range of the float32-weight
 * network; with inflate = 0 the arithmetic follows the paper's formulas without that term.
 * n = 0 is valid and enqueues nothing. */
isx_status isx_bound_cells(isx_inr inr, const float* d_lo, const float* d_hi, int64_t n,
                           isx_bound_mode mode, isx_precision prec, int inflate,
                           float* d_center, float* d_spread, void* stream);

/* Allocation-free variant of isx_bound_cells with prec = ISX_PREC_BF16 (the paper has no
 * counterpart; this is a deployment convenience).  Some callers cannot allocate device memory once
 * they are running: a process whose device memory is owned by a framework's caching allocator,
 * or a latency-critical loop that must not take the device-wide synchronisation that cudaMalloc
 * and cudaFree imply.  This entry point allocates nothing: the per-cell tensor-core kernel takes its
 * per-CTA coefficient slices and its status word from a 16 MiB array compiled into the library
 * (every device that loads the library holds that array until the process exits).  Arguments
 * are those of isx_bound_cells.  Each cell is bounded by one CTA from start to end, so the results
 * do not depend on the grid: they are bit-identical from call to call, and agree with
 * isx_bound_cells within the BF16 band.  The grid is min(n, SMs, slices that fit in the array),
 * one slice being max(128, w (H - 3)) rows x w x 2 bytes (63 slices for a 256-wide, 5-hidden-layer
 * network), so it can be slower than isx_bound_cells.
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *    that device current and keeps it for the process; make that first call before any stream
 *    capture.  The address belongs to the device's context: after cudaDeviceReset on a device, do
 *    not call this entry point on that device again in the same process.
 *  - All calls share the array, which keeps the last call's contents; the call clears the status
 *    word itself.  Calls that overlap on the GPU (several streams or threads) race on the array:
 *    serialise them.
 *  - Errors: those of isx_bound_cells, ISX_ERR_UNSUPPORTED for widths other than 128 / 256, and
 *    ISX_ERR_CAPACITY if one CTA's slice would not fit in the array.  Synchronises `stream`. */
isx_status isx_bound_cells_noalloc(isx_inr inr, const float* d_lo, const float* d_hi, int64_t n,
                                   isx_bound_mode mode, int inflate, float* d_center, float* d_spread,
                                   void* stream);

/* Evaluates the INR at n points (device float32 [n][3]) into d_out (device float32 [n]).
 * ISX_PREC_FP32: FP32 FMAs on the CUDA cores.  ISX_PREC_BF16: tcgen05 tensor cores with every operand
 * split into two BF16 terms (x = x_hi + x_lo) and three products per multiply-add
 * (a_hi b_hi + a_hi b_lo + a_lo b_hi), FP32 accumulation: relative error per layer below about
 * 2^-15 of the absolute-value propagation, i.e. FP32-class; widths 128 and 256 only
 * (ISX_ERR_UNSUPPORTED otherwise). */
isx_status isx_eval_points(isx_inr inr, const float* d_xyz, int64_t n, isx_precision prec,
                           float* d_out, void* stream);

typedef struct {
  int max_level;                 /* finest grid: 2^max_level cells per axis over [-1, 1]^3     */
  int n_iso;                     /* 1 .. ISX_MAX_ISO                                            */
  float iso[ISX_MAX_ISO];        /* iso-values c (Algorithm 1)                                  */
  isx_bound_mode mode;
  float k;                       /* confidence multiplier t of Algorithm 1 (CLT, RAUA)          */
  isx_precision prec;
  int inflate;                   /* SOUND only: rounding-error inflation (see isx_bound_cells)  */
  int bound_stop_level;          /* levels deeper than this keep every child without bounding;
                                    < 0 or >= max_level: bound every level (the paper's setting) */
  /* learned proposal (no counterpart in the paper; NULL: plain range analysis at every level).
     At levels >= proposer_level (>= 1) every (cell, iso) pair of a cell's mask is scored first:
     p <= tau_lo drops the iso, p >= tau_hi keeps it without a bound, and a cell with any pair in
     between is bounded, its bound then deciding all of its isos. */
  isx_proposer proposer;
  int proposer_level;
  float tau_lo, tau_hi;
  /* corner / lattice evaluation: ISX_PREC_FP32 (CUDA cores, the default) or ISX_PREC_BF16
     (tensor cores with two-term BF16 operands, FP32-class accuracy; see isx_eval_points) */
  isx_precision eval_prec;
  /* 0: octree (every level splits all three axes; the default). 1: the k-d tree of Algorithm 1: every
     depth bisects the widest side (x, then y, then z on ties), depths 0 .. 3 max_level, so every third
     depth and the leaves are cubes; bound_stop_level counts octree levels (depth 3 x level).
     cells_visited / bounded / kept of depth d are added to octree level (d + 2) / 3.  With a
     proposer: ISX_ERR_UNSUPPORTED. */
  int kd_tree;
  /* optional record of the level loop (NULL: none); see isx_level_record */
  struct isx_level_record_s* record;
} isx_extract_params;

/* Record of the level loop of one hierarchical extraction (no counterpart in the paper: it exposes
 * the per-node state of Algorithm 1 so that callers, e.g. the proposer's label generation, need not
 * re-run the cull test and the subdivision themselves).  With params->record set,
 * isx_extract_isosurface appends, level after level from the root, every visited cell: its packed
 * code, the iso mask it inherited from its parent (all isos at the root), and the bound computed for
 * it (centre, spread as in isx_bound_cells; NaN at levels deeper than bound_stop_level).  Within a
 * level, cells are in the extraction's own order (children of surviving cells, in parent order,
 * child c = 2 (i, j, k) + the bits of c).  Buffers are caller-owned device arrays of `cap` entries;
 * level_off[l] .. level_off[l + 1] - 1 are level l's entries, filled in for levels 0 .. max_level.
 * If the total exceeds `cap`, nothing past `cap` is written, the extraction completes and the call
 * returns ISX_ERR_CAPACITY with level_off holding the required sizes.  Octree extraction without a
 * proposer only (ISX_ERR_UNSUPPORTED otherwise). */
typedef struct isx_level_record_s {
  uint32_t* d_code;
  uint32_t* d_mask;
  float* d_center;
  float* d_spread;
  int64_t cap;
  int64_t level_off[ISX_MAX_LEVEL + 2];   /* filled in by the call */
} isx_level_record;

typedef struct {
  /* caller-owned device outputs and capacities (in elements of the first dimension) */
  uint32_t* d_active_code;       /* [active_cap] packed codes of the predicted active cells      */
  uint32_t* d_active_mask;       /* [active_cap] bit q set: cell predicted active for iso q       */
  int64_t active_cap;
  float* d_tri_vert;             /* [tri_cap][3][3] triangle vertex positions                     */
  int64_t* d_tri_edge;           /* [tri_cap][3] global lattice-edge id of each vertex            */
  int32_t* d_tri_iso;            /* [tri_cap] iso-value index of each triangle                    */
  uint32_t* d_tri_cell;          /* [tri_cap] packed code of each triangle's cell (may be NULL)   */
  int64_t tri_cap;
  /* filled in by the call */
  int64_t n_active;              /* predicted active cells                                        */
  int64_t n_tris;                /* triangles over all iso-values                                 */
  int64_t n_points;              /* distinct lattice corners evaluated                            */
  int64_t cells_bounded[ISX_MAX_LEVEL + 1];   /* cells whose affine bound was computed        */
  int64_t cells_kept[ISX_MAX_LEVEL + 1];
  float ms_acp, ms_inr, ms_mc, ms_total;   /* active-cell prediction, corner evaluation, marching
                                              cubes, whole call (CUDA events on `stream`)        */
  int64_t cells_visited[ISX_MAX_LEVEL + 1];   /* cells considered per level (>= cells_bounded)  */
} isx_mesh;

/* Hierarchical extraction (Algorithm 1 run level by level over octree cubes, then corner queries
 * and marching cubes in the predicted active cells, Sec. IV-D).  The root cell [-1,1]^3 is bounded
 * first; a cell keeps iso q iff lower <= c_q <= upper and survives while any iso remains; at
 * max_level the survivors are the active cells.  Their distinct corners are evaluated and
 * triangulated per iso-value (inside = value < c).  Triangles are written in cell order.
 * Synchronises `stream`.  Errors: ISX_ERR_ARG, ISX_ERR_CAPACITY (n_active / n_tris hold the
 * required sizes), ISX_ERR_UNSUPPORTED (e.g. BF16 for an unsupported width), ISX_ERR_CUDA. */
isx_status isx_extract_isosurface(isx_inr inr, const isx_extract_params* params, isx_mesh* mesh,
                                  void* stream);

/* ---- batched extraction ----------------------------------------------------------------------
 * Many extractions in flight together (no counterpart in the paper, which extracts one INR at a
 * time).  Every entry runs exactly isx_extract_isosurface with its own INR and parameters (any mode,
 * precision, k, isos, max_level, bound_stop_level, k-d tree, proposer, level record), so its outputs
 * are bit-identical to that single call.  isx_batch_run hands the entries to `workers` host threads
 * (0: 8), each with its own non-blocking CUDA stream created by isx_batch_create; the level loops of
 * several extractions then overlap on the GPU, which pays where an extraction is too small to fill
 * it.  Each worker owns a workspace (grown with cudaMalloc on first use, freed by isx_batch_destroy)
 * and lends it to the INR of the entry it runs, so a batch holds `workers` workspaces however many
 * INRs it has, and an INR's own workspace is left as it was; with several workers the row-batched
 * bound works in smaller chunks (no cell's result depends on the chunking).  Entries that share an
 * INR handle run on one worker in entry order; different handles run concurrently, and no other call
 * may use the batch's INRs while isx_batch_run runs.  The workers start after the work queued on `stream`, and
 * `stream` waits for all of them.  Outputs per entry are those of isx_extract_isosurface (meshes[i]
 * for entry i, its caller-owned buffers).  The INRs must outlive the batch.  Errors: ISX_ERR_ARG
 * (a malformed entry, INRs on another device, workers outside 0..64, n outside 1..65535); otherwise
 * every entry runs and the first failing entry's status is returned (ISX_ERR_CAPACITY fills that
 * entry's required counts), with isx_last_error naming the entry.  isx_batch_run synchronises every
 * worker stream. */
typedef struct isx_batch_s* isx_batch;
isx_status isx_batch_create(const isx_inr* inrs, const isx_extract_params* params, int n, int workers,
                            isx_batch* out);
isx_status isx_batch_run(isx_batch batch, isx_mesh* meshes, void* stream);
isx_status isx_batch_destroy(isx_batch batch);

/* The dense baseline of Sec. V-A.4: evaluates every lattice point of the (2^max_level + 1)^3 grid
 * and runs marching cubes in every cell.  n_active = cells with at least one triangle; when
 * d_active_code and d_active_mask are given and n_active <= active_cap, those cells are written
 * there in cell order (i fastest, then j, then k) with bit q of the mask set iff the cell has a
 * triangle of iso q (the cells that truly cross each iso-surface on this grid).  mode, k, inflate
 * and bound_stop_level are ignored. */
isx_status isx_extract_dense(isx_inr inr, const isx_extract_params* params, isx_mesh* mesh,
                             void* stream);

/* The library's marching-cubes case table (host memory): ntri[256] triangle counts and
 * tris[256][ISX_MC_MAX_TRI][3] local edge numbers (-1 = unused).  Corner c of a cell sits at
 * (c & 1, c >> 1 & 1, c >> 2 & 1); edge 4a + t runs along axis a from the corner with bit a clear;
 * the two other axes p < q take bits t & 1 and t >> 1.  Host-only; needs no GPU. */
isx_status isx_mc_table(int8_t* ntri, int8_t* tris);

/* ---- learned proposal ------------------------------------------------------------------------
 * A cell-subdivision proposer (an addition; the paper decides by range analysis alone): an
 * 8 -> 64 -> 64 -> 64 -> 1 ReLU MLP with a sigmoid output giving, for a (cell, iso) pair, the
 * probability that the cell's subtree holds a finest cell crossed by that iso-surface.  BF16 weights
 * and activations with FP32 accumulation; FP32 master weights and Adam state on the device.
 * Parameters are packed FP32, row-major [out][in] weights each followed by its bias:
 * W1[64][8] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[1][64] b4[1].
 * Feature rows (float32 [n][8]): cell centre x, y, z; log2 of the half-width (= -level); iso-value
 * c; (centre of the nearest bounded ancestor's bound) - c; that bound's spread (radius or sigma);
 * level gap to that ancestor.  Features are standardised with (x - mean) / std before layer 1. */
#define ISX_PROPOSER_NPARAM 8961
/* Copies `params` (host, ISX_PROPOSER_NPARAM floats) and the standardisation (host, 8 + 8 floats,
 * std > 0) to the current device; Adam state starts at zero.  Synchronous. */
isx_status isx_proposer_create(const float* params, const float* feat_mean, const float* feat_std,
                               isx_proposer* out);
isx_status isx_proposer_destroy(isx_proposer p);
/* Current FP32 master parameters into host memory (ISX_PROPOSER_NPARAM floats).  Synchronous. */
isx_status isx_proposer_get_params(isx_proposer p, float* host_out);
/* Logits of n feature rows (device float32 [n][8]) into d_logit (device float32 [n]). */
isx_status isx_proposer_predict(isx_proposer p, const float* d_feat, int64_t n, float* d_logit,
                                void* stream);
/* Gradient of the mean binary cross-entropy over n labelled rows (labels device float32 [n], 0 or 1)
 * into d_grad (device float32 [ISX_PROPOSER_NPARAM], overwritten) and the loss into d_loss (device
 * float32 [1], overwritten).  The parameters are not changed. */
isx_status isx_proposer_grad(isx_proposer p, const float* d_feat, const float* d_label, int64_t n,
                             float* d_grad, float* d_loss, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on the mean BCE of n labelled rows;
 * d_loss (nullable, device float32 [1]) receives the loss before the step. */
isx_status isx_proposer_train_step(isx_proposer p, const float* d_feat, const float* d_label, int64_t n,
                                   float lr, float* d_loss, void* stream);

/* ---- measurement ----------------------------------------------------------------------------
 * Per-kernel accounting.  Launch counts and the algorithmic work of every launch (FLOPs and bytes
 * the method needs, excluding padding and recomputation) are always accumulated; with profiling
 * enabled every launch is also bracketed by CUDA events on its stream, and isx_profile_read
 * synchronises on them.  Counters are process-wide. */
typedef struct {
  const char* name;              /* kernel name (static string)                                   */
  int64_t launches;
  double ms;                     /* summed event time (0 unless profiling was enabled)            */
  double flops;                  /* summed algorithmic FLOPs                                       */
  double bytes;                  /* summed algorithmic HBM bytes                                   */
} isx_kernel_stats;

void isx_profile_enable(int on);
void isx_profile_reset(void);
/* Fills up to `max` entries and returns how many kernels the library knows. */
int isx_profile_read(isx_kernel_stats* out, int max);

/* ---- launch-shape autotuner ------------------------------------------------------------------
 * Kernels with interchangeable tile shapes (the FP32 coefficient GEMM of the FP32 bound: 64x64,
 * 32x64, 16x64, 128x64 and 64x128 output tiles, identical results) time every shape once per key
 * (kernel, hidden width, row-count bucket) on the real operands and keep the fastest for the process;
 * ISX_TUNE=0 in the environment disables tuning (first shape always).  isx_tune_read fills up to
 * `max` entries and returns how many keys are cached; strings stay valid until isx_tune_reset. */
typedef struct {
  const char* key;               /* e.g. "gemm_fp32 w=64 rows<=128"                              */
  const char* choice;            /* chosen tile shape                                             */
  int variant, n_variants;
  float ms_best, ms_first;       /* timed launch of the chosen and of the first shape            */
} isx_tune_entry;
int isx_tune_read(isx_tune_entry* out, int max);
void isx_tune_reset(void);

/* Self-check of the bounded device-side wait that every persistent kernel of the library uses
 * (tcgen05 producer / MMA / epilogue hand-offs on mbarriers): one CTA waits on an mbarrier that
 * nothing completes, with a limit of `limit_ns` nanoseconds, then records ISX_ERR_TIMEOUT and
 * returns, as the real kernels do when a wait expires.  Returns ISX_ERR_TIMEOUT (the expected
 * outcome; the context stays usable) or ISX_ERR_ARG for a limit outside [1000, 10^10] ns.
 * Synchronises `stream`.  No counterpart in the paper. */
isx_status isx_check_bounded_wait(int64_t limit_ns, void* stream);

/* Message describing the last failure on the calling thread ("" if none). */
const char* isx_last_error(void);

/* Library version: 100 * major + minor. */
int isx_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ISX_H */
