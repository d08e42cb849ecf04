/*
 * adjtx.h — C ABI of the GB300 (sm_103a) adjusted-transform library.
 *
 * The library computes batched, separable 2-D "adjusted" trigonometric
 * transforms of residual blocks, after A. Said, H. E. Egilmez, Y.-H. Chao,
 * "Low-complexity transform adjustments for video coding":
 *
 *   1-D transform of length N (Eq. 1):  H = C B A
 *     B  fast core, one of DCT-2, DCT-3, DST-2, DST-3 (Section 2.1: DCT-3 = DCT-2^T,
 *        DST-2 = R DCT-2 S, DST-3 = S DCT-2^T R), orthonormal;
 *     A  band pre-adjustment (Section 2, after Eq. 2; Section 2.2, item 1): layers of
 *        disjoint adjacent-pair Givens rotations, layer 0 applied first; an even layer
 *        rotates pairs (0,1),(2,3),..., an odd layer (1,2),(3,4),...,(N-3,N-2); the
 *        rotation by theta maps (x_i, x_{i+1}) to (c x_i - s x_{i+1}, s x_i + c x_{i+1});
 *     C  post-adjustment diag(Q, I_{N-K}) with Q a K x K orthogonal matrix acting on the K
 *        lowest-frequency outputs (Section 2.2, item 2; Section 2.3).
 *   2-D forward of an h x w row-major block X (Section 2.2: the adjustments act
 *   horizontally and vertically on the whole block):  Y = H_v X H_h^T  (row pass with
 *   the horizontal transform H_h of length w, column pass with the vertical H_v of length h);
 *   2-D inverse:  X = H_v^T Y H_h.
 *
 * Everything runs on one GPU in hand-written CUDA.  There is no CPU fallback: every
 * call that computes launches kernels, and fails with ADJ_ERR_CUDA when no usable
 * device is present.
 *
 * Conventions
 *   - All calls return ADJ_OK (0) or a negative ADJ_ERR_* code; nothing aborts or
 *     throws across this boundary.  adj_last_error() returns a message for the last
 *     failing call of the calling thread.  Calls that build host-side tables (plan
 *     creation and updates, block lists, tuning, graphs, the *_host entry points and
 *     adj_layout_preview) also return ADJ_ERR_NO_MEMORY when host memory runs out.
 *   - "stream" arguments are cudaStream_t values passed as void* (NULL = legacy
 *     default stream).  Device entry points are asynchronous with respect to the host:
 *     a kernel fault surfaces at the caller's next synchronisation.
 *   - Device buffers are owned by the caller; the library never allocates or frees
 *     them.  A plan owns its parameter tables, tile lists and work counters, all
 *     allocated by adj_plan_create / adj_plan_set_blocks, and the staging buffers of
 *     the *_host entry points (allocated on their first call).
 *   - Calls that use one plan must not run concurrently on the GPU (one stream, or
 *     serialised by the caller): the plan's work counters are shared by its launches.
 */
#ifndef ADJTX_H
#define ADJTX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ADJ_OK = 0,
  ADJ_ERR_INVALID_ARG = -1,      /* null pointer, bad enum, bad count, overlapping blocks */
  ADJ_ERR_UNSUPPORTED_SIZE = -2, /* N or block side not in {4, 8, 16, 32, 64}, K > N, too many layers */
  ADJ_ERR_PARAM_MISMATCH = -3,   /* block side != its transform's N; angle count; non-orthogonal Q;
                                    update_params that changes structure */
  ADJ_ERR_MISALIGNED = -4,       /* block offset not a multiple of 16 samples; buffer not 16-B aligned */
  ADJ_ERR_CUDA = -5,             /* a CUDA runtime call failed (message in adj_last_error) */
  ADJ_ERR_NO_BLOCKS = -6,        /* transform called before adj_plan_set_blocks */
  ADJ_ERR_NO_MEMORY = -7         /* host memory allocation failed; a plan the call was changing
                                    keeps its parameters but loses its block list */
};

/* Core B (Section 2.1). */
typedef enum { ADJ_CORE_DCT2 = 0, ADJ_CORE_DCT3 = 1, ADJ_CORE_DST2 = 2, ADJ_CORE_DST3 = 3 } adj_core_t;
/* Adjustment (Section 2.2): none, band pre-adjustment A, or top-left post-adjustment C.
 * ADJ_ADJ_DENSE is the reference the adjustments approximate: the 1-D transform is the given
 * dense orthogonal n x n matrix (q, k = n; e.g. the exact DST-7 or DCT-8 of Section 2.2,
 * Eq. 3) applied by a full matrix-vector product, with no fast core. */
typedef enum { ADJ_ADJ_NONE = 0, ADJ_ADJ_PRE_BAND = 1, ADJ_ADJ_POST_BLOCK = 2, ADJ_ADJ_DENSE = 3 } adj_kind_t;

#define ADJ_MAX_LAYERS 64

/* One 1-D adjusted transform H = C B A of length n.  Host memory, read during the call
 * that receives it (copied; the caller may free it afterwards). */
typedef struct {
  int32_t n;                    /* 4, 8, 16, 32 or 64 */
  int32_t core;                 /* adj_core_t */
  int32_t kind;                 /* adj_kind_t */
  int32_t n_layers;             /* band: number of rotation layers, 0..ADJ_MAX_LAYERS */
  const uint8_t* layer_parity;  /* band: n_layers entries, 0 = even pairs, 1 = odd pairs */
  const double* angles;         /* band: angles of layer 0 first; n/2 per even layer,
                                   n/2 - 1 per odd layer */
  int32_t k;                    /* post: size K of Q, 1 <= K <= n; dense: k = n */
  const double* q;              /* post / dense: K x K row-major, orthogonal to 1e-6 */
} adj_1d_desc_t;

/* One residual block: h rows x w columns, row-major, starting at element `offset` of
 * the packed buffers.  tf_h / tf_v index the plan's 1-D transforms (tfs[tf_h].n == w,
 * tfs[tf_v].n == h).  16 bytes. */
typedef struct {
  int64_t offset;  /* in samples; multiple of 16 */
  uint16_t w, h;
  uint16_t tf_h, tf_v;
} adj_block_t;

typedef struct adj_plan adj_plan_t;

/* Launch and tiling choices of a plan (see adj_plan_autotune).
 * cap_div[(log2 w - 2) * 5 + (log2 h - 2)]: a tile of w x h blocks holds 1/cap_div of the
 * most that fit (1, 2, 4 or 8); ctas_per_sm: persistent CTAs per SM (0 = as many as fit);
 * ranges_per_sm: scheduling ranges of the class-sorted tile list per SM (1..4);
 * tail_pct: the cheapest tiles, this percentage of the estimated run time, are dealt over
 * the ends of all ranges instead of staying with their class (0..50), so that the tiles
 * CTAs hold when the work runs out are short ones.  A new plan has every cap_div 1,
 * ctas_per_sm 0, ranges_per_sm 1 and tail_pct 10. */
typedef struct {
  int32_t cap_div[25];
  int32_t ctas_per_sm;
  int32_t ranges_per_sm;
  int32_t tail_pct;
} adj_tuning_t;

/* Plan flags. */
#define ADJ_PLAN_DEFAULT 0

/*
 * Create a plan for a table of 1-D transforms (Eq. 1 per entry).
 * Validates every entry, materialises the parameters on the host in FP64 (cos/sin of
 * each angle; Q padded to a power of two with the identity, i.e. the top-left block of
 * C = diag(Q, I)) and uploads them as FP32 to the current device.
 * Errors: INVALID_ARG, UNSUPPORTED_SIZE, PARAM_MISMATCH, CUDA.  On error *plan is NULL.
 */
int adj_plan_create(adj_plan_t** plan, const adj_1d_desc_t* tfs, int32_t n_tfs, int32_t flags);

/*
 * Give the plan its block list (host memory, n_blocks records) for buffers of
 * total_coefs samples: the W x H residual blocks a codec transforms (Section 2.2).  Validates sizes, transform indices, alignment, bounds and
 * non-overlap; groups blocks of equal (w, h, tf_h, tf_v) into shared-memory tiles in
 * storage order, sorts the tiles by the code they run and cuts them into one scheduling
 * range per SM of about equal estimated run time (most expensive tiles first in each),
 * and uploads the tile list.  May be called again to replace the list; the previous
 * list's device tables are freed then, so no launch of this plan may still be running.
 * A list with more blocks than total_coefs / 16 is rejected before it is read.
 * Errors: INVALID_ARG, UNSUPPORTED_SIZE, PARAM_MISMATCH, MISALIGNED, CUDA, NO_MEMORY.
 */
int adj_plan_set_blocks(adj_plan_t* plan, const adj_block_t* blocks, int64_t n_blocks,
                        int64_t total_coefs);

/*
 * The scheduling layout adj_plan_set_blocks builds, computed on the host alone (no device is
 * used): the transforms and blocks are validated as by adj_plan_create and
 * adj_plan_set_blocks, then grouped into tiles and cut into ranges for a GPU of n_sm SMs
 * under the default tuning.  Outputs (each optional; the counts are always written):
 *   tiles[t]    tile t in launch order: its first entry in `list`, block count, w, h, tf_h, tf_v;
 *   costs[t]    its estimated run time (microseconds, the planner's model);
 *   list        block offsets / 16 of every tile, each tile's run 4-entry aligned, 4 spare
 *               entries at the end (*list_len entries);
 *   range_begin first tile of each range, *n_ranges + 1 entries (the last one = *n_tiles).
 * tiles and costs hold tiles_cap records, list list_cap entries, range_begin ranges_cap + 1.
 * Errors: as those two calls; INVALID_ARG also when an output array is too small (the counts
 * are still written) or n_sm is outside 1..256.
 */
typedef struct {
  uint32_t list_begin;            /* first entry of the tile's block list */
  uint16_t nblk, w, h, tf_h, tf_v, pad;
} adj_tile_info_t;
int adj_layout_preview(const adj_1d_desc_t* tfs, int32_t n_tfs, const adj_block_t* blocks, int64_t n_blocks,
                       int64_t total_coefs, int32_t n_sm, adj_tile_info_t* tiles, double* costs,
                       int64_t tiles_cap, int64_t* n_tiles, uint32_t* list, int64_t list_cap, int64_t* list_len,
                       uint32_t* range_begin, int32_t ranges_cap, int32_t* n_ranges);

/*
 * Replace the parameter values (angles, Q) of all transforms without changing their
 * structure (n, core, kind, layer parities, K).  The upload is a synchronous cudaMemcpy
 * that has completed when the call returns.  It is ordered after earlier work on the
 * legacy default stream and on blocking streams only: launches of this plan on a
 * non-blocking stream must have finished before the call (synchronise that stream).
 * After a validation error the plan keeps its previous values.
 * Errors: INVALID_ARG, PARAM_MISMATCH, CUDA, NO_MEMORY.
 */
int adj_plan_update_params(adj_plan_t* plan, const adj_1d_desc_t* tfs, int32_t n_tfs);

/*
 * Forward 2-D transform of every block: d_resid (int16, device, total_coefs samples,
 * 16-B aligned) -> d_coef (FP32, device, total_coefs, 16-B aligned), Y = H_v X H_h^T with
 * H = C B A of Eq. 1 in each direction, applied horizontally and vertically to the whole
 * block (Section 2.2).  Samples outside every block are not written.  One persistent
 * kernel launch, asynchronous on `stream`.
 * Errors: INVALID_ARG, NO_BLOCKS, MISALIGNED, CUDA.
 */
int adj_transform_fwd(adj_plan_t* plan, const int16_t* d_resid, float* d_coef, void* stream);

/*
 * Inverse 2-D transform: d_coef (FP32, device) -> d_resid_out (FP32, device, not
 * rounded), X = H_v^T Y H_h: every factor of Eq. 1 is orthogonal, so H^-1 = A^T B^T C^T
 * (the inverse core, the transposed post block, the band layers reversed with -theta).
 * Same layout, alignment, launch and error rules as adj_transform_fwd.
 */
int adj_transform_inv(adj_plan_t* plan, const float* d_coef, float* d_resid_out, void* stream);

/*
 * Forward 2-D transform of FP32 blocks (Eq. 1 applied to inputs that are not int16
 * residuals, e.g. the FP32 input of a gradient computation): d_x (FP32, device, total_coefs,
 * 16-B aligned) -> d_coef as adj_transform_fwd.  Same kernel design with FP32 staging, one
 * persistent launch, asynchronous on `stream`.  Errors: INVALID_ARG, NO_BLOCKS, MISALIGNED,
 * CUDA.
 */
int adj_transform_fwd_f32(adj_plan_t* plan, const float* d_x, float* d_coef, void* stream);

/*
 * Blocks inside a frame.  The adjustments act on W x B and B x H regions of a frame
 * (Section 2.2); a codec keeps its residual and its reconstruction as frames, so these calls
 * read each block from its place in a residual frame and write it back to its place,
 * without a packing step.
 *
 * adj_plan_set_frame_blocks gives the plan n_blocks blocks (host memory) of a frame of
 * frame_w x frame_h samples whose rows are `stride` samples apart (stride >= frame_w, a
 * multiple of 8; frame buffers 16-B aligned).  A batch of equal frames stored one after
 * another with the same stride is one frame of (frames x frame_h) rows: one launch then
 * covers the whole batch.  Block positions (x, y) are multiples of 4, blocks
 * lie inside the frame and do not overlap; sizes and transform indices follow the rules of
 * adj_block_t.  The coefficients of the blocks are packed: block i's h x w coefficients
 * (row-major) start at sample sum_{j<i} w_j h_j, and total_coefs is that sum over all blocks.
 * (The packed entry points adj_transform_fwd/_inv and the host-buffer ones then work on that
 * packed layout.)  Errors: INVALID_ARG (also overlaps, blocks outside the frame),
 * UNSUPPORTED_SIZE, PARAM_MISMATCH, MISALIGNED (positions, stride), CUDA.
 *
 * adj_transform_fwd_frame: d_frame (int16 residual frame, device) -> d_coef (FP32, packed as
 * above, device).  adj_transform_inv_frame: d_coef -> exactly one of d_frame_f32 (FP32) or
 * d_frame_i16 (rounded to nearest, ties to even, saturated to int16); samples outside every
 * block are not written.  One persistent launch each, asynchronous on `stream`.
 * Errors: INVALID_ARG (also: the plan has no frame blocks, both or neither output given),
 * NO_BLOCKS, MISALIGNED, CUDA.
 */
typedef struct {
  int32_t x, y;    /* top-left sample of the block in the frame */
  uint16_t w, h;
  uint16_t tf_h, tf_v;
} adj_frame_block_t;
int adj_plan_set_frame_blocks(adj_plan_t* plan, const adj_frame_block_t* blocks, int64_t n_blocks, int32_t frame_w,
                              int32_t frame_h, int32_t stride);
int adj_transform_fwd_frame(adj_plan_t* plan, const int16_t* d_frame, float* d_coef, void* stream);
int adj_transform_inv_frame(adj_plan_t* plan, const float* d_coef, float* d_frame_f32, int16_t* d_frame_i16,
                            void* stream);

/*
 * Simultaneous DST-7 / DCT-8 adjustments for an encoder's transform search ("Multiple",
 * Section 2.3).  With a post-adjustment after the DCT-2, S T^(C2) = T^(C2) R turns the
 * DCT-8 flip of Eq. 3 into Eq. 5: if C^(S7) = diag(Q, I) adjusts the DCT-2 towards the
 * DST-7, then C^(C8) = S C^(S7) S adjusts it towards the DCT-8 (Q with its signs flipped in
 * a chessboard pattern).  The encoder wants, per block, the 2-D DCT-2 and the four
 * (vertical a, horizontal b) pairings of the two adjusted transforms,
 *   Y_DD = T_v X T_h^T,   Y_ab = H_a,v X H_b,h^T   (a, b in {S = DST-7, C = DCT-8}),
 * and only the first K lines of an adjusted transform differ from the DCT-2, so each
 * distinct coefficient is computed and stored once: Y_DD in place, plus per block these
 * side regions (kh, kv = the K of the horizontal / vertical transform, 0 when it has no
 * adjustment; a, b = 0 for DST-7, 1 for DCT-8; each region row-major, in this order):
 *   R_0, R_1           rows < kv, columns >= kh of the pairings with vertical a: kv x (w - kh)
 *   L_0, L_1           rows >= kv, columns < kh of the pairings with horizontal b: (h - kv) x kh
 *   X_00, X_01, X_10, X_11   rows < kv, columns < kh of pairing (a, b): kv x kh
 * that is 2 kv w + 2 h kh floats, rounded up to a multiple of 4.  Every other coefficient
 * of Y_ab equals Y_DD.  The even/odd split of Q gives both adjustments of a line for the
 * multiplications of one K x K product.
 *
 * adj_plan_prepare_multiple validates the current block list for this form: every
 * transform a block uses must have core ADJ_CORE_DCT2 and kind ADJ_ADJ_NONE or
 * ADJ_ADJ_POST_BLOCK with 2K <= n (INVALID_ARG / UNSUPPORTED_SIZE otherwise; the q of the
 * transform is Q of C^(S7)).  Side regions follow the order of the block list given to
 * adj_plan_set_blocks: block i starts at side_offsets[i] floats (host array of n_blocks + 1
 * entries, optional; the last entry is the total), *side_total = total floats (optional).
 * Call it again after adj_plan_set_blocks; adj_plan_set_tuning and adj_plan_autotune keep it.
 *
 * adj_transform_fwd_multiple: d_resid (int16, device) -> d_coef (FP32, device, Y_DD in the
 * layout of adj_transform_fwd) and d_side (FP32, device, side_total floats; may be NULL
 * when side_total is 0); all 16-B aligned.  One persistent kernel launch, asynchronous
 * on `stream`.  Errors: INVALID_ARG (also: not prepared), NO_BLOCKS, MISALIGNED, CUDA.
 * The inverse of a chosen pairing is adj_transform_inv with post transforms Q or S Q S.
 */
int adj_plan_prepare_multiple(adj_plan_t* plan, int64_t* side_offsets, int64_t* side_total);
int adj_transform_fwd_multiple(adj_plan_t* plan, const int16_t* d_resid, float* d_coef, float* d_side,
                               void* stream);

/*
 * Backward of adj_transform_fwd for fitting the adjustments (the paper designs them by a
 * constrained least-squares fit, Eq. 2, through the Givens factorisation after it).
 * Given the forward input d_x (int16 or FP32 per x_dtype, device, the same layout) and
 * d_gy = dL/dY (FP32, device), writes
 *   d_gx      (optional, FP32, device, total_coefs): dL/dX = H_v^T G H_h per block;
 *   d_gparams (optional, FP32, device): the gradients of every transform's parameters,
 *             transform i at offsets[i] (adj_plan_param_layout): band -> one entry per angle
 *             (same order as the angles), post -> K x K entries of dL/dQ (row major),
 *             dense -> n x n entries, none -> nothing.
 * Sums over blocks are formed per CTA in a fixed assignment and added in a fixed order, so
 * repeated calls give bit-identical gradients.  Asynchronous on `stream`.
 */
#define ADJ_DTYPE_INT16 0
#define ADJ_DTYPE_FP32 1
int adj_transform_bwd(adj_plan_t* plan, const void* d_x, int32_t x_dtype, const float* d_gy, float* d_gx,
                      float* d_gparams, void* stream);
/* offsets[i] = first gradient entry of transform i; offsets[n_tfs] = total (n_tfs + 1 entries). */
int adj_plan_param_layout(const adj_plan_t* plan, int32_t* offsets);

/*
 * Coding-gain proxy of coefficient blocks, the objective beside Eq. 2 that the fitter
 * minimises: for n_blocks blocks of hw coefficients stored back to back in d_y (FP32,
 * device), var[p] = mean_b Y_b[p]^2, *d_loss = (1/hw) sum_p log var[p] (FP64, device), and,
 * if d_gy is given, dL/dY = 2 Y / (hw n var) (FP32, device, same layout as d_y).  d_work is
 * caller-owned device scratch of 65 * hw doubles.  Sums are in a fixed order.
 * Errors: INVALID_ARG (hw not in 1..4096), CUDA.
 */
int adj_coding_gain_proxy(const float* d_y, int64_t n_blocks, int32_t hw, double* d_work, double* d_loss, float* d_gy,
                          void* stream);

/*
 * Plain (unfused) form of the same transforms, the baseline the fused path is measured
 * against: for every block size present, one launch per step of the chain (band, core,
 * post) along the rows, then along the columns (forward; the inverse runs the transposed
 * steps in reverse order), each step reading and writing FP32 lines in global memory.
 * Same arguments, layout and results (up to FP32 rounding) as adj_transform_fwd/_inv;
 * up to 150 launches per call.
 */
int adj_transform_fwd_plain(adj_plan_t* plan, const int16_t* d_resid, float* d_coef, void* stream);
int adj_transform_inv_plain(adj_plan_t* plan, const float* d_coef, float* d_resid_out, void* stream);

/*
 * Host-buffer variants: copy the input from host memory to plan-owned device staging
 * buffers, transform, copy the result back and wait for it.  The block list (in storage
 * order) is cut into chunks of up to about 4 M samples, shorter at both ends; each chunk's
 * input copy, kernel launch and output copy run on three streams, so the copies of one chunk
 * overlap the kernel and copies of the others.  Page-locked host memory gives full copy bandwidth.
 * Samples of h_out outside every block are left unchanged or set to zero.  The staging
 * buffers, chunk tile lists, two streams and their events are allocated on the first call
 * (and the chunk lists again after the block list or the tuning changes).
 */
int adj_transform_fwd_host(adj_plan_t* plan, const int16_t* h_resid, float* h_coef, void* stream);
int adj_transform_inv_host(adj_plan_t* plan, const float* h_coef, float* h_resid_out, void* stream);

/*
 * Forward transform of a uniform batch that allocates nothing.
 * The paper has no counterpart to this entry point; it exists for callers that cannot
 * allocate device memory on their processing path: a real-time encoder that reserves all
 * of its GPU memory at start-up and must not call cudaMalloc/cudaFree per frame (they
 * can synchronise the device and stall the rest of the pipeline), or a plug-in inside a
 * host framework that owns the device memory and offers plug-ins no allocator.
 *
 * Computes the same transform as adj_transform_fwd with the same fused kernel, for
 * n_blocks blocks of tf_v->n rows x tf_h->n columns stored back to back (block b starts
 * at sample b * w * h), all using tf_h horizontally and tf_v vertically.  d_resid (int16)
 * and d_coef (FP32) are caller-owned device buffers, 16-B aligned.  The transform runs
 * asynchronously on `stream`, but the transform records and parameters are uploaded from
 * pageable host memory that lives only for the call, so the call may block the host until
 * the work already queued on `stream` has finished (adj_transform_fwd, whose parameters
 * were uploaded at plan creation, does not).  For the same reason the call cannot be
 * recorded into a CUDA graph: while `stream` is capturing it returns INVALID_ARG and
 * enqueues nothing.
 *
 * Scratch: the work counter, the two transform records, their FP32 parameters and the
 * tile list live in one static device array of ADJ_NOALLOC_SCRATCH_BYTES that every
 * device loading the library holds until the process exits.  No cudaMalloc, cudaFree or
 * other allocating routine is called.  The first call on a device (with that device
 * current) looks up the array's device address once; make that first call before any
 * stream capture on that device.  Every call shares the array: it clears the work counter and rewrites
 * the rest, and calls that overlap on the GPU (other streams or host threads) race on it,
 * so the caller must serialise them.
 * Errors: INVALID_ARG (also a call on a capturing stream), UNSUPPORTED_SIZE (also
 * n_blocks > ADJ_NOALLOC_MAX_BLOCKS), PARAM_MISMATCH, MISALIGNED, CUDA.
 */
#define ADJ_NOALLOC_SCRATCH_BYTES (3u << 20)
#define ADJ_NOALLOC_MAX_BLOCKS 131072
int adj_transform_fwd_uniform_noalloc(const adj_1d_desc_t* tf_h, const adj_1d_desc_t* tf_v, int64_t n_blocks,
                                      const int16_t* d_resid, float* d_coef, void* stream);

/*
 * CUDA graphs of a plan's launches for fixed buffers (captured once, replayed by
 * adj_graph_launch).  `what` selects the launches:
 *   ADJ_GRAPH_FWD / ADJ_GRAPH_INV              the fused kernel (d_in -> d_out)
 *   ADJ_GRAPH_FWD_PLAIN / ADJ_GRAPH_INV_PLAIN  the plain form (d_in -> d_out)
 *   ADJ_GRAPH_ROUNDTRIP                        fused forward d_in -> d_out, then fused
 *                                              inverse d_out -> d_out2
 *   ADJ_GRAPH_FWD_MULTIPLE                     Multiple forward d_in -> d_out (Y_DD) and
 *                                              d_out2 (side regions)
 * The graph refers to the plan's tables: replace neither the block list nor the plan while
 * it exists (adj_plan_update_params is fine).  Errors: INVALID_ARG, NO_BLOCKS, MISALIGNED, CUDA.
 */
typedef struct adj_graph adj_graph_t;
enum { ADJ_GRAPH_FWD = 0, ADJ_GRAPH_INV = 1, ADJ_GRAPH_FWD_PLAIN = 2, ADJ_GRAPH_INV_PLAIN = 3,
       ADJ_GRAPH_ROUNDTRIP = 4, ADJ_GRAPH_FWD_MULTIPLE = 5 };
int adj_graph_create(adj_plan_t* plan, int32_t what, const void* d_in, float* d_out, float* d_out2,
                     adj_graph_t** graph);
int adj_graph_launch(adj_graph_t* graph, void* stream);
void adj_graph_destroy(adj_graph_t* graph);

/* Read / replace a plan's tuning; replacing rebuilds its tile layout (no graph made from the
 * plan may be launched afterwards).  Errors: INVALID_ARG (values out of range), CUDA. */
int adj_plan_get_tuning(const adj_plan_t* plan, adj_tuning_t* tuning);
int adj_plan_set_tuning(adj_plan_t* plan, const adj_tuning_t* tuning);

/*
 * Autotuner: times forward + inverse on the plan's own blocks (d_resid int16 input,
 * d_coef and d_recon FP32 scratch of total_coefs samples, all device) for candidate
 * tunings and keeps the fastest: the tail share, CTAs per SM, ranges per SM, then the tile capacity of each
 * block size in order of its share of the coefficients (coordinate descent).  If
 * cache_path is given, a result stored there for this device and this workload signature
 * (block sizes and transform kinds) is applied without measuring, and a new result is
 * appended.  max_evals bounds the number of timed candidates (0: no bound).  Synchronises
 * `stream`.  Errors: INVALID_ARG, NO_BLOCKS, MISALIGNED, CUDA.
 */
int adj_plan_autotune(adj_plan_t* plan, const int16_t* d_resid, float* d_coef, float* d_recon,
                      const char* cache_path, int32_t max_evals, void* stream);

/* Launch geometry and tile statistics of a plan (for benchmarks and tests). */
typedef struct {
  int64_t n_blocks;
  int64_t total_coefs;
  int32_t n_tiles;
  int32_t grid_fwd, grid_inv;   /* persistent CTAs per launch */
  int32_t threads;              /* threads per CTA */
  int32_t smem_bytes;           /* dynamic shared memory per CTA */
  int32_t n_sm;
} adj_plan_info_t;
int adj_plan_info(const adj_plan_t* plan, adj_plan_info_t* info);

/* Release everything the plan owns.  Safe on NULL. */
void adj_plan_destroy(adj_plan_t* plan);

/* Message of the last failing call on this thread ("" if none). */
const char* adj_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ADJTX_H */
