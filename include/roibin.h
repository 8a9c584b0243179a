/*
 * roibin.h - C ABI of the GB300 ROIBIN-SZ compression library (libroibin).
 *
 * ROIBIN-SZ (arXiv 2206.11297) compresses serial-crystallography detector
 * frames: a peak finder marks Bragg spots (§4.2), a window around each spot is
 * kept losslessly (§4, §4.1), the whole frame is binned (§4.1, §6) and the
 * binned background is coded with an absolute error bound (§5.3.3) by an
 * SZ-style predictor/quantiser/entropy coder (§5.3.2).  Every step runs in
 * CUDA kernels for sm_103a; this header is the only boundary.
 *
 * Conventions (all entry points):
 *  - Pointers named d_* are device pointers, h_* host pointers.  The caller
 *    owns every buffer it passes; the context owns only its own scratch.
 *  - A frame is float32[n_panels][rows][cols], little-endian, contiguous;
 *    frames of a batch follow each other (4-D events x panel x row x col,
 *    the panel-aware layout of §4.1).
 *  - Calls taking a stream enqueue asynchronously on it (cudaStream_t passed
 *    as void*; NULL = legacy default stream) unless stated otherwise.
 *  - Every call returns a status (ROIBIN_OK or a negative ROIBIN_ERR_*).
 *    Argument errors are detected on the host before anything is enqueued.
 *    Per-frame conditions found on the device (too many peaks, output too
 *    small, corrupt input stream) are written to the caller's per-frame status
 *    array; they never trap the GPU.
 *  - One call at a time per context: calls on the same context must be ordered
 *    (same stream, or synchronised), since they share its scratch; one host
 *    thread drives a context.
 *
 * Stream format (version 1, little-endian; the paper defines no container):
 *   [0,96)  header: u32 magic "RBSZ" | u32 version | u32 n_panels, rows, cols |
 *           u16 roi_h, roi_w, bin_h, bin_w | f32 abs_eb | u32 quant_radius |
 *           u32 n_peaks | u32 n_lorenzo_outliers | u32 n_prequant_outliers |
 *           u32 n_symbols | u32 chunk_symbols (4096) | u32 n_chunks |
 *           u32 bitstream_words | u64 total_bytes | u32 lorenzo dimension
 *           (0 for the default 2, else 1 or 3) | u32 roi coding | u32 roi
 *           section bytes | u32 roi section words | u32 code-length back
 *           reference (0: this stream keeps its code lengths; b > 0: they are
 *           in the stream of the frame b frames earlier in the same call, the
 *           head of its chunk) | 4 zero bytes
 *   then, each starting on a 16-byte boundary, zero padded:
 *     peaks       u16[n_peaks][3] (panel, row, col)
 *     roi         f32[n_peaks][roi_h][roi_w] (roi coding 0; empty otherwise)
 *     lengths     u8[2 * quant_radius]        Huffman code length per symbol
 *                                             (back reference 0 only; absent otherwise)
 *     chunk index u32[n_chunks]               word offset of each 4096-symbol chunk
 *     lorenzo     (u32 bin index, i32 delta)[n_lorenzo_outliers], ascending
 *     prequant    (u32 bin index, u32 float bits)[n_prequant_outliers], ascending
 *     bitstream   u32[bitstream_words]; inside a chunk, codeword bits are
 *                 appended MSB first, stream bit b is bit 31-(b%32) of word b/32;
 *                 every chunk starts on a word boundary.
 *     roi section (roi coding 1 or 2 only; roi section bytes long):
 *                 coding 2: f32[n_peaks][roi_h][roi_w], the raw windows;
 *                 coding 1: the windows coded losslessly (paper §4 keeps them
 *                 with fpzip; this coder is our own of that kind):
 *                   u8[33] Huffman code length per class, zero padded to 48;
 *                   u32[n_peaks] first word of each window, padded to 16;
 *                   u32[roi section words], padded to 16.
 *                 In a window, row-major, each float's bits u become
 *                 m = u + 2^31 (sign 0) or NOT u (sign 1); m is predicted mod
 *                 2^32 by m[i-1][j] + m[i][j-1] - m[i-1][j-1] (0 outside the
 *                 window; the first value by 2^31); the residual r (int32) is
 *                 folded to z = 2r or -2r-1; z is written as the Huffman code
 *                 of its bit length c (0..32), then its c-1 bits below the
 *                 leading one, MSB first.  Each window starts on a word.
 *                 The coder stores coding 2 whenever coding 1 would not be
 *                 smaller, so a stream never exceeds roibin_compress_bound.
 */
#ifndef ROIBIN_H
#define ROIBIN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define ROIBIN_OK 0
#define ROIBIN_ERR_INVALID_ARG (-1)    /* bad pointer, geometry or parameter          */
#define ROIBIN_ERR_CAPACITY (-2)       /* > max_peaks peaks, or frame > output stride */
#define ROIBIN_ERR_CORRUPT_STREAM (-3) /* decompression input fails validation       */
#define ROIBIN_ERR_OUT_OF_BUDGET (-4)  /* scratch would exceed the HBM budget         */
#define ROIBIN_ERR_CUDA (-5)           /* a CUDA runtime call failed                  */
#define ROIBIN_ERR_TIMEOUT (-6)        /* a bounded device-side wait gave up          */
#define ROIBIN_ERR_CODE_LENGTH (-7)    /* Huffman code > 32 bits (cannot occur for
                                          frames below 5,702,887 bins)                */
#define ROIBIN_ERR_CHECK (-8)          /* checks build: a device bounds check failed
                                          or a scratch guard band was overwritten     */
/* Per-frame outcome that is not an error: non-hit rejection (paper §1, §4:
 * frames with too few peaks to index are dropped before compression).  The
 * frame has fewer peaks than nhr_min_peaks; nothing is written for it and its
 * size is 0. */
#define ROIBIN_REJECTED 1

/* ---- execution paths for roibin_compress ----------------------------- */
#define ROIBIN_PATH_AUTO 0  /* fused when the geometry and parameters allow it, else
                               plain                                                 */
#define ROIBIN_PATH_PLAIN 1 /* one kernel per stage, intermediates in device memory  */
#define ROIBIN_PATH_FUSED 2 /* one persistent kernel per batch: work items of a few
                               panels each, then each frame's coding stages        */

/* Decompression paths (roibin_ctx_set_decompress_path). */
#define ROIBIN_DEC_AUTO 0      /* PANEL when the geometry and lorenzo_dims (2) allow it,
                                  else MULTIPASS                                         */
#define ROIBIN_DEC_PANEL 1     /* prefix-table decode to symbols, then one block per
                                  (frame, panel) rebuilds the panel in shared memory
                                  and writes its pixels once; needs bins per panel row
                                  (cols / bin_w rounded up) <= 4096                     */
#define ROIBIN_DEC_MULTIPASS 2 /* one kernel per step of the inverse, intermediates in
                                  device memory                                         */

typedef struct roibin_ctx roibin_ctx;

/* Detector geometry: every frame is n_panels panels of rows x cols pixels
 * (CSPAD 32x185x388, epix10k 16x352x384, JUNGFRAU 8x512x1024; §4.2). */
typedef struct {
  uint32_t n_panels, rows, cols;
} roibin_geometry;

/* Method parameters.  All are user-configurable (§4.2); defaults from
 * roibin_default_params are the paper's values where it gives one.
 *   Peak finder (§4.2): a pixel is a candidate when it is the maximum of its
 *   (2 rank + 1)^2 window clipped to the panel (ties: the first pixel in
 *   row-major order wins) and >= amax_thr (300).  The background is the mean
 *   and population standard deviation of the in-panel ring
 *   ring_r0^2 <= di^2 + dj^2 < (ring_r0 + ring_dr)^2 (5, 2), both in float32:
 *   every add, subtract, multiply, divide and sqrt rounds once to nearest, and
 *   the sums run in row-major order over the ring.  Peak pixels are
 *   window pixels with I - bkg > pix_nsigma * sigma (3; 0 = the paper's plain
 *   above-zero test).  A candidate is kept when npix_min <= npix <= npix_max
 *   (2, 30), atot > atot_thr (600) and atot > son_min * sigma * sqrt(npix) (10).
 *   ROI (§4): roi_h x roi_w window centred on each peak (17 x 17), fill 0 past
 *   the panel edge.  Binning (§4.1, §6): bin_h x bin_w mean per panel (2 x 2).
 *   Coding (§5.3.3): |b - b^| <= abs_eb on every binned value; quant_radius R
 *   gives 2R symbols (512 -> 1024); max_peaks (2048, §4) caps the peak list.
 *   lorenzo_dims (§6, the "dimension" of the quality search: the row of
 *   pixels, the panel, the stack of panels) is the order of the Lorenzo
 *   predictor on the binned array [n_panels][rows/bin_h][cols/bin_w]:
 *     1: the whole frame as one row-major run, delta = q[k] - q[k-1];
 *     2: each panel on its own, the 2-D predictor (default);
 *     3: the panels as a volume, the 3-D predictor (seven neighbours in the
 *        previous panel, row and column);
 *   neighbours outside the array count as 0.  Only 2 runs on the fused path
 *   and on the PANEL decompression path; 1 and 3 take the plain path and the
 *   multi-pass decompression path.
 *   nhr_min_peaks (§1, §4, non-hit rejection): frames whose peak list (found
 *   or given) has fewer entries are not compressed; their status is
 *   ROIBIN_REJECTED and their size 0.  0 (default) keeps every frame.  A frame
 *   with more than max_peaks peaks still reports ROIBIN_ERR_CAPACITY.
 *   roi_coder (§4, the ROI kept losslessly): 0 (default) stores the ROI
 *   windows as raw float32 in the roi section; 1 codes them with the
 *   predictive lossless coder described above (roi section after the
 *   bitstream).  Either way the windows come back bit for bit.
 *   chunk_frames (§5.3.4, events per compressor call): frames f of one
 *   roibin_compress call with the same f / chunk_frames form a chunk, and the
 *   chunk's coded frames (those still OK after the peak stage: not rejected,
 *   no error) share one Huffman code, built from the sum of their histograms.
 *   The chunk's first coded frame (its head) keeps the code lengths; each
 *   later one keeps a back reference instead and saves those 2R bytes.  A
 *   stream with a back reference decodes only in a roibin_decompress call that
 *   also holds its head at that many frames before it.  1 (default): every
 *   frame has its own code, and every stream decodes alone.  Chunks follow the
 *   frame index within the call, so a frame's bytes depend on the other
 *   frames of its chunk (and on nothing else). */
typedef struct {
  float amax_thr, atot_thr, son_min, pix_nsigma;
  int32_t rank, ring_r0, ring_dr, npix_min, npix_max;
  int32_t roi_h, roi_w, bin_h, bin_w;
  float abs_eb;
  int32_t quant_radius, max_peaks;
  int32_t lorenzo_dims;
  int32_t nhr_min_peaks;
  int32_t roi_coder;
  int32_t chunk_frames;
} roibin_params;

/* Fills *p with the defaults listed above.  Never fails for non-NULL p. */
int roibin_default_params(roibin_params* p);

/* Validates geometry + parameters without creating anything.  Limits:
 * 1 <= n_panels, rows, cols <= 65535; cols/bin_w <= 8192; 1 <= bin <= 8;
 * 1 <= roi <= 63; 1 <= rank <= 7; ring_r0, ring_dr >= 1, r0 + dr <= 16;
 * 2 <= quant_radius <= 512; 0 <= max_peaks <= 8192; pix_nsigma >= 0;
 * lorenzo_dims 1, 2 or 3; 0 <= nhr_min_peaks <= 8192; roi_coder 0 or 1;
 * 1 <= chunk_frames <= 64;
 * abs_eb > 0 with 2 abs_eb and 1/(2 abs_eb) finite; binned size below
 * 5,702,887 (so that no Huffman code exceeds 32 bits). */
int roibin_validate(const roibin_geometry* g, const roibin_params* p);

/* Worst-case compressed size of one frame (bytes, a multiple of 16); 0 when
 * the arguments are invalid.  An output stride of this size never overflows. */
uint64_t roibin_compress_bound(const roibin_geometry* g, const roibin_params* p);

/* Creates a context on CUDA device `device` for frames of geometry g and
 * parameters p, with preallocated device scratch for up to
 * max_frames_per_call frames per call (the zero-allocation principle of §4.1:
 * no call below allocates).  hbm_budget_bytes caps the scratch (0 = no cap);
 * ROIBIN_ERR_OUT_OF_BUDGET when it would be exceeded.  *out is NULL on error.
 * The context keeps its own copies of g and p. */
int roibin_ctx_create(roibin_ctx** out, const roibin_geometry* g, const roibin_params* p,
                      uint32_t max_frames_per_call, uint64_t hbm_budget_bytes, int device);

/* Frees the context and its scratch.  Synchronises the device first.  NULL ok.
 * In a checks build (below) it first runs roibin_ctx_debug_status and returns
 * ROIBIN_ERR_CHECK if that finds a failure (the context is freed all the
 * same). */
int roibin_ctx_destroy(roibin_ctx* ctx);

/* Checks build.  The library built with -DROIBIN_CHECKS stands in for a
 * memory checker, which cannot run on every GPU (the paper has no
 * counterpart):
 *  - device code checks the bounds of its stores into the caller's output
 *    buffers and into offset-computed scratch; a failing check records its id
 *    (ROIBIN_CHECK_*) and a count in the context's scratch and skips the store,
 *    instead of trapping;
 *  - the context's scratch sections are separated by 256-byte guard bands
 *    filled with 0xA5 bytes at creation.
 * roibin_ctx_debug_status synchronises the device and reports: *checks_build
 * (1 in a checks build, else 0 and nothing else is examined), *first_check
 * (id of the first failed check, 0 if none), *failed (failed checks so far)
 * and *bad_guard (byte offset in the scratch of the first overwritten guard
 * band, UINT64_MAX if none).  Returns ROIBIN_ERR_CHECK if a check failed or a
 * guard was overwritten, else ROIBIN_OK (also in other builds).  Any output
 * pointer may be NULL.  roibin_ctx_debug_poke_guard (checks builds only; else
 * ROIBIN_ERR_INVALID_ARG) overwrites one word of guard band `index` from the
 * host, so that a test can see the guard check report it. */
#define ROIBIN_CHECK_PLAN_TOTAL 1   /* a frame's planned stream exceeds its output slot  */
#define ROIBIN_CHECK_BITSTREAM 2    /* a bitstream word past the frame's word count      */
#define ROIBIN_CHECK_OUTLIERS 3     /* an outlier record past the frame's outlier count  */
#define ROIBIN_CHECK_ROI 4          /* an ROI window past the frame's stream             */
#define ROIBIN_CHECK_CODES 5        /* a code byte past the frame's code area            */
#define ROIBIN_CHECK_ROI_WORDS 6    /* coded ROI words past a window's or frame's share  */
#define ROIBIN_CHECK_STREAM_READ 7  /* a decoder read past a frame's compressed stream    */
int roibin_ctx_debug_status(roibin_ctx* ctx, uint32_t* checks_build, uint32_t* first_check, uint32_t* failed,
                            uint64_t* bad_guard);
int roibin_ctx_debug_poke_guard(roibin_ctx* ctx, uint32_t index);

/* Bytes of device scratch the context holds. */
uint64_t roibin_ctx_scratch_bytes(const roibin_ctx* ctx);

/* Selects the kernel path for later roibin_compress calls (ROIBIN_PATH_*).
 * ROIBIN_ERR_INVALID_ARG when FUSED is asked for a shape it does not cover
 * (it needs bin 2x2, cols % 4 == 0 and cols <= 868).  Both paths write
 * identical bytes. */
int roibin_ctx_set_path(roibin_ctx* ctx, int path);
/* The path AUTO resolves to for this context (PLAIN or FUSED): FUSED when the
 * shape allows it, unless the autotuner found PLAIN faster on this context. */
int roibin_ctx_resolved_path(const roibin_ctx* ctx);

/* Tuning hook of the fused path: ctas_per_sm resident CTAs per SM (1..8,
 * capped by what fits) stream rows_per_step binned rows per step (0 = the
 * most that fits the shared memory, else 2 or 3) through a ring of `stages` TMA
 * bulk-copy slots (1..8).  ROIBIN_ERR_INVALID_ARG when the shape does not fit
 * or the context has no fused path; the previous shape is then kept.
 * Results are identical for every shape; only speed changes. */
int roibin_ctx_set_fused_shape(roibin_ctx* ctx, uint32_t ctas_per_sm, uint32_t rows_per_step,
                               uint32_t stages);
/* Autotuner of the path the context resolves to, on the caller's batch
 * (arguments as roibin_compress, which it calls three times per shape), with
 * CUDA events on `stream`; keeps the fastest shape for later calls.
 *   fused: every fused shape that fits this GPU (CTAs per SM 2..4, rows per
 *          step 2..3, ring slots 2..4), then the best one in both peak
 *          variants (roibin_ctx_set_fused_dense_peaks);
 *   plain: rows per step 1, 2, 4, 8, 16 (those that fit) times bands per
 *          panel 1, 2, 4, 8, 16 (up to half the binned rows).
 * A context left on ROIBIN_PATH_AUTO that has both paths gets both tuned;
 * the two winners are then timed again three times in alternation (so that
 * clocks still ramping during the first search favour neither), and AUTO
 * takes the faster one for later calls (roibin_ctx_resolved_path reports it;
 * roibin_ctx_set_path still overrides it).
 * Synchronous.  *best_ms (optional) receives the best time per call.  Every
 * shape and path writes identical bytes, so the choice only changes speed. */
int roibin_ctx_autotune(roibin_ctx* ctx, const float* d_frames, uint32_t n_frames, uint8_t* d_out,
                        uint64_t out_stride, uint64_t* d_frame_bytes, int32_t* d_frame_status, void* stream,
                        float* best_ms);

/* Variant of the fused kernel for frames with many peak candidates (hot
 * pixels).  Its warp tests first try an exact rejection screen (interval
 * bounds on the ring statistics; a candidate that could pass still gets the
 * full evaluation), and a work item whose candidates overflow its list
 * evaluates them one per lane instead of one per warp.  It pays on such frames
 * and costs a little on frames with few candidates; both variants write the
 * same bytes.  Off by default; the autotuner tries both on its best fused
 * shape.  ROIBIN_ERR_INVALID_ARG when the context has no fused path. */
int roibin_ctx_set_fused_dense_peaks(roibin_ctx* ctx, int on);
/* 1 if the fused kernel's dense-peaks variant is selected, else 0. */
int roibin_ctx_fused_dense_peaks(const roibin_ctx* ctx);

/* Shape of the plain path: binned rows per step of its streaming kernel
 * (1..16, as fit its shared memory) and bands per panel (1 .. ceil(rows /
 * bin_h / 2)); 0 for either leaves that choice to each call (rows from the
 * panel width, bands from the batch size).  ROIBIN_ERR_INVALID_ARG for a
 * value out of range.  Results are identical for every shape. */
int roibin_ctx_set_plain_shape(roibin_ctx* ctx, uint32_t rows_per_step, uint32_t bands_per_panel);
/* The plain-path shape set on the context (0: chosen per call).  Either
 * output pointer may be NULL. */
int roibin_ctx_plain_shape(const roibin_ctx* ctx, uint32_t* rows_per_step, uint32_t* bands_per_panel);

/* Current fused shape: CTAs per SM, rows per step, ring stages, grid size,
 * shared memory bytes per CTA.  Any output pointer may be NULL. */
int roibin_ctx_fused_shape(const roibin_ctx* ctx, uint32_t* ctas_per_sm, uint32_t* rows_per_step,
                           uint32_t* stages, uint32_t* grid_ctas, uint32_t* smem_bytes);

/* Failure-detection hook of the fused path.  Its later stages hand over
 * through flags in device memory, and every wait on a flag is bounded: after
 * `polls` unsuccessful polls (about 130 ns apart) the waiting work item gives
 * up and marks its frame ROIBIN_ERR_TIMEOUT in the frame status, instead of
 * waiting forever.  polls < 0 restores the default (4,194,304 polls, about
 * half a second); polls = 0 makes every flag wait give up at once, which a
 * test uses to see the timeout reach the caller.  A waiting item only ever
 * waits for work handed out before it, so with the default limit a wait
 * always ends first.  Affects later roibin_compress calls on the fused path. */
int roibin_ctx_set_wait_limit(roibin_ctx* ctx, int64_t polls);

/* Phase trace of the fused path: for frames f < n_frames of later calls the
 * kernel writes 16 u64 words at d_trace[f * 16 + i] (globaltimer ns):
 * 0 codebook stage start, 1 peak list gathered, 2 codebook built, 3 plan
 * start, 4 plan done (head written); summed over the frame's chunk items:
 * 5 size items, 6 write items, 7 size waits, 8 write waits, 9 size chunk
 * loops, 10 write chunk loops, 11 write ROI copies (12..15 unused).  After
 * the n_frames * 16 words, every streaming item u of a traced frame f (items
 * are groups of consecutive panels, fewer than P per frame) writes 4 stamps
 * at index n_frames * 16 + (f * P + u) * 4: start, streaming done, peaks done
 * (3 unused; slots of items that do not exist stay zero).  The caller zeroes d_trace before the call and owns
 * it (device u64[n_frames * (16 + 4 P)]); n_frames = 0 switches tracing off.
 */
int roibin_ctx_set_trace(roibin_ctx* ctx, uint64_t* d_trace, uint32_t n_frames);

/* Compresses n_frames frames (1 <= n_frames <= max_frames_per_call).
 *   d_frames        float32[n_frames][P][H][W], 16-byte aligned.
 *   d_peaks,d_npeaks optional caller-supplied peak lists (§4.2 allows the
 *                   regions of interest to be given as coordinates): d_peaks is
 *                   u16[n_frames][max_peaks][3] (panel,row,col), d_npeaks
 *                   u32[n_frames].  Both NULL -> the peak finder runs.  User
 *                   peaks are stored in the order given; out-of-range
 *                   coordinates give the frame ROIBIN_ERR_INVALID_ARG and more
 *                   than max_peaks gives ROIBIN_ERR_CAPACITY.
 *   d_out           u8; frame k's stream is written at d_out + k*out_stride.
 *   out_stride      bytes per frame slot, a multiple of 16.
 *   d_frame_bytes   u64[n_frames] out: stream size of each frame (on CAPACITY
 *                   because of out_stride: the size it needs; else 0 on error).
 *   d_frame_status  i32[n_frames] out: ROIBIN_OK, ROIBIN_REJECTED (non-hit
 *                   rejection, size 0) or the frame's error.
 *   stream          cudaStream_t as void*.
 * With roi_coder = 1 the windows are coded by three more kernels after the
 * main ones (classes and counts per window, one codebook and layout per
 * frame, the bits), on both paths.
 * Returns ROIBIN_OK when the work was enqueued. */
int roibin_compress(roibin_ctx* ctx, const float* d_frames, uint32_t n_frames,
                    const uint16_t* d_peaks, const uint32_t* d_npeaks, uint8_t* d_out,
                    uint64_t out_stride, uint64_t* d_frame_bytes, int32_t* d_frame_status,
                    void* stream);

/* Decompresses n_frames streams back to float32 frames (the round trip of
 * §4.1: ROIs restored exactly over the up-sampled background).
 *   d_in             u8 buffer of in_bytes bytes holding the streams.
 *   d_frame_offsets  u64[n_frames]: byte offset of each frame's stream in d_in
 *                    (16-byte aligned).
 *   d_frames_out     float32[n_frames][P][H][W].
 *   d_frame_status   i32[n_frames] out: ROIBIN_OK or ROIBIN_ERR_CORRUPT_STREAM
 *                    (header, geometry, size, index or code mismatch; outlier
 *                    lists out of order, past the frame or off their code-0
 *                    bins; a peak outside the frame).  The panel path may also
 *                    report ROIBIN_ERR_TIMEOUT (a bulk copy of symbols that did
 *                    not land within its bounded wait).  A frame's output is
 *                    unspecified unless its status is ROIBIN_OK.
 * Paths (roibin_ctx_set_decompress_path): the panel path decodes through a
 * prefix table into symbols and rebuilds each panel in shared memory, writing
 * every pixel once; the multi-pass path runs one kernel per step.  Both write
 * the same frames and statuses.
 * Streams must come from a context of the same geometry (other parameters are
 * read from each header). */
int roibin_decompress(roibin_ctx* ctx, const uint8_t* d_in, uint64_t in_bytes,
                      const uint64_t* d_frame_offsets, uint32_t n_frames, float* d_frames_out,
                      int32_t* d_frame_status, void* stream);

/* Selects the kernel path for later roibin_decompress calls (ROIBIN_DEC_*).
 * ROIBIN_ERR_INVALID_ARG for an unknown path or PANEL on a geometry it does
 * not cover.  Both paths write identical frames and statuses. */
int roibin_ctx_set_decompress_path(roibin_ctx* ctx, int path);
/* The decompression path AUTO resolves to (PANEL or MULTIPASS). */
int roibin_ctx_resolved_decompress_path(const roibin_ctx* ctx);

/* Reserves the device staging area that roibin_compress_host needs:
 * max_frames_per_call input frames, the same number of output slots of
 * roibin_compress_bound bytes, and a packed output buffer.  This is the only
 * call besides roibin_ctx_create that allocates; calling it again is a no-op.
 * ROIBIN_ERR_OUT_OF_BUDGET when the context budget would be exceeded. */
int roibin_ctx_reserve_host_path(roibin_ctx* ctx);

/* End-to-end compression from HOST memory: copies h_frames (pinned memory
 * recommended) to the context's device staging area, compresses, packs the
 * streams back to back on the device and copies them to h_out.  Synchronous:
 * returns after h_out, h_frame_bytes and h_frame_status are written.
 *   h_out            receives the streams packed back to back (each padded to
 *                    16 bytes); frame k starts at the sum of the sizes before it.
 *   h_out_capacity   bytes available at h_out; ROIBIN_ERR_CAPACITY if the packed
 *                    total is larger (h_frame_bytes still filled).
 * The copies are pipelined with compression in slices of the batch.  Needs
 * roibin_ctx_reserve_host_path first and n_frames <= max_frames_per_call. */
int roibin_compress_host(roibin_ctx* ctx, const float* h_frames, uint32_t n_frames,
                         uint8_t* h_out, uint64_t h_out_capacity, uint64_t* h_frame_bytes,
                         int32_t* h_frame_status, void* stream);

/* ROI mask of each frame: u8 per pixel, 1 where some peak's window covers an
 * in-panel pixel (the pixels the round trip restores exactly), else 0.
 *   d_peaks u16[n_frames][max_peaks][3], d_npeaks u32[n_frames] (clamped to
 *   max_peaks), d_mask u8[n_frames][P][H][W]. */
int roibin_roi_mask(roibin_ctx* ctx, const uint16_t* d_peaks, const uint32_t* d_npeaks,
                    uint32_t n_frames, uint8_t* d_mask, void* stream);

/* Peak lists found by the last roibin_compress call on this context, copied
 * to caller buffers (d_peaks as above, d_npeaks may exceed max_peaks when the
 * frame overflowed).  Enqueued on `stream`, which must be ordered after that
 * call. */
int roibin_last_peaks(roibin_ctx* ctx, uint16_t* d_peaks, uint32_t* d_npeaks, uint32_t n_frames,
                      void* stream);

/* Per-kernel timing with CUDA events on the launch stream.  While enabled,
 * every compress call records an event pair around each of its kernels.
 * roibin_ctx_kernel_times synchronises, writes up to max_kernels entries
 * (kernel name, total ms, launches) summed over the calls since the last
 * read, and resets the sums.  Names are static strings owned by the library. */
int roibin_ctx_enable_timing(roibin_ctx* ctx, int enable);
int roibin_ctx_kernel_times(roibin_ctx* ctx, const char** names, double* total_ms,
                            uint32_t* launches, int max_kernels, int* n_kernels);

/* Number of kernels the last compress or decompress call launched (memsets
 * not counted). */
uint32_t roibin_ctx_last_launch_count(const roibin_ctx* ctx);

/* Bytes of device memory the library sets aside, per device, for
 * roibin_compress_frame_static (a fixed array in its device code). */
#define ROIBIN_STATIC_SCRATCH_BYTES (16ull << 20)

/* Compresses ONE frame with the per-stage kernels, taking its scratch from a
 * fixed area in the library's static device memory: this call allocates
 * nothing (no cudaMalloc, no allocating library routine).  It is for callers
 * that cannot allocate at the point of the call: the allocator may
 * synchronise the device and stall other streams, a process may run under a
 * hard memory budget that was spent up front, or the caller holds no
 * context object.  The paper has no counterpart of this call; it produces the
 * same bytes as roibin_compress on a one-frame batch.
 *   g, p            geometry and parameters (validated on every call).
 *   d_frame         float32[P][H][W] on the current device, 16-byte aligned.
 *   d_peaks,d_npeaks optional caller-supplied peak list as in roibin_compress
 *                   (u16[max_peaks][3] and one u32), both or neither.
 *   d_out           u8[out_capacity], 16-byte aligned; out_capacity a
 *                   multiple of 16 (roibin_compress_bound is always enough).
 *   d_frame_bytes   u64, d_frame_status i32: as roibin_compress for one frame.
 *   stream          cudaStream_t (0 = legacy default stream).
 * Limit: the frame's scratch (about 10 bytes per bin plus the peak and
 * codebook tables) must fit ROIBIN_STATIC_SCRATCH_BYTES; otherwise the call
 * returns ROIBIN_ERR_OUT_OF_BUDGET before touching the GPU.  A 32 x 185 x 388
 * frame at bin 2x2 needs about 7.3 MB.
 * Setup: the first call in each CUDA context (normally one per device, the
 * device's primary context) looks the area's address up
 * (cudaGetSymbolAddress) with that context current, which may load the
 * library's device code; make one call per device before any stream capture
 * or latency-critical section.  A context that is reset or replaced
 * (cudaDeviceReset, a caller's own driver context) gets its own lookup on its
 * first call, since the area then lives at a new address.  ROIBIN_ERR_CUDA if
 * the lookup fails.
 * Nothing has to start at zero: the call's first kernel clears the counters
 * the later ones accumulate into.
 * Overlap: every call on a device uses the same area, so two calls in flight
 * at once on one device (other streams, other threads) corrupt each other's
 * results.  The caller orders them (one stream, or events between streams). */
int roibin_compress_frame_static(const roibin_geometry* g, const roibin_params* p, const float* d_frame,
                                 const uint16_t* d_peaks, const uint32_t* d_npeaks, uint8_t* d_out,
                                 uint64_t out_capacity, uint64_t* d_frame_bytes, int32_t* d_frame_status,
                                 void* stream);

/* ---- Mixed batches under one CUDA graph ---------------------------------
 * One compression job: the arguments of roibin_compress, with its context.
 * Jobs of one graph may have different geometries and parameters (one
 * context each). */
typedef struct {
  roibin_ctx* ctx;
  const float* d_frames;
  uint32_t n_frames;
  const uint16_t* d_peaks;   /* optional, as in roibin_compress */
  const uint32_t* d_npeaks;  /* optional, as in roibin_compress */
  uint8_t* d_out;
  uint64_t out_stride;
  uint64_t* d_frame_bytes;
  int32_t* d_frame_status;
} roibin_job;

typedef struct roibin_graph roibin_graph;

#define ROIBIN_GRAPH_SERIAL 0     /* the jobs run one after another (a chain)        */
#define ROIBIN_GRAPH_CONCURRENT 1 /* each job on its own branch, free to overlap     */
#define ROIBIN_GRAPH_FUSED 2      /* the fused-path jobs in ONE persistent launch    */

/* Captures the jobs' compression launches into one CUDA graph and
 * instantiates it.  A launch of the graph runs every job once, in the order
 * given (ROIBIN_GRAPH_SERIAL) or on independent branches the GPU may run
 * concurrently (ROIBIN_GRAPH_CONCURRENT; a persistent fused kernel only ever
 * waits for work handed out at an earlier ticket of its own launch, so
 * concurrent branches cannot block one another).  Which is faster depends on
 * the mix: a persistent kernel that fills the GPU leaves little for a
 * concurrent branch to overlap with.
 * ROIBIN_GRAPH_FUSED runs the jobs whose contexts take the fused path (at most
 * 16) in one persistent kernel launch (§4.1, §5.3.5: the work of many events,
 * here of several detectors, spread over the device at once).  Their work
 * items take consecutive runs of one ticket counter, in the order given, so
 * a job's work fills the tail of the one before it; each keeps its own
 * geometry, parameters, scratch and outputs, and every frame's bytes equal
 * those of compressing its job alone.  The jobs share the CTAs per SM and ring slots
 * of the first (CTAs per SM, slots) pair all of them fit, at two binned rows
 * per step; each keeps its dense-peaks choice and wait limit.  The ROI coder
 * (if a context has it) follows the launch, then the jobs on the plain path,
 * one after another.  The graph owns a small device buffer (the launch's
 * ticket counter and sync words) that every launch zeroes first;
 * ROIBIN_ERR_INVALID_ARG if the jobs have no common shape.
 * Each context compiles into the graph with its path and fused shape at
 * capture time (tune them first, e.g. with roibin_ctx_autotune).
 * The graph keeps the job pointers: the caller refills d_frames (and the
 * peak lists) between launches, keeps every buffer alive, and does not use a
 * job's context for anything else while a launch may be in flight.
 * Contexts must be distinct and on one device; ROIBIN_ERR_INVALID_ARG
 * otherwise or for any job roibin_compress would reject; ROIBIN_ERR_CUDA if
 * capture or instantiation fails.  Allocates (the graph), so call it at
 * setup, not per batch. */
int roibin_graph_create(roibin_graph** out, const roibin_job* jobs, uint32_t n_jobs, int flags);
/* Launches the graph on `stream`; asynchronous; per-frame results as
 * roibin_compress writes them. */
int roibin_graph_launch(roibin_graph* g, void* stream);
/* Kernel launches one graph launch performs (memset nodes not counted). */
int roibin_graph_launch_count(const roibin_graph* g);
/* Frees the graph.  Synchronises the device first.  NULL ok. */
int roibin_graph_destroy(roibin_graph* g);

/* Human-readable text for a status code (static string). */
const char* roibin_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* ROIBIN_H */
