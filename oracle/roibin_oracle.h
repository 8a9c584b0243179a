/*
 * ROIBIN-SZ oracle: plain, slow, single-threaded CPU definition of the
 * compression hot path (ROI extraction + binning + SZ-style background coding).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link or
 * call this code: only tests/, the smoke check and the benchmark's CPU-baseline
 * leg use it.  It shares no source with the CUDA library.
 *
 * All entry points use plain C types so they can be called through ctypes.
 * Arrays are row-major; a frame is float32[n_panels][rows][cols].
 */
#ifndef ROIBIN_ORACLE_H
#define ROIBIN_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORC_OK = 0,
  ORC_ERR_INVALID_ARG = -1,
  ORC_ERR_CAPACITY = -2,
  ORC_ERR_CORRUPT_STREAM = -3,
  ORC_ERR_CODE_LENGTH = -7, /* a Huffman code longer than 32 bits (cannot occur below 5,702,887 symbols) */
  ORC_REJECTED = 1          /* non-hit rejection: fewer than nhr_min_peaks peaks, nothing written */
};

/* Format version 1 constants (the paper defines no container; this one is ours). */
#define ORC_MAGIC 0x5A534252u        /* bytes "RBSZ" */
#define ORC_VERSION 1u
#define ORC_HEADER_BYTES 96u
#define ORC_CHUNK_SYMBOLS 4096u
#define ORC_CANONICAL_NAN 0x7FC00000u /* bits stored for a NaN bin */
#define ORC_PQ_LIMIT 268435456.0f    /* 2^28: |q| must stay below it */
#define ORC_MAX_SYMBOLS_PER_FRAME 5702886u /* F(34) - 1: keeps every code length <= 32 */

typedef struct {
  uint32_t n_panels, rows, cols;
} orc_geometry;

typedef struct {
  float amax_thr;   /* local maximum must be >= this (300 ADU)          */
  float atot_thr;   /* total peak intensity must be > this (600 ADU)     */
  float son_min;    /* signal-to-noise ratio must be > this (10)         */
  float pix_nsigma; /* peak pixel: I - bkg > pix_nsigma * sigma (>= 0)   */
  int32_t rank;     /* local-maximum window is (2 rank + 1)^2 (3 -> 7x7) */
  int32_t ring_r0;  /* background ring: r0^2 <= di^2+dj^2 < (r0+dr)^2   */
  int32_t ring_dr;
  int32_t npix_min; /* 2 <= npix <= 30 */
  int32_t npix_max;
  int32_t roi_h;    /* ROI window, 17 x 17 */
  int32_t roi_w;
  int32_t bin_h;    /* binning factor, 2 x 2 */
  int32_t bin_w;
  float abs_eb;     /* absolute error bound on binned values */
  int32_t quant_radius; /* R: codes 1..2R-1 hold |delta| < R, code 0 = outlier */
  int32_t max_peaks;    /* 2048 */
  int32_t lorenzo_dims; /* 1: the frame as one row-major run; 2: each panel (default); 3: the panel stack */
  int32_t nhr_min_peaks; /* non-hit rejection: frames with fewer peaks are dropped (0 = off) */
  int32_t roi_coder;     /* 0: raw float32 ROI windows; 1: the predictive lossless ROI coder */
  int32_t chunk_frames;  /* frames per chunk sharing one codebook (1..64; 1 = a codebook per frame) */
} orc_params;

/* ---- step-level entry points (each is one row of the method) ---- */
int orc_is_peak_candidate(const float* panel, uint32_t rows, uint32_t cols, uint32_t r,
                          uint32_t c, int32_t rank, float amax_thr);
int orc_evaluate_peak(const float* panel, uint32_t rows, uint32_t cols, uint32_t r, uint32_t c,
                      const orc_params* p);
int orc_find_peaks(const float* frame, const orc_geometry* g, const orc_params* p,
                   uint16_t* peaks_out, uint32_t peaks_capacity, uint32_t* n_found);
void orc_roi_extract(const float* frame, const orc_geometry* g, const orc_params* p,
                     const uint16_t* peaks, uint32_t n_peaks, float* roi_out);
void orc_roi_mask(const orc_geometry* g, const orc_params* p, const uint16_t* peaks,
                  uint32_t n_peaks, uint8_t* mask_out);
void orc_bin(const float* frame, const orc_geometry* g, int32_t bin_h, int32_t bin_w,
             float* binned_out);
void orc_prequantize(const float* binned, uint64_t m, float abs_eb, int32_t* q_out,
                     uint8_t* outlier_out);
void orc_lorenzo(const int32_t* q, uint32_t n_panels, uint32_t hb, uint32_t wb,
                 int32_t* delta_out);
/* a6 in dimension 1, 2 or 3 (§6: along the row of pixels, the panel, the
 * stack of panels); 2 is orc_lorenzo. */
void orc_lorenzo_nd(const int32_t* q, uint32_t n_panels, uint32_t hb, uint32_t wb, int32_t dims,
                    int32_t* delta_out);
void orc_quant_codes(const int32_t* delta, uint64_t m, int32_t radius, uint16_t* codes_out);
void orc_histogram(const uint16_t* codes, uint64_t m, uint32_t n_symbols, uint64_t* hist_out);
int orc_huffman_lengths(const uint64_t* hist, uint32_t n_symbols, uint8_t* len_out);
void orc_canonical_codes(const uint8_t* len, uint32_t n_symbols, uint32_t* code_out);
uint32_t orc_pack_chunks(const uint16_t* codes, uint64_t m, const uint8_t* len,
                         const uint32_t* codewords, uint32_t* chunk_index_out,
                         uint32_t* words_out);

/* ---- lossless ROI coding (fpzip-style; see the source) ---- */
uint32_t orc_roi_order_bits(float x);
void orc_roi_residuals(const float* win, int32_t h, int32_t w, uint32_t* z_out);
uint32_t orc_roi_class(uint32_t z);
uint64_t orc_roi_encode(const float* windows, uint32_t n_windows, int32_t h, int32_t w, uint8_t* out,
                        uint32_t* coding, uint32_t* n_words);
int orc_roi_decode(const uint8_t* sec, uint64_t bytes, uint32_t coding, uint32_t n_words, uint32_t n_windows,
                   int32_t h, int32_t w, float* windows_out);

/* ---- whole-frame entry points ---- */
uint64_t orc_compress_bound(const orc_geometry* g, const orc_params* p);
int orc_compress_frame(const float* frame, const orc_geometry* g, const orc_params* p,
                       const uint16_t* user_peaks, int64_t n_user_peaks, uint8_t* out,
                       uint64_t capacity, uint64_t* out_bytes);
int orc_decompress_frame(const uint8_t* in, uint64_t in_bytes, const orc_geometry* g,
                         float* frame_out);
/* A call of frames sharing chunk codebooks (see the source). */
int orc_compress_frames(const float* frames, uint32_t n_frames, const orc_geometry* g, const orc_params* p,
                        const uint16_t* user_peaks, const int64_t* n_user_peaks, uint8_t* outs, uint64_t stride,
                        uint64_t* out_bytes, int32_t* status);
int orc_decompress_frames(const uint8_t* in, uint64_t in_bytes, const uint64_t* offsets, uint32_t n_frames,
                          const orc_geometry* g, float* frames_out, int32_t* status);

#ifdef __cplusplus
}
#endif
#endif
