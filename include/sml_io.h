/*
 * sml_io.h -- stack input pipeline of the GB300 localization library.
 *
 * The paper's inference frame (Sec. 2.2) overlaps loading images from disk with inference
 * and keeps images preloaded in host memory ahead of the network.  Here that is:
 *   * a reader: one host thread per open stack reads raw frames with pread into a ring of
 *     pinned host buffers, ahead of their use;
 *   * sml_localize_file: batches flow reader -> H2D copy (copy stream) -> localization
 *     (the context's stream) -> D2H of the batch's records (copy stream).  Batch k's
 *     compute overlaps batch k+1's copy in and batch k-1's records coming back, while the
 *     reader thread keeps reading ahead.
 *
 * Stack file format: T frames of H x W uint16 (little-endian, row-major, frame after frame),
 * starting `offset` bytes into the file; nothing else is interpreted.
 */
#ifndef SML_IO_H
#define SML_IO_H

#include <stddef.h>
#include <stdint.h>

#include "sml.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sml_reader sml_reader;

/* Reading statistics: bytes read from the file, seconds the reader thread spent in reads,
 * and (sml_localize_file) wall seconds of the whole call and frames localized. */
typedef struct {
  double bytes_read;
  double read_seconds;
  double wall_seconds;
  long long frames;
} sml_io_stats;

/* Open the stack and start reading ahead: n_buffers (2..16) buffers of `batch` (>= 1) frames
 * each.  Buffers are pinned (page-locked) when a CUDA device is present, ordinary host
 * memory otherwise.  Errors: SML_ERR_BAD_ARG (bad sizes, unreadable file, or a file shorter
 * than offset + T*H*W*2 bytes), SML_ERR_OOM.  The caller owns *out (sml_reader_close). */
int sml_reader_open(const char* path, long long offset, int T, int H, int W, int batch, int n_buffers,
                    sml_reader** out);

/* The next batch in file order: *frames points to n_frames frames (the last batch may be
 * short; *n_frames == 0 after the last one), *first_frame is the index of its first frame
 * in the stack.  Waits up to timeout_ms for the reader.  The buffer stays valid until
 * sml_reader_release.  Errors: SML_ERR_BAD_ARG (a read failed), SML_ERR_CUDA (timeout:
 * nothing arrived in time). */
int sml_reader_next(sml_reader* r, const uint16_t** frames, int* n_frames, long long* first_frame, int timeout_ms);

/* Give a batch's buffer back to the reader, in the order the batches were handed out. */
int sml_reader_release(sml_reader* r, const uint16_t* frames);

/* Statistics so far (wall_seconds and frames are 0 for a bare reader). */
int sml_reader_stats(const sml_reader* r, sml_io_stats* out);

/* Stop the reader thread and free its buffers (waits for a read in progress). */
void sml_reader_close(sml_reader* r);

/* Localize a whole stack file in batches of `batch` frames (see the pipeline above).
 * Records go to `out` (host memory, `capacity` records) in (frame, row, column) order with
 * frame = index in the stack, exactly as sml_localize on all T frames returns them.
 * Three-frame nets (in_ch = 3) read the frame before and after each batch from the
 * neighbouring batches (copied on the device), so their records too equal sml_localize on
 * all T frames; each batch is then localized once its successor has been read.
 * CAPACITY sets *n_out to the needed count (records beyond capacity are not written).
 * stats may be NULL. */
int sml_localize_file(sml_ctx* ctx, const char* path, long long offset, int T, int H, int W, const sml_camera* cam,
                      const sml_thresholds* thr, int batch, sml_record* out, size_t capacity, size_t* n_out,
                      sml_io_stats* stats);

#ifdef __cplusplus
}
#endif

#endif
