// Internal declarations shared by the libjl.so translation units (not part of
// the public ABI; see include/jl.h for that).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/jl.h"

namespace jl {

// Device-side description of one frame.  The host fills it; kernels read it
// from a table in global memory (batches) or from the launch parameters.
struct Frame {
    double cr, ci;                 // C for Julia frames (binary64)
    float cr32, ci32;              // the same C rounded once to binary32 on the host (kernels
                                   // must not convert per pixel: binary64 ops are slow here)
    double xmin, ymin, dx, dy;     // region covering in binary64 (Sec. 2)
    int32_t W, H, max_iter, mode;  // mode: JL_JULIA / JL_MANDELBROT
    int32_t count_type;            // JL_COUNT_*
    int32_t chunks_per_row;        // ceil(W / chunk_len) (rows_per_chunk == 1)
    int32_t chunk_len;             // target pixels per work chunk (<= 1024)
    int32_t rows_per_chunk;        // > 1: each chunk is this many whole rows (W < chunk_len)
    uint32_t span_magic;           // ceil(2^20 / W) when rows_per_chunk > 1, else 0
    int32_t chunk_count;           // chunks of this frame
    int32_t tiles_x;               // static kernel: 32 x 32 pixel tiles per tile row
    int32_t tile_count;            // static kernel: tiles of this frame
    int32_t pad2;
    uint64_t tiles_x_magic;        // floor(2^40 / tiles_x) + 1: exact t / tiles_x for t < 2^29
    int64_t tile_begin;            // static kernel: index of this frame's first tile in the launch
    int32_t safe;                  // 1: escape is monotone for every pixel (see escape kernels)
    int32_t precision;             // JL_FP32 / JL_FP64 (working type of xs/ys)
    int32_t pad0;
    uint64_t colour_magic;         // floor(2^40 / max_iter) + 1 (exact count*255/max_iter)
    int64_t chunk_begin;           // index of this frame's first chunk in the launch
    uint8_t *counts;               // device or NULL
    uint32_t *rgba;                // device or NULL (one RGBA8 word per pixel)
    uint32_t *hist_bins;           // device uint32[max_iter + 1] or NULL
    const void *xs;                // coordinate table: W values of the working type
    const void *ys;                // coordinate table: H values of the working type
    const float *xs32;             // binary64 frames: the tables rounded once to binary32 (certified
    const float *ys32;             // binary32 pass), written with xs/ys; NULL: no certified pass
    float cert_ec;                 // binary64 Julia frames: per-step error constant of the certified pass
    float cr_lo32, ci_lo32;        // binary64 Julia frames: C - (cr32, ci32) rounded to binary32 (C as
                                   // float pairs for the double-float pass)
    float cert2_kc;                // binary64 Julia frames: per-step constant of the double-float pass
    int32_t pad4;
    const float *xs32lo;           // binary64 frames: x - xs32 and y - ys32 rounded to binary32 (the
    const float *ys32lo;           // coordinates as float pairs for the double-float pass), with xs32
};

// Launch parameters of the escape kernels (passed by value as a grid constant).
struct EscapeArgs {
    const Frame *frames;               // device table, or NULL to use `single`
    const int32_t *chunk_frame;        // device: frame index of every chunk (batches)
    const int32_t *tile_frame;         // device: frame of every 32x32 tile (tile kernels, batches)
    const int32_t *tile_local;         // device: index of every tile within its frame (tile kernels, batches)
    int64_t total_tiles;               // static kernel: tiles in the launch
    int32_t n_frames;
    int32_t hist_smem;                 // 1: accumulate histogram bins in shared memory (one frame)
    int64_t total_chunks;
    unsigned long long *chunk_counter; // zeroed before the launch
    int32_t *status;                   // device status word (0 = ok), may be NULL
    long long cycle_budget;            // per-CTA clock64 budget; <= 0: unlimited
    int32_t claim;                     // tile kernels: 8 x 16 parts per counter claim (set by the launcher)
    int32_t out_mode;                  // batches: 1 = uint16 counts + RGBA8, 2 = RGBA8 only, 3 = uint8 counts + RGBA8 (every frame, no histograms)
    // binary64 frames: the certified binary32 pass appends the pixels it could
    // not decide to cert_list ((frame << 32) | (row << 16) | column, at most
    // cert_cap entries; the count in *cert_count), which the binary64 kernel
    // then renders, taking 32-entry pieces from *list_counter.  cert_list NULL:
    // no certified pass (the binary64 kernels cover every pixel).
    uint64_t *cert_list;
    int64_t cert_cap;
    unsigned long long *cert_count;    // zeroed before the launch
    unsigned long long *list_counter;  // zeroed before the launch
    unsigned long long *list_iters;    // zeroed before the launch, or NULL: iterations of the listed pixels
    // second certified pass (double-float) over cert_list: the pixels it cannot
    // settle go to cert_list2 (cap cert_cap, count *cert_count2), which the
    // binary64 kernel then renders instead of cert_list; it takes 32-entry
    // pieces of cert_list from *list2_counter.  NULL: no second pass.
    uint64_t *cert_list2;
    unsigned long long *cert_count2;   // zeroed before the launch
    unsigned long long *list2_counter; // zeroed before the launch
    unsigned long long *cert2_iters;   // zeroed before the launch, or NULL: iterations the second pass settles
    unsigned long long *cert_steps;    // zeroed before the launch, or NULL: tests the binary32 pass decided
    unsigned long long *cert2_steps;   // zeroed before the launch, or NULL: tests the double-float pass decided
    uint32_t palette[256];
    Frame single;
};

// Kernel variant knobs (chosen by the autotuner or the defaults).
struct Variant {
    int ppt;      // independent pixels per thread (ILP slots); 0 = static kernel (one pixel per thread)
    int unroll;   // steps per block between service points
    int threads;  // threads per CTA
    int ctas_per_sm;
};

// Thread-local last error.
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

// Launchers implemented in jl_escape.cu.
// `frames_dev` is a device table of n frames, or NULL with `single` used instead.
cudaError_t launch_coords(const Frame *frames_dev, const Frame *single, int n, cudaStream_t st);
// A binary64 launch with the certified passes records `mid` (when not NULL)
// after the binary32 pass and `mid2` after the double-float pass (external
// event nodes when captured, for timing), and `done` (a plain record, for a
// dependency of other work) after the passes.
cudaError_t launch_escape(const EscapeArgs &args, int precision, const Variant &v, int num_sms,
                          cudaStream_t st, cudaEvent_t mid = nullptr, cudaEvent_t mid2 = nullptr,
                          cudaEvent_t done = nullptr);
cudaError_t launch_hist_finalize(const Frame *frames_dev, const Frame *single, int n, cudaStream_t st);
cudaError_t launch_hist_zero(const Frame *frames_dev, int n, cudaStream_t st);
bool variant_supported(int precision, int ppt, int unroll);
int variant_list(int precision, int32_t *pairs, int cap);
int device_sm_count();
cudaError_t occupancy_per_sm(const void *kern, int threads, size_t smem, int *out);
cudaError_t launch_dbl2(const double *in, double *out, int n, cudaStream_t st);

// Validates a frame request and fills F (outputs and coordinate tables are
// left NULL).  chunk_len: target pixels per work chunk (16 .. 1024).
int make_frame(double cr, double ci, const jl_rect &rect, int W, int H, int max_iter, int precision, int mode,
               int count_type, bool has_counts, bool has_rgba, bool has_hist, Frame *F, int *prec_out,
               int chunk_len = 256);
int default_palette_bytes(uint8_t *out);
int select_precision(const jl_rect &r, int W, int H);

// Launches the escape kernel of one frame whose coordinate tables are filled:
// clears the 48-byte control block `ctl` (work counter, status, the certified
// passes' list counts and list counters) and the histogram, runs the tuned (or
// `vopt`'s) variant, finalises the histogram.  Binary64 frames with binary32
// tables (F.xs32) and a list of cert_cap >= W * H entries take the certified
// binary32 pass first, and the double-float pass when a second list of the
// same capacity is given.  Allocates nothing.
int launch_frame(Frame &F, int prec, const uint8_t *palette, void *ctl, cudaStream_t st, const Variant *vopt,
                 uint64_t *cert_list = nullptr, int64_t cert_cap = 0, uint64_t *cert_list2 = nullptr);

// Per-step error constant of the certified binary32 pass for a binary64
// Julia frame (see jl_escape.cu), rounded up to binary32.
float cert_error_constant(double cr, double ci, float cr32, float ci32);
// The low parts and the per-step constant of the double-float pass for a
// binary64 Julia frame (see jl_escape.cu).
void cert2_frame_constants(double cr, double ci, float cr32, float ci32, float *cr_lo, float *ci_lo, float *kc);

// Default variants, and the autotuned one when the tuner has run.
Variant default_variant(int precision, int max_iter);
Variant tuned_variant(int precision, int max_iter);

}  // namespace jl
