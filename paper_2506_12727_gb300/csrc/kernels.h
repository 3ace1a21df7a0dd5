// Host-side launchers of the sm_103a kernels (internal to libmvgs).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "common.cuh"

namespace mvgs {

// Process-wide count of kernels launched by the library (api.cu).
void note_launches(int k);

// Sets the calling thread's last error message (api.cu) and returns `st`.
int record_error(int st, const char* msg);

// Records events around one stage on `s` while stage timing is enabled
// (mvgs_profile_enable); the totals are read by mvgs_profile_read (api.cu).
class StageTimer {
  public:
    StageTimer(int stage, cudaStream_t s);
    ~StageTimer();
    StageTimer(const StageTimer&) = delete;
    StageTimer& operator=(const StageTimer&) = delete;

  private:
    int stage_;
    cudaStream_t s_;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
};

// ---- preprocess.cu -------------------------------------------------------
void upload_cams(const DevCam* host, int V, DevCam* dst, cudaStream_t s);

struct SceneArgs {
    long long n;
    int sh_degree;
    const float* means;
    const float* log_scales;
    const float* quats;
    const float* logits;
    const float* sh;
};

// Records of the visible (Gaussian, view) pairs, Gaussian-major.
struct RecordArgs {
    long long* rec_off;  // [n + 1]
    int* rec_g;
    int* rec_v;
    float2* xy;
    float4* conic_o;
    float4* rgb_r;       // rgb, radius
    int* clamp;
    float* depth;
    short4* rect;
    long long cap;       // records the arrays hold: no record index reaches it
};

// Per Gaussian: visible views and covered tiles (sizing only; no records).
void launch_count_keys(const SceneArgs& sc, const DevCam* cams, int V, int tw, int th, int* recs, uint32_t* keys,
                       cudaStream_t s);
// vis: [n * V] bytes, 1 where (g, v) is visible; counts: visible views per Gaussian.
void launch_count_visible(const SceneArgs& sc, const DevCam* cams, int V, int tw, int th, int* counts, uint8_t* vis,
                          cudaStream_t s);
// Writes all records of the visible pairs, the number of tiles each record
// touches and its tile descriptor (pack_tile_desc).
void launch_preprocess(const SceneArgs& sc, const DevCam* cams, int V, int tw, int th, const uint8_t* vis,
                       const RecordArgs& rec, uint32_t* tiles_touched, unsigned long long* tile_desc,
                       cudaStream_t s);
void launch_zero_f32(float* p, size_t count, cudaStream_t s);
// rec_grad: [records, kGradStride] float (mean2d x, y, opacity, rgb, e1 at
// 0, 1, 2, 3..5, 6); rec_conic: [records, 3] double (conic A, B, C).
void launch_preprocess_backward(const SceneArgs& sc, const DevCam* cams, int V, const RecordArgs& rec,
                                const float* rec_grad, const double* rec_conic, float* g_means,
                                float* g_log_scales, float* g_quats, float* g_logits, float* g_sh,
                                float* out_mean2d, float* out_e1, cudaStream_t s);
// records at or past *rec_count are ignored
void launch_adc_accumulate(const long long* rec_off, const long long* rec_count, long long n, const float* g_mean2d,
                           const float* e1, float* accum_e1, float* accum_e2, float* denom, cudaStream_t s);

// ---- sort.cu ---------------------------------------------------------------
size_t scan_temp_bytes(uint64_t n);
// out[0..n] = exclusive prefix sums of in[0..n), out[n] = total.
void scan_i32_to_i64(const int* in, long long* out, uint64_t n, void* tmp, cudaStream_t s);
// scans in[i] & mask
void scan_masked_i32_to_i64(const int* in, int mask, long long* out, uint64_t n, void* tmp, cudaStream_t s);
void scan_u32_to_u64(const uint32_t* in, unsigned long long* out, uint64_t n, void* tmp, cudaStream_t s);
// gathered variant: scans in[idx[i]]
// (also the total into *total when given; n may be a device count)
void scan_u32_to_u64_count(const uint32_t* in, unsigned long long* out, Count n, unsigned long long* total,
                           void* tmp, cudaStream_t s);
void scan_gather_u32_to_u64(const uint32_t* in, const uint32_t* idx, unsigned long long* out, Count n,
                            unsigned long long* total, void* tmp, cudaStream_t s);

size_t radix_temp_bytes(uint64_t n);
size_t tile_sort_temp_bytes(uint64_t K);
// Stable LSD sort of (key, value) pairs on key bits [0, bits).  Input in
// (keys0, vals0), read only; vals0 == nullptr sorts the identity permutation
// (values generated, not read).  keys_a/b and vals_a/b are scratch; the sorted
// values end in vals_out.  With gather_src, the last pass also writes
// gather_out[i] = gather_src[vals_out[i]] (gather_out may be vals_a).
void radix_sort_pairs(const uint32_t* keys0, const uint32_t* vals0, uint32_t* keys_a, uint32_t* vals_a,
                      uint32_t* keys_b, uint32_t* vals_b, uint32_t* vals_out, Count n, int bits, void* tmp,
                      cudaStream_t s, const uint32_t* gather_src = nullptr, uint32_t* gather_out = nullptr);

// Stable sort, by global (view, tile) id, of one entry per (record, covered
// tile) taken in the order of `order` (records sorted by depth); tile_off is
// the exclusive scan of the records' tile counts in that order; desc holds the
// records' tile descriptors (pack_tile_desc, record order).  The entries
// are generated by the first pass's histogram kernel (the duplication) and
// written to keys_a / vals_a (16-bit tile ids when the sort runs packed).
// Sorted record ids end in vals_out; keys_a/b and vals_a/b are scratch of K
// entries.
void tile_sort(const uint32_t* order, const unsigned long long* tile_off, Count R, Count K,
               const unsigned long long* desc, const DevCam* cams, long long tiles, int bits, uint32_t* keys_a,
               uint32_t* vals_a, uint32_t* keys_b, uint32_t* vals_b, uint32_t* vals_out, void* tmp, cudaStream_t s);

// Tiles ordered by decreasing list length (the blend's processing order).
size_t tile_order_temp_bytes(long long tiles);
void tile_order(const long long* ranges, long long tiles, uint32_t* order, void* tmp, cudaStream_t s);

// Per-tile [start, end) of the sorted list, from the records' rectangles.
size_t tile_count_temp_bytes(const DevCam* host_cams, int V, long long tiles);
void tile_ranges_from_rects(const short4* rect, const int* rec_v, Count R, Count K, const DevCam* cams,
                            const DevCam* host_cams, int V, long long tiles, long long* ranges, void* tmp,
                            cudaStream_t s);

// ---- blend.cu --------------------------------------------------------------
struct BlendArgs {
    const DevCam* cams;
    int V;
    int tw, th;
    int ppt;                 // pixels per lane (resolved, 1..8)
    int wbatch;              // Gaussians per warp batch in shared memory (64, 128 or 192; 128 unless ppt 4)
    int sw;                  // columns of a warp's strip (blend_strip_width)
    int strip_h;             // rows of a warp's strip: (32 / sw) * ppt
    int strips;              // strips per tile: (tw / sw) * (th / strip_h)
    long long tiles;
    const long long* ranges;
    const uint32_t* order;   // tiles in processing order (longest lists first)
    const uint32_t* sorted;
    const float2* xy;
    const float4* conic_o;
    const float4* rgb_r;
    float bg[3];
    // sampled mode (thread-efficient partial rendering, Alg. 3); s_off null
    // for the full render
    const long long* s_off;      // [tiles + 1] samples of global tile t: [s_off[t], s_off[t + 1])
    const uint16_t* s_pix;       // pixel index inside the tile, ly * tw + lx
    const long long* chunk_off;  // [tiles + 1] first run of order position i; [tiles] = total runs
    const int* chunk_map;        // [total runs] order position of each run
    long long chunk_cap;         // entries of chunk_map (runs beyond it are not rendered)
    // naive partial rendering (Fig. 3b): full strips, pixels with a zero byte idle
    const uint8_t* pixel_mask;   // [pixels] or null
    // optional expected depth sum_i alpha_i T_i z_i per pixel (forward only)
    const float* rec_depth;      // [records] camera depth
    float* depth_out;            // [pixels] or null
};
// Columns of a blend strip for a tile width (8: strips tile a 16- or 32-wide
// tile two or four across).
int blend_strip_width(int tw);
// Pixels per lane for a tile size (req > 0: the caller's choice, checked).
int blend_pixels_per_thread(int tw, int th, int req);
// Persistent launches; `counter` is one device int of scratch (reset here).
void launch_blend_forward(const BlendArgs& a, int* counter, float* img, float* final_T, uint32_t* n_contrib,
                          uint2* pixel_stats, cudaStream_t s);
void launch_blend_backward(const BlendArgs& a, int* counter, const float* dimg, const float* final_T,
                           const uint32_t* n_contrib, float* rec_grad, double* rec_conic, cudaStream_t s);

// ---- partial.cu ------------------------------------------------------------
// Pixel selection of the partial render: view v takes pixel (x, y) when the
// SplitMix64 hash of (seed, x, y) falls in slot v mod `group` of `group`.
size_t sample_temp_bytes(long long tiles);
void launch_partial_samples(const DevCam* cams, int V, long long tiles, int tw, int th, int group, int cw, int ch,
                            unsigned long long seed, long long* s_off, uint16_t* s_pix, void* tmp, cudaStream_t s);
// Runs of 32 * ppt samples per tile in the blend's tile order.
size_t chunk_temp_bytes(long long tiles);
void launch_sample_chunks(const uint32_t* order, const long long* s_off, long long tiles, int run,
                          long long* chunk_off, int* chunk_map, long long map_cap, void* tmp, cudaStream_t s);
// Byte mask [pixels] of the sampled pixels (zeroed first).
void launch_samples_to_mask(const DevCam* cams, int V, long long tiles, long long pixels, int tw, int th,
                            const long long* s_off, const uint16_t* s_pix, uint8_t* mask, cudaStream_t s);

// ---- dssim3d.cu -------------------------------------------------------------
size_t dssim3d_temp_bytes(const int* hw, int M);
void launch_dssim3d(const float* img, const float* target, const float* points, const float* sigma, const int* hw,
                    int M, float lambda, float* loss, float* dimg, void* tmp, cudaStream_t s);
// mbase: device [M + 1] first pixel of each merged image; cams: device, all V views
void launch_merge_views(const DevCam* cams, int group, int cw, int ch, unsigned long long seed, float sigma_px,
                        long long merged_pix,
                        const long long* mbase, int M, const float* images, const float* targets,
                        const float* depth_acc, const float* final_T, float* out_img, float* out_tgt, float* out_pts,
                        float* out_sig, cudaStream_t s);
void launch_split_merged(const DevCam* cams, int group, int cw, int ch, unsigned long long seed, long long merged_pix,
                         const long long* mbase, int M, const float* dmerged, float* dimg, cudaStream_t s);

// ---- train.cu ---------------------------------------------------------------
struct DensifyArgs {
    long long n;
    const float* means;
    const float* log_scales;
    const float* quats;
    const float* logits;
    const float* sh;
    int nk;                   // floats of SH per Gaussian
    const float* e1;
    const float* e2;
    const float* denom;
    const float* normals;     // [n, 2, 3] standard normal samples for split children
    double split_threshold, clone_threshold, prune_logit, log_dense_extent;
};
struct DensifyOut {
    float* means;
    float* log_scales;
    float* quats;
    float* logits;
    float* sh;
    long long* src;           // or null
    int* kind;                // or null
};
constexpr float kLogSplitDiv = 0.47000362924573558f;  // ln 1.6
size_t densify_temp_bytes(long long n);
const long long* launch_densify_plan(const DensifyArgs& a, void* tmp, cudaStream_t s);
void launch_densify_write(const DensifyArgs& a, const DensifyOut& o, void* tmp, cudaStream_t s);
void launch_carry(long long n_out, const long long* src, const int* kind, int width, const float* in, float* out,
                  cudaStream_t s);
void launch_adam(long long count, float* p, const float* g, float* m, float* v, float lr, float b1, float b2,
                 float eps, int step, cudaStream_t s);

// ---- dssim.cu --------------------------------------------------------------
size_t dssim_temp_bytes(const int* hw, int V);
void launch_dssim(const float* img, const float* target, const int* hw, int V, float lambda, float* loss_per_view,
                  float* dimg, void* tmp, cudaStream_t s);

}  // namespace mvgs
