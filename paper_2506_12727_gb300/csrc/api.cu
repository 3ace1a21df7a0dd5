// C ABI of libmvgs (declared in include/mvgs.h): argument checks, buffer
// layout, and the launch sequence of each call.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mvgs.h"
#include "kernels.h"

using namespace mvgs;

namespace mvgs {
static std::atomic<long long> g_launches{0};
void note_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
}  // namespace mvgs

namespace {
thread_local std::string g_last_error;
}  // namespace

namespace mvgs {
int record_error(int st, const char* msg) {
    g_last_error = msg;
    return st;
}
}  // namespace mvgs

namespace {

mvgs_status fail(mvgs_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
mvgs_status fail(mvgs_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

mvgs_status cuda_check(const char* where) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(MVGS_ECUDA, "%s: %s", where, cudaGetErrorString(e));
    return MVGS_OK;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// ---- optional stage timing -------------------------------------------------
struct Pending {
    int stage;
    cudaEvent_t a, b;
};
struct Profiler {
    std::mutex mu;
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<Pending> pending;
    double total[MVGS_STAGE_COUNT] = {};
    long long calls[MVGS_STAGE_COUNT] = {};
    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
};
Profiler& profiler() {
    static Profiler p;
    return p;
}

}  // namespace

mvgs::StageTimer::StageTimer(int stage, cudaStream_t s) : stage_(stage), s_(s) {
    Profiler& p = profiler();
    std::lock_guard<std::mutex> lk(p.mu);
    if (!p.on) return;
    a_ = p.get();
    b_ = p.get();
    cudaEventRecord(a_, s_);
}

mvgs::StageTimer::~StageTimer() {
    if (!a_) return;
    Profiler& p = profiler();
    std::lock_guard<std::mutex> lk(p.mu);
    cudaEventRecord(b_, s_);
    p.pending.push_back({stage_, a_, b_});
}

namespace {

const char* kStageNames[MVGS_STAGE_COUNT] = {"count_visible", "scan_records", "preprocess", "depth_sort",
                                             "scan_tiles", "tile_sort", "ranges", "blend_forward",
                                             "zero_grads", "blend_backward", "preprocess_backward", "dssim", "adc"};

// Sub-allocation of one caller buffer.
struct Carver {
    size_t off = 0;
    size_t take(size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    }
};

struct Plan {
    int V = 0;
    long long n = 0;
    std::vector<DevCam> cams;
    long long tiles = 0, pixels = 0;
    mvgs_layout L{};
    // workspace offsets (forward)
    size_t w_cams = 0, w_counts = 0, w_vis = 0, w_scan = 0, w_dkeys_a = 0, w_dkeys_b = 0, w_ids_a = 0, w_ids_b = 0,
           w_order = 0, w_tiles = 0, w_desc = 0, w_tile_off = 0, w_keys_a = 0, w_keys_b = 0, w_vals_a = 0, w_vals_b = 0,
           w_radix = 0, w_tcount = 0, w_torder = 0, w_counter = 0, w_dcount = 0;
    // workspace offsets of the sampled blend (forward and backward each carve their own)
    size_t w_chunk_off = 0, w_chunk_map = 0, w_chunk_tmp = 0, w_mask = 0;
    size_t b_chunk_off = 0, b_chunk_map = 0, b_chunk_tmp = 0, b_mask = 0;
    long long chunk_cap = 0;
    // workspace offsets (backward)
    size_t b_cams = 0, b_grad = 0, b_counter = 0;
};

mvgs_status check_config(const mvgs_config* cfg) {
    if (!cfg) return fail(MVGS_EINVAL, "config is NULL");
    const int tw = cfg->tile_w, th = cfg->tile_h;
    const bool side_ok = (tw == 8 || tw == 16 || tw == 32) && (th == 8 || th == 16 || th == 32 || th == 64);
    if (!side_ok) return fail(MVGS_EINVAL, "unsupported tile %dx%d (width 8, 16 or 32; height 8 to 64)", tw, th);
    if (cfg->flags & ~(uint32_t)(MVGS_FLAG_MASKED_PARTIAL | MVGS_FLAG_DEPTH | MVGS_FLAG_CAPTURABLE |
                                 MVGS_FLAG_PIXEL_STATS))
        return fail(MVGS_EINVAL, "unknown flags 0x%x", cfg->flags);
    if (!(cfg->smem_batch == 0 || cfg->smem_batch == 64 || cfg->smem_batch == 128 || cfg->smem_batch == 192))
        return fail(MVGS_EINVAL, "smem_batch must be 0, 64, 128 or 192");
    const int ppt = cfg->pixels_per_thread;
    if (ppt != 0) {
        // a warp covers a strip of blend_strip_width(tile_w) columns and
        // (32 / that width) * ppt rows of a tile
        if (!(ppt == 1 || ppt == 2 || ppt == 4 || ppt == 8) || th % ((32 / blend_strip_width(tw)) * ppt))
            return fail(MVGS_EINVAL, "pixels_per_thread %d does not fit a %dx%d tile", ppt, tw, th);
    }
    return MVGS_OK;
}

mvgs_status make_plan(long long n, const mvgs_camera* cams, int V, const mvgs_config* cfg, const mvgs_capacity* cap,
                      Plan& P) {
    if (n < 0) return fail(MVGS_EINVAL, "n < 0");
    if (V < 1 || !cams) return fail(MVGS_EINVAL, "need at least one camera");
    if (V > 65535) return fail(MVGS_EOVERFLOW, "at most 65535 views per call");
    if (!cap || cap->records < 0 || cap->keys < 0) return fail(MVGS_EINVAL, "bad capacity");
    mvgs_status st = check_config(cfg);
    if (st != MVGS_OK) return st;
    if (cap->records >= (1LL << 31)) return fail(MVGS_EOVERFLOW, "record capacity must be < 2^31");
    if (cap->keys >= (1LL << 32)) return fail(MVGS_EOVERFLOW, "key capacity must be < 2^32");
    const int tw = cfg->tile_w, th = cfg->tile_h;
    P.V = V;
    P.n = n;
    P.cams.resize(V);
    long long tiles = 0, pixels = 0, cells = 0;
    for (int v = 0; v < V; v++) {
        const mvgs_camera& c = cams[v];
        if (c.width < 1 || c.height < 1) return fail(MVGS_EINVAL, "view %d: empty image", v);
        if (!(c.fx > 0.f) || !(c.fy > 0.f)) return fail(MVGS_EINVAL, "view %d: focal lengths must be > 0", v);
        const int txs = (c.width + tw - 1) / tw, tys = (c.height + th - 1) / th;
        // tile coordinates travel in 12-bit fields of the duplication's record descriptors
        if (txs > 4095 || tys > 4095) return fail(MVGS_EOVERFLOW, "view %d: more than 4095 tiles per axis", v);
        DevCam& d = P.cams[v];
        for (int i = 0; i < 3; i++) {
            for (int j = 0; j < 3; j++) d.R[3 * i + j] = c.viewmat[4 * i + j];
            d.t[i] = c.viewmat[4 * i + 3];
            d.campos[i] = c.campos[i];
        }
        d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy;
        d.near_z = c.near_z;
        d.limx = kGuard * 0.5f * (float)c.width / c.fx;
        d.limy = kGuard * 0.5f * (float)c.height / c.fy;
        d.W = c.width; d.H = c.height;
        d.tiles_x = txs; d.tiles_y = tys;
        d.tile_base = tiles;
        d.pix_base = pixels;
        d.diff_base = cells;
        cells += (long long)(txs + 1) * (tys + 1);
        tiles += (long long)txs * tys;
        pixels += (long long)c.width * c.height;
    }
    if (tiles >= (1LL << 32)) return fail(MVGS_EOVERFLOW, "more than 2^32 tiles over all views");
    P.tiles = tiles;
    P.pixels = pixels;

    const size_t R = (size_t)cap->records, K = (size_t)cap->keys;
    mvgs_layout& L = P.L;
    std::memset(&L, 0, sizeof(L));
    Carver s;
    L.off_counts = s.take(4 * sizeof(long long));
    L.off_rec_offsets = s.take((size_t)(n + 1) * sizeof(long long));
    L.off_rec_gauss = s.take(R * sizeof(int));
    L.off_rec_view = s.take(R * sizeof(int));
    L.off_rec_xy = s.take(R * sizeof(float2));
    L.off_rec_conic_opacity = s.take(R * sizeof(float4));
    L.off_rec_rgb = s.take(R * sizeof(float4));
    L.off_rec_clamp = s.take(R * sizeof(int));
    L.off_rec_depth = s.take(R * sizeof(float));
    L.off_rec_rect = s.take(R * sizeof(short4));
    L.off_sorted_records = s.take(K * sizeof(uint32_t));
    L.off_tile_ranges = s.take((size_t)tiles * 2 * sizeof(long long));
    L.off_tile_order = s.take((size_t)tiles * sizeof(uint32_t));
    L.off_final_T = s.take((size_t)pixels * sizeof(float));
    L.off_n_contrib = s.take((size_t)pixels * sizeof(uint32_t));
    L.off_pixel_stats = s.take((size_t)pixels * 2 * sizeof(uint32_t));
    L.off_pixel_depth = s.take((size_t)pixels * sizeof(float));
    L.state_bytes = s.off;
    L.tiles = tiles;
    L.pixels = pixels;

    Carver w;
    P.w_cams = w.take((size_t)V * sizeof(DevCam));
    P.w_counts = w.take((size_t)(n > 0 ? n : 1) * sizeof(int));
    P.w_vis = w.take((size_t)(n > 0 ? n : 1) * V);
    const size_t big = R > K ? R : K;
    P.w_scan = w.take(scan_temp_bytes(big > (size_t)n ? big : (size_t)n));
    P.w_dkeys_a = w.take(R * sizeof(uint32_t));
    P.w_dkeys_b = w.take(R * sizeof(uint32_t));
    P.w_ids_a = w.take(R * sizeof(uint32_t));
    P.w_ids_b = w.take(R * sizeof(uint32_t));
    P.w_order = w.take(R * sizeof(uint32_t));
    P.w_tiles = w.take(R * sizeof(uint32_t));
    P.w_desc = w.take(R * sizeof(unsigned long long));
    P.w_tile_off = w.take((R + 1) * sizeof(unsigned long long));
    P.w_keys_a = w.take(K * sizeof(uint32_t));
    P.w_keys_b = w.take(K * sizeof(uint32_t));
    P.w_vals_a = w.take(K * sizeof(uint32_t));
    P.w_vals_b = w.take(K * sizeof(uint32_t));
    P.w_radix = w.take(radix_temp_bytes(big) > tile_sort_temp_bytes(K) ? radix_temp_bytes(big)
                                                                          : tile_sort_temp_bytes(K));
    P.w_tcount = w.take(tile_count_temp_bytes(P.cams.data(), V, tiles));
    P.w_torder = w.take(tile_order_temp_bytes(tiles));
    P.w_counter = w.take(sizeof(int));
    P.w_dcount = w.take(4 * sizeof(unsigned long long));
    // runs of at least 32 samples: at most one partial run per tile
    P.chunk_cap = tiles + pixels / 32 + 1;
    P.w_chunk_off = w.take((size_t)(tiles + 1) * sizeof(long long));
    P.w_chunk_map = w.take((size_t)P.chunk_cap * sizeof(int));
    P.w_chunk_tmp = w.take(chunk_temp_bytes(tiles));
    P.w_mask = w.take((size_t)pixels);
    const size_t fwd_bytes = w.off;
    Carver b;
    P.b_cams = b.take((size_t)V * sizeof(DevCam));
    P.b_grad = b.take(R * kGradStride * sizeof(float) + R * 3 * sizeof(double));
    P.b_counter = b.take(sizeof(int));
    P.b_chunk_off = b.take((size_t)(tiles + 1) * sizeof(long long));
    P.b_chunk_map = b.take((size_t)P.chunk_cap * sizeof(int));
    P.b_chunk_tmp = b.take(chunk_temp_bytes(tiles));
    P.b_mask = b.take((size_t)pixels);
    L.workspace_bytes = fwd_bytes > b.off ? fwd_bytes : b.off;
    return MVGS_OK;
}

mvgs_status check_scene(const mvgs_scene* sc) {
    if (!sc) return fail(MVGS_EINVAL, "scene is NULL");
    if (sc->n < 0) return fail(MVGS_EINVAL, "scene n < 0");
    if (sc->sh_degree < 0 || sc->sh_degree > 3) return fail(MVGS_EINVAL, "sh_degree must be 0..3");
    if (sc->n > 0 && (!sc->means || !sc->log_scales || !sc->quats || !sc->opacity_logits || !sc->sh))
        return fail(MVGS_EINVAL, "scene has a NULL parameter array");
    if (sc->n >= (1LL << 31)) return fail(MVGS_EOVERFLOW, "at most 2^31 - 1 Gaussians");
    return MVGS_OK;
}

template <class T>
T* at(void* base, size_t off) {
    return reinterpret_cast<T*>(static_cast<char*>(base) + off);
}
template <class T>
const T* at(const void* base, size_t off) {
    return reinterpret_cast<const T*>(static_cast<const char*>(base) + off);
}

RecordArgs record_args(void* state, const mvgs_layout& L) {
    RecordArgs r;
    r.rec_off = at<long long>(state, L.off_rec_offsets);
    r.rec_g = at<int>(state, L.off_rec_gauss);
    r.rec_v = at<int>(state, L.off_rec_view);
    r.xy = at<float2>(state, L.off_rec_xy);
    r.conic_o = at<float4>(state, L.off_rec_conic_opacity);
    r.rgb_r = at<float4>(state, L.off_rec_rgb);
    r.clamp = at<int>(state, L.off_rec_clamp);
    r.depth = at<float>(state, L.off_rec_depth);
    r.rect = at<short4>(state, L.off_rec_rect);
    r.cap = 0;
    return r;
}

SceneArgs scene_args(const mvgs_scene* sc) {
    SceneArgs a;
    a.n = sc->n;
    a.sh_degree = sc->sh_degree;
    a.means = sc->means;
    a.log_scales = sc->log_scales;
    a.quats = sc->quats;
    a.logits = sc->opacity_logits;
    a.sh = sc->sh;
    return a;
}

// counts block of the state: records and keys in the arrays, tiles, pixels,
// records and keys the batch needed (larger only after a capturable call ran
// out of capacity)
__global__ void set_counts_kernel(long long* c, long long R, long long K, long long T, long long P) {
    c[0] = R;
    c[1] = K;
    c[2] = T;
    c[3] = P;
    c[4] = R;
    c[5] = K;
}

// capturable mode: the counts stay on the device
__global__ void clamp_records_kernel(const long long* rec_total, long long cap, unsigned long long* dcnt) {
    const long long R = *rec_total;
    dcnt[0] = (unsigned long long)(R < cap ? R : cap);
}

__global__ void clamp_keys_kernel(long long cap, unsigned long long* dcnt) {
    const unsigned long long K = dcnt[1];
    dcnt[2] = K < (unsigned long long)cap ? K : (unsigned long long)cap;
}

__global__ void set_counts_dev_kernel(long long* c, const long long* rec_total, const unsigned long long* dcnt,
                                      long long T, long long P) {
    c[0] = (long long)dcnt[0];
    c[1] = (long long)dcnt[2];
    c[2] = T;
    c[3] = P;
    c[4] = *rec_total;
    c[5] = (long long)dcnt[1];
}

int bits_for(long long tiles) {
    int b = 0;
    while (b < 63 && (1LL << b) < tiles) b++;
    return b;
}

// Points the blend at a sample set: sampled runs (Alg. 3) or, with the
// masked-partial flag, the full strips with unsampled pixels idle (Fig. 3b).
void attach_samples(BlendArgs& ba, const mvgs_samples* smp, const mvgs_config* cfg, const Plan& P, void* ws,
                    size_t off_chunk, size_t off_map, size_t off_tmp, size_t off_mask, cudaStream_t s) {
    ba.s_off = nullptr;
    ba.s_pix = nullptr;
    ba.chunk_off = nullptr;
    ba.chunk_map = nullptr;
    ba.chunk_cap = 0;
    ba.pixel_mask = nullptr;
    if (!smp) return;
    const long long* s_off = reinterpret_cast<const long long*>(smp->offsets);
    if (cfg->flags & MVGS_FLAG_MASKED_PARTIAL) {
        uint8_t* mask = at<uint8_t>(ws, off_mask);
        launch_samples_to_mask(ba.cams, ba.V, P.tiles, P.pixels, ba.tw, ba.th, s_off, smp->pixels, mask, s);
        ba.pixel_mask = mask;
        return;
    }
    long long* chunk_off = at<long long>(ws, off_chunk);
    int* chunk_map = at<int>(ws, off_map);
    launch_sample_chunks(ba.order, s_off, P.tiles, 32 * ba.ppt, chunk_off, chunk_map, P.chunk_cap,
                         at<void>(ws, off_tmp), s);
    ba.s_off = s_off;
    ba.s_pix = smp->pixels;
    ba.chunk_off = chunk_off;
    ba.chunk_map = chunk_map;
    ba.chunk_cap = P.chunk_cap;
}

mvgs_status check_samples(const mvgs_samples* smp) {
    if (smp && (!smp->offsets || !smp->pixels)) return fail(MVGS_EINVAL, "sample set with a NULL array");
    return MVGS_OK;
}

}  // namespace

extern "C" {

const char* mvgs_last_error(void) { return g_last_error.c_str(); }

mvgs_status mvgs_profile_enable(int32_t on) {
    Profiler& p = profiler();
    std::lock_guard<std::mutex> lk(p.mu);
    p.on = on != 0;
    return MVGS_OK;
}

int32_t mvgs_profile_read(float* total_ms, int64_t* launches, int32_t max_stages) {
    Profiler& p = profiler();
    std::lock_guard<std::mutex> lk(p.mu);
    for (const Pending& e : p.pending) {
        float ms = 0.f;
        cudaEventSynchronize(e.b);
        if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) {
            p.total[e.stage] += ms;
            p.calls[e.stage] += 1;
        }
        p.pool.push_back(e.a);
        p.pool.push_back(e.b);
    }
    p.pending.clear();
    const int n = max_stages < MVGS_STAGE_COUNT ? max_stages : MVGS_STAGE_COUNT;
    for (int i = 0; i < n; i++) {
        if (total_ms) total_ms[i] = (float)p.total[i];
        if (launches) launches[i] = p.calls[i];
    }
    for (int i = 0; i < MVGS_STAGE_COUNT; i++) {
        p.total[i] = 0.0;
        p.calls[i] = 0;
    }
    return MVGS_STAGE_COUNT;
}

int64_t mvgs_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

const char* mvgs_stage_name(int32_t stage) {
    return stage >= 0 && stage < MVGS_STAGE_COUNT ? kStageNames[stage] : "";
}

mvgs_status mvgs_render_layout(int64_t n, const mvgs_camera* cams, int32_t V, const mvgs_config* cfg,
                               const mvgs_capacity* cap, mvgs_layout* out) {
    if (!out) return fail(MVGS_EINVAL, "layout output is NULL");
    Plan P;
    const mvgs_status st = make_plan(n, cams, V, cfg, cap, P);
    if (st != MVGS_OK) return st;
    *out = P.L;
    return MVGS_OK;
}

static mvgs_status render_impl(const mvgs_scene* scene, const mvgs_camera* cams, int32_t V, const mvgs_config* cfg,
                               const mvgs_capacity* cap, float* images, void* state, size_t state_bytes,
                               void* workspace, size_t workspace_bytes, mvgs_capacity* needed,
                               const mvgs_samples* smp, mvgs_stream stream) {
    mvgs_status st = check_scene(scene);
    if (st != MVGS_OK) return st;
    if ((st = check_samples(smp)) != MVGS_OK) return st;
    Plan P;
    st = make_plan(scene->n, cams, V, cfg, cap, P);
    if (st != MVGS_OK) return st;
    const mvgs_layout& L = P.L;
    if (!images || !state || !workspace) return fail(MVGS_EINVAL, "NULL images, state or workspace");
    if (state_bytes < L.state_bytes || workspace_bytes < L.workspace_bytes)
        return fail(MVGS_ENOSPACE, "state %zu < %zu or workspace %zu < %zu bytes", state_bytes, L.state_bytes,
                    workspace_bytes, L.workspace_bytes);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const long long n = scene->n;
    const int tw = cfg->tile_w, th = cfg->tile_h;
    DevCam* dcams = at<DevCam>(workspace, P.w_cams);
    upload_cams(P.cams.data(), V, dcams, s);
    const SceneArgs sc = scene_args(scene);
    RecordArgs rec = record_args(state, L);
    long long* counts_dev = at<long long>(state, L.off_counts);

    // participation: which (Gaussian, view) pairs are visible, Gaussian-major
    int* counts = at<int>(workspace, P.w_counts);
    {
        StageTimer t(MVGS_STAGE_COUNT_VISIBLE, s);
        launch_count_visible(sc, dcams, V, tw, th, counts, at<uint8_t>(workspace, P.w_vis), s);
    }
    {
        StageTimer t(MVGS_STAGE_SCAN_RECORDS, s);
        scan_i32_to_i64(counts, rec.rec_off, (uint64_t)n, at<void>(workspace, P.w_scan), s);
    }
    // Without MVGS_FLAG_CAPTURABLE the record and key counts are read back to
    // size the sorts exactly; with it they stay on the device and every
    // launch is sized by the capacity (the kernels stop at the device count),
    // so the call can be captured in a CUDA graph.
    const bool capt = (cfg->flags & MVGS_FLAG_CAPTURABLE) != 0;
    unsigned long long* dcnt = at<unsigned long long>(workspace, P.w_dcount);
    long long R = 0;
    if (!capt) {
        if (cudaMemcpyAsync(&R, rec.rec_off + n, sizeof(long long), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return cuda_check("record count read-back");
        if ((st = cuda_check("participation")) != MVGS_OK) return st;
        if (needed) {
            needed->records = R;
            needed->keys = 0;
        }
        if (R > cap->records)
            return fail(MVGS_ENOSPACE, "%lld visible records exceed the capacity of %lld", R,
                        (long long)cap->records);
        rec.cap = R;
    } else {
        clamp_records_kernel<<<1, 1, 0, s>>>(rec.rec_off + n, cap->records, dcnt);
        note_launches(1);
        rec.cap = cap->records;
        if (needed) {
            needed->records = -1;  // on the device: counts block of the state
            needed->keys = -1;
        }
    }
    const Count Rc = capt ? Count((unsigned long long)cap->records, dcnt) : Count((unsigned long long)R);

    // projection, colour, radius and tile rectangle of every record, its tile
    // count and its tile descriptor (rectangle and view in 8 bytes)
    uint32_t* tiles = at<uint32_t>(workspace, P.w_tiles);
    unsigned long long* desc = at<unsigned long long>(workspace, P.w_desc);
    {
        StageTimer t(MVGS_STAGE_PREPROCESS, s);
        launch_preprocess(sc, dcams, V, tw, th, at<uint8_t>(workspace, P.w_vis), rec, tiles, desc, s);
    }

    // records by depth (the keys are the records' float32 depths, positive, so
    // their bits sort as unsigned integers; the values the record indices),
    // with each record's tile count carried into depth order by the last pass;
    // then keys per covered tile in that order
    uint32_t* order = at<uint32_t>(workspace, P.w_order);
    uint32_t* tiles_by_depth = at<uint32_t>(workspace, P.w_ids_a);
    {
        StageTimer t(MVGS_STAGE_DEPTH_SORT, s);
        radix_sort_pairs(reinterpret_cast<const uint32_t*>(rec.depth), nullptr, at<uint32_t>(workspace, P.w_dkeys_a),
                         tiles_by_depth, at<uint32_t>(workspace, P.w_dkeys_b), at<uint32_t>(workspace, P.w_ids_b),
                         order, Rc, 32, at<void>(workspace, P.w_radix), s, tiles, tiles_by_depth);
    }
    unsigned long long* tile_off = at<unsigned long long>(workspace, P.w_tile_off);
    {
        StageTimer t(MVGS_STAGE_SCAN_TILES, s);
        scan_u32_to_u64_count(tiles_by_depth, tile_off, Rc, capt ? dcnt + 1 : nullptr, at<void>(workspace, P.w_scan),
                              s);
    }
    unsigned long long K = 0;
    if (!capt) {
        if (cudaMemcpyAsync(&K, tile_off + R, sizeof(K), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return cuda_check("key count read-back");
        if ((st = cuda_check("preprocess")) != MVGS_OK) return st;
        if (needed) needed->keys = (long long)K;
        if (K >= (1ULL << 32)) return fail(MVGS_EOVERFLOW, "%llu keys do not fit 32-bit positions", K);
        if ((long long)K > cap->keys)
            return fail(MVGS_ENOSPACE, "%llu keys exceed the capacity of %lld", K, (long long)cap->keys);
    } else {
        clamp_keys_kernel<<<1, 1, 0, s>>>(cap->keys, dcnt);
        note_launches(1);
    }
    const Count Kc = capt ? Count((unsigned long long)cap->keys, dcnt + 2) : Count(K);

    uint32_t* sorted = at<uint32_t>(state, L.off_sorted_records);
    {
        StageTimer t(MVGS_STAGE_TILE_SORT, s);
        tile_sort(order, tile_off, Rc, Kc, desc, dcams, P.tiles, bits_for(P.tiles),
                  at<uint32_t>(workspace, P.w_keys_a), at<uint32_t>(workspace, P.w_vals_a),
                  at<uint32_t>(workspace, P.w_keys_b), at<uint32_t>(workspace, P.w_vals_b), sorted,
                  at<void>(workspace, P.w_radix), s);
    }
    long long* ranges = at<long long>(state, L.off_tile_ranges);
    {
        StageTimer t(MVGS_STAGE_RANGES, s);
        tile_ranges_from_rects(rec.rect, rec.rec_v, Rc, Kc, dcams, P.cams.data(), V, P.tiles, ranges,
                               at<void>(workspace, P.w_tcount), s);
        tile_order(ranges, P.tiles, at<uint32_t>(state, L.off_tile_order), at<void>(workspace, P.w_torder), s);
    }
    if (capt)
        set_counts_dev_kernel<<<1, 1, 0, s>>>(counts_dev, rec.rec_off + n, dcnt, P.tiles, P.pixels);
    else
        set_counts_kernel<<<1, 1, 0, s>>>(counts_dev, R, (long long)K, P.tiles, P.pixels);
    note_launches(1);

    BlendArgs ba;
    ba.cams = dcams;
    ba.V = V;
    ba.tw = tw;
    ba.th = th;
    ba.ppt = blend_pixels_per_thread(tw, th, cfg->pixels_per_thread);
    ba.wbatch = cfg->smem_batch ? cfg->smem_batch : 128;
    ba.sw = blend_strip_width(tw);
    ba.strip_h = (32 / ba.sw) * ba.ppt;
    ba.strips = (tw / ba.sw) * (th / ba.strip_h);
    ba.tiles = P.tiles;
    ba.ranges = ranges;
    ba.order = at<uint32_t>(state, L.off_tile_order);
    ba.sorted = sorted;
    ba.xy = rec.xy;
    ba.conic_o = rec.conic_o;
    ba.rgb_r = rec.rgb_r;
    for (int i = 0; i < 3; i++) ba.bg[i] = cfg->bg[i];
    ba.rec_depth = rec.depth;
    ba.depth_out = (cfg->flags & MVGS_FLAG_DEPTH) ? at<float>(state, L.off_pixel_depth) : nullptr;
    {
        StageTimer t(MVGS_STAGE_BLEND_FORWARD, s);
        attach_samples(ba, smp, cfg, P, workspace, P.w_chunk_off, P.w_chunk_map, P.w_chunk_tmp, P.w_mask, s);
        launch_blend_forward(ba, at<int>(workspace, P.w_counter), images, at<float>(state, L.off_final_T),
                             at<uint32_t>(state, L.off_n_contrib),
                             (cfg->flags & MVGS_FLAG_PIXEL_STATS) ? at<uint2>(state, L.off_pixel_stats) : nullptr,
                             s);
    }
    return cuda_check("render");
}

static mvgs_status backward_impl(const mvgs_scene* scene, const mvgs_camera* cams, int32_t V,
                                 const mvgs_config* cfg, const mvgs_capacity* cap, const float* dL_dimages,
                                 const void* state, size_t state_bytes, void* workspace, size_t workspace_bytes,
                                 float* g_means, float* g_log_scales, float* g_quats, float* g_opacity_logits,
                                 float* g_sh, float* g_mean2d, float* e1, const mvgs_samples* smp,
                                 mvgs_stream stream) {
    mvgs_status st = check_scene(scene);
    if (st != MVGS_OK) return st;
    if ((st = check_samples(smp)) != MVGS_OK) return st;
    Plan P;
    st = make_plan(scene->n, cams, V, cfg, cap, P);
    if (st != MVGS_OK) return st;
    const mvgs_layout& L = P.L;
    if (!dL_dimages || !state || !workspace) return fail(MVGS_EINVAL, "NULL gradient, state or workspace");
    if (scene->n > 0 && (!g_means || !g_log_scales || !g_quats || !g_opacity_logits || !g_sh))
        return fail(MVGS_EINVAL, "NULL parameter gradient");
    if (state_bytes < L.state_bytes || workspace_bytes < L.workspace_bytes)
        return fail(MVGS_ENOSPACE, "state %zu < %zu or workspace %zu < %zu bytes", state_bytes, L.state_bytes,
                    workspace_bytes, L.workspace_bytes);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DevCam* dcams = at<DevCam>(workspace, P.b_cams);
    upload_cams(P.cams.data(), V, dcams, s);
    void* st_mut = const_cast<void*>(state);  // read only below; RecordArgs carries non-const pointers
    RecordArgs rec = record_args(st_mut, L);
    rec.cap = cap->records;
    float* rec_grad = at<float>(workspace, P.b_grad);
    double* rec_conic = reinterpret_cast<double*>(rec_grad + (size_t)cap->records * kGradStride);
    {
        StageTimer t(MVGS_STAGE_ZERO_GRADS, s);
        launch_zero_f32(rec_grad, (size_t)cap->records * (kGradStride + 6), s);  // floats, then the doubles
    }

    BlendArgs ba;
    ba.cams = dcams;
    ba.V = V;
    ba.tw = cfg->tile_w;
    ba.th = cfg->tile_h;
    ba.ppt = blend_pixels_per_thread(ba.tw, ba.th, cfg->pixels_per_thread);
    ba.wbatch = cfg->smem_batch ? cfg->smem_batch : 128;
    ba.sw = blend_strip_width(ba.tw);
    ba.strip_h = (32 / ba.sw) * ba.ppt;
    ba.strips = (ba.tw / ba.sw) * (ba.th / ba.strip_h);
    ba.tiles = P.tiles;
    ba.ranges = at<long long>(state, L.off_tile_ranges);
    ba.order = at<uint32_t>(state, L.off_tile_order);
    ba.sorted = at<uint32_t>(state, L.off_sorted_records);
    ba.xy = rec.xy;
    ba.conic_o = rec.conic_o;
    ba.rgb_r = rec.rgb_r;
    for (int i = 0; i < 3; i++) ba.bg[i] = cfg->bg[i];
    ba.rec_depth = rec.depth;
    ba.depth_out = nullptr;
    {
        StageTimer t(MVGS_STAGE_BLEND_BACKWARD, s);
        attach_samples(ba, smp, cfg, P, workspace, P.b_chunk_off, P.b_chunk_map, P.b_chunk_tmp, P.b_mask, s);
        launch_blend_backward(ba, at<int>(workspace, P.b_counter), dL_dimages, at<float>(state, L.off_final_T),
                              at<uint32_t>(state, L.off_n_contrib), rec_grad, rec_conic, s);
    }
    {
        StageTimer t(MVGS_STAGE_PREPROCESS_BACKWARD, s);
        launch_preprocess_backward(scene_args(scene), dcams, V, rec, rec_grad, rec_conic, g_means, g_log_scales, g_quats,
                                   g_opacity_logits, g_sh, g_mean2d, e1, s);
    }
    return cuda_check("render backward");
}

mvgs_status mvgs_render_views(const mvgs_scene* scene, const mvgs_camera* cams, int32_t V, const mvgs_config* cfg,
                              const mvgs_capacity* cap, float* images, void* state, size_t state_bytes,
                              void* workspace, size_t workspace_bytes, mvgs_capacity* needed, mvgs_stream stream) {
    return render_impl(scene, cams, V, cfg, cap, images, state, state_bytes, workspace, workspace_bytes, needed,
                       nullptr, stream);
}

mvgs_status mvgs_render_views_backward(const mvgs_scene* scene, const mvgs_camera* cams, int32_t V,
                                       const mvgs_config* cfg, const mvgs_capacity* cap, const float* dL_dimages,
                                       const void* state, size_t state_bytes, void* workspace,
                                       size_t workspace_bytes, float* g_means, float* g_log_scales, float* g_quats,
                                       float* g_opacity_logits, float* g_sh, float* g_mean2d, float* e1,
                                       mvgs_stream stream) {
    return backward_impl(scene, cams, V, cfg, cap, dL_dimages, state, state_bytes, workspace, workspace_bytes,
                         g_means, g_log_scales, g_quats, g_opacity_logits, g_sh, g_mean2d, e1, nullptr, stream);
}

mvgs_status mvgs_render_views_sampled(const mvgs_scene* scene, const mvgs_camera* cams, int32_t V,
                                      const mvgs_config* cfg, const mvgs_capacity* cap, const mvgs_samples* samples,
                                      float* images, void* state, size_t state_bytes, void* workspace,
                                      size_t workspace_bytes, mvgs_capacity* needed, mvgs_stream stream) {
    if (!samples) return fail(MVGS_EINVAL, "samples is NULL");
    return render_impl(scene, cams, V, cfg, cap, images, state, state_bytes, workspace, workspace_bytes, needed,
                       samples, stream);
}

mvgs_status mvgs_render_views_sampled_backward(const mvgs_scene* scene, const mvgs_camera* cams, int32_t V,
                                               const mvgs_config* cfg, const mvgs_capacity* cap,
                                               const mvgs_samples* samples, const float* dL_dimages,
                                               const void* state, size_t state_bytes, void* workspace,
                                               size_t workspace_bytes, float* g_means, float* g_log_scales,
                                               float* g_quats, float* g_opacity_logits, float* g_sh,
                                               float* g_mean2d, float* e1, mvgs_stream stream) {
    if (!samples) return fail(MVGS_EINVAL, "samples is NULL");
    return backward_impl(scene, cams, V, cfg, cap, dL_dimages, state, state_bytes, workspace, workspace_bytes,
                         g_means, g_log_scales, g_quats, g_opacity_logits, g_sh, g_mean2d, e1, samples, stream);
}

// ---- participation pre-count -------------------------------------------------
static size_t count_ws_parts(long long n, size_t* a, size_t* b, size_t* c) {
    const long long nn = n > 0 ? n : 1;
    *a = ((size_t)nn * sizeof(int) + 255) / 256 * 256;
    *b = ((size_t)(nn + 1) * sizeof(long long) + 255) / 256 * 256;
    // rounded up: the camera table (16-byte aligned structs) follows it
    *c = (scan_temp_bytes((uint64_t)nn) + 255) / 256 * 256;
    return 256 + 2 * *a + 2 * *b + *c;
}

size_t mvgs_count_workspace_size(int64_t n, int32_t V) {
    size_t a, b, c;
    return count_ws_parts(n, &a, &b, &c) + ((size_t)(V > 0 ? V : 1) * sizeof(DevCam) + 255) / 256 * 256;
}

mvgs_status mvgs_count_views(const mvgs_scene* scene, const mvgs_camera* cams, int32_t V, const mvgs_config* cfg,
                             mvgs_capacity* needed, void* workspace, size_t workspace_bytes, mvgs_stream stream) {
    mvgs_status st = check_scene(scene);
    if (st != MVGS_OK) return st;
    Plan P;
    const mvgs_capacity cap{0, 0};
    if ((st = make_plan(scene->n, cams, V, cfg, &cap, P)) != MVGS_OK) return st;
    if (!needed || !workspace) return fail(MVGS_EINVAL, "NULL needed or workspace");
    if (workspace_bytes < mvgs_count_workspace_size(scene->n, V))
        return fail(MVGS_ENOSPACE, "workspace %zu < %zu bytes", workspace_bytes,
                    mvgs_count_workspace_size(scene->n, V));
    size_t a, b, c;
    count_ws_parts(scene->n, &a, &b, &c);
    char* base = reinterpret_cast<char*>(((uintptr_t)workspace + 255) / 256 * 256);
    int* recs = reinterpret_cast<int*>(base);
    uint32_t* keys = reinterpret_cast<uint32_t*>(base + a);
    long long* roff = reinterpret_cast<long long*>(base + 2 * a);
    unsigned long long* koff = reinterpret_cast<unsigned long long*>(base + 2 * a + b);
    void* scan_tmp = base + 2 * a + 2 * b;
    DevCam* dcams = reinterpret_cast<DevCam*>(base + 2 * a + 2 * b + c);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    upload_cams(P.cams.data(), V, dcams, s);
    const long long n = scene->n;
    launch_count_keys(scene_args(scene), dcams, V, cfg->tile_w, cfg->tile_h, recs, keys, s);
    scan_i32_to_i64(recs, roff, (uint64_t)n, scan_tmp, s);
    scan_u32_to_u64(keys, koff, (uint64_t)n, scan_tmp, s);
    long long R = 0;
    unsigned long long K = 0;
    if (cudaMemcpyAsync(&R, roff + n, sizeof(R), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&K, koff + n, sizeof(K), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return cuda_check("count read-back");
    needed->records = R;
    needed->keys = (long long)K;
    return cuda_check("count views");
}

static bool bad_sampling(const mvgs_sampling* sp) {
    return !sp || sp->group < 1 || sp->cell_w < 1 || sp->cell_h < 1;
}

size_t mvgs_partial_samples_workspace_size(const mvgs_camera* cams, int32_t V, const mvgs_config* cfg) {
    Plan P;
    const mvgs_capacity cap{0, 0};
    if (make_plan(0, cams, V, cfg, &cap, P) != MVGS_OK) return 0;
    return 256 + ((size_t)V * sizeof(DevCam) + 255) / 256 * 256 + sample_temp_bytes(P.tiles);
}

mvgs_status mvgs_partial_samples(const mvgs_camera* cams, int32_t V, const mvgs_config* cfg,
                                 const mvgs_sampling* sampling, int64_t* offsets, uint16_t* pixels, void* workspace,
                                 size_t workspace_bytes, mvgs_stream stream) {
    Plan P;
    const mvgs_capacity cap{0, 0};
    mvgs_status st = make_plan(0, cams, V, cfg, &cap, P);
    if (st != MVGS_OK) return st;
    if (bad_sampling(sampling)) return fail(MVGS_EINVAL, "sampling: group and cell sides must be >= 1");
    if (!offsets || !pixels || !workspace) return fail(MVGS_EINVAL, "NULL offsets, pixels or workspace");
    const size_t cam_bytes = ((size_t)V * sizeof(DevCam) + 255) / 256 * 256;
    const size_t need = 256 + cam_bytes + sample_temp_bytes(P.tiles);
    if (workspace_bytes < need) return fail(MVGS_ENOSPACE, "workspace %zu < %zu bytes", workspace_bytes, need);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // 256-byte aligned pieces of the caller's workspace
    char* base = reinterpret_cast<char*>(((uintptr_t)workspace + 255) / 256 * 256);
    DevCam* dcams = reinterpret_cast<DevCam*>(base);
    upload_cams(P.cams.data(), V, dcams, s);
    launch_partial_samples(dcams, V, P.tiles, cfg->tile_w, cfg->tile_h, sampling->group, sampling->cell_w,
                           sampling->cell_h, (unsigned long long)sampling->seed, reinterpret_cast<long long*>(offsets),
                           pixels, base + cam_bytes, s);
    return cuda_check("partial samples");
}

// ---- merged images and the 3D distance-aware D-SSIM -------------------------
static mvgs_status merge_plan(const mvgs_camera* cams, int32_t V, int32_t group, Plan& P, std::vector<long long>& mb) {
    if (group < 1 || V < 1 || !cams || V % group) return fail(MVGS_EINVAL, "V must be a positive multiple of group");
    mvgs_config cfg{};
    cfg.tile_w = cfg.tile_h = 16;
    const mvgs_capacity cap{0, 0};
    mvgs_status st = make_plan(0, cams, V, &cfg, &cap, P);
    if (st != MVGS_OK) return st;
    const int M = V / group;
    mb.assign(M + 1, 0);
    for (int m = 0; m < M; m++) {
        for (int k = 1; k < group; k++)
            if (cams[m * group + k].width != cams[m * group].width || cams[m * group + k].height != cams[m * group].height)
                return fail(MVGS_EINVAL, "views %d..%d of group %d differ in resolution", m * group, m * group + group - 1, m);
        mb[m + 1] = mb[m] + (long long)cams[m * group].width * cams[m * group].height;
    }
    return MVGS_OK;
}

size_t mvgs_merge_workspace_size(int32_t V) {
    if (V < 1) return 0;
    return 256 + ((size_t)V * sizeof(DevCam) + 255) / 256 * 256 + (size_t)(V + 1) * sizeof(long long);
}

static mvgs_status merge_upload(const Plan& P, const std::vector<long long>& mb, void* workspace,
                                size_t workspace_bytes, cudaStream_t s, DevCam** dcams, long long** dmb) {
    if (!workspace || workspace_bytes < mvgs_merge_workspace_size(P.V))
        return fail(MVGS_ENOSPACE, "workspace %zu < %zu bytes", workspace_bytes, mvgs_merge_workspace_size(P.V));
    char* base = reinterpret_cast<char*>(((uintptr_t)workspace + 255) / 256 * 256);
    *dcams = reinterpret_cast<DevCam*>(base);
    *dmb = reinterpret_cast<long long*>(base + ((size_t)P.V * sizeof(DevCam) + 255) / 256 * 256);
    upload_cams(P.cams.data(), P.V, *dcams, s);
    if (cudaMemcpyAsync(*dmb, mb.data(), mb.size() * sizeof(long long), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return cuda_check("merge upload");
    return MVGS_OK;
}

mvgs_status mvgs_merge_views(const mvgs_camera* cams, int32_t V, const mvgs_sampling* sampling, float sigma_px,
                             const float* images, const float* targets, const float* depth_acc, const float* final_T,
                             float* merged_img, float* merged_tgt, float* points, float* sigma, void* workspace,
                             size_t workspace_bytes, mvgs_stream stream) {
    if (bad_sampling(sampling)) return fail(MVGS_EINVAL, "sampling: group and cell sides must be >= 1");
    const int group = sampling->group;
    Plan P;
    std::vector<long long> mb;
    mvgs_status st = merge_plan(cams, V, group, P, mb);
    if (st != MVGS_OK) return st;
    if ((merged_img && !images) || (merged_tgt && !targets)) return fail(MVGS_EINVAL, "NULL input for a requested output");
    if ((points != nullptr) != (sigma != nullptr)) return fail(MVGS_EINVAL, "points and sigma go together");
    if (points && (!depth_acc || !final_T)) return fail(MVGS_EINVAL, "points need depth_acc and final_T");
    if (points && !(sigma_px > 0.f)) return fail(MVGS_EINVAL, "sigma_px must be > 0");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DevCam* dcams;
    long long* dmb;
    if ((st = merge_upload(P, mb, workspace, workspace_bytes, s, &dcams, &dmb)) != MVGS_OK) return st;
    launch_merge_views(dcams, group, sampling->cell_w, sampling->cell_h, (unsigned long long)sampling->seed, sigma_px,
                       mb.back(), dmb, V / group, images, targets, depth_acc, final_T, merged_img, merged_tgt, points,
                       sigma, s);
    return cuda_check("merge views");
}

mvgs_status mvgs_split_merged_grad(const mvgs_camera* cams, int32_t V, const mvgs_sampling* sampling,
                                   const float* dL_dmerged, float* dL_dimages, void* workspace,
                                   size_t workspace_bytes, mvgs_stream stream) {
    if (bad_sampling(sampling)) return fail(MVGS_EINVAL, "sampling: group and cell sides must be >= 1");
    const int group = sampling->group;
    Plan P;
    std::vector<long long> mb;
    mvgs_status st = merge_plan(cams, V, group, P, mb);
    if (st != MVGS_OK) return st;
    if (!dL_dmerged || !dL_dimages) return fail(MVGS_EINVAL, "NULL gradient");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DevCam* dcams;
    long long* dmb;
    if ((st = merge_upload(P, mb, workspace, workspace_bytes, s, &dcams, &dmb)) != MVGS_OK) return st;
    launch_split_merged(dcams, group, sampling->cell_w, sampling->cell_h, (unsigned long long)sampling->seed, mb.back(),
                        dmb, V / group, dL_dmerged, dL_dimages, s);
    return cuda_check("split merged gradient");
}

size_t mvgs_dssim3d_workspace_size(const int32_t* hw, int32_t M) {
    if (!hw || M < 1) return 0;
    return dssim3d_temp_bytes(hw, M);
}

mvgs_status mvgs_dssim3d_loss(const float* img, const float* target, const float* points, const float* sigma,
                              const int32_t* hw, int32_t M, float lambda, float* loss_per_image, float* dL_dimg,
                              void* workspace, size_t workspace_bytes, mvgs_stream stream) {
    if (!img || !target || !points || !sigma || !hw || !loss_per_image || !workspace)
        return fail(MVGS_EINVAL, "NULL argument");
    if (M < 1) return fail(MVGS_EINVAL, "need at least one image");
    for (int i = 0; i < M; i++)
        if (hw[2 * i] < 1 || hw[2 * i + 1] < 1) return fail(MVGS_EINVAL, "image %d: empty", i);
    if (!(lambda >= 0.f && lambda <= 1.f)) return fail(MVGS_EINVAL, "lambda must be in [0, 1]");
    const size_t need = dssim3d_temp_bytes(hw, M);
    if (workspace_bytes < need) return fail(MVGS_ENOSPACE, "workspace %zu < %zu bytes", workspace_bytes, need);
    {
        StageTimer t(MVGS_STAGE_DSSIM, reinterpret_cast<cudaStream_t>(stream));
        launch_dssim3d(img, target, points, sigma, hw, M, lambda, loss_per_image, dL_dimg, workspace,
                       reinterpret_cast<cudaStream_t>(stream));
    }
    return cuda_check("dssim3d");
}

// ---- densification and Adam -------------------------------------------------
size_t mvgs_densify_workspace_size(int64_t n) { return n < 0 ? 0 : densify_temp_bytes(n); }

mvgs_status mvgs_densify(const mvgs_scene* scene, const float* accum_e1, const float* accum_e2, const float* denom,
                         const float* normals, const mvgs_densify_params* params, int64_t capacity,
                         float* out_means, float* out_log_scales, float* out_quats, float* out_opacity_logits,
                         float* out_sh, int64_t* out_src, int32_t* out_kind, int64_t* n_out, void* workspace,
                         size_t workspace_bytes, mvgs_stream stream) {
    mvgs_status st = check_scene(scene);
    if (st != MVGS_OK) return st;
    if (!params || !n_out || !workspace) return fail(MVGS_EINVAL, "NULL params, n_out or workspace");
    if (scene->n > 0 && (!accum_e1 || !accum_e2 || !denom || !normals))
        return fail(MVGS_EINVAL, "NULL statistics or normals");
    if (capacity < 0) return fail(MVGS_EINVAL, "capacity < 0");
    if (capacity > 0 && (!out_means || !out_log_scales || !out_quats || !out_opacity_logits || !out_sh))
        return fail(MVGS_EINVAL, "NULL output array");
    if (workspace_bytes < densify_temp_bytes(scene->n))
        return fail(MVGS_ENOSPACE, "workspace %zu < %zu bytes", workspace_bytes, densify_temp_bytes(scene->n));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DensifyArgs a;
    a.n = scene->n;
    a.means = scene->means;
    a.log_scales = scene->log_scales;
    a.quats = scene->quats;
    a.logits = scene->opacity_logits;
    a.sh = scene->sh;
    a.nk = 3 * (scene->sh_degree + 1) * (scene->sh_degree + 1);
    a.e1 = accum_e1;
    a.e2 = accum_e2;
    a.denom = denom;
    a.normals = normals;
    a.split_threshold = params->split_threshold;
    a.clone_threshold = params->clone_threshold;
    a.prune_logit = params->prune_logit;
    a.log_dense_extent = params->log_dense_extent;
    const long long* total_dev = launch_densify_plan(a, workspace, s);
    long long total = 0;
    if (cudaMemcpyAsync(&total, total_dev, sizeof(long long), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return cuda_check("densify count read-back");
    *n_out = total;
    if (total > capacity)
        return fail(MVGS_ENOSPACE, "%lld output Gaussians exceed the capacity of %lld", total, (long long)capacity);
    DensifyOut o{out_means, out_log_scales, out_quats, out_opacity_logits, out_sh,
                 reinterpret_cast<long long*>(out_src), out_kind};
    launch_densify_write(a, o, workspace, s);
    return cuda_check("densify");
}

mvgs_status mvgs_densify_carry(int64_t n_out, const int64_t* src, const int32_t* kind, int32_t width,
                               const float* in, float* out, mvgs_stream stream) {
    if (n_out < 0 || width < 1) return fail(MVGS_EINVAL, "n_out < 0 or width < 1");
    if (n_out > 0 && (!src || !kind || !in || !out)) return fail(MVGS_EINVAL, "NULL argument");
    launch_carry(n_out, reinterpret_cast<const long long*>(src), kind, width, in, out,
                 reinterpret_cast<cudaStream_t>(stream));
    return cuda_check("densify carry");
}

mvgs_status mvgs_adam_step(int64_t count, float* param, const float* grad, float* m, float* v, float lr, float beta1,
                           float beta2, float eps, int32_t step, mvgs_stream stream) {
    if (count < 0 || step < 1) return fail(MVGS_EINVAL, "count < 0 or step < 1");
    if (count > 0 && (!param || !grad || !m || !v)) return fail(MVGS_EINVAL, "NULL argument");
    if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f)) return fail(MVGS_EINVAL, "betas in [0, 1)");
    launch_adam(count, param, grad, m, v, lr, beta1, beta2, eps, step, reinterpret_cast<cudaStream_t>(stream));
    return cuda_check("adam");
}

size_t mvgs_dssim_workspace_size(const int32_t* hw, int32_t V) {
    if (!hw || V < 1) return 0;
    return dssim_temp_bytes(hw, V);
}

mvgs_status mvgs_dssim_loss(const float* img, const float* target, const int32_t* hw, int32_t V, float lambda,
                            float* loss_per_view, float* dL_dimg, void* workspace, size_t workspace_bytes,
                            mvgs_stream stream) {
    if (!img || !target || !hw || !loss_per_view || !workspace) return fail(MVGS_EINVAL, "NULL argument");
    if (V < 1) return fail(MVGS_EINVAL, "need at least one view");
    for (int v = 0; v < V; v++)
        if (hw[2 * v] < 1 || hw[2 * v + 1] < 1) return fail(MVGS_EINVAL, "view %d: empty image", v);
    if (!(lambda >= 0.f && lambda <= 1.f)) return fail(MVGS_EINVAL, "lambda must be in [0, 1]");
    const size_t need = dssim_temp_bytes(hw, V);
    if (workspace_bytes < need) return fail(MVGS_ENOSPACE, "workspace %zu < %zu bytes", workspace_bytes, need);
    {
        StageTimer t(MVGS_STAGE_DSSIM, reinterpret_cast<cudaStream_t>(stream));
        launch_dssim(img, target, hw, V, lambda, loss_per_view, dL_dimg, workspace,
                     reinterpret_cast<cudaStream_t>(stream));
    }
    return cuda_check("dssim");
}

mvgs_status mvgs_adc_accumulate(const void* state, int64_t n, const float* g_mean2d, const float* e1,
                                float* accum_e1, float* accum_e2, float* denom, mvgs_stream stream) {
    if (!state || !g_mean2d || !e1 || !accum_e1 || !accum_e2 || !denom) return fail(MVGS_EINVAL, "NULL argument");
    if (n < 0) return fail(MVGS_EINVAL, "n < 0");
    // the record offsets sit right after the 256-byte count block of the state
    const long long* rec_off = at<long long>(state, 256);
    {
        StageTimer t(MVGS_STAGE_ADC, reinterpret_cast<cudaStream_t>(stream));
        launch_adc_accumulate(rec_off, at<long long>(state, 0), n, g_mean2d, e1, accum_e1, accum_e2, denom,
                              reinterpret_cast<cudaStream_t>(stream));
    }
    return cuda_check("adc");
}

}  // extern "C"
