// Tile-based alpha blending (Eq. 1) and its backward.
//
// In the supplement's rasterizer every (tile, view) pair gets its own thread
// block, and Alg. 2 has a tile's threads fetch its depth-sorted Gaussians
// into shared memory batch by batch and blend them.  Here the unit of work is a strip of
// a (tile, view) pair -- 8 columns (blend_strip_width) by (32 / 8) * PPT rows,
// strips side by side across wider tiles -- owned by one warp: each lane owns
// PPT pixels of one column, the warp stages batches
// of the tile's list in its own slice of shared memory, and leaves the strip
// as soon as all its pixels have stopped.  Warps of a persistent launch take
// strips from a queue that lists the tiles with the longest lists first, so
// the whole batch of views (any mix of resolutions) is one launch without a
// tail of heavy tiles, and no block-wide barrier couples unrelated strips.
//
// Each staged batch keeps only the Gaussians whose support and alpha >= 1/255
// region reach a pixel centre of the strip (an exact test of the quadratic
// form over the strip's rectangle), compacted with a ballot; the list
// positions are kept for the per-pixel bookkeeping.
//
// Forward per pixel (front to back): alpha = min(0.99, o G), skip alpha <
// 1/255, stop before T (1 - alpha) < 1e-4, C += c alpha T, T *= 1 - alpha;
// output C + T bg.  G is evaluated in base 2 from the staged coefficients
// and the column terms of the lane's pixel column (pair_eval).
//
// Backward per pixel (back to front from the last contributor), with T
// recovered by an (approximate) reciprocal:  dC/dc_i = alpha_i T_i,
// dC/dalpha_i = c_i T_i - S_i / (1 - alpha_i), S_i the colour blended behind
// i plus T_final bg.  The gradients of one Gaussian are summed over the
// lane's pixels (in a strip, as sums of dL/dpower times 1, dy, dy^2 for the
// lane's one column), then over the
// warp by a reduce-scatter (12 shuffles for 10 values), and one lane per
// value adds it with one atomic.
#include <mutex>
#include <unordered_map>

#include "kernels.h"

namespace mvgs {
namespace {

constexpr unsigned kFull = 0xffffffffu;

constexpr int WBATCH_DEFAULT = 128;  // Gaussians per warp batch in shared memory (64 and 192 with 4 px/lane)
constexpr int WARPS_PER_BLOCK = 4;

// One warp's work item: PPT pixels per lane of one (view, tile) pair -- a
// strip of the tile, or (sampled mode) a run of 32 * PPT of the tile's pixel
// samples.
template <int PPT>
struct Work {
    long long gt;               // global (view, tile) id, -1 when the queue is empty
    const DevCam* cam;
    float fx[PPT], fy[PPT];     // pixel centres (strips: one column, fx[k] all equal)
    int pix[PPT];               // pixel index in the view (y W + x); -1 for an idle slot
    float sx0, sx1, sy0, sy1;   // bounds of the warp's pixel centres
};

__device__ __forceinline__ int take_item(int* counter, int lane) {
    int item = 0;
    if (lane == 0) item = atomicAdd(counter, 1);
    return __shfl_sync(kFull, item, 0);
}

__device__ __forceinline__ const DevCam* view_of(const BlendArgs& a, long long gt, int lane) {
    int v = 0;
    if (lane == 0) v = find_view(a.cams, a.V, gt);
    v = __shfl_sync(kFull, v, 0);
    return &a.cams[v];
}

// Next strip for the warp.  With a pixel mask (the naive partial rendering
// of Fig. 3b) masked pixels are idle slots of their lanes.
template <int PPT>
__device__ __forceinline__ bool next_strip(const BlendArgs& a, int* counter, int lane, Work<PPT>& w) {
    const int item = take_item(counter, lane);
    if ((long long)item >= a.tiles * a.strips) return false;
    w.gt = (long long)a.order[item / a.strips];
    const int strip = item % a.strips;
    w.cam = view_of(a, w.gt, lane);
    const DevCam& cam = *w.cam;
    const long long local = w.gt - cam.tile_base;
    const int tx = (int)(local % cam.tiles_x), ty = (int)(local / cam.tiles_x);
    const int across = a.tw / a.sw;  // strips side by side in a tile
    const int step = 32 / a.sw;      // thread rows of the warp
    const int x0 = tx * a.tw + (strip % across) * a.sw, y0 = ty * a.th + (strip / across) * a.strip_h;
    const int px = x0 + lane % a.sw;
    const int py0 = y0 + lane / a.sw;
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        const int py = py0 + k * step;
        w.fx[k] = px + 0.5f;
        w.fy[k] = py + 0.5f;
        int p = -1;
        if (px < cam.W && py < cam.H) {
            p = py * cam.W + px;
            if (a.pixel_mask && !a.pixel_mask[cam.pix_base + p]) p = -1;
        }
        w.pix[k] = p;
    }
    w.sx0 = x0 + 0.5f;
    w.sx1 = (float)min(x0 + a.sw, cam.W) - 0.5f;
    w.sy0 = y0 + 0.5f;
    w.sy1 = (float)min(y0 + a.strip_h, cam.H) - 0.5f;
    return true;
}

// Next run of pixel samples (Alg. 3): lanes take consecutive samples of the
// tile's list, so every lane of the warp has a pixel to blend except in the
// tile's last run.  Runs whose samples are all invalid are skipped.
template <int PPT>
__device__ __forceinline__ bool next_samples(const BlendArgs& a, int* counter, int lane, long long total,
                                             Work<PPT>& w) {
    for (;;) {
        const int item = take_item(counter, lane);
        if ((long long)item >= total) return false;
        const int i = a.chunk_map[item];
        w.gt = (long long)a.order[i];
        const long long chunk = (long long)item - a.chunk_off[i];
        w.cam = view_of(a, w.gt, lane);
        const DevCam& cam = *w.cam;
        const long long local = w.gt - cam.tile_base;
        const int tx = (int)(local % cam.tiles_x), ty = (int)(local / cam.tiles_x);
        const long long s0 = a.s_off[w.gt] + chunk * 32 * PPT, s1 = a.s_off[w.gt + 1];
        int xmin = 0x7fffffff, ymin = 0x7fffffff, xmax = -1, ymax = -1;
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            const long long si = s0 + k * 32 + lane;
            int p = -1, px = 0, py = 0;
            if (si < s1) {
                const int li = a.s_pix[si];
                const int lx = li % a.tw, ly = li / a.tw;
                px = tx * a.tw + lx;
                py = ty * a.th + ly;
                if (ly < a.th && px < cam.W && py < cam.H) {
                    p = py * cam.W + px;
                    xmin = min(xmin, px);
                    xmax = max(xmax, px);
                    ymin = min(ymin, py);
                    ymax = max(ymax, py);
                }
            }
            w.fx[k] = px + 0.5f;
            w.fy[k] = py + 0.5f;
            w.pix[k] = p;
        }
        xmax = __reduce_max_sync(kFull, xmax);
        if (xmax < 0) continue;  // no valid sample in this run
        xmin = __reduce_min_sync(kFull, xmin);
        ymin = __reduce_min_sync(kFull, ymin);
        ymax = __reduce_max_sync(kFull, ymax);
        w.sx0 = xmin + 0.5f;
        w.sx1 = xmax + 0.5f;
        w.sy0 = ymin + 0.5f;
        w.sy1 = ymax + 0.5f;
        return true;
    }
}

template <int PPT, bool SAMPLED>
__device__ __forceinline__ bool next_work(const BlendArgs& a, int* counter, int lane, long long total,
                                          Work<PPT>& w) {
    if constexpr (SAMPLED) return next_samples<PPT>(a, counter, lane, total, w);
    else return next_strip<PPT>(a, counter, lane, w);
}

// Resident blocks per SM the forward is compiled for: six (at most 80
// registers) for 4 pixels per lane without the depth and statistics outputs
// (strips and sample runs), where the extra warps hide more latency than the
// registers given up cost (3-4% faster); no bound elsewhere (more state
// there, and a bound spills it).
constexpr int fwd_min_blocks(int ppt, bool extra) { return ppt == 4 && !extra ? 6 : 1; }

// DEPTH: also the expected depth per pixel; STATS: also the per-pixel
// statistics (list position where the pixel stopped, Gaussians blended).
template <int PPT, bool SAMPLED, int WBATCH, bool DEPTH, bool STATS>
__global__ void __launch_bounds__(32 * WARPS_PER_BLOCK, fwd_min_blocks(PPT, DEPTH || STATS))
    blend_forward_kernel(BlendArgs a, int* __restrict__ counter,
                                                                             float* __restrict__ img,
                                                                             float* __restrict__ final_T,
                                                                             uint32_t* __restrict__ n_contrib,
                                                                             uint2* __restrict__ pixel_stats) {
    __shared__ float2 s_xy[WARPS_PER_BLOCK][WBATCH];
    __shared__ float4 s_co[WARPS_PER_BLOCK][WBATCH];
    __shared__ float4 s_rgb[WARPS_PER_BLOCK][WBATCH];
    __shared__ uint32_t s_pos[WARPS_PER_BLOCK][WBATCH];
    __shared__ float s_dep[WARPS_PER_BLOCK][DEPTH ? WBATCH : 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    float2* wxy = s_xy[w];
    float4* wco = s_co[w];
    float4* wrgb = s_rgb[w];
    uint32_t* wpos = s_pos[w];
    float* wdep = s_dep[w];
    constexpr uint32_t ALL = (1u << PPT) - 1u;
    const long long total = SAMPLED ? min(a.chunk_off[a.tiles], a.chunk_cap) : 0;
    Work<PPT> st;
    while (next_work<PPT, SAMPLED>(a, counter, lane, total, st)) {
        const DevCam& cam = *st.cam;
        const long long start = a.ranges[2 * st.gt], end = a.ranges[2 * st.gt + 1];
        float T[PPT], C0[PPT], C1[PPT], C2[PPT], D[PPT];
        uint32_t last[PPT], stop[PPT], nblend[PPT];
        uint32_t done = 0;
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            T[k] = 1.f;
            C0[k] = C1[k] = C2[k] = D[k] = 0.f;
            last[k] = 0;
            stop[k] = (uint32_t)(end - start);  // list position where the pixel stopped
            nblend[k] = 0;
            if (st.pix[k] < 0) done |= 1u << k;
        }
        for (long long b = start; b < end; b += WBATCH) {
            if (__all_sync(kFull, done == ALL)) break;
            // stage the Gaussians of this batch that can reach a pixel of the work item
            __syncwarp();
            int n = 0;
            for (int i0 = 0; i0 < WBATCH; i0 += 32) {
                const long long idx = b + i0 + lane;
                bool hit = false;
                float2 m;
                float4 co, cr;
                uint32_t r = 0;
                if (idx < end) {
                    r = a.sorted[idx];
                    m = a.xy[r];
                    co = a.conic_o[r];
                    cr = a.rgb_r[r];
                    hit = rect_reaches(st.sx0 - m.x, st.sx1 - m.x, st.sy0 - m.y, st.sy1 - m.y, co, cr.w);
                }
                const uint32_t bal = __ballot_sync(kFull, hit);
                if (hit) {
                    const int slot = n + __popc(bal & lt);
                    wxy[slot] = m;
                    wco[slot] = exp2_coeffs(co);
                    wrgb[slot] = cr;
                    wpos[slot] = (uint32_t)(idx - start);
                    if (DEPTH) wdep[slot] = a.rec_depth[r];
                }
                n += __popc(bal);
            }
            __syncwarp();
            for (int j = 0; j < n; j++) {
                const float2 m = wxy[j];
                const float4 cr = wrgb[j];
                const float dx0 = st.fx[0] - m.x;
                if (!SAMPLED && fabsf(dx0) > cr.w) continue;  // outside the support for the whole column
                const float4 q = wco[j];
                const uint32_t pos = wpos[j];
                const float dep = DEPTH ? wdep[j] : 0.f;
                const ColTerms ct0 = col_terms(dx0, q);
#pragma unroll
                for (int k = 0; k < PPT; k++) {
                    if ((done >> k) & 1u) continue;
                    const float dx = SAMPLED ? st.fx[k] - m.x : dx0;
                    const ColTerms ct = SAMPLED ? col_terms(dx, q) : ct0;
                    float alpha, G;
                    if (!pair_eval(dx, st.fy[k] - m.y, ct, q, cr.w, alpha, G)) continue;
                    const float Tn = __fmul_rn(T[k], __fsub_rn(1.f, alpha));
                    if (Tn < kTMin) {
                        done |= 1u << k;
                        if (STATS) stop[k] = pos + 1;
                        continue;
                    }
                    const float wgt = __fmul_rn(alpha, T[k]);
                    C0[k] = __fmaf_rn(cr.x, wgt, C0[k]);
                    C1[k] = __fmaf_rn(cr.y, wgt, C1[k]);
                    C2[k] = __fmaf_rn(cr.z, wgt, C2[k]);
                    if (DEPTH) D[k] = __fmaf_rn(dep, wgt, D[k]);
                    T[k] = Tn;
                    last[k] = pos + 1;
                    if (STATS) nblend[k]++;
                }
                if (done == ALL) break;
            }
        }
        const long long HW = (long long)cam.W * cam.H;
        float* out = img + 3 * cam.pix_base;
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            const long long p = st.pix[k];
            if (p >= 0) {
                out[p] = __fmaf_rn(T[k], a.bg[0], C0[k]);
                out[HW + p] = __fmaf_rn(T[k], a.bg[1], C1[k]);
                out[2 * HW + p] = __fmaf_rn(T[k], a.bg[2], C2[k]);
                final_T[cam.pix_base + p] = T[k];
                n_contrib[cam.pix_base + p] = last[k];
                if (STATS) pixel_stats[cam.pix_base + p] = make_uint2(stop[k], nblend[k]);
                if (DEPTH) a.depth_out[cam.pix_base + p] = D[k];
            }
        }
    }
}

// Sum over the warp of 10 values per lane, scattered: 12 shuffles in five
// halving steps (5 + 3 + 2 + 1 + 1), after which every lane holds the full sum
// of one value, value_of_lane(lane).
__device__ __forceinline__ int value_of_lane(int lane) {
    const int b4 = (lane >> 4) & 1, b3 = (lane >> 3) & 1, b2 = (lane >> 2) & 1, b1 = (lane >> 1) & 1;
    return 5 * b4 + (b3 ? 3 + b2 : (b2 ? 2 : b1));
}

__device__ __forceinline__ float warp_reduce_scatter10(const float (&g)[10], int lane) {
    const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0, b2 = (lane & 4) != 0, b1 = (lane & 2) != 0;
    // step 1 (lanes l, l^16): values 0-4 stay in the lower, 5-9 in the upper half
    float a[5];
#pragma unroll
    for (int i = 0; i < 5; i++) {
        const float send = b4 ? g[i] : g[i + 5];
        const float keep = b4 ? g[i + 5] : g[i];
        a[i] = keep + __shfl_xor_sync(kFull, send, 16);
    }
    // step 2 (l^8): a0-a2 stay in the lower, a3-a4 in the upper half
    float b[3];
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const float send = b3 ? a[i] : a[3 + i];
        const float keep = b3 ? a[3 + i] : a[i];
        b[i] = keep + __shfl_xor_sync(kFull, send, 8);
    }
    b[2] = a[2] + __shfl_xor_sync(kFull, a[2], 8);
    // step 3 (l^4): three values split 2 + 1, two values 1 + 1
    const float send0 = b2 ? b[0] : (b3 ? b[1] : b[2]);
    const float keep0 = b2 ? (b3 ? b[1] : b[2]) : b[0];
    const float c0 = keep0 + __shfl_xor_sync(kFull, send0, 4);
    const float c1 = b[1] + __shfl_xor_sync(kFull, b[1], 4);
    // step 4 (l^2): the two-value lanes split 1 + 1, the others add
    const bool two = !b3 && !b2;
    const float send = (two && !b1) ? c1 : c0;
    const float keep = (two && b1) ? c1 : c0;
    const float d = keep + __shfl_xor_sync(kFull, send, 2);
    return d + __shfl_xor_sync(kFull, d, 1);
}

template <int PPT, bool SAMPLED, int WBATCH>
__global__ void __launch_bounds__(32 * WARPS_PER_BLOCK) blend_backward_kernel(BlendArgs a, int* __restrict__ counter,
                                                                              const float* __restrict__ dimg,
                                                                              const float* __restrict__ final_T,
                                                                              const uint32_t* __restrict__ n_contrib,
                                                                              float* __restrict__ rec_grad,
                                                                              double* __restrict__ rec_conic) {
    __shared__ float2 s_xy[WARPS_PER_BLOCK][WBATCH];
    __shared__ float4 s_co[WARPS_PER_BLOCK][WBATCH];
    __shared__ float4 s_rgb[WARPS_PER_BLOCK][WBATCH];
    __shared__ uint32_t s_rid[WARPS_PER_BLOCK][WBATCH];
    __shared__ uint32_t s_pos[WARPS_PER_BLOCK][WBATCH];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    float2* wxy = s_xy[w];
    float4* wco = s_co[w];
    float4* wrgb = s_rgb[w];
    uint32_t* wrid = s_rid[w];
    uint32_t* wpos = s_pos[w];
    // the value this lane holds after the reduce-scatter
    const int my_val = value_of_lane(lane);
    // one lane per value: value_of_lane is the same for lanes l, l^1 and, where
    // it ignores bit 1, for l^2
    const bool adder = (lane & 1) == 0 && ((lane & 12) == 0 || (lane & 2) == 0);
    const long long total = SAMPLED ? min(a.chunk_off[a.tiles], a.chunk_cap) : 0;
    Work<PPT> st;
    while (next_work<PPT, SAMPLED>(a, counter, lane, total, st)) {
        const DevCam& cam = *st.cam;
        const long long HW = (long long)cam.W * cam.H;
        const float* din = dimg + 3 * cam.pix_base;
        // per pixel: T in front of the current Gaussian, dL/dC, and
        // U = dL/dC . (colour blended behind the current Gaussian + T_final bg)
        float T[PPT], d0[PPT], d1[PPT], d2[PPT], U[PPT];
        uint32_t last[PPT];
        uint32_t mylast = 0;
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            T[k] = 1.f;
            d0[k] = d1[k] = d2[k] = 0.f;
            last[k] = 0;
            const long long p = st.pix[k];
            if (p >= 0) {
                d0[k] = din[p];
                d1[k] = din[HW + p];
                d2[k] = din[2 * HW + p];
                T[k] = final_T[cam.pix_base + p];
                last[k] = n_contrib[cam.pix_base + p];
            }
            U[k] = T[k] * (d0[k] * a.bg[0] + d1[k] * a.bg[1] + d2[k] * a.bg[2]);
            mylast = last[k] > mylast ? last[k] : mylast;
        }
        const uint32_t maxlast = __reduce_max_sync(kFull, mylast);
        const long long start = a.ranges[2 * st.gt];
        for (uint32_t b = 0; b < maxlast; b += WBATCH) {
            // stage, back to front, the Gaussians that can reach the work item
            __syncwarp();
            int n = 0;
            for (int i0 = 0; i0 < WBATCH; i0 += 32) {
                const long long pos = (long long)maxlast - 1 - b - i0 - lane;
                bool hit = false;
                uint32_t r = 0;
                float2 m;
                float4 co, cr;
                if (pos >= 0) {
                    r = a.sorted[start + pos];
                    m = a.xy[r];
                    co = a.conic_o[r];
                    cr = a.rgb_r[r];
                    hit = rect_reaches(st.sx0 - m.x, st.sx1 - m.x, st.sy0 - m.y, st.sy1 - m.y, co, cr.w);
                }
                const uint32_t bal = __ballot_sync(kFull, hit);
                if (hit) {
                    const int slot = n + __popc(bal & lt);
                    wrid[slot] = r;
                    wxy[slot] = m;
                    wco[slot] = exp2_coeffs(co);
                    wrgb[slot] = cr;
                    wpos[slot] = (uint32_t)pos;
                }
                n += __popc(bal);
            }
            __syncwarp();
            // two Gaussians per loop trip: one's reduce-scatter overlaps the next one's pixels
#pragma unroll 2
            for (int j = 0; j < n; j++) {
                const uint32_t pos = wpos[j];
                float g[10];
#pragma unroll
                for (int i = 0; i < 10; i++) g[i] = 0.f;
                bool any = false;
                const float2 m = wxy[j];
                const float4 cr = wrgb[j];
                const float dx0 = st.fx[0] - m.x;
                if (pos < mylast && (SAMPLED || fabsf(dx0) <= cr.w)) {
                    const float4 q = wco[j];
                    const float3 cn = conic_of(q);  // (A, B, C)
                    const ColTerms ct0 = col_terms(dx0, q);
                    const float adx0 = cn.x * dx0, bdx0 = cn.y * dx0;
                    // strips (one column per lane): sums over the lane's pixels of
                    // dL/dpower times 1, dy and dy^2, turned into the mean and conic
                    // gradients once per Gaussian below
                    float P0 = 0.f, P1 = 0.f, P2 = 0.f;
#pragma unroll
                    for (int k = 0; k < PPT; k++) {
                        if (pos >= last[k]) continue;
                        const float dx = SAMPLED ? st.fx[k] - m.x : dx0;
                        const float dy = st.fy[k] - m.y;
                        const ColTerms ct = SAMPLED ? col_terms(dx, q) : ct0;
                        float alpha, G;
                        if (!pair_eval(dx, dy, ct, q, cr.w, alpha, G)) continue;
                        any = true;
                        const float inv = rcp_approx(1.f - alpha);
                        T[k] *= inv;  // transmittance in front of this Gaussian
                        const float wgt = alpha * T[k];
                        g[6] += d0[k] * wgt;
                        g[7] += d1[k] * wgt;
                        g[8] += d2[k] * wgt;
                        const float dc = d0[k] * cr.x + d1[k] * cr.y + d2[k] * cr.z;
                        const float dLda = T[k] * dc - U[k] * inv;
                        U[k] += dc * wgt;
                        if (alpha < kAlphaMax) {  // below the clamp alpha = o G
                            const float dLdp = dLda * alpha;  // dL/d power = dL/dalpha o G
                            // d power / d mean2d = (ax, ay) = (A dx + B dy, B dx + C dy)
                            const float ax = fmaf(cn.y, dy, SAMPLED ? cn.x * dx : adx0);
                            const float ay = fmaf(cn.z, dy, SAMPLED ? cn.y * dx : bdx0);
                            if (SAMPLED) {
                                const float h = -0.5f * dLdp;
                                g[0] += dLdp * ax;
                                g[1] += dLdp * ay;
                                g[2] += h * dx * dx;
                                g[3] += 2.f * h * dx * dy;
                                g[4] += h * dy * dy;
                            } else {
                                const float e = dLdp * dy;
                                P0 += dLdp;
                                P1 += e;
                                P2 = fmaf(e, dy, P2);
                            }
                            g[5] += dLda * G;
                            g[9] += fabsf(dLdp) * sqrt_approx(ax * ax + ay * ay);
                        }
                    }
                    if (!SAMPLED) {
                        // sum_k dL/dpower_k (ax_k, ay_k) and -1/2 sum_k dL/dpower_k (dx^2, 2 dx dy_k, dy_k^2)
                        g[0] = fmaf(adx0, P0, cn.y * P1);
                        g[1] = fmaf(bdx0, P0, cn.z * P1);
                        g[2] = -0.5f * dx0 * dx0 * P0;
                        g[3] = -dx0 * P1;
                        g[4] = -0.5f * P2;
                    }
                }
                if (__ballot_sync(kFull, any) == 0u) continue;
                const float sum = warp_reduce_scatter10(g, lane);
                if (adder) {
                    // the conic gradients sum terms weighted by dx^2 ~ 1e4 px^2 of both
                    // signs: they are added across warps in double precision
                    if (my_val >= 2 && my_val <= 4)
                        atomicAdd(rec_conic + (size_t)3 * wrid[j] + (my_val - 2), (double)sum);
                    else
                        atomicAdd(rec_grad + (size_t)kGradStride * wrid[j] + grad_slot(my_val), sum);
                }
            }
        }
    }
}

// Resident blocks over the whole GPU for a kernel (cached per kernel).
int persistent_blocks(const void* kernel) {
    static std::mutex mu;
    static std::unordered_map<const void*, int> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(kernel);
    if (it != cache.end()) return it->second;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32 * WARPS_PER_BLOCK, 0);
    const int n = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    cache[kernel] = n;
    return n;
}

template <class K>
unsigned grid_for(K kernel, long long items) {
    const long long blocks = (items + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK;
    const long long n = persistent_blocks(reinterpret_cast<const void*>(kernel));
    return (unsigned)(blocks < n ? blocks : n);
}

}  // namespace

// Strips are 8 columns wide whatever the tile width: with 4 pixels per lane
// an 8 x 16 strip, whose perimeter (and so the Gaussians that cross into it)
// is smaller than that of a full-width 32 x 4 strip of the same 128 pixels
// (3M Gaussians x 8 views at 32 x 64 tiles: blend forward + backward 16.7 ->
// 13.6 ms; 16-column strips 13.9 ms, 4-column 15.4 ms).
int blend_strip_width(int tw) { return tw > 8 ? 8 : tw; }

int blend_pixels_per_thread(int tw, int th, int req) {
    if (req > 0) return req;
    for (int p = 4; p >= 1; p >>= 1)
        if (th % ((32 / blend_strip_width(tw)) * p) == 0) return p;
    return 1;
}

void launch_blend_forward(const BlendArgs& a, int* counter, float* img, float* final_T, uint32_t* n_contrib,
                          uint2* pixel_stats, cudaStream_t s) {
    if (a.tiles == 0) return;
    cudaMemsetAsync(counter, 0, sizeof(int), s);
    const bool sampled = a.s_off != nullptr;
    // sampled mode: the number of runs is only known on the device; launch a
    // full persistent grid
    const bool depth = a.depth_out != nullptr, stats = pixel_stats != nullptr;
    const long long items = sampled ? (1LL << 40) : a.tiles * a.strips;
#define MVGS_BF1(P, S, B, D, ST)                                                                  \
    blend_forward_kernel<P, S, B, D, ST><<<grid_for(blend_forward_kernel<P, S, B, D, ST>, items),          \
                                           32 * WARPS_PER_BLOCK, 0, s>>>(a, counter, img, final_T, n_contrib, \
                                                                         pixel_stats)
#define MVGS_BF(P, S, B)                        \
    do {                                        \
        if (depth && stats)                     \
            MVGS_BF1(P, S, B, true, true);      \
        else if (depth)                         \
            MVGS_BF1(P, S, B, true, false);     \
        else if (stats)                         \
            MVGS_BF1(P, S, B, false, true);     \
        else                                    \
            MVGS_BF1(P, S, B, false, false);    \
    } while (0)
#define MVGS_BF2(P, B)              \
    do {                            \
        if (sampled)                \
            MVGS_BF(P, true, B);    \
        else                        \
            MVGS_BF(P, false, B);   \
    } while (0)
    switch (a.ppt) {
        case 1: MVGS_BF2(1, WBATCH_DEFAULT); break;
        case 2: MVGS_BF2(2, WBATCH_DEFAULT); break;
        case 8: MVGS_BF2(8, WBATCH_DEFAULT); break;
        default:
            if (a.wbatch == 64) MVGS_BF2(4, 64);
            else if (a.wbatch == 192) MVGS_BF2(4, 192);
            else MVGS_BF2(4, WBATCH_DEFAULT);
            break;
    }
#undef MVGS_BF2
#undef MVGS_BF
#undef MVGS_BF1
    note_launches(1);
}

void launch_blend_backward(const BlendArgs& a, int* counter, const float* dimg, const float* final_T,
                           const uint32_t* n_contrib, float* rec_grad, double* rec_conic, cudaStream_t s) {
    if (a.tiles == 0) return;
    cudaMemsetAsync(counter, 0, sizeof(int), s);
    const bool sampled = a.s_off != nullptr;
    const long long items = sampled ? (1LL << 40) : a.tiles * a.strips;
#define MVGS_BB(P, S, B)                                                                                         \
    blend_backward_kernel<P, S, B><<<grid_for(blend_backward_kernel<P, S, B>, items), 32 * WARPS_PER_BLOCK, 0,   \
                                     s>>>(a, counter, dimg, final_T, n_contrib, rec_grad, rec_conic)
#define MVGS_BB2(P, B) if (sampled) MVGS_BB(P, true, B); else MVGS_BB(P, false, B)
    switch (a.ppt) {
        case 1: MVGS_BB2(1, WBATCH_DEFAULT); break;
        case 2: MVGS_BB2(2, WBATCH_DEFAULT); break;
        case 8: MVGS_BB2(8, WBATCH_DEFAULT); break;
        default:
            if (a.wbatch == 64) MVGS_BB2(4, 64);
            else if (a.wbatch == 192) MVGS_BB2(4, 192);
            else MVGS_BB2(4, WBATCH_DEFAULT);
            break;
    }
#undef MVGS_BB2
#undef MVGS_BB
    note_launches(1);
}

}  // namespace mvgs
