// Tile-based alpha blending (Eq. 1) and its backward.
//
// One block renders one (tile, view) pair at a time: the supplement allocates
// "one block for each viewpoint" per tile, and Alg. 2 has the block's threads
// fetch the tile's depth-sorted Gaussians into shared memory batch by batch,
// blend, and synchronise.  The whole batch of views is a single persistent
// launch over the global (view, tile) list, whatever the views' resolutions:
// resident blocks take tiles from a queue in an order that puts the longest
// lists first, so the heavy tiles do not form a tail.
//
// Each thread owns PPT pixels of one tile column (rows ly0, ly0 + R, ...), so
// one shared-memory read of a Gaussian serves PPT pixels; pixels that have
// stopped, or that a Gaussian does not reach, are skipped.
//
// Forward per pixel (front to back): alpha = min(0.99, o G), skip alpha <
// 1/255, stop before T (1 - alpha) < 1e-4, C += c alpha T, T *= 1 - alpha;
// output C + T bg.  A block leaves a tile once all its pixels have stopped.
//
// Backward per pixel (back to front from the last contributor), with T
// recovered by division:  dC/dc_i = alpha_i T_i,  dC/dalpha_i = c_i T_i -
// S_i / (1 - alpha_i), S_i the colour blended behind i plus T_final bg.  The
// gradients of one Gaussian are summed over the thread's pixels, then over
// the warp by a reduce-scatter (16 shuffles for 10 values), and each lane
// pair adds one value with one atomic.
#include <mutex>
#include <unordered_map>

#include "kernels.h"

namespace mvgs {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int BATCH = 256;  // Gaussians per shared-memory batch

struct PixelGeom {
    int px, py0, rows;  // rows: distance between a thread's pixels
    const DevCam* cam;
};

__device__ __forceinline__ PixelGeom pixel_geom(const BlendArgs& a, long long gt, int v) {
    PixelGeom g;
    g.cam = &a.cams[v];
    const long long local = gt - g.cam->tile_base;
    const int tx = (int)(local % g.cam->tiles_x), ty = (int)(local / g.cam->tiles_x);
    g.rows = blockDim.x / a.tw;
    g.px = tx * a.tw + (int)(threadIdx.x % a.tw);
    g.py0 = ty * a.th + (int)(threadIdx.x / a.tw);
    return g;
}

// Next tile of the queue for the whole block (-1 when the queue is empty).
__device__ __forceinline__ long long next_tile(const BlendArgs& a, int* counter, int* s_slot, int* s_v) {
    __syncthreads();  // every thread is done with the previous tile's shared values
    if (threadIdx.x == 0) {
        const int it = atomicAdd(counter, 1);
        *s_slot = it;
        if (it < a.tiles) *s_v = find_view(a.cams, a.V, a.order[it]);
    }
    __syncthreads();
    const int it = *s_slot;
    const long long gt = it < a.tiles ? (long long)a.order[it] : -1;
    return gt;
}

template <int PPT>
__global__ void __launch_bounds__(PPT >= 4 ? 128 : 256) blend_forward_kernel(BlendArgs a, int* __restrict__ counter,
                                                           float* __restrict__ img, float* __restrict__ final_T,
                                                           uint32_t* __restrict__ n_contrib,
                                                           uint2* __restrict__ pixel_stats) {
    __shared__ float2 s_xy[BATCH];
    __shared__ float4 s_co[BATCH];
    __shared__ float4 s_rgb[BATCH];
    __shared__ int s_slot, s_v;
    const int NT = blockDim.x;
    constexpr uint32_t ALL = (1u << PPT) - 1u;
    for (;;) {
        const long long gt = next_tile(a, counter, &s_slot, &s_v);
        if (gt < 0) break;
        const PixelGeom pg = pixel_geom(a, gt, s_v);
        const DevCam& cam = *pg.cam;
        const float fx = pg.px + 0.5f;
        float fy[PPT], T[PPT], C0[PPT], C1[PPT], C2[PPT];
        uint32_t last[PPT], stop[PPT], nblend[PPT];
        uint32_t done = 0;
        const long long start = a.ranges[2 * gt], end = a.ranges[2 * gt + 1];
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            const int py = pg.py0 + k * pg.rows;
            fy[k] = py + 0.5f;
            T[k] = 1.f;
            C0[k] = C1[k] = C2[k] = 0.f;
            last[k] = 0;
            stop[k] = (uint32_t)(end - start);  // list position where the pixel stopped
            nblend[k] = 0;
            if (!(pg.px < cam.W && py < cam.H)) done |= 1u << k;
        }
        for (long long b = start; b < end; b += BATCH) {
            if (__syncthreads_count(done == ALL) == NT) break;
            for (int i = threadIdx.x; i < BATCH; i += NT) {
                const long long idx = b + i;
                if (idx < end) {
                    const uint32_t r = a.sorted[idx];
                    s_xy[i] = a.xy[r];
                    s_co[i] = a.conic_o[r];
                    s_rgb[i] = a.rgb_r[r];
                }
            }
            __syncthreads();
            const int cnt = (int)(end - b < (long long)BATCH ? end - b : (long long)BATCH);
            const uint32_t base = (uint32_t)(b - start);
            for (int j = 0; j < cnt; j++) {
                const float2 m = s_xy[j];
                const float4 cr = s_rgb[j];
                const float dx = fx - m.x;
                if (fabsf(dx) > cr.w) continue;  // outside the support for the whole column
                const float4 co = s_co[j];
#pragma unroll
                for (int k = 0; k < PPT; k++) {
                    if ((done >> k) & 1u) continue;
                    float alpha, G;
                    if (!pair_eval(dx, fy[k] - m.y, co, cr.w, alpha, G)) continue;
                    const float Tn = T[k] * (1.f - alpha);
                    if (Tn < kTMin) {
                        done |= 1u << k;
                        stop[k] = base + j + 1;
                        continue;
                    }
                    const float w = alpha * T[k];
                    C0[k] += cr.x * w;
                    C1[k] += cr.y * w;
                    C2[k] += cr.z * w;
                    T[k] = Tn;
                    last[k] = base + j + 1;
                    nblend[k]++;
                }
                if (done == ALL) break;
            }
        }
        const long long HW = (long long)cam.W * cam.H;
        float* out = img + 3 * cam.pix_base;
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            const int py = pg.py0 + k * pg.rows;
            if (pg.px < cam.W && py < cam.H) {
                const long long p = (long long)py * cam.W + pg.px;
                out[p] = C0[k] + T[k] * a.bg[0];
                out[HW + p] = C1[k] + T[k] * a.bg[1];
                out[2 * HW + p] = C2[k] + T[k] * a.bg[2];
                final_T[cam.pix_base + p] = T[k];
                n_contrib[cam.pix_base + p] = last[k];
                pixel_stats[cam.pix_base + p] = make_uint2(stop[k], nblend[k]);
            }
        }
    }
}

// Sum over the warp of 16 values per lane, scattered: afterwards lane l holds
// the full sum of value 8 b4 + 4 b3 + 2 b2 + b1 (b_i the bits of l), in both
// lanes of each pair (l, l ^ 1).
__device__ __forceinline__ float warp_reduce_scatter16(float (&g)[16], int lane) {
#pragma unroll
    for (int h = 8, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; i++) {
            const float send = up ? g[i] : g[i + h];
            const float keep = up ? g[i + h] : g[i];
            g[i] = keep + __shfl_xor_sync(kFull, send, o);
        }
    }
    return g[0] + __shfl_xor_sync(kFull, g[0], 1);
}

template <int PPT>
__global__ void __launch_bounds__(PPT >= 4 ? 128 : 256) blend_backward_kernel(BlendArgs a, int* __restrict__ counter,
                                                            const float* __restrict__ dimg,
                                                            const float* __restrict__ final_T,
                                                            const uint32_t* __restrict__ n_contrib,
                                                            float* __restrict__ rec_grad) {
    __shared__ float2 s_xy[BATCH];
    __shared__ float4 s_co[BATCH];
    __shared__ float4 s_rgb[BATCH];
    __shared__ uint32_t s_rid[BATCH];
    __shared__ int s_slot, s_v;
    __shared__ uint32_t s_max;
    const int NT = blockDim.x;
    const int lane = threadIdx.x & 31;
    // value this lane adds after the reduce-scatter (lane pairs share one)
    const int my_val = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
    const bool adder = (lane & 1) == 0 && my_val < 10;
    for (;;) {
        const long long gt = next_tile(a, counter, &s_slot, &s_v);
        if (gt < 0) break;
        if (threadIdx.x == 0) s_max = 0;
        __syncthreads();
        const PixelGeom pg = pixel_geom(a, gt, s_v);
        const DevCam& cam = *pg.cam;
        const float fx = pg.px + 0.5f;
        const long long HW = (long long)cam.W * cam.H;
        const float* din = dimg + 3 * cam.pix_base;
        float fy[PPT], T[PPT], d0[PPT], d1[PPT], d2[PPT], S0[PPT], S1[PPT], S2[PPT];
        uint32_t last[PPT];
        uint32_t mylast = 0;
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            const int py = pg.py0 + k * pg.rows;
            fy[k] = py + 0.5f;
            T[k] = 1.f;
            d0[k] = d1[k] = d2[k] = 0.f;
            last[k] = 0;
            if (pg.px < cam.W && py < cam.H) {
                const long long p = (long long)py * cam.W + pg.px;
                d0[k] = din[p];
                d1[k] = din[HW + p];
                d2[k] = din[2 * HW + p];
                T[k] = final_T[cam.pix_base + p];
                last[k] = n_contrib[cam.pix_base + p];
            }
            // colour blended behind the current Gaussian, starting with the background
            S0[k] = T[k] * a.bg[0];
            S1[k] = T[k] * a.bg[1];
            S2[k] = T[k] * a.bg[2];
            mylast = last[k] > mylast ? last[k] : mylast;
        }
        atomicMax(&s_max, mylast);
        __syncthreads();
        const uint32_t maxlast = s_max;
        const long long start = a.ranges[2 * gt];
        for (uint32_t b = 0; b < maxlast; b += BATCH) {
            __syncthreads();
            for (int i = threadIdx.x; i < BATCH; i += NT) {
                const long long pos = (long long)maxlast - 1 - b - i;  // list position of slot i
                if (pos >= 0) {
                    const uint32_t r = a.sorted[start + pos];
                    s_rid[i] = r;
                    s_xy[i] = a.xy[r];
                    s_co[i] = a.conic_o[r];
                    s_rgb[i] = a.rgb_r[r];
                }
            }
            __syncthreads();
            const int cnt = (int)(maxlast - b < (uint32_t)BATCH ? maxlast - b : (uint32_t)BATCH);
            for (int j = 0; j < cnt; j++) {
                const uint32_t pos = maxlast - 1 - b - j;
                float g[16];
#pragma unroll
                for (int i = 0; i < 16; i++) g[i] = 0.f;
                bool any = false;
                const float2 m = s_xy[j];
                const float4 cr = s_rgb[j];
                const float dx = fx - m.x;
                if (pos < mylast && fabsf(dx) <= cr.w) {
                    const float4 co = s_co[j];
#pragma unroll
                    for (int k = 0; k < PPT; k++) {
                        if (pos >= last[k]) continue;
                        const float dy = fy[k] - m.y;
                        float alpha, G;
                        if (!pair_eval(dx, dy, co, cr.w, alpha, G)) continue;
                        any = true;
                        const float inv = __frcp_rn(1.f - alpha);
                        T[k] *= inv;  // transmittance in front of this Gaussian
                        const float w = alpha * T[k];
                        g[6] += d0[k] * w;
                        g[7] += d1[k] * w;
                        g[8] += d2[k] * w;
                        const float dLda = d0[k] * (cr.x * T[k] - S0[k] * inv) + d1[k] * (cr.y * T[k] - S1[k] * inv) +
                                           d2[k] * (cr.z * T[k] - S2[k] * inv);
                        S0[k] += cr.x * w;
                        S1[k] += cr.y * w;
                        S2[k] += cr.z * w;
                        if (co.w * G < kAlphaMax) {  // below the clamp alpha = o G
                            const float dLdp = dLda * alpha;  // dL/d power = dL/dalpha o G
                            const float gx = dLdp * (co.x * dx + co.y * dy);
                            const float gy = dLdp * (co.z * dy + co.y * dx);
                            g[0] += gx;
                            g[1] += gy;
                            g[2] += -0.5f * dLdp * dx * dx;
                            g[3] += -dLdp * dx * dy;
                            g[4] += -0.5f * dLdp * dy * dy;
                            g[5] += dLda * G;
                            g[9] += sqrtf(gx * gx + gy * gy);
                        }
                    }
                }
                if (__ballot_sync(kFull, any) == 0u) continue;
                const float sum = warp_reduce_scatter16(g, lane);
                if (adder) atomicAdd(rec_grad + (size_t)kGradStride * s_rid[j] + my_val, sum);
            }
        }
    }
}

// threads per block and pixels per thread for a tile size (tile sides 8, 16
// or 32 with at most 512 pixels: the thread count is a multiple of 32 and
// divides evenly into tile rows); a requested pixels-per-thread was checked
// by the caller
void blend_shape(int tw, int th, int req, int& threads, int& ppt) {
    const int pix = tw * th;
    ppt = req > 0 ? req : (pix >= 128 ? 4 : 2);
    threads = pix / ppt;
}

// Resident blocks over the whole GPU for a kernel at a block size (cached).
int persistent_blocks(const void* kernel, int threads) {
    static std::mutex mu;
    static std::unordered_map<const void*, int> cache;
    std::lock_guard<std::mutex> lk(mu);
    const auto key = static_cast<const void*>(static_cast<const char*>(kernel) + threads);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    const int n = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    cache[key] = n;
    return n;
}

template <class K>
unsigned grid_for(K kernel, int threads, long long tiles) {
    const long long n = persistent_blocks(reinterpret_cast<const void*>(kernel), threads);
    return (unsigned)(tiles < n ? tiles : n);
}

}  // namespace

void launch_blend_forward(const BlendArgs& a, int* counter, float* img, float* final_T, uint32_t* n_contrib,
                          uint2* pixel_stats, cudaStream_t s) {
    if (a.tiles == 0) return;
    int threads, ppt;
    blend_shape(a.tw, a.th, a.ppt, threads, ppt);
    cudaMemsetAsync(counter, 0, sizeof(int), s);
#define MVGS_BF(P)                                                                                               \
    blend_forward_kernel<P><<<grid_for(blend_forward_kernel<P>, threads, a.tiles), threads, 0, s>>>(            \
        a, counter, img, final_T, n_contrib, pixel_stats)
    switch (ppt) {
        case 1: MVGS_BF(1); break;
        case 2: MVGS_BF(2); break;
        case 8: MVGS_BF(8); break;
        default: MVGS_BF(4); break;
    }
#undef MVGS_BF
    note_launches(1);
}

void launch_blend_backward(const BlendArgs& a, int* counter, const float* dimg, const float* final_T,
                           const uint32_t* n_contrib, float* rec_grad, cudaStream_t s) {
    if (a.tiles == 0) return;
    int threads, ppt;
    blend_shape(a.tw, a.th, a.ppt, threads, ppt);
    cudaMemsetAsync(counter, 0, sizeof(int), s);
#define MVGS_BB(P)                                                                                               \
    blend_backward_kernel<P><<<grid_for(blend_backward_kernel<P>, threads, a.tiles), threads, 0, s>>>(          \
        a, counter, dimg, final_T, n_contrib, rec_grad)
    switch (ppt) {
        case 1: MVGS_BB(1); break;
        case 2: MVGS_BB(2); break;
        case 8: MVGS_BB(8); break;
        default: MVGS_BB(4); break;
    }
#undef MVGS_BB
    note_launches(1);
}

}  // namespace mvgs
