// Tile-based alpha blending (Eq. 1) and its backward.
//
// One block renders one (tile, view) pair: the supplement allocates "one block
// for each viewpoint" per tile, and Alg. 2 has the block's threads fetch the
// tile's depth-sorted Gaussians into shared memory batch by batch, blend, and
// synchronise.  The whole batch of views is a single launch over the global
// (view, tile) list, whatever the views' resolutions.
//
// Each thread owns PPT pixels of one tile column (rows ly0, ly0 + R, ...), so
// one shared-memory read of a Gaussian serves PPT pixels and, in the backward,
// PPT per-pixel gradients are summed in registers before the warp reduction.
//
// Forward per pixel (front to back): alpha = min(0.99, o G), skip alpha <
// 1/255, stop before T (1 - alpha) < 1e-4, C += c alpha T, T *= 1 - alpha;
// output C + T bg.  The block leaves the loop once every pixel has stopped.
//
// Backward per pixel (back to front from the last contributor), with T
// recovered by division:  dC/dc_i = alpha_i T_i,  dC/dalpha_i = c_i T_i -
// S_i / (1 - alpha_i), S_i the colour blended behind i plus T_final bg.  The
// gradients of one Gaussian are summed over the thread's pixels, then across
// the warp with shuffles, before one atomic add per warp and value.
#include "kernels.h"

namespace mvgs {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int BATCH = 256;  // Gaussians per shared-memory batch

struct PixelGeom {
    int px, py0, rows;  // rows: distance between a thread's pixels
    const DevCam* cam;
};

__device__ __forceinline__ PixelGeom pixel_geom(const BlendArgs& a, int v) {
    PixelGeom g;
    g.cam = &a.cams[v];
    const long long local = (long long)blockIdx.x - g.cam->tile_base;
    const int tx = (int)(local % g.cam->tiles_x), ty = (int)(local / g.cam->tiles_x);
    g.rows = blockDim.x / a.tw;
    g.px = tx * a.tw + (int)(threadIdx.x % a.tw);
    g.py0 = ty * a.th + (int)(threadIdx.x / a.tw);
    return g;
}

template <int PPT>
__global__ void __launch_bounds__(128) blend_forward_kernel(BlendArgs a, float* __restrict__ img,
                                                           float* __restrict__ final_T,
                                                           uint32_t* __restrict__ n_contrib) {
    __shared__ float2 s_xy[BATCH];
    __shared__ float4 s_co[BATCH];
    __shared__ float4 s_rgb[BATCH];
    __shared__ int s_v;
    const int NT = blockDim.x;
    const long long gt = blockIdx.x;
    if (threadIdx.x == 0) s_v = find_view(a.cams, a.V, gt);
    __syncthreads();
    const PixelGeom pg = pixel_geom(a, s_v);
    const DevCam& cam = *pg.cam;
    const float fx = pg.px + 0.5f;
    float fy[PPT], T[PPT], C0[PPT], C1[PPT], C2[PPT];
    uint32_t last[PPT];
    constexpr uint32_t ALL = (1u << PPT) - 1u;
    uint32_t done = 0;
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        const int py = pg.py0 + k * pg.rows;
        fy[k] = py + 0.5f;
        T[k] = 1.f;
        C0[k] = C1[k] = C2[k] = 0.f;
        last[k] = 0;
        if (!(pg.px < cam.W && py < cam.H)) done |= 1u << k;
    }
    const long long start = a.ranges[2 * gt], end = a.ranges[2 * gt + 1];
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
        for (int j = 0; done != ALL && j < cnt; j++) {
            const float2 m = s_xy[j];
            const float4 cr = s_rgb[j];
            const float dx = fx - m.x;
            if (fabsf(dx) > cr.w) continue;  // outside the support for the whole column
            const float4 co = s_co[j];
#pragma unroll
            for (int k = 0; k < PPT; k++) {
                if ((done >> k) & 1u) continue;
                float alpha, G;
                if (!pair_alpha(dx, fy[k] - m.y, co, cr.w, alpha, G)) continue;
                const float Tn = T[k] * (1.f - alpha);
                if (Tn < kTMin) {
                    done |= 1u << k;
                    continue;
                }
                const float w = alpha * T[k];
                C0[k] += cr.x * w;
                C1[k] += cr.y * w;
                C2[k] += cr.z * w;
                T[k] = Tn;
                last[k] = base + j + 1;
            }
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
        }
    }
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

template <int PPT>
__global__ void __launch_bounds__(128) blend_backward_kernel(BlendArgs a, const float* __restrict__ dimg,
                                                            const float* __restrict__ final_T,
                                                            const uint32_t* __restrict__ n_contrib,
                                                            float* __restrict__ rec_grad) {
    __shared__ float2 s_xy[BATCH];
    __shared__ float4 s_co[BATCH];
    __shared__ float4 s_rgb[BATCH];
    __shared__ uint32_t s_rid[BATCH];
    __shared__ int s_v;
    __shared__ uint32_t s_max;
    const int NT = blockDim.x;
    const long long gt = blockIdx.x;
    if (threadIdx.x == 0) {
        s_v = find_view(a.cams, a.V, gt);
        s_max = 0;
    }
    __syncthreads();
    const PixelGeom pg = pixel_geom(a, s_v);
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
    const int lane = threadIdx.x & 31;
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
            float g[10];
#pragma unroll
            for (int i = 0; i < 10; i++) g[i] = 0.f;
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
                    if (!pair_alpha(dx, dy, co, cr.w, alpha, G)) continue;
                    any = true;
                    const float om = 1.f - alpha;
                    T[k] = T[k] / om;  // transmittance in front of this Gaussian
                    const float w = alpha * T[k];
                    g[6] += d0[k] * w;
                    g[7] += d1[k] * w;
                    g[8] += d2[k] * w;
                    const float dLda = d0[k] * (cr.x * T[k] - S0[k] / om) + d1[k] * (cr.y * T[k] - S1[k] / om) +
                                       d2[k] * (cr.z * T[k] - S2[k] / om);
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
#pragma unroll
            for (int i = 0; i < 10; i++) g[i] = warp_sum(g[i]);
            // lanes 0..9 each add one value of the warp's sum
            float mine = 0.f;
#pragma unroll
            for (int i = 0; i < 10; i++) mine = lane == i ? g[i] : mine;
            if (lane < 10) atomicAdd(rec_grad + (size_t)kGradStride * s_rid[j] + lane, mine);
        }
    }
}

// threads per block and pixels per thread for a tile size (tile sides 8, 16
// or 32 with at most 512 pixels: the thread count is a multiple of 32 and
// divides evenly into tile rows)
void blend_shape(int tw, int th, int& threads, int& ppt) {
    const int pix = tw * th;
    ppt = pix >= 128 ? 4 : 2;
    threads = pix / ppt;
}

}  // namespace

void launch_blend_forward(const BlendArgs& a, float* img, float* final_T, uint32_t* n_contrib, cudaStream_t s) {
    if (a.tiles == 0) return;
    int threads, ppt;
    blend_shape(a.tw, a.th, threads, ppt);
    if (ppt == 4) blend_forward_kernel<4><<<(unsigned)a.tiles, threads, 0, s>>>(a, img, final_T, n_contrib);
    else blend_forward_kernel<2><<<(unsigned)a.tiles, threads, 0, s>>>(a, img, final_T, n_contrib);
    note_launches(1);
}

void launch_blend_backward(const BlendArgs& a, const float* dimg, const float* final_T, const uint32_t* n_contrib,
                           float* rec_grad, cudaStream_t s) {
    if (a.tiles == 0) return;
    int threads, ppt;
    blend_shape(a.tw, a.th, threads, ppt);
    if (ppt == 4) blend_backward_kernel<4><<<(unsigned)a.tiles, threads, 0, s>>>(a, dimg, final_T, n_contrib, rec_grad);
    else blend_backward_kernel<2><<<(unsigned)a.tiles, threads, 0, s>>>(a, dimg, final_T, n_contrib, rec_grad);
    note_launches(1);
}

}  // namespace mvgs
