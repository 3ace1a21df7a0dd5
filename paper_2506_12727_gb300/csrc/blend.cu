// Tile-based alpha blending (Eq. 1) and its backward.
//
// One block renders one (tile, view) pair: the supplement allocates "one block
// for each viewpoint" per tile, and Alg. 2 has the block's threads fetch the
// tile's depth-sorted Gaussians into shared memory batch by batch, blend, and
// synchronise.  The whole batch of views is a single launch over the global
// (view, tile) list, whatever the views' resolutions.
//
// Forward per pixel (front to back): alpha = min(0.99, o G), skip alpha <
// 1/255, stop before T (1 - alpha) < 1e-4, C += c alpha T, T *= 1 - alpha;
// output C + T bg.  The block leaves the loop once every pixel has stopped.
//
// Backward per pixel (back to front from the last contributor), with T
// recovered by division:  dC/dc_i = alpha_i T_i,  dC/dalpha_i = c_i T_i -
// S_i / (1 - alpha_i), S_i the colour blended behind i plus T_final bg.  The
// per-pixel gradients of one Gaussian are summed across the warp with
// shuffles before one atomic add per warp and value.
#include "kernels.h"

namespace mvgs {
namespace {

constexpr unsigned kFull = 0xffffffffu;

template <int MAXB>
__global__ void __launch_bounds__(MAXB) blend_forward_kernel(BlendArgs a, float* __restrict__ img,
                                                            float* __restrict__ final_T,
                                                            uint32_t* __restrict__ n_contrib) {
    __shared__ float2 s_xy[MAXB];
    __shared__ float4 s_co[MAXB];
    __shared__ float4 s_rgb[MAXB];
    __shared__ int s_v;
    const int B = blockDim.x;
    const long long gt = blockIdx.x;
    if (threadIdx.x == 0) s_v = find_view(a.cams, a.V, gt);
    __syncthreads();
    const DevCam& cam = a.cams[s_v];
    const long long local = gt - cam.tile_base;
    const int tx = (int)(local % cam.tiles_x), ty = (int)(local / cam.tiles_x);
    const int px = tx * a.tw + (int)(threadIdx.x % a.tw);
    const int py = ty * a.th + (int)(threadIdx.x / a.tw);
    const bool inside = px < cam.W && py < cam.H;
    const float fx = px + 0.5f, fy = py + 0.5f;
    const long long start = a.ranges[2 * gt], end = a.ranges[2 * gt + 1];
    bool done = !inside;
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t last = 0;
    for (long long b = start; b < end; b += B) {
        if (__syncthreads_count(done) == B) break;
        const long long idx = b + threadIdx.x;
        if (idx < end) {
            const uint32_t r = a.sorted[idx];
            s_xy[threadIdx.x] = a.xy[r];
            s_co[threadIdx.x] = a.conic_o[r];
            s_rgb[threadIdx.x] = a.rgb_r[r];
        }
        __syncthreads();
        const int cnt = (int)(end - b < (long long)B ? end - b : (long long)B);
        for (int j = 0; !done && j < cnt; j++) {
            const float2 m = s_xy[j];
            const float4 cr = s_rgb[j];
            float alpha, G;
            if (!pair_alpha(fx - m.x, fy - m.y, s_co[j], cr.w, alpha, G)) continue;
            const float Tn = T * (1.f - alpha);
            if (Tn < kTMin) {
                done = true;
                break;
            }
            const float w = alpha * T;
            C0 += cr.x * w;
            C1 += cr.y * w;
            C2 += cr.z * w;
            T = Tn;
            last = (uint32_t)(b - start) + j + 1;
        }
    }
    if (inside) {
        const long long HW = (long long)cam.W * cam.H;
        const long long p = (long long)py * cam.W + px;
        float* out = img + 3 * cam.pix_base;
        out[p] = C0 + T * a.bg[0];
        out[HW + p] = C1 + T * a.bg[1];
        out[2 * HW + p] = C2 + T * a.bg[2];
        final_T[cam.pix_base + p] = T;
        n_contrib[cam.pix_base + p] = last;
    }
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

template <int MAXB>
__global__ void __launch_bounds__(MAXB) blend_backward_kernel(BlendArgs a, const float* __restrict__ dimg,
                                                             const float* __restrict__ final_T,
                                                             const uint32_t* __restrict__ n_contrib,
                                                             float* __restrict__ rec_grad) {
    __shared__ float2 s_xy[MAXB];
    __shared__ float4 s_co[MAXB];
    __shared__ float4 s_rgb[MAXB];
    __shared__ uint32_t s_rid[MAXB];
    __shared__ int s_v;
    __shared__ uint32_t s_max;
    const int B = blockDim.x;
    const long long gt = blockIdx.x;
    if (threadIdx.x == 0) {
        s_v = find_view(a.cams, a.V, gt);
        s_max = 0;
    }
    __syncthreads();
    const DevCam& cam = a.cams[s_v];
    const long long local = gt - cam.tile_base;
    const int tx = (int)(local % cam.tiles_x), ty = (int)(local / cam.tiles_x);
    const int px = tx * a.tw + (int)(threadIdx.x % a.tw);
    const int py = ty * a.th + (int)(threadIdx.x / a.tw);
    const bool inside = px < cam.W && py < cam.H;
    const float fx = px + 0.5f, fy = py + 0.5f;
    const long long start = a.ranges[2 * gt];
    float T = 1.f, d0 = 0.f, d1 = 0.f, d2 = 0.f;
    uint32_t last = 0;
    if (inside) {
        const long long HW = (long long)cam.W * cam.H;
        const long long p = (long long)py * cam.W + px;
        const float* din = dimg + 3 * cam.pix_base;
        d0 = din[p];
        d1 = din[HW + p];
        d2 = din[2 * HW + p];
        T = final_T[cam.pix_base + p];
        last = n_contrib[cam.pix_base + p];
        atomicMax(&s_max, last);
    }
    // colour blended behind the current Gaussian, starting with the background
    float S0 = T * a.bg[0], S1 = T * a.bg[1], S2 = T * a.bg[2];
    __syncthreads();
    const uint32_t maxlast = s_max;
    const int lane = threadIdx.x & 31;
    for (uint32_t b = 0; b < maxlast; b += B) {
        __syncthreads();
        const long long pos = (long long)maxlast - 1 - b - threadIdx.x;  // list position loaded by this thread
        if (pos >= 0) {
            const uint32_t r = a.sorted[start + pos];
            s_rid[threadIdx.x] = r;
            s_xy[threadIdx.x] = a.xy[r];
            s_co[threadIdx.x] = a.conic_o[r];
            s_rgb[threadIdx.x] = a.rgb_r[r];
        }
        __syncthreads();
        const int cnt = (int)(maxlast - b < (uint32_t)B ? maxlast - b : (uint32_t)B);
        for (int j = 0; j < cnt; j++) {
            const uint32_t mypos = maxlast - 1 - b - j;
            float g[10];
#pragma unroll
            for (int i = 0; i < 10; i++) g[i] = 0.f;
            bool contrib = false;
            if (mypos < last) {
                const float2 m = s_xy[j];
                const float4 co = s_co[j];
                const float4 cr = s_rgb[j];
                const float dx = fx - m.x, dy = fy - m.y;
                float alpha, G;
                if (pair_alpha(dx, dy, co, cr.w, alpha, G)) {
                    contrib = true;
                    const float om = 1.f - alpha;
                    T = T / om;  // transmittance in front of this Gaussian
                    const float w = alpha * T;
                    g[6] = d0 * w;
                    g[7] = d1 * w;
                    g[8] = d2 * w;
                    const float dLda = d0 * (cr.x * T - S0 / om) + d1 * (cr.y * T - S1 / om) +
                                       d2 * (cr.z * T - S2 / om);
                    S0 += cr.x * w;
                    S1 += cr.y * w;
                    S2 += cr.z * w;
                    if (co.w * G < kAlphaMax) {  // below the clamp alpha = o G
                        const float dLdp = dLda * alpha;  // dL/d power = dL/dalpha o G
                        const float gx = dLdp * (co.x * dx + co.y * dy);
                        const float gy = dLdp * (co.z * dy + co.y * dx);
                        g[0] = gx;
                        g[1] = gy;
                        g[2] = -0.5f * dLdp * dx * dx;
                        g[3] = -dLdp * dx * dy;
                        g[4] = -0.5f * dLdp * dy * dy;
                        g[5] = dLda * G;
                        g[9] = sqrtf(gx * gx + gy * gy);
                    }
                }
            }
            if (__ballot_sync(kFull, contrib) == 0u) continue;
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

}  // namespace

void launch_blend_forward(const BlendArgs& a, float* img, float* final_T, uint32_t* n_contrib, cudaStream_t s) {
    if (a.tiles == 0) return;
    const int B = a.tw * a.th;
    if (B <= 64) blend_forward_kernel<64><<<(unsigned)a.tiles, B, 0, s>>>(a, img, final_T, n_contrib);
    else if (B <= 128) blend_forward_kernel<128><<<(unsigned)a.tiles, B, 0, s>>>(a, img, final_T, n_contrib);
    else if (B <= 256) blend_forward_kernel<256><<<(unsigned)a.tiles, B, 0, s>>>(a, img, final_T, n_contrib);
    else blend_forward_kernel<512><<<(unsigned)a.tiles, B, 0, s>>>(a, img, final_T, n_contrib);
    note_launches(1);
}

void launch_blend_backward(const BlendArgs& a, const float* dimg, const float* final_T, const uint32_t* n_contrib,
                           float* rec_grad, cudaStream_t s) {
    if (a.tiles == 0) return;
    const int B = a.tw * a.th;
    if (B <= 64) blend_backward_kernel<64><<<(unsigned)a.tiles, B, 0, s>>>(a, dimg, final_T, n_contrib, rec_grad);
    else if (B <= 128) blend_backward_kernel<128><<<(unsigned)a.tiles, B, 0, s>>>(a, dimg, final_T, n_contrib, rec_grad);
    else if (B <= 256) blend_backward_kernel<256><<<(unsigned)a.tiles, B, 0, s>>>(a, dimg, final_T, n_contrib, rec_grad);
    else blend_backward_kernel<512><<<(unsigned)a.tiles, B, 0, s>>>(a, dimg, final_T, n_contrib, rec_grad);
    note_launches(1);
}

}  // namespace mvgs
