// Photometric l1 + D-SSIM loss per view, forward and gradient.
//
// Sec. 5.1.2: SSIM(I1, I2) = (2 mu1 mu2 + C1)(2 tau12 + C2) /
// ((mu1^2 + mu2^2 + C1)(tau1^2 + tau2^2 + C2)) with local moments against a
// Gaussian kernel; D-SSIM = 1 - SSIM.  Window 11x11, sigma 1.5, normalised
// to sum 1 and applied separably; zero padding; C1 = 0.01^2, C2 = 0.03^2.
//
// Kernel 1 computes, per 32x32 output tile of one channel plane, the five
// blurred moments from a 42x42 staged input, the SSIM map, and the three
// partial derivatives of SSIM with respect to the blurred moments m1 =
// K*I1, m11 = K*I1^2, m12 = K*(I1 I2); it also writes per-block sums of SSIM
// and |I1 - I2|.  Kernel 2 blurs those partials again (the filter is its own
// adjoint) to get dSSIM/dI1 = K*(dS/dm1) + 2 I1 K*(dS/dm11) + I2 K*(dS/dm12)
// and forms the gradient of the view-averaged loss.  Kernel 3 reduces the
// block sums per view in a fixed order (deterministic).
#include <cmath>
#include <vector>

#include "kernels.h"

namespace mvgs {
namespace {

// 32 x 32 outputs per block of 256 threads (four rows per thread): the staged
// halo is 1.7x the outputs instead of 2.6x with 16 x 16
constexpr int TSX = 32, TSY = 32;
constexpr int ROWS = TSY / 8;  // output rows per thread
constexpr int RADIUS = 5;            // 11 taps
constexpr int TAPS = 2 * RADIUS + 1;
constexpr int HSX = TSX + 2 * RADIUS, HSY = TSY + 2 * RADIUS;  // staged 42 x 42
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;
constexpr int kMaxViews = 64;

struct Views {
    int count;
    int H[kMaxViews], W[kMaxViews];
    int tiles_x[kMaxViews];
    long long pix[kMaxViews];     // first pixel of the view in the packed layout
    long long blk[kMaxViews + 1]; // first block of the view (3 channel planes)
    int first_view;               // global index of views[0]
    float w[TAPS];
};

__device__ __forceinline__ int block_view(const Views& vw, long long b) {
    int v = 0;
    while (v + 1 < vw.count && vw.blk[v + 1] <= b) v++;
    return v;
}

struct BlockPos {
    int v, ch, x0, y0, H, W;
    long long plane;  // offset of the channel plane in the packed image
};

__device__ __forceinline__ BlockPos block_pos(const Views& vw) {
    BlockPos p;
    const long long b = blockIdx.x;
    p.v = block_view(vw, b);
    const long long lb = b - vw.blk[p.v];
    p.H = vw.H[p.v];
    p.W = vw.W[p.v];
    const int tiles = vw.tiles_x[p.v] * ((p.H + TSY - 1) / TSY);
    p.ch = (int)(lb / tiles);
    const int t = (int)(lb % tiles);
    p.x0 = (t % vw.tiles_x[p.v]) * TSX;
    p.y0 = (t / vw.tiles_x[p.v]) * TSY;
    p.plane = 3 * vw.pix[p.v] + (long long)p.ch * p.H * p.W;
    return p;
}

__global__ void __launch_bounds__(256) dssim_forward_kernel(Views vw, const float* __restrict__ img,
                                                           const float* __restrict__ tgt,
                                                           float* __restrict__ dm1, float* __restrict__ dm11,
                                                           float* __restrict__ dm12, float2* __restrict__ bsum,
                                                           long long blk_offset) {
    // rows of 44 floats: 16-byte aligned, for the vector reads of the row pass
    __shared__ __align__(16) float s1[HSY][HSX + 2], s2[HSY][HSX + 2];
    __shared__ float h[5][HSY][TSX + 1];
    __shared__ float red[2][8];
    const BlockPos p = block_pos(vw);
    for (int i = threadIdx.x; i < HSY * HSX; i += blockDim.x) {
        const int r = i / HSX, c = i % HSX;
        const int y = p.y0 + r - RADIUS, x = p.x0 + c - RADIUS;
        const bool in = x >= 0 && y >= 0 && x < p.W && y < p.H;
        const long long o = p.plane + (long long)y * p.W + x;
        s1[r][c] = in ? img[o] : 0.f;
        s2[r][c] = in ? tgt[o] : 0.f;
    }
    __syncthreads();
    // row pass, four adjacent outputs per item: their 14 inputs come in four
    // 16-byte reads instead of 44 scalar ones
    for (int i = threadIdx.x; i < HSY * (TSX / 4); i += blockDim.x) {
        const int r = i / (TSX / 4), c0 = 4 * (i % (TSX / 4));
        float x1[16], x2[16];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const float4 u = reinterpret_cast<const float4*>(&s1[r][c0])[q];
            const float4 v = reinterpret_cast<const float4*>(&s2[r][c0])[q];
            x1[4 * q] = u.x; x1[4 * q + 1] = u.y; x1[4 * q + 2] = u.z; x1[4 * q + 3] = u.w;
            x2[4 * q] = v.x; x2[4 * q + 1] = v.y; x2[4 * q + 2] = v.z; x2[4 * q + 3] = v.w;
        }
#pragma unroll
        for (int o = 0; o < 4; o++) {
            float a = 0.f, b = 0.f, aa = 0.f, bb = 0.f, ab = 0.f;
#pragma unroll
            for (int k = 0; k < TAPS; k++) {
                const float u = x1[o + k], v = x2[o + k], w = vw.w[k];
                a += w * u;
                b += w * v;
                aa += w * u * u;
                bb += w * v * v;
                ab += w * u * v;
            }
            const int c = c0 + o;
            h[0][r][c] = a; h[1][r][c] = b; h[2][r][c] = aa; h[3][r][c] = bb; h[4][r][c] = ab;
        }
    }
    __syncthreads();
    float ssim = 0.f, l1 = 0.f;
    const int c = threadIdx.x % TSX;
    // a thread's ROWS consecutive output rows share ROWS + TAPS - 1 staged rows:
    // each staged value is read once and used for every output it reaches
    const int r0 = (threadIdx.x / TSX) * ROWS;
    float mv[ROWS][5];
#pragma unroll
    for (int q = 0; q < ROWS; q++)
#pragma unroll
        for (int i = 0; i < 5; i++) mv[q][i] = 0.f;
#pragma unroll
    for (int k = 0; k < ROWS + TAPS - 1; k++) {
        float hv[5];
#pragma unroll
        for (int i = 0; i < 5; i++) hv[i] = h[i][r0 + k][c];
#pragma unroll
        for (int q = 0; q < ROWS; q++) {
            const int t = k - q;
            if (t >= 0 && t < TAPS) {
                const float w = vw.w[t];
#pragma unroll
                for (int i = 0; i < 5; i++) mv[q][i] += w * hv[i];
            }
        }
    }
#pragma unroll
    for (int q = 0; q < ROWS; q++) {
        const int r = r0 + q;
        const float m1 = mv[q][0], m2 = mv[q][1], m11 = mv[q][2], m22 = mv[q][3], m12 = mv[q][4];
        const int x = p.x0 + c, y = p.y0 + r;
        if (x < p.W && y < p.H) {
            const float t11 = m11 - m1 * m1, t22 = m22 - m2 * m2, t12 = m12 - m1 * m2;
            const float a1 = 2.f * m1 * m2 + kC1, a2 = 2.f * t12 + kC2;
            const float b1 = m1 * m1 + m2 * m2 + kC1, b2 = t11 + t22 + kC2;
            // only the denominators b1, b2 (>= C1, C2 > 0) are inverted: S / a_k
            // is written as a product, so a vanishing a2 = 2 cov + C2 is harmless
            const float ib1 = rcp_approx(b1), ib2 = rcp_approx(b2), q = ib1 * ib2;
            const float sv = a1 * a2 * q;
            ssim += sv;
            const long long o = p.plane + (long long)y * p.W + x;
            dm1[o] = 2.f * (m2 * (a2 - a1) * q + m1 * sv * (ib2 - ib1));
            dm11[o] = -sv * ib2;
            dm12[o] = 2.f * a1 * q;
            l1 += fabsf(s1[r + RADIUS][c + RADIUS] - s2[r + RADIUS][c + RADIUS]);
        }
    }
    // block sums of SSIM and |I1 - I2|
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ssim += __shfl_xor_sync(0xffffffffu, ssim, o);
        l1 += __shfl_xor_sync(0xffffffffu, l1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = ssim;
        red[1][threadIdx.x >> 5] = l1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f, b = 0.f;
        for (int i = 0; i < 8; i++) {
            a += red[0][i];
            b += red[1][i];
        }
        bsum[blk_offset + blockIdx.x] = make_float2(a, b);
    }
}

__global__ void __launch_bounds__(256) dssim_backward_kernel(Views vw, const float* __restrict__ img,
                                                            const float* __restrict__ tgt,
                                                            const float* __restrict__ dm1,
                                                            const float* __restrict__ dm11,
                                                            const float* __restrict__ dm12, float lambda,
                                                            float inv_views, float* __restrict__ dimg) {
    __shared__ __align__(16) float s[3][HSY][HSX + 2];
    __shared__ float h[3][HSY][TSX + 1];
    const BlockPos p = block_pos(vw);
    for (int i = threadIdx.x; i < HSY * HSX; i += blockDim.x) {
        const int r = i / HSX, c = i % HSX;
        const int y = p.y0 + r - RADIUS, x = p.x0 + c - RADIUS;
        const bool in = x >= 0 && y >= 0 && x < p.W && y < p.H;
        const long long o = p.plane + (long long)y * p.W + x;
        s[0][r][c] = in ? dm1[o] : 0.f;
        s[1][r][c] = in ? dm11[o] : 0.f;
        s[2][r][c] = in ? dm12[o] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < HSY * (TSX / 4); i += blockDim.x) {
        const int r = i / (TSX / 4), c0 = 4 * (i % (TSX / 4));
        float x[3][16];
#pragma unroll
        for (int m = 0; m < 3; m++)
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const float4 u = reinterpret_cast<const float4*>(&s[m][r][c0])[q];
                x[m][4 * q] = u.x; x[m][4 * q + 1] = u.y; x[m][4 * q + 2] = u.z; x[m][4 * q + 3] = u.w;
            }
#pragma unroll
        for (int o = 0; o < 4; o++) {
            float a = 0.f, b = 0.f, d = 0.f;
#pragma unroll
            for (int k = 0; k < TAPS; k++) {
                const float w = vw.w[k];
                a += w * x[0][o + k];
                b += w * x[1][o + k];
                d += w * x[2][o + k];
            }
            const int c = c0 + o;
            h[0][r][c] = a; h[1][r][c] = b; h[2][r][c] = d;
        }
    }
    __syncthreads();
    const int c = threadIdx.x % TSX;
    const float inv_n = 1.f / (3.f * (float)p.H * (float)p.W);
    const int r0 = (threadIdx.x / TSX) * ROWS;
    float bv[ROWS][3];
#pragma unroll
    for (int q = 0; q < ROWS; q++) bv[q][0] = bv[q][1] = bv[q][2] = 0.f;
#pragma unroll
    for (int k = 0; k < ROWS + TAPS - 1; k++) {
        const float h0 = h[0][r0 + k][c], h1 = h[1][r0 + k][c], h2 = h[2][r0 + k][c];
#pragma unroll
        for (int q = 0; q < ROWS; q++) {
            const int t = k - q;
            if (t >= 0 && t < TAPS) {
                const float w = vw.w[t];
                bv[q][0] += w * h0;
                bv[q][1] += w * h1;
                bv[q][2] += w * h2;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < ROWS; q++) {
        const int r = r0 + q;
        const int x = p.x0 + c, y = p.y0 + r;
        if (x >= p.W || y >= p.H) continue;
        const float B1 = bv[q][0], B11 = bv[q][1], B12 = bv[q][2];
        const long long o = p.plane + (long long)y * p.W + x;
        const float i1 = img[o], i2 = tgt[o];
        const float diff = i1 - i2;
        const float sgn = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
        const float dssim = B1 + 2.f * i1 * B11 + i2 * B12;
        dimg[o] = inv_views * inv_n * ((1.f - lambda) * sgn - lambda * dssim);
    }
}

__global__ void dssim_reduce_kernel(Views vw, const float2* __restrict__ bsum, long long blk_offset, float lambda,
                                    float* __restrict__ loss) {
    const int v = blockIdx.x;
    const long long b0 = vw.blk[v], b1 = vw.blk[v + 1];
    __shared__ double red[2][256];
    double a = 0.0, b = 0.0;
    for (long long i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        const float2 s = bsum[blk_offset + i];
        a += s.x;
        b += s.y;
    }
    red[0][threadIdx.x] = a;
    red[1][threadIdx.x] = b;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double n = 3.0 * vw.H[v] * (double)vw.W[v];
        loss[vw.first_view + v] = (float)((1.0 - lambda) * red[1][0] / n + lambda * (1.0 - red[0][0] / n));
    }
}

Views make_views(const int* hw, int first, int count) {
    Views vw{};
    vw.count = count;
    vw.first_view = first;
    long long pix = 0, blk = 0;
    for (int v = 0; v < first; v++) pix += (long long)hw[2 * v] * hw[2 * v + 1];
    for (int i = 0; i < count; i++) {
        const int H = hw[2 * (first + i)], W = hw[2 * (first + i) + 1];
        vw.H[i] = H;
        vw.W[i] = W;
        vw.tiles_x[i] = (W + TSX - 1) / TSX;
        vw.pix[i] = pix;
        vw.blk[i] = blk;
        pix += (long long)H * W;
        blk += 3LL * vw.tiles_x[i] * ((H + TSY - 1) / TSY);
    }
    vw.blk[count] = blk;
    // 1D Gaussian taps, normalised to sum 1 (double on the host)
    double tap[TAPS], sum = 0.0;
    for (int k = 0; k < TAPS; k++) {
        const double x = k - RADIUS;
        tap[k] = std::exp(-x * x / (2.0 * 1.5 * 1.5));
        sum += tap[k];
    }
    for (int k = 0; k < TAPS; k++) vw.w[k] = (float)(tap[k] / sum);
    return vw;
}

long long total_blocks(const int* hw, int V) {
    long long blk = 0;
    for (int v = 0; v < V; v++) blk += 3LL * ((hw[2 * v + 1] + TSX - 1) / TSX) * ((hw[2 * v] + TSY - 1) / TSY);
    return blk;
}

long long total_pixels(const int* hw, int V) {
    long long p = 0;
    for (int v = 0; v < V; v++) p += (long long)hw[2 * v] * hw[2 * v + 1];
    return p;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

size_t dssim_temp_bytes(const int* hw, int V) {
    const long long P = total_pixels(hw, V);
    return 3 * align256(3 * P * sizeof(float)) + align256(total_blocks(hw, V) * sizeof(float2));
}

void launch_dssim(const float* img, const float* target, const int* hw, int V, float lambda, float* loss_per_view,
                  float* dimg, void* tmp, cudaStream_t s) {
    const long long P = total_pixels(hw, V);
    char* base = static_cast<char*>(tmp);
    float* dm1 = reinterpret_cast<float*>(base);
    float* dm11 = reinterpret_cast<float*>(base + align256(3 * P * sizeof(float)));
    float* dm12 = reinterpret_cast<float*>(base + 2 * align256(3 * P * sizeof(float)));
    float2* bsum = reinterpret_cast<float2*>(base + 3 * align256(3 * P * sizeof(float)));
    long long blk_offset = 0;
    for (int first = 0; first < V; first += kMaxViews) {
        const int count = V - first < kMaxViews ? V - first : kMaxViews;
        const Views vw = make_views(hw, first, count);
        const long long nb = vw.blk[count];
        if (nb > 0) {
            dssim_forward_kernel<<<(unsigned)nb, 256, 0, s>>>(vw, img, target, dm1, dm11, dm12, bsum, blk_offset);
            note_launches(1);
            if (dimg)
                dssim_backward_kernel<<<(unsigned)nb, 256, 0, s>>>(vw, img, target, dm1, dm11, dm12, lambda,
                                                                   1.f / (float)V, dimg);
            if (dimg) note_launches(1);
        }
        dssim_reduce_kernel<<<count, 256, 0, s>>>(vw, bsum, blk_offset, lambda, loss_per_view);
        note_launches(1);
        blk_offset += nb;
    }
}

}  // namespace mvgs
