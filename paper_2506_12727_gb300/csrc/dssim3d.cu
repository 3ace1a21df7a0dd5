// 3D distance-aware D-SSIM (Sec. 5.1.2) on the merged images of a partially
// rendered batch (Fig. 3c), and the two copies around it.
//
// merge:  for every pixel of merged image m (views m*group .. m*group+group-1,
//         one resolution), the owner view v = m*group + slot(x, y) -- the view
//         that rendered the pixel in the partial render -- gives the merged
//         colour and target, and the pixel's surface point: the expected depth
//         z = D / (1 - T_final) (D = sum alpha T z_i from the forward) lifted
//         through the pixel centre of v's camera, X = R^T (z K^-1 (x+.5, y+.5,
//         1) - t), with the kernel width s = sigma_px z / f_x (the window's
//         sigma in pixels carried to the surface).  1 - T_final < 1e-3: no
//         surface point (s = 0).
// loss:   K*(p, q) = exp(-|X_q - X_p|^2 / (2 s_p^2)) over the 11x11 window of
//         the centre p, normalised to sum 1 over the neighbours inside the
//         image that have a surface point (a centre without one keeps only
//         itself); SSIM with K* in place of the 2D window, C1 = 0.01^2,
//         C2 = 0.03^2; L_m = (1 - lambda) mean|I - I*| + lambda (1 - mean SSIM),
//         the weights held constant.
//         Kernel 1 (per 32x8 block, halo 42x18 in shared memory) forms the
//         weights, the moments, SSIM and, per centre p and channel, the
//         coefficients A_p, B_p, C_p / Z_p of dSSIM_p/dI1(q) = w_pq (A + 2 B
//         I1(q) + C I2(q)) / Z_p; kernel 2 gathers them back per pixel q over
//         the centres whose window holds q; kernel 3 reduces the block sums per
//         image in a fixed order.
// split:  dL/d(merged pixel) goes to the owner view's pixel, 0 to the group's
//         other views there.
#include <cmath>

#include "kernels.h"

namespace mvgs {
namespace {

// 32 x 8 pixels per block: a warp holds one row of 32 pixels, so its
// shared-memory reads of a neighbour offset fall in 32 different banks
constexpr int TSX = 32, TSY = 8;
constexpr int RAD = 5;
constexpr int HSX = TSX + 2 * RAD, HSY = TSY + 2 * RAD;  // 42 x 18 staged
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;
constexpr int kMaxImages = 64;
constexpr float kMinOpacity = 1e-3f;

struct Images {
    int count;
    int H[kMaxImages], W[kMaxImages], tiles_x[kMaxImages];
    long long pix[kMaxImages];      // first pixel of the image in the packed layout
    long long blk[kMaxImages + 1];  // first block of the image
    int first;                      // global index of image 0
};

__device__ __forceinline__ int image_of(const Images& im, long long b) {
    int i = 0;
    while (i + 1 < im.count && im.blk[i + 1] <= b) i++;
    return i;
}

// Kernel weight of neighbour q for centre p (p == q: 1).  Forward and
// backward evaluate it with this one function.
__device__ __forceinline__ float k3d(float px, float py, float pz, float sp, float qx, float qy, float qz, float sq,
                                     bool same) {
    if (same) return 1.f;
    if (!(sp > 0.f) || !(sq > 0.f)) return 0.f;
    const float dx = qx - px, dy = qy - py, dz = qz - pz;
    const float d2 = dx * dx + dy * dy + dz * dz;
    return __expf(-d2 / (2.f * sp * sp));
}

struct Blk {
    int i, H, W, x0, y0;
    long long pix;
};

__device__ __forceinline__ Blk block_of(const Images& im) {
    Blk b;
    b.i = image_of(im, blockIdx.x);
    const long long t = blockIdx.x - im.blk[b.i];
    b.H = im.H[b.i];
    b.W = im.W[b.i];
    b.x0 = (int)(t % im.tiles_x[b.i]) * TSX;
    b.y0 = (int)(t / im.tiles_x[b.i]) * TSY;
    b.pix = im.pix[b.i];
    return b;
}

__global__ void __launch_bounds__(256) dssim3d_forward_kernel(Images im, long long P, const float* __restrict__ img,
                                                             const float* __restrict__ tgt,
                                                             const float* __restrict__ pts,
                                                             const float* __restrict__ sig,
                                                             float* __restrict__ coef, float2* __restrict__ bsum,
                                                             long long blk_offset) {
    __shared__ float sX[3][HSY][HSX + 1], sS[HSY][HSX + 1], s1[3][HSY][HSX + 1], s2[3][HSY][HSX + 1];
    __shared__ float red[2][8];
    const Blk b = block_of(im);
    const long long HW = (long long)b.H * b.W;
    for (int k = threadIdx.x; k < HSX * HSY; k += blockDim.x) {
        const int r = k / HSX, c = k % HSX;
        const int y = b.y0 + r - RAD, x = b.x0 + c - RAD;
        const bool in = x >= 0 && y >= 0 && x < b.W && y < b.H;
        const long long o = (long long)y * b.W + x;
        sS[r][c] = in ? sig[b.pix + o] : -1.f;  // < 0: outside the image
#pragma unroll
        for (int ch = 0; ch < 3; ch++) {
            sX[ch][r][c] = in ? pts[3 * b.pix + ch * HW + o] : 0.f;
            s1[ch][r][c] = in ? img[3 * b.pix + ch * HW + o] : 0.f;
            s2[ch][r][c] = in ? tgt[3 * b.pix + ch * HW + o] : 0.f;
        }
    }
    __syncthreads();
    const int r = threadIdx.x / TSX + RAD, c = threadIdx.x % TSX + RAD;
    const int x = b.x0 + c - RAD, y = b.y0 + r - RAD;
    float ssim = 0.f, l1 = 0.f;
    if (x < b.W && y < b.H) {
        const float px = sX[0][r][c], py = sX[1][r][c], pz = sX[2][r][c], sp = sS[r][c];
        float Z = 0.f, m1[3] = {0.f, 0.f, 0.f}, m2[3] = {0.f, 0.f, 0.f}, e11[3] = {0.f, 0.f, 0.f},
              e22[3] = {0.f, 0.f, 0.f}, e12[3] = {0.f, 0.f, 0.f};
        for (int dv = -RAD; dv <= RAD; dv++) {
            for (int du = -RAD; du <= RAD; du++) {
                const int rr = r + dv, cc = c + du;
                const float sq = sS[rr][cc];
                if (sq < 0.f && !(du == 0 && dv == 0)) continue;  // outside the image
                const float w = k3d(px, py, pz, sp, sX[0][rr][cc], sX[1][rr][cc], sX[2][rr][cc], sq,
                                    du == 0 && dv == 0);
                if (w == 0.f) continue;
                Z += w;
#pragma unroll
                for (int ch = 0; ch < 3; ch++) {
                    const float a = s1[ch][rr][cc], q = s2[ch][rr][cc];
                    m1[ch] += w * a;
                    m2[ch] += w * q;
                    e11[ch] += w * a * a;
                    e22[ch] += w * q * q;
                    e12[ch] += w * a * q;
                }
            }
        }
        const float iZ = 1.f / Z;
        const long long p = b.pix + (long long)y * b.W + x;
#pragma unroll
        for (int ch = 0; ch < 3; ch++) {
            const float mu1 = m1[ch] * iZ, mu2 = m2[ch] * iZ;
            const float s11 = e11[ch] * iZ - mu1 * mu1, s22 = e22[ch] * iZ - mu2 * mu2;
            const float s12 = e12[ch] * iZ - mu1 * mu2;
            const float a1 = 2.f * mu1 * mu2 + kC1, a2 = 2.f * s12 + kC2;
            const float b1 = mu1 * mu1 + mu2 * mu2 + kC1, b2 = s11 + s22 + kC2;
            const float S = a1 * a2 / (b1 * b2);
            const float dmu1 = 2.f * mu2 * S / a1 - 2.f * mu1 * S / b1;
            const float ds11 = -S / b2;
            const float ds12 = 2.f * S / a2;
            coef[(0 * 3 + ch) * P + p] = (dmu1 - 2.f * mu1 * ds11 - mu2 * ds12) * iZ;
            coef[(1 * 3 + ch) * P + p] = ds11 * iZ;
            coef[(2 * 3 + ch) * P + p] = ds12 * iZ;
            ssim += S;
            l1 += fabsf(s1[ch][r][c] - s2[ch][r][c]);
        }
    }
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
        float a = 0.f, q = 0.f;
        for (int k = 0; k < 8; k++) {
            a += red[0][k];
            q += red[1][k];
        }
        bsum[blk_offset + blockIdx.x] = make_float2(a, q);
    }
}

__global__ void __launch_bounds__(256) dssim3d_backward_kernel(Images im, long long P, const float* __restrict__ img,
                                                              const float* __restrict__ tgt,
                                                              const float* __restrict__ pts,
                                                              const float* __restrict__ sig,
                                                              const float* __restrict__ coef, float lambda,
                                                              float inv_images, float* __restrict__ dimg) {
    __shared__ float sX[3][HSY][HSX + 1], sS[HSY][HSX + 1], sC[9][HSY][HSX + 1];
    const Blk b = block_of(im);
    const long long HW = (long long)b.H * b.W;
    for (int k = threadIdx.x; k < HSX * HSY; k += blockDim.x) {
        const int r = k / HSX, c = k % HSX;
        const int y = b.y0 + r - RAD, x = b.x0 + c - RAD;
        const bool in = x >= 0 && y >= 0 && x < b.W && y < b.H;
        const long long o = (long long)y * b.W + x;
        sS[r][c] = in ? sig[b.pix + o] : -1.f;
#pragma unroll
        for (int ch = 0; ch < 3; ch++) sX[ch][r][c] = in ? pts[3 * b.pix + ch * HW + o] : 0.f;
#pragma unroll
        for (int j = 0; j < 9; j++) sC[j][r][c] = in ? coef[j * P + b.pix + o] : 0.f;
    }
    __syncthreads();
    const int r = threadIdx.x / TSX + RAD, c = threadIdx.x % TSX + RAD;
    const int x = b.x0 + c - RAD, y = b.y0 + r - RAD;
    if (x >= b.W || y >= b.H) return;
    const float qx = sX[0][r][c], qy = sX[1][r][c], qz = sX[2][r][c], sq = sS[r][c];
    const long long o = (long long)y * b.W + x;
    float i1[3], i2[3];
#pragma unroll
    for (int ch = 0; ch < 3; ch++) {
        i1[ch] = img[3 * b.pix + ch * HW + o];
        i2[ch] = tgt[3 * b.pix + ch * HW + o];
    }
    float g[3] = {0.f, 0.f, 0.f};
    // centres p = q - (du, dv) whose window holds q
    for (int dv = -RAD; dv <= RAD; dv++) {
        for (int du = -RAD; du <= RAD; du++) {
            const int rr = r - dv, cc = c - du;
            const float sp = sS[rr][cc];
            if (sp < 0.f && !(du == 0 && dv == 0)) continue;
            const float w = k3d(sX[0][rr][cc], sX[1][rr][cc], sX[2][rr][cc], sp, qx, qy, qz, sq, du == 0 && dv == 0);
            if (w == 0.f) continue;
#pragma unroll
            for (int ch = 0; ch < 3; ch++)
                g[ch] += w * (sC[ch][rr][cc] + 2.f * sC[3 + ch][rr][cc] * i1[ch] + sC[6 + ch][rr][cc] * i2[ch]);
        }
    }
    const float inv_n = 1.f / (3.f * (float)b.H * (float)b.W);
#pragma unroll
    for (int ch = 0; ch < 3; ch++) {
        const float d = i1[ch] - i2[ch];
        const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
        dimg[3 * b.pix + ch * HW + o] = inv_images * inv_n * ((1.f - lambda) * sgn - lambda * g[ch]);
    }
}

__global__ void dssim3d_reduce_kernel(Images im, const float2* __restrict__ bsum, long long blk_offset,
                                      float lambda, float* __restrict__ loss) {
    const int i = blockIdx.x;
    __shared__ double red[2][256];
    double a = 0.0, q = 0.0;
    for (long long k = im.blk[i] + threadIdx.x; k < im.blk[i + 1]; k += blockDim.x) {
        const float2 s = bsum[blk_offset + k];
        a += s.x;
        q += s.y;
    }
    red[0][threadIdx.x] = a;
    red[1][threadIdx.x] = q;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double n = 3.0 * im.H[i] * (double)im.W[i];
        loss[im.first + i] = (float)((1.0 - lambda) * red[1][0] / n + lambda * (1.0 - red[0][0] / n));
    }
}

// ---- merge / split ---------------------------------------------------------
__global__ void merge_kernel(const DevCam* __restrict__ cams, int group, int cw, int ch, unsigned long long seed,
                             float sigma_px,
                             long long merged_pix, const long long* __restrict__ mbase, int M,
                             const float* __restrict__ images, const float* __restrict__ targets,
                             const float* __restrict__ depth_acc, const float* __restrict__ final_T,
                             float* __restrict__ out_img, float* __restrict__ out_tgt, float* __restrict__ out_pts,
                             float* __restrict__ out_sig) {
    const long long gp = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gp >= merged_pix) return;
    int m = 0;
    while (m + 1 < M && mbase[m + 1] <= gp) m++;
    const DevCam& c0 = cams[m * group];
    const long long local = gp - mbase[m];
    const int x = (int)(local % c0.W), y = (int)(local / c0.W);
    const int v = m * group + sample_slot(seed, x / cw, y / ch, group);
    const DevCam& cam = cams[v];
    const long long HW = (long long)cam.W * cam.H;
    const long long src = (long long)y * cam.W + x;
    const long long dst3 = 3 * mbase[m];
    for (int ch = 0; ch < 3; ch++) {
        if (out_img) out_img[dst3 + ch * HW + local] = images[3 * cam.pix_base + ch * HW + src];
        if (out_tgt) out_tgt[dst3 + ch * HW + local] = targets[3 * cam.pix_base + ch * HW + src];
    }
    if (!out_pts) return;
    const float opac = 1.f - final_T[cam.pix_base + src];
    float X[3] = {0.f, 0.f, 0.f}, s = 0.f;
    if (opac >= kMinOpacity) {
        const float z = depth_acc[cam.pix_base + src] / opac;
        const float pc[3] = {z * (x + 0.5f - cam.cx) / cam.fx - cam.t[0], z * (y + 0.5f - cam.cy) / cam.fy - cam.t[1],
                             z - cam.t[2]};
        for (int i = 0; i < 3; i++) X[i] = cam.R[i] * pc[0] + cam.R[3 + i] * pc[1] + cam.R[6 + i] * pc[2];
        s = sigma_px * z / cam.fx;
    }
    for (int i = 0; i < 3; i++) out_pts[dst3 + i * HW + local] = X[i];
    out_sig[gp] = s;
}

__global__ void split_kernel(const DevCam* __restrict__ cams, int group, int cw, int ch, unsigned long long seed,
                             long long merged_pix, const long long* __restrict__ mbase, int M,
                             const float* __restrict__ dmerged, float* __restrict__ dimg) {
    const long long gp = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gp >= merged_pix) return;
    int m = 0;
    while (m + 1 < M && mbase[m + 1] <= gp) m++;
    const DevCam& c0 = cams[m * group];
    const long long local = gp - mbase[m];
    const int x = (int)(local % c0.W), y = (int)(local / c0.W);
    const int owner = sample_slot(seed, x / cw, y / ch, group);
    const long long HW = (long long)c0.W * c0.H;
    for (int k = 0; k < group; k++) {
        const DevCam& cam = cams[m * group + k];
        for (int ch = 0; ch < 3; ch++)
            dimg[3 * cam.pix_base + ch * HW + local] = k == owner ? dmerged[3 * mbase[m] + ch * HW + local] : 0.f;
    }
}

Images make_images(const int* hw, int first, int count) {
    Images im{};
    im.count = count;
    im.first = first;
    long long pix = 0, blk = 0;
    for (int i = 0; i < first; i++) pix += (long long)hw[2 * i] * hw[2 * i + 1];
    for (int i = 0; i < count; i++) {
        const int H = hw[2 * (first + i)], W = hw[2 * (first + i) + 1];
        im.H[i] = H;
        im.W[i] = W;
        im.tiles_x[i] = (W + TSX - 1) / TSX;
        im.pix[i] = pix;
        im.blk[i] = blk;
        pix += (long long)H * W;
        blk += (long long)im.tiles_x[i] * ((H + TSY - 1) / TSY);
    }
    im.blk[count] = blk;
    return im;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

size_t dssim3d_temp_bytes(const int* hw, int M) {
    long long P = 0, blocks = 0;
    for (int i = 0; i < M; i++) {
        P += (long long)hw[2 * i] * hw[2 * i + 1];
        blocks += (long long)((hw[2 * i + 1] + TSX - 1) / TSX) * ((hw[2 * i] + TSY - 1) / TSY);
    }
    return align256(9 * (size_t)P * sizeof(float)) + align256((size_t)blocks * sizeof(float2));
}

void launch_dssim3d(const float* img, const float* target, const float* points, const float* sigma, const int* hw,
                    int M, float lambda, float* loss, float* dimg, void* tmp, cudaStream_t s) {
    long long P = 0;
    for (int i = 0; i < M; i++) P += (long long)hw[2 * i] * hw[2 * i + 1];
    char* base = static_cast<char*>(tmp);
    float* coef = reinterpret_cast<float*>(base);
    float2* bsum = reinterpret_cast<float2*>(base + align256(9 * (size_t)P * sizeof(float)));
    long long blk_offset = 0;
    for (int first = 0; first < M; first += kMaxImages) {
        const int count = M - first < kMaxImages ? M - first : kMaxImages;
        const Images im = make_images(hw, first, count);
        const long long nb = im.blk[count];
        if (nb > 0) {
            dssim3d_forward_kernel<<<(unsigned)nb, 256, 0, s>>>(im, P, img, target, points, sigma, coef, bsum,
                                                                blk_offset);
            note_launches(1);
            if (dimg) {
                dssim3d_backward_kernel<<<(unsigned)nb, 256, 0, s>>>(im, P, img, target, points, sigma, coef, lambda,
                                                                     1.f / (float)M, dimg);
                note_launches(1);
            }
        }
        dssim3d_reduce_kernel<<<count, 256, 0, s>>>(im, bsum, blk_offset, lambda, loss);
        note_launches(1);
        blk_offset += nb;
    }
}

void launch_merge_views(const DevCam* cams, int group, int cw, int ch, unsigned long long seed, float sigma_px,
                        long long merged_pix,
                        const long long* mbase, int M, const float* images, const float* targets,
                        const float* depth_acc, const float* final_T, float* out_img, float* out_tgt, float* out_pts,
                        float* out_sig, cudaStream_t s) {
    if (merged_pix <= 0) return;
    merge_kernel<<<(unsigned)((merged_pix + 255) / 256), 256, 0, s>>>(cams, group, cw, ch, seed, sigma_px, merged_pix,
                                                                       mbase, M, images, targets, depth_acc, final_T,
                                                                       out_img, out_tgt, out_pts, out_sig);
    note_launches(1);
}

void launch_split_merged(const DevCam* cams, int group, int cw, int ch, unsigned long long seed, long long merged_pix,
                         const long long* mbase, int M, const float* dmerged, float* dimg, cudaStream_t s) {
    if (merged_pix <= 0) return;
    split_kernel<<<(unsigned)((merged_pix + 255) / 256), 256, 0, s>>>(cams, group, cw, ch, seed, merged_pix, mbase, M,
                                                                       dmerged, dimg);
    note_launches(1);
}

}  // namespace mvgs
