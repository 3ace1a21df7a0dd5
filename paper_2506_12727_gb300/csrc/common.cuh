// Shared definitions of the sm_103a kernels (device side of libmvgs).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mvgs {

// Rasterizer constants the paper inherits from 3DGS without printing them
// (Sec. 3 cites the 3DGS rasterizer and EWA splatting): low-pass dilation of
// the projected covariance, alpha clamp, alpha skip threshold, transmittance
// cutoff, guard band of the projection Jacobian, 3-sigma radius and the
// eigenvalue floor used for it.
constexpr float kDilation = 0.3f;
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;
constexpr float kGuard = 1.3f;
constexpr float kSigmas = 3.0f;
constexpr float kEigFloor = 0.1f;

// Per-view camera table entry, built on the host from mvgs_camera and
// uploaded once per call; every kernel reads it from global memory.
struct __align__(16) DevCam {
    float R[9];      // world -> camera rotation, row-major
    float t[3];
    float fx, fy, cx, cy;
    float campos[3];
    float near_z;
    float limx, limy;  // guard band on x/z and y/z
    int W, H, tiles_x, tiles_y;
    long long tile_base;  // first global tile id of the view
    long long pix_base;   // first pixel of the view in the packed layout
    long long diff_base;  // first cell of the view's (tiles_y + 1) x (tiles_x + 1) count grid
};
static_assert(sizeof(DevCam) == 128, "camera table entry is 128 bytes");

constexpr int kCamChunk = 32;
struct CamChunk {
    DevCam c[kCamChunk];
};

// Per-record gradient slots written by the blend backward and read by the
// preprocessing backward: mean2d (2), conic A B C (3), opacity (1), rgb (3),
// E_1 term (1), padding (2).
constexpr int kGradStride = 12;

// Global tile ids index the view-major list of (view, tile) pairs.
__device__ __forceinline__ int find_view(const DevCam* cams, int V, long long gt) {
    int lo = 0, hi = V - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (cams[mid].tile_base <= gt) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The blend decision and opacity of one (pixel, Gaussian) pair (Eq. 1 with
// the 3DGS clamp and skip rules and the per-pixel support rule).  Everything
// is evaluated unconditionally so callers can stay branch-free; the return
// value says whether the Gaussian takes part at this pixel, alpha and the
// Gaussian falloff G are valid when it does.  The forward and the backward
// call this same function, so both take the same decision for every pair.
__device__ __forceinline__ bool pair_eval(float dx, float dy, float4 co, float radius, float& alpha, float& G) {
    const float power = -0.5f * (co.x * dx * dx + co.z * dy * dy) - co.y * dx * dy;
    G = __expf(power);
    alpha = fminf(kAlphaMax, co.w * G);
    return fabsf(dx) <= radius && fabsf(dy) <= radius && power <= 0.f && alpha >= kAlphaMin;
}

}  // namespace mvgs
