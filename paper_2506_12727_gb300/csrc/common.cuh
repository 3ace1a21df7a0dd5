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

// An element count: known on the host (max), or -- in the capturable mode,
// where no count is read back -- held in device memory and bounded by the
// capacity the buffers were sized for: min(max, *dev).
struct Count {
    unsigned long long max;
    const unsigned long long* dev;
    __host__ __device__ Count(unsigned long long m = 0, const unsigned long long* d = nullptr) : max(m), dev(d) {}
    __device__ __forceinline__ unsigned long long get() const {
        if (!dev) return max;
        const unsigned long long v = *dev;
        return v < max ? v : max;
    }
};

constexpr int kCamChunk = 32;
struct CamChunk {
    DevCam c[kCamChunk];
};

// Per-record float gradient slots written by the blend backward and read by
// the preprocessing backward: mean2d x, y, opacity, r, g, b, E_1 term,
// padding (the conic's three go to a separate double array).  The blend
// backward's reduced value v (0, 1 mean2d; 2..4 conic; 5 opacity; 6..8 rgb;
// 9 E_1) goes to float slot grad_slot(v).
constexpr int kGradStride = 8;
__host__ __device__ constexpr int grad_slot(int v) { return v < 2 ? v : v - 3; }

// Global tile ids index the view-major list of (view, tile) pairs.
// Single-instruction approximations (PTX rcp.approx / sqrt.approx, about
// 1 ulp; flush-to-zero) for per-pair arithmetic, where the correctly rounded
// forms (__frcp_rn, IEEE sqrtf and division) are instruction sequences with a
// slow path.  The blend backward recovers T by a reciprocal and sums
// |dL/dmean2d| with a square root on every blended pair: the exact forms cost
// a fifth of that kernel, and the approximations are far inside the gradient
// tolerance of 1e-3 relative.
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ int find_view(const DevCam* cams, int V, long long gt) {
    int lo = 0, hi = V - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (cams[mid].tile_base <= gt) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): output number k of the
// stream seeded with s is mix(s + k * 0x9e3779b97f4a7c15).  The partial-render
// sample slot of cell (x, y) in a group of `group` views is
// floor(group * (h >> 32) / 2^32) with h output number 2^32 y + x + 1; a
// pixel's cell is (px / cell_w, py / cell_h).
__device__ __forceinline__ unsigned long long splitmix64_mix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ int sample_slot(unsigned long long seed, int x, int y, int group) {
    const unsigned long long c = ((unsigned long long)y << 32) | (unsigned)x;
    const unsigned long long h = splitmix64_mix(seed + (c + 1ULL) * 0x9e3779b97f4a7c15ULL);
    return (int)(((h >> 32) * (unsigned long long)group) >> 32);
}

// 2^x for the blend exponent (PTX ex2.approx, relative error near 2^-22;
// results below 2^-126 flush to zero, far under the 1/255 skip threshold).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The blend exponent in base 2.  With conic (A, B, C), d = pixel centre
// minus projected mean and L = log2 e,
//   power L = -(A dx^2 + 2 B dx dy + C dy^2) L / 2 = qa dx^2 + qb dx dy + qc dy^2,
// q = (qa, qb, qc) = (-A L / 2, -B L, -C L / 2), so G = exp(power) is one
// ex2 of a two-FMA polynomial in dy once the column terms (qa dx^2, qb dx)
// of the pixel's column are known.  A lane of a strip owns one column: it
// computes the column terms once per Gaussian and reuses them for its PPT
// pixels.
__device__ __forceinline__ float4 exp2_coeffs(float4 co) {
    constexpr float L = 1.4426950408889634f;
    return make_float4(__fmul_rn(-0.5f * L, co.x), __fmul_rn(-L, co.y), __fmul_rn(-0.5f * L, co.z), co.w);
}

// Conic (A, B, C) back from the base-2 coefficients (gradients need it).
__device__ __forceinline__ float3 conic_of(float4 q) {
    constexpr float LN2 = 0.6931471805599453f;
    return make_float3(-2.f * LN2 * q.x, -LN2 * q.y, -2.f * LN2 * q.z);
}

// A record's tile rectangle and view for the duplication, in 8 bytes: the
// corners x0, y0, x1, y1 (tile coordinates, end exclusive, each below 2^12)
// in bits 0-47 and the view in bits 48-63.
__device__ __forceinline__ unsigned long long pack_tile_desc(short4 rc, int view) {
    return (unsigned long long)(uint16_t)rc.x | (unsigned long long)(uint16_t)rc.y << 12 |
           (unsigned long long)(uint16_t)rc.z << 24 | (unsigned long long)(uint16_t)rc.w << 36 |
           (unsigned long long)view << 48;
}
__device__ __forceinline__ short4 tile_desc_rect(unsigned long long d) {
    return make_short4((short)(d & 0xfffu), (short)(d >> 12 & 0xfffu), (short)(d >> 24 & 0xfffu),
                       (short)(d >> 36 & 0xfffu));
}
__device__ __forceinline__ int tile_desc_view(unsigned long long d) { return (int)(d >> 48); }

struct ColTerms {
    float xx, x;  // qa dx^2 and qb dx
};

__device__ __forceinline__ ColTerms col_terms(float dx, float4 q) {
    return ColTerms{__fmul_rn(__fmul_rn(q.x, dx), dx), __fmul_rn(q.y, dx)};
}

// The blend decision and opacity of one (pixel, Gaussian) pair (Eq. 1 with
// the 3DGS clamp and skip rules and the per-pixel support rule); q holds the
// base-2 coefficients and the opacity (q.w), ct the column terms of dx.
// Everything is evaluated unconditionally; the return value says whether the
// Gaussian takes part at this pixel, and alpha and G = exp(power) are valid
// when it does.  The forward and the backward call this same function with
// the same inputs, so both take the same decision for every pair.  The
// products and fused multiply-adds are spelled out (no contraction left to
// the compiler), and the column terms are the same products whether a lane
// reuses them (strips) or computes them per pixel (sample runs), so every
// kernel rounds a pair the same way.
__device__ __forceinline__ bool pair_eval(float dx, float dy, ColTerms ct, float4 q, float radius, float& alpha,
                                          float& G) {
    const float e = __fmaf_rn(dy, __fmaf_rn(q.z, dy, ct.x), ct.xx);
    G = ex2_approx(e);
    alpha = fminf(kAlphaMax, __fmul_rn(q.w, G));
    return fabsf(dx) <= radius && fabsf(dy) <= radius && e <= 0.f && alpha >= kAlphaMin;
}

// Whether a Gaussian can pass the support rule and alpha >= 1/255 at any
// pixel centre of the rectangle [x0, x1] x [y0, y1] (centre coordinates,
// relative to the projected mean).  The exponent is largest where the
// quadratic form q = A dx^2 + 2 B dx dy + C dy^2 is smallest; over a
// rectangle that is 0 if it holds the mean, else on an edge, where q is a
// 1D quadratic minimised in closed form.  alpha >= 1/255 needs
// q <= 2 ln(255 o); the margin keeps the test a superset of what any pixel's
// float32 evaluation lets through.  The edge minimisers use approximate
// reciprocals: a point off the minimiser by a relative 1e-7 raises q by a
// second-order amount, far inside the margin.
__device__ __forceinline__ bool rect_reaches(float x0, float x1, float y0, float y1, float4 co, float radius) {
    if (x0 > radius || x1 < -radius || y0 > radius || y1 < -radius) return false;
    const float lvl = 2.f * __logf(255.f * co.w);
    if (!(lvl > 0.f)) return false;
    if (x0 <= 0.f && x1 >= 0.f && y0 <= 0.f && y1 >= 0.f) return true;
    const float A = co.x, B = co.y, C = co.z;
    auto q = [&](float x, float y) { return A * x * x + 2.f * B * x * y + C * y * y; };
    // edges x = x0, x = x1: minimise over y in [y0, y1]
    const float iC = rcp_approx(C), iA = rcp_approx(A);
    float best = 3.4e38f;
    {
        const float ya = fminf(fmaxf(-B * x0 * iC, y0), y1);
        const float yb = fminf(fmaxf(-B * x1 * iC, y0), y1);
        best = fminf(best, fminf(q(x0, ya), q(x1, yb)));
    }
    {
        const float xa = fminf(fmaxf(-B * y0 * iA, x0), x1);
        const float xb = fminf(fmaxf(-B * y1 * iA, x0), x1);
        best = fminf(best, fminf(q(xa, y0), q(xb, y1)));
    }
    return best <= lvl * 1.001f + 1e-3f;
}

}  // namespace mvgs
