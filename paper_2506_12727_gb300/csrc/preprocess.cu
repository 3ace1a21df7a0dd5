// Per-(Gaussian, view) preprocessing and its backward, plus the multi-view
// densification statistics.
//
// Sec. 3: Sigma = R S S^T R^T; the mean and covariance are projected to the
// image plane with the EWA local affine approximation (Zwicker et al.):
// Sigma' = J W Sigma W^T J^T, W the camera rotation and J the Jacobian of the
// perspective map at the mean.  The supplement ("Rasterization in multi-view
// training") decides which Gaussians take part in each view before anything
// is allocated, then culls, projects and duplicates only those; here a count
// pass over every (Gaussian, view) pair sizes a Gaussian-major record list and
// a second pass fills it.
#include "kernels.h"

namespace mvgs {
namespace {

// ---- spherical harmonics ---------------------------------------------------
// Real spherical harmonics up to degree 3 with the Condon-Shortley sign
// (-1)^m kept, index k = l^2 + l + m.  The normalisation constants are the
// closed forms sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!), times sqrt(2) for m != 0,
// written per term and evaluated at compile time.
constexpr double kPi = 3.14159265358979323846;

constexpr double const_sqrt(double x) {
    double r = x > 1.0 ? x : 1.0;
    for (int i = 0; i < 100; i++) r = 0.5 * (r + x / r);
    return r;
}

constexpr float Y00 = (float)(0.5 * const_sqrt(1.0 / kPi));
constexpr float Y1 = (float)const_sqrt(3.0 / (4.0 * kPi));
constexpr float Y2a = (float)(0.5 * const_sqrt(15.0 / kPi));
constexpr float Y2b = (float)(0.25 * const_sqrt(5.0 / kPi));
constexpr float Y2c = (float)(0.25 * const_sqrt(15.0 / kPi));
constexpr float Y3a = (float)(0.25 * const_sqrt(35.0 / (2.0 * kPi)));
constexpr float Y3b = (float)(0.5 * const_sqrt(105.0 / kPi));
constexpr float Y3c = (float)(0.25 * const_sqrt(21.0 / (2.0 * kPi)));
constexpr float Y3d = (float)(0.25 * const_sqrt(7.0 / kPi));
constexpr float Y3e = (float)(0.25 * const_sqrt(105.0 / kPi));

template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y) {
    Y[0] = Y00;
    if (DEG < 1) return;
    Y[1] = -Y1 * y;
    Y[2] = Y1 * z;
    Y[3] = -Y1 * x;
    if (DEG < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = Y2a * x * y;
    Y[5] = -Y2a * y * z;
    Y[6] = Y2b * (2.f * zz - xx - yy);
    Y[7] = -Y2a * x * z;
    Y[8] = Y2c * (xx - yy);
    if (DEG < 3) return;
    Y[9] = -Y3a * y * (3.f * xx - yy);
    Y[10] = Y3b * x * y * z;
    Y[11] = -Y3c * y * (4.f * zz - xx - yy);
    Y[12] = Y3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -Y3c * x * (4.f * zz - xx - yy);
    Y[14] = Y3e * z * (xx - yy);
    Y[15] = -Y3a * x * (xx - 3.f * yy);
}

// Gradient of sum_k w_k Y_k(x, y, z) with respect to (x, y, z), the basis
// taken as polynomials in the direction components.
template <int DEG>
__device__ __forceinline__ float3 sh_basis_grad(float x, float y, float z, const float* w) {
    float3 g = make_float3(0.f, 0.f, 0.f);
    if (DEG < 1) return g;
    g.y += -Y1 * w[1];
    g.z += Y1 * w[2];
    g.x += -Y1 * w[3];
    if (DEG < 2) return g;
    g.x += Y2a * y * w[4];
    g.y += Y2a * x * w[4];
    g.y += -Y2a * z * w[5];
    g.z += -Y2a * y * w[5];
    g.x += -2.f * Y2b * x * w[6];
    g.y += -2.f * Y2b * y * w[6];
    g.z += 4.f * Y2b * z * w[6];
    g.x += -Y2a * z * w[7];
    g.z += -Y2a * x * w[7];
    g.x += 2.f * Y2c * x * w[8];
    g.y += -2.f * Y2c * y * w[8];
    if (DEG < 3) return g;
    const float xx = x * x, yy = y * y, zz = z * z;
    g.x += -6.f * Y3a * x * y * w[9];
    g.y += -3.f * Y3a * (xx - yy) * w[9];
    g.x += Y3b * y * z * w[10];
    g.y += Y3b * x * z * w[10];
    g.z += Y3b * x * y * w[10];
    g.x += 2.f * Y3c * x * y * w[11];
    g.y += -Y3c * (4.f * zz - xx - 3.f * yy) * w[11];
    g.z += -8.f * Y3c * y * z * w[11];
    g.x += -6.f * Y3d * x * z * w[12];
    g.y += -6.f * Y3d * y * z * w[12];
    g.z += Y3d * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
    g.x += -Y3c * (4.f * zz - 3.f * xx - yy) * w[13];
    g.y += 2.f * Y3c * x * y * w[13];
    g.z += -8.f * Y3c * x * z * w[13];
    g.x += 2.f * Y3e * x * z * w[14];
    g.y += -2.f * Y3e * y * z * w[14];
    g.z += Y3e * (xx - yy) * w[14];
    g.x += -3.f * Y3a * (xx - yy) * w[15];
    g.y += 6.f * Y3a * x * y * w[15];
    return g;
}

// ---- Gaussian activation and projection -----------------------------------
struct Gauss {
    float mu[3];
    float s[3];
    float q[4];    // normalised (w, x, y, z)
    float qnorm;
    float R[9];    // rotation of q
    float M[9];    // R diag(s)
    float Sig[6];  // xx, xy, xz, yy, yz, zz
    float o;
};

__device__ __forceinline__ void load_gauss(const SceneArgs& sc, long long g, Gauss& G, bool need_opacity) {
    const float* m = sc.means + 3 * g;
    const float* ls = sc.log_scales + 3 * g;
    const float4 qr = *reinterpret_cast<const float4*>(sc.quats + 4 * g);
#pragma unroll
    for (int i = 0; i < 3; i++) {
        G.mu[i] = m[i];
        G.s[i] = __expf(ls[i]);
    }
    G.qnorm = sqrtf(qr.x * qr.x + qr.y * qr.y + qr.z * qr.z + qr.w * qr.w);
    const float inv = 1.f / G.qnorm;
    const float w = qr.x * inv, x = qr.y * inv, y = qr.z * inv, z = qr.w * inv;
    G.q[0] = w; G.q[1] = x; G.q[2] = y; G.q[3] = z;
    G.R[0] = 1.f - 2.f * (y * y + z * z); G.R[1] = 2.f * (x * y - w * z); G.R[2] = 2.f * (x * z + w * y);
    G.R[3] = 2.f * (x * y + w * z); G.R[4] = 1.f - 2.f * (x * x + z * z); G.R[5] = 2.f * (y * z - w * x);
    G.R[6] = 2.f * (x * z - w * y); G.R[7] = 2.f * (y * z + w * x); G.R[8] = 1.f - 2.f * (x * x + y * y);
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) G.M[3 * i + j] = G.R[3 * i + j] * G.s[j];
    auto dot3 = [&](int i, int j) {
        return G.M[3 * i] * G.M[3 * j] + G.M[3 * i + 1] * G.M[3 * j + 1] + G.M[3 * i + 2] * G.M[3 * j + 2];
    };
    G.Sig[0] = dot3(0, 0); G.Sig[1] = dot3(0, 1); G.Sig[2] = dot3(0, 2);
    G.Sig[3] = dot3(1, 1); G.Sig[4] = dot3(1, 2); G.Sig[5] = dot3(2, 2);
    G.o = need_opacity ? 1.f / (1.f + __expf(-sc.logits[g])) : 0.f;
}

struct Proj {
    float t[3];
    float depth;        // correctly rounded float32 of the camera depth (sort key)
    float ux, uy;       // t_x / t_z, t_y / t_z (unclamped)
    int clx, cly;       // guard-band clamp: 0 or +-1
    float J00, J02, J11, J12;
    float T[6];         // J W, 2x3
    float a, b, c, det; // Sigma' with dilation
    float2 xy;
    int radius;
    short4 rect;
};

__device__ __forceinline__ float sig_at(const float* S, int i, int j) {
    // symmetric 3x3 stored as xx, xy, xz, yy, yz, zz
    const int lo = i < j ? i : j, hi = i < j ? j : i;
    return lo == 0 ? S[hi] : (lo == 1 ? S[2 + hi] : S[5]);
}

// Projects one Gaussian into one view; false if culled (behind the near
// plane, degenerate covariance, or no tile of the image within its radius).
__device__ __forceinline__ bool project(const Gauss& G, const DevCam& cam, int tw, int th, Proj& P) {
#pragma unroll
    for (int i = 0; i < 3; i++)
        P.t[i] = cam.R[3 * i] * G.mu[0] + cam.R[3 * i + 1] * G.mu[1] + cam.R[3 * i + 2] * G.mu[2] + cam.t[i];
    const float tz = P.t[2];
    if (!(tz > cam.near_z)) return false;
    // The depth key must not depend on the evaluation order of this sum: take
    // it in double precision and round once, which gives the correctly rounded
    // float32 depth (ties in the sort are then exact ties).
    P.depth = __double2float_rn((double)cam.R[6] * G.mu[0] + (double)cam.R[7] * G.mu[1] +
                                (double)cam.R[8] * G.mu[2] + (double)cam.t[2]);
    const float iz = 1.f / tz;
    P.ux = P.t[0] * iz;
    P.uy = P.t[1] * iz;
    P.clx = P.ux > cam.limx ? 1 : (P.ux < -cam.limx ? -1 : 0);
    P.cly = P.uy > cam.limy ? 1 : (P.uy < -cam.limy ? -1 : 0);
    const float cux = P.clx ? P.clx * cam.limx : P.ux;
    const float cuy = P.cly ? P.cly * cam.limy : P.uy;
    P.J00 = cam.fx * iz;
    P.J02 = -cam.fx * cux * iz;
    P.J11 = cam.fy * iz;
    P.J12 = -cam.fy * cuy * iz;
#pragma unroll
    for (int j = 0; j < 3; j++) {
        P.T[j] = P.J00 * cam.R[j] + P.J02 * cam.R[6 + j];
        P.T[3 + j] = P.J11 * cam.R[3 + j] + P.J12 * cam.R[6 + j];
    }
    float TS[6];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            TS[3 * i + j] = P.T[3 * i] * sig_at(G.Sig, 0, j) + P.T[3 * i + 1] * sig_at(G.Sig, 1, j) +
                            P.T[3 * i + 2] * sig_at(G.Sig, 2, j);
    P.a = TS[0] * P.T[0] + TS[1] * P.T[1] + TS[2] * P.T[2] + kDilation;
    P.b = TS[0] * P.T[3] + TS[1] * P.T[4] + TS[2] * P.T[5];
    P.c = TS[3] * P.T[3] + TS[4] * P.T[4] + TS[5] * P.T[5] + kDilation;
    P.det = P.a * P.c - P.b * P.b;
    if (!(P.det > 0.f)) return false;
    P.xy = make_float2(cam.fx * P.ux + cam.cx, cam.fy * P.uy + cam.cy);
    const float mid = 0.5f * (P.a + P.c);
    const float lam = mid + sqrtf(fmaxf(kEigFloor, mid * mid - P.det));
    P.radius = (int)ceilf(kSigmas * sqrtf(lam));
    if (P.radius <= 0) return false;
    // The tiles the Gaussian covers: those holding a pixel centre where it
    // passes both the support rule (|d| <= r per axis) and alpha >= 1/255.
    // The second needs d^T Sigma'^-1 d <= 2 ln(255 o), an ellipse whose
    // bounding box has half-widths sqrt(2 ln(255 o) Sigma'_xx) and
    // sqrt(2 ln(255 o) Sigma'_yy); the margins keep the box a superset of the
    // pixels any float32 evaluation of alpha lets through.
    const float lo = logf(255.f * G.o);
    if (!(lo > 0.f)) return false;  // o <= 1/255: no pixel reaches 1/255
    const float ext = 2.f * lo * 1.001f + 1e-3f;
    const float r = (float)P.radius;
    const float hx = fminf(r, sqrtf(ext * P.a) + 1e-2f), hy = fminf(r, sqrtf(ext * P.c) + 1e-2f);
    // floor on both ends keeps at least half a pixel of slack
    const float x0 = fminf(fmaxf(floorf((P.xy.x - hx) / tw), 0.f), (float)cam.tiles_x);
    const float x1 = fminf(fmaxf(floorf((P.xy.x + hx) / tw) + 1.f, 0.f), (float)cam.tiles_x);
    const float y0 = fminf(fmaxf(floorf((P.xy.y - hy) / th), 0.f), (float)cam.tiles_y);
    const float y1 = fminf(fmaxf(floorf((P.xy.y + hy) / th) + 1.f, 0.f), (float)cam.tiles_y);
    P.rect = make_short4((short)x0, (short)y0, (short)x1, (short)y1);
    return x0 < x1 && y0 < y1;
}

// ---- kernels ---------------------------------------------------------------
__global__ void upload_cams_kernel(CamChunk chunk, int count, DevCam* dst) {
    if ((int)threadIdx.x < count) dst[threadIdx.x] = chunk.c[threadIdx.x];
}

// Visibility of every (Gaussian, view) pair: one byte per pair (view-minor)
// and the count per Gaussian.  The fill pass reads these bytes instead of
// deciding again, so the record count is exact by construction.
__global__ void __launch_bounds__(256) count_visible_kernel(SceneArgs sc, const DevCam* __restrict__ cams, int V,
                                                            int tw, int th, int* __restrict__ counts,
                                                            uint8_t* __restrict__ vis) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= sc.n) return;
    Gauss G;
    load_gauss(sc, g, G, true);
    int cnt = 0;
    for (int v = 0; v < V; v++) {
        Proj P;
        const bool ok = project(G, cams[v], tw, th, P);
        vis[g * V + v] = ok ? 1 : 0;
        cnt += ok ? 1 : 0;
    }
    counts[g] = cnt;
}

// SH coefficients of one Gaussian ([NK, 3], channel-minor) read as float4
// vectors when the row allows it (12 instead of 48 loads at degree 3), else
// one by one.  f(e, value) receives flat element e = 3 k + ch.
template <int NK, class F>
__device__ __forceinline__ void for_each_sh(const float* __restrict__ row, bool vec_ok, F f) {
    constexpr int E = NK * 3;
    if constexpr (E % 4 == 0) {
        if (vec_ok) {
            const float4* r4 = reinterpret_cast<const float4*>(row);
#pragma unroll
            for (int q = 0; q < E / 4; q++) {
                const float4 v = __ldg(r4 + q);
                f(4 * q, v.x);
                f(4 * q + 1, v.y);
                f(4 * q + 2, v.z);
                f(4 * q + 3, v.w);
            }
            return;
        }
    }
#pragma unroll
    for (int e = 0; e < E; e++) f(e, __ldg(row + e));
}

// A thread's SH coefficients staged once in shared memory, in a column of
// its own (element e of thread t at e * BS + t: consecutive threads hit
// consecutive banks), so the walk over the Gaussian's views reads them from
// shared memory instead of re-reading the 48-float row through L1 for every
// view -- at degree 3 the rows of all resident threads do not fit L1, and the
// re-reads went to L2 and HBM.  Only the owning thread reads its column: no
// block barrier is needed.
template <int NK, int BS>
__device__ __forceinline__ float* stage_sh(const float* __restrict__ row, bool vec_ok, float* smem) {
    float* col = smem + threadIdx.x;
    for_each_sh<NK>(row, vec_ok, [&](int e, float c) { col[e * BS] = c; });
    return col;
}

// Participation pre-count for sizing: per Gaussian, the visible views and the
// tiles they cover (the same projection as the render, so the totals are the
// render's record and key counts exactly).
__global__ void __launch_bounds__(256) count_keys_kernel(SceneArgs sc, const DevCam* __restrict__ cams, int V, int tw,
                                                         int th, int* __restrict__ recs,
                                                         uint32_t* __restrict__ keys) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= sc.n) return;
    Gauss G;
    load_gauss(sc, g, G, true);
    int r = 0;
    unsigned long long k = 0;
    for (int v = 0; v < V; v++) {
        Proj P;
        if (!project(G, cams[v], tw, th, P)) continue;
        r++;
        k += (unsigned long long)((P.rect.z - P.rect.x) * (P.rect.w - P.rect.y));
    }
    recs[g] = r;
    keys[g] = (uint32_t)(k < 0xffffffffull ? k : 0xffffffffull);
}

constexpr int PRE_THREADS = 128;

// One lane per (Gaussian, view) pair: a warp takes 32 / VG consecutive
// Gaussians with VG = min(V, 32) lanes each (views in order; more than 32
// views go in chunks of 32), so a warp's visible pairs are consecutive records
// of the Gaussian-major list and every record field is stored coalesced (one
// thread per Gaussian stored its records about V records apart from the next
// thread's: partly written sectors).  The lanes of a Gaussian read the same
// parameters (broadcast loads).  Compiled for 8 resident blocks per SM (64
// registers): the kernel waits mostly on its loads, and the extra warps hide
// more of them.
template <int DEG>
__global__ void __launch_bounds__(PRE_THREADS, 8) preprocess_kernel(SceneArgs sc, const DevCam* __restrict__ cams, int V,
                                                                 int tw, int th, const uint8_t* __restrict__ vis,
                                                                 RecordArgs rec, uint32_t* __restrict__ tiles_touched,
                                                                 unsigned long long* __restrict__ tile_desc) {
    constexpr int NK = (DEG + 1) * (DEG + 1);
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const int VG = V < 32 ? V : 32;
    const int GPW = 32 / VG;
    const long long g0 = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * GPW;
    if (g0 >= sc.n) return;  // the whole warp
    const int gi = lane / VG, vl = lane - gi * VG;
    const long long g = g0 + gi;
    const bool mine = gi < GPW && g < sc.n;
    // the warp's Gaussians' SH rows (consecutive in memory) copied once into
    // shared memory by all lanes, with loads issued before any arithmetic
    constexpr int E = NK * 3;
    __shared__ float s_sh[PRE_THREADS / 32][32 * E];
    float* wsh = s_sh[threadIdx.x >> 5];
    const int gcount = (int)(sc.n - g0 < GPW ? sc.n - g0 : GPW);
    const float* rows = sc.sh + (size_t)g0 * E;
    for (int i = lane; i < gcount * E; i += 32) wsh[i] = __ldg(rows + i);
    Gauss G;
    if (mine) load_gauss(sc, g, G, true);
    __syncwarp();
    const float* shc = wsh + (mine ? gi : 0) * E;
    long long rbase = rec.rec_off[g0];
    for (int c = 0; c < V; c += VG) {
        const int v = c + vl;
        const bool on = mine && v < V && vis[g * V + v];
        const uint32_t bal = __ballot_sync(0xffffffffu, on);
        const long long r = rbase + __popc(bal & lt);
        rbase += __popc(bal);
        // capturable mode past its record capacity: not written (reported through the counts)
        if (!on || r >= rec.cap) continue;
        const DevCam& cam = cams[v];
        Proj P;
        const bool ok = project(G, cam, tw, th, P);
        if (!ok) P.rect = make_short4(0, 0, 0, 0);  // same decision as the count pass, kept safe regardless
        const float inv = 1.f / P.det;
        rec.rec_g[r] = (int)g;
        rec.rec_v[r] = v;
        rec.xy[r] = P.xy;
        rec.conic_o[r] = make_float4(P.c * inv, -P.b * inv, P.a * inv, G.o);
        // colour from the direction camera -> mean
        float dx = G.mu[0] - cam.campos[0], dy = G.mu[1] - cam.campos[1], dz = G.mu[2] - cam.campos[2];
        const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
        dx *= il; dy *= il; dz *= il;
        float Y[NK];
        sh_basis<DEG>(dx, dy, dz, Y);
        float rgb[3] = {0.5f, 0.5f, 0.5f};
        int clamp = 0;
#pragma unroll
        for (int e = 0; e < E; e++) rgb[e % 3] += Y[e / 3] * shc[e];
#pragma unroll
        for (int ch = 0; ch < 3; ch++) {
            if (rgb[ch] < 0.f) { clamp |= 1 << ch; rgb[ch] = 0.f; }
        }
        rec.rgb_r[r] = make_float4(rgb[0], rgb[1], rgb[2], (float)P.radius);
        rec.clamp[r] = clamp;
        rec.depth[r] = P.depth;
        rec.rect[r] = P.rect;
        tiles_touched[r] = (uint32_t)((P.rect.z - P.rect.x) * (P.rect.w - P.rect.y));
        tile_desc[r] = pack_tile_desc(P.rect, v);
    }
}

// Chain rule from the per-record 2D gradients to the Gaussian parameters;
// one thread per Gaussian walks its records (one per view it is visible in)
// and sums the view contributions in registers, so every parameter gradient
// is written exactly once, without atomics.
template <int DEG>
__global__ void __launch_bounds__(128, 3) preprocess_backward_kernel(SceneArgs sc, const DevCam* __restrict__ cams,
                                                                  RecordArgs rec, const float* __restrict__ rg,
                                                                  const double* __restrict__ rc,
                                                                  float* __restrict__ g_means,
                                                                  float* __restrict__ g_log_scales,
                                                                  float* __restrict__ g_quats,
                                                                  float* __restrict__ g_logits,
                                                                  float* __restrict__ g_sh,
                                                                  float* __restrict__ out_mean2d,
                                                                  float* __restrict__ out_e1) {
    constexpr int NK = (DEG + 1) * (DEG + 1);
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= sc.n) return;
    Gauss G;
    load_gauss(sc, g, G, true);
    const float* shg = sc.sh + (size_t)g * NK * 3;
    const bool sh_vec = (reinterpret_cast<uintptr_t>(sc.sh) & 15) == 0;  // rows of 48 floats stay 16-byte aligned
    __shared__ float s_sh[NK * 3 * 128];
    const float* shc = stage_sh<NK, 128>(shg, sh_vec, s_sh);
    float gmu[3] = {0.f, 0.f, 0.f};
    float gS[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // dL/dSigma, symmetric (xx, xy, xz, yy, yz, zz)
    float go = 0.f;
    float gsh[NK * 3];
#pragma unroll
    for (int i = 0; i < NK * 3; i++) gsh[i] = 0.f;
    const long long r0 = rec.rec_off[g], r1 = min(rec.rec_off[g + 1], rec.cap);
    for (long long r = r0; r < r1; r++) {
        const DevCam& cam = cams[rec.rec_v[r]];
        Proj P;
        project(G, cam, 1, 1, P);  // same arithmetic as the forward; the tile size only affects the rect
        const float4 q0 = *reinterpret_cast<const float4*>(rg + kGradStride * r);      // x, y, opacity, r
        const float4 q1 = *reinterpret_cast<const float4*>(rg + kGradStride * r + 4);  // g, b, E_1, -
        const float gx = q0.x, gy = q0.y, gop = q0.z;
        const float gA = (float)rc[3 * r], gB = (float)rc[3 * r + 1], gC = (float)rc[3 * r + 2];
        const float grgb_raw[3] = {q0.w, q1.x, q1.y};
        if (out_mean2d) {
            out_mean2d[2 * r] = gx;
            out_mean2d[2 * r + 1] = gy;
        }
        if (out_e1) out_e1[r] = q1.z;
        // conic Q = Sigma'^-1 = [[A, B], [B, C]] = [[c, -b], [-b, a]] / det; with
        // dQ = -Q dSigma' Q, dL/dSigma' = -Q G Q for G = [[gA, gB/2], [gB/2, gC]]
        // (gB is the derivative w.r.t. B filling both off-diagonal entries, and
        // gb likewise w.r.t. b).  Written in Q, no term cancels as the
        // expansion in (a, b, c) / det does when b is small.
        const float id = 1.f / P.det;
        const float QA = P.c * id, QB = -P.b * id, QC = P.a * id;
        const float ga = -(QA * QA * gA + QA * QB * gB + QB * QB * gC);
        const float gb = -(2.f * QA * QB * gA + (QA * QC + QB * QB) * gB + 2.f * QB * QC * gC);
        const float gc = -(QB * QB * gA + QB * QC * gB + QC * QC * gC);
        // Sigma' = T Sigma T^T: dL/dSigma += T^T G2 T with G2 = [[ga, gb/2], [gb/2, gc]]
        const float h = 0.5f * gb;
        float GT[6];  // G2 T (2x3)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            GT[j] = ga * P.T[j] + h * P.T[3 + j];
            GT[3 + j] = h * P.T[j] + gc * P.T[3 + j];
        }
        gS[0] += P.T[0] * GT[0] + P.T[3] * GT[3];
        gS[1] += P.T[0] * GT[1] + P.T[3] * GT[4];
        gS[2] += P.T[0] * GT[2] + P.T[3] * GT[5];
        gS[3] += P.T[1] * GT[1] + P.T[4] * GT[4];
        gS[4] += P.T[1] * GT[2] + P.T[4] * GT[5];
        gS[5] += P.T[2] * GT[2] + P.T[5] * GT[5];
        // dL/dT = 2 G2 T Sigma, then dL/dJ = dL/dT W^T (only J00, J02, J11, J12 vary)
        float gT[6];
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int j = 0; j < 3; j++)
                gT[3 * i + j] = 2.f * (GT[3 * i] * sig_at(G.Sig, 0, j) + GT[3 * i + 1] * sig_at(G.Sig, 1, j) +
                                       GT[3 * i + 2] * sig_at(G.Sig, 2, j));
        const float gJ00 = gT[0] * cam.R[0] + gT[1] * cam.R[1] + gT[2] * cam.R[2];
        const float gJ02 = gT[0] * cam.R[6] + gT[1] * cam.R[7] + gT[2] * cam.R[8];
        const float gJ11 = gT[3] * cam.R[3] + gT[4] * cam.R[4] + gT[5] * cam.R[5];
        const float gJ12 = gT[3] * cam.R[6] + gT[4] * cam.R[7] + gT[5] * cam.R[8];
        const float tz = P.t[2], iz = 1.f / tz, iz2 = iz * iz;
        float gt0 = 0.f, gt1 = 0.f, gt2 = 0.f;
        gt2 += -(gJ00 * cam.fx + gJ11 * cam.fy) * iz2;
        // J02 = -fx * clamp(tx/tz) / tz: unclamped -fx tx / tz^2, clamped -fx (+-lim) / tz
        if (P.clx == 0) {
            gt0 += -gJ02 * cam.fx * iz2;
            gt2 += 2.f * gJ02 * cam.fx * P.ux * iz2;
        } else {
            gt2 += gJ02 * cam.fx * (P.clx * cam.limx) * iz2;
        }
        if (P.cly == 0) {
            gt1 += -gJ12 * cam.fy * iz2;
            gt2 += 2.f * gJ12 * cam.fy * P.uy * iz2;
        } else {
            gt2 += gJ12 * cam.fy * (P.cly * cam.limy) * iz2;
        }
        // mean2d = (fx tx / tz + cx, fy ty / tz + cy)
        gt0 += gx * cam.fx * iz;
        gt1 += gy * cam.fy * iz;
        gt2 += -(gx * cam.fx * P.ux + gy * cam.fy * P.uy) * iz;
#pragma unroll
        for (int j = 0; j < 3; j++) gmu[j] += cam.R[j] * gt0 + cam.R[3 + j] * gt1 + cam.R[6 + j] * gt2;
        // colour: rgb = sum_k Y_k(dir) sh_k + 0.5, clamped at 0
        const int cm = rec.clamp[r];
        float grgb[3];
#pragma unroll
        for (int ch = 0; ch < 3; ch++) grgb[ch] = (cm >> ch) & 1 ? 0.f : grgb_raw[ch];
        float dx = G.mu[0] - cam.campos[0], dy = G.mu[1] - cam.campos[1], dz = G.mu[2] - cam.campos[2];
        const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
        dx *= il; dy *= il; dz *= il;
        float Y[NK];
        sh_basis<DEG>(dx, dy, dz, Y);
        float wk[NK];
#pragma unroll
        for (int k = 0; k < NK; k++) {
            wk[k] = 0.f;
#pragma unroll
            for (int ch = 0; ch < 3; ch++) gsh[3 * k + ch] += Y[k] * grgb[ch];
        }
#pragma unroll
        for (int e = 0; e < NK * 3; e++) wk[e / 3] += shc[e * 128] * grgb[e % 3];
        const float3 gd = sh_basis_grad<DEG>(dx, dy, dz, wk);
        const float dd = gd.x * dx + gd.y * dy + gd.z * dz;
        gmu[0] += (gd.x - dx * dd) * il;
        gmu[1] += (gd.y - dy * dd) * il;
        gmu[2] += (gd.z - dz * dd) * il;
        go += gop;
    }
#pragma unroll
    for (int j = 0; j < 3; j++) g_means[3 * g + j] = gmu[j];
    g_logits[g] = go * G.o * (1.f - G.o);
    float* gshg = g_sh + (size_t)g * NK * 3;
    if constexpr ((NK * 3) % 4 == 0) {
        if ((reinterpret_cast<uintptr_t>(g_sh) & 15) == 0) {
#pragma unroll
            for (int q = 0; q < NK * 3 / 4; q++)
                reinterpret_cast<float4*>(gshg)[q] = make_float4(gsh[4 * q], gsh[4 * q + 1], gsh[4 * q + 2], gsh[4 * q + 3]);
        } else {
#pragma unroll
            for (int i = 0; i < NK * 3; i++) gshg[i] = gsh[i];
        }
    } else {
#pragma unroll
        for (int i = 0; i < NK * 3; i++) gshg[i] = gsh[i];
    }
    // Sigma = M M^T, M = R diag(s): dL/dM = 2 dL/dSigma M
    float gM[9];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            gM[3 * i + j] = 2.f * (sig_at(gS, i, 0) * G.M[j] + sig_at(gS, i, 1) * G.M[3 + j] +
                                   sig_at(gS, i, 2) * G.M[6 + j]);
    float gR[9];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const float gs = gM[j] * G.R[j] + gM[3 + j] * G.R[3 + j] + gM[6 + j] * G.R[6 + j];
        g_log_scales[3 * g + j] = gs * G.s[j];
#pragma unroll
        for (int i = 0; i < 3; i++) gR[3 * i + j] = gM[3 * i + j] * G.s[j];
    }
    const float w = G.q[0], x = G.q[1], y = G.q[2], z = G.q[3];
    float gq[4];
    gq[0] = 2.f * (-z * gR[1] + y * gR[2] + z * gR[3] - x * gR[5] - y * gR[6] + x * gR[7]);
    gq[1] = 2.f * (y * gR[1] + z * gR[2] + y * gR[3] - 2.f * x * gR[4] - w * gR[5] + z * gR[6] + w * gR[7] -
                   2.f * x * gR[8]);
    gq[2] = 2.f * (-2.f * y * gR[0] + x * gR[1] + w * gR[2] + x * gR[3] + z * gR[5] - w * gR[6] + z * gR[7] -
                   2.f * y * gR[8]);
    gq[3] = 2.f * (-2.f * z * gR[0] - w * gR[1] + x * gR[2] + w * gR[3] - 2.f * z * gR[4] + y * gR[5] + x * gR[6] +
                   y * gR[7]);
    const float dq = gq[0] * w + gq[1] * x + gq[2] * y + gq[3] * z;
    const float iq = 1.f / G.qnorm;
    *reinterpret_cast<float4*>(g_quats + 4 * g) =
        make_float4((gq[0] - w * dq) * iq, (gq[1] - x * dq) * iq, (gq[2] - y * dq) * iq, (gq[3] - z * dq) * iq);
}

// E_1 (norm per pixel, then add) and E_2 (add per view, then norm) of
// Sec. 5.2.2, accumulated over calls; one thread per Gaussian.
__global__ void adc_kernel(const long long* __restrict__ rec_off, const long long* __restrict__ rec_count, long long n,
                           const float* __restrict__ g_mean2d, const float* __restrict__ e1,
                           float* __restrict__ acc_e1, float* __restrict__ acc_e2, float* __restrict__ denom) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const long long rc = *rec_count;
    const long long r0 = min(rec_off[g], rc), r1 = min(rec_off[g + 1], rc);
    float s1 = 0.f, s2 = 0.f;
    for (long long r = r0; r < r1; r++) {
        const float2 m = *reinterpret_cast<const float2*>(g_mean2d + 2 * r);
        s1 += e1[r];
        s2 += sqrtf(m.x * m.x + m.y * m.y);
    }
    acc_e1[g] += s1;
    acc_e2[g] += s2;
    denom[g] += (float)(r1 - r0);
}

unsigned blocks_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

void upload_cams(const DevCam* host, int V, DevCam* dst, cudaStream_t s) {
    for (int start = 0; start < V; start += kCamChunk) {
        CamChunk chunk;
        const int cnt = V - start < kCamChunk ? V - start : kCamChunk;
        for (int i = 0; i < cnt; i++) chunk.c[i] = host[start + i];
        upload_cams_kernel<<<1, kCamChunk, 0, s>>>(chunk, cnt, dst + start);
        note_launches(1);
    }
}

void launch_count_keys(const SceneArgs& sc, const DevCam* cams, int V, int tw, int th, int* recs, uint32_t* keys,
                       cudaStream_t s) {
    if (sc.n == 0) return;
    count_keys_kernel<<<blocks_for(sc.n, 256), 256, 0, s>>>(sc, cams, V, tw, th, recs, keys);
    note_launches(1);
}

void launch_count_visible(const SceneArgs& sc, const DevCam* cams, int V, int tw, int th, int* counts,
                          uint8_t* vis, cudaStream_t s) {
    if (sc.n == 0) return;
    count_visible_kernel<<<blocks_for(sc.n, 256), 256, 0, s>>>(sc, cams, V, tw, th, counts, vis);
    note_launches(1);
}

void launch_preprocess(const SceneArgs& sc, const DevCam* cams, int V, int tw, int th, const uint8_t* vis,
                       const RecordArgs& rec, uint32_t* tiles_touched, unsigned long long* tile_desc,
                       cudaStream_t s) {
    if (sc.n == 0) return;
    const long long gpw = V < 32 ? 32 / V : 1;  // Gaussians per warp
    const long long warps = (sc.n + gpw - 1) / gpw;
    const unsigned nb = (unsigned)((warps + PRE_THREADS / 32 - 1) / (PRE_THREADS / 32));
#define MVGS_PP(D) \
    preprocess_kernel<D><<<nb, PRE_THREADS, 0, s>>>(sc, cams, V, tw, th, vis, rec, tiles_touched, tile_desc)
    switch (sc.sh_degree) {
        case 0: MVGS_PP(0); break;
        case 1: MVGS_PP(1); break;
        case 2: MVGS_PP(2); break;
        default: MVGS_PP(3); break;
    }
#undef MVGS_PP
    note_launches(1);
}

void launch_zero_f32(float* p, size_t count, cudaStream_t s) {
    // the runtime's fill: 6.6 TB/s on the per-record gradient slots (1.5 GB at
    // 3M x 8 views), against 5.0 TB/s for a grid of float4 stores
    if (count == 0) return;
    cudaMemsetAsync(p, 0, count * sizeof(float), s);
}

void launch_preprocess_backward(const SceneArgs& sc, const DevCam* cams, int V, const RecordArgs& rec,
                                const float* rec_grad, const double* rec_conic, float* g_means,
                                float* g_log_scales, float* g_quats, float* g_logits, float* g_sh, float* out_mean2d,
                                float* out_e1, cudaStream_t s) {
    (void)V;
    if (sc.n == 0) return;
    const unsigned nb = blocks_for(sc.n, 128);
#define MVGS_PB(D)                                                                                                 \
    preprocess_backward_kernel<D><<<nb, 128, 0, s>>>(sc, cams, rec, rec_grad, rec_conic, g_means, g_log_scales,    \
                                                     g_quats, g_logits, g_sh, out_mean2d, out_e1)
    switch (sc.sh_degree) {
        case 0: MVGS_PB(0); break;
        case 1: MVGS_PB(1); break;
        case 2: MVGS_PB(2); break;
        default: MVGS_PB(3); break;
    }
    note_launches(1);
#undef MVGS_PB
}

void launch_adc_accumulate(const long long* rec_off, const long long* rec_count, long long n, const float* g_mean2d,
                           const float* e1, float* accum_e1, float* accum_e2, float* denom, cudaStream_t s) {
    if (n == 0) return;
    adc_kernel<<<blocks_for(n, 256), 256, 0, s>>>(rec_off, rec_count, n, g_mean2d, e1, accum_e1, accum_e2, denom);
    note_launches(1);
}

}  // namespace mvgs
