// Training-loop pieces around the rasterizer: the multi-view densification
// step (Sec. 5.2.2; supplement "Experiment details") and a fused Adam update.
//
// Densification decides every Gaussian on its own, in double precision from
// the float32 inputs (so the decision is exact and reproducible):
//   mean E_k = accum_E_k / denom (0 where denom = 0);
//   large    = max_i log_scale_i > log_dense_extent;
//   pruned   = logit < prune_logit (the opacity threshold, multiplied by the
//              views per iteration, in logit space);
//   split    = !pruned && large && mean E_1 >= split_threshold;
//   cloned   = !pruned && !large && mean E_2 >= clone_threshold;
// outputs, ordered by source Gaussian: none if pruned; two children if split
// (mean mu + R(q)(s * z_k) with the caller's standard normal samples z,
// log-scale - ln 1.6, the rest copied); the Gaussian and a copy if cloned;
// else the Gaussian.  Kind per output: 0 the Gaussian itself, 1 a copy, 2 a
// split child; carried per-Gaussian arrays (optimiser moments) are copied for
// kind 0 and zeroed for kinds 1 and 2.
//
// Adam (Kingma & Ba, ICLR 2015) with bias correction, one read and one write
// of parameter, gradient and both moments per element.
#include "kernels.h"

namespace mvgs {
namespace {

__global__ void densify_count_kernel(DensifyArgs a, int* __restrict__ counts) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.n) return;
    const double den = (double)a.denom[g];
    const double m1 = den > 0.0 ? (double)a.e1[g] / den : 0.0;
    const double m2 = den > 0.0 ? (double)a.e2[g] / den : 0.0;
    const float* ls = a.log_scales + 3 * g;
    const double mx = (double)fmaxf(ls[0], fmaxf(ls[1], ls[2]));
    const bool large = mx > a.log_dense_extent;
    const bool pruned = (double)a.logits[g] < a.prune_logit;
    const bool split = !pruned && large && m1 >= a.split_threshold;
    const bool cloned = !pruned && !large && m2 >= a.clone_threshold;
    counts[g] = pruned ? 0 : ((split || cloned) ? 2 : 1) | (split ? 4 : 0);
}

// counts carry the split bit (4) next to the output count (bits 0-1); the
// scan reads the count through the mask 3
__global__ void densify_write_kernel(DensifyArgs a, const int* __restrict__ counts,
                                     const long long* __restrict__ off, DensifyOut o) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.n) return;
    const int c = counts[g];
    const int cnt = c & 3;
    if (cnt == 0) return;
    const bool split = (c & 4) != 0;
    const long long d0 = off[g];
    float q[4];
    float nq = 0.f;
    for (int i = 0; i < 4; i++) {
        q[i] = a.quats[4 * g + i];
        nq += q[i] * q[i];
    }
    const float inv = rsqrtf(nq);
    const float w = q[0] * inv, x = q[1] * inv, y = q[2] * inv, z = q[3] * inv;
    const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                        2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                        2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
    for (int k = 0; k < cnt; k++) {
        const long long d = d0 + k;
        const int kind = split ? 2 : k;  // cloned: the Gaussian (0), then its copy (1)
        if (o.src) o.src[d] = g;
        if (o.kind) o.kind[d] = kind;
        for (int i = 0; i < 3; i++) {
            float m = a.means[3 * g + i];
            float l = a.log_scales[3 * g + i];
            if (split) {
                float off_i = 0.f;
                for (int j = 0; j < 3; j++)
                    off_i += R[3 * i + j] * (expf(a.log_scales[3 * g + j]) * a.normals[6 * g + 3 * k + j]);
                m += off_i;
                l -= kLogSplitDiv;
            }
            o.means[3 * d + i] = m;
            o.log_scales[3 * d + i] = l;
        }
        for (int i = 0; i < 4; i++) o.quats[4 * d + i] = a.quats[4 * g + i];
        o.logits[d] = a.logits[g];
        for (int i = 0; i < a.nk; i++) o.sh[(long long)a.nk * d + i] = a.sh[(long long)a.nk * g + i];
    }
}

__global__ void carry_kernel(long long n_out, const long long* __restrict__ src, const int* __restrict__ kind,
                             int width, const float* __restrict__ in, float* __restrict__ out) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_out * width) return;
    const long long d = e / width;
    const int i = (int)(e % width);
    out[e] = kind[d] == 0 ? in[src[d] * width + i] : 0.f;
}

__global__ void adam_kernel(long long count, float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        // p -= lr * (m / c1) / (sqrt(v / c2) + eps), c_k = 1 - beta_k^t
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// The same update on float4 vectors (count4 = count / 4, all pointers 16-byte
// aligned); the caller handles a tail of count % 4 elements with adam_kernel.
__device__ __forceinline__ void adam1(float& p, float g, float& m, float& v, float lr, float b1, float b2, float eps,
                                      float c1, float c2) {
    m = b1 * m + (1.f - b1) * g;
    v = b2 * v + (1.f - b2) * g * g;
    p -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

__global__ void adam4_kernel(long long count4, float4* __restrict__ p, const float4* __restrict__ g,
                             float4* __restrict__ m, float4* __restrict__ v, float lr, float b1, float b2, float eps,
                             float c1, float c2) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count4;
         i += (long long)gridDim.x * blockDim.x) {
        float4 pp = p[i], mm = m[i], vv = v[i];
        const float4 gg = g[i];
        adam1(pp.x, gg.x, mm.x, vv.x, lr, b1, b2, eps, c1, c2);
        adam1(pp.y, gg.y, mm.y, vv.y, lr, b1, b2, eps, c1, c2);
        adam1(pp.z, gg.z, mm.z, vv.z, lr, b1, b2, eps, c1, c2);
        adam1(pp.w, gg.w, mm.w, vv.w, lr, b1, b2, eps, c1, c2);
        p[i] = pp;
        m[i] = mm;
        v[i] = vv;
    }
}

}  // namespace

size_t densify_temp_bytes(long long n) {
    const size_t a = ((size_t)(n > 0 ? n : 1) * sizeof(int) + 255) / 256 * 256;
    const size_t b = ((size_t)(n + 1) * sizeof(long long) + 255) / 256 * 256;
    return a + b + scan_temp_bytes((uint64_t)(n > 0 ? n : 1));
}

// Pass 1: decisions and output offsets; returns the device pointer of the
// output count (off[n]).
const long long* launch_densify_plan(const DensifyArgs& a, void* tmp, cudaStream_t s) {
    char* base = static_cast<char*>(tmp);
    int* counts = reinterpret_cast<int*>(base);
    base += ((size_t)(a.n > 0 ? a.n : 1) * sizeof(int) + 255) / 256 * 256;
    long long* off = reinterpret_cast<long long*>(base);
    base += ((size_t)(a.n + 1) * sizeof(long long) + 255) / 256 * 256;
    if (a.n > 0) {
        densify_count_kernel<<<(unsigned)((a.n + 255) / 256), 256, 0, s>>>(a, counts);
        note_launches(1);
    }
    scan_masked_i32_to_i64(counts, 3, off, (uint64_t)a.n, base, s);
    return off + a.n;
}

void launch_densify_write(const DensifyArgs& a, const DensifyOut& o, void* tmp, cudaStream_t s) {
    if (a.n <= 0) return;
    char* base = static_cast<char*>(tmp);
    const int* counts = reinterpret_cast<const int*>(base);
    base += ((size_t)a.n * sizeof(int) + 255) / 256 * 256;
    const long long* off = reinterpret_cast<const long long*>(base);
    densify_write_kernel<<<(unsigned)((a.n + 255) / 256), 256, 0, s>>>(a, counts, off, o);
    note_launches(1);
}

void launch_carry(long long n_out, const long long* src, const int* kind, int width, const float* in, float* out,
                  cudaStream_t s) {
    const long long total = n_out * width;
    if (total <= 0) return;
    carry_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(n_out, src, kind, width, in, out);
    note_launches(1);
}

void launch_adam(long long count, float* p, const float* g, float* m, float* v, float lr, float b1, float b2,
                 float eps, int step, cudaStream_t s) {
    if (count <= 0) return;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    const bool aligned = ((reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(g) |
                           reinterpret_cast<uintptr_t>(m) | reinterpret_cast<uintptr_t>(v)) & 15) == 0;
    long long head = 0;
    if (aligned && count >= 4) {
        const long long c4 = count / 4;
        long long blocks = (c4 + 255) / 256;
        if (blocks > 152 * 8) blocks = 152 * 8;
        adam4_kernel<<<(unsigned)blocks, 256, 0, s>>>(c4, reinterpret_cast<float4*>(p),
                                                      reinterpret_cast<const float4*>(g),
                                                      reinterpret_cast<float4*>(m), reinterpret_cast<float4*>(v),
                                                      lr, b1, b2, eps, c1, c2);
        note_launches(1);
        head = 4 * c4;
    }
    if (head < count) {
        long long blocks = (count - head + 255) / 256;
        if (blocks > 152 * 16) blocks = 152 * 16;
        adam_kernel<<<(unsigned)blocks, 256, 0, s>>>(count - head, p + head, g + head, m + head, v + head, lr, b1,
                                                     b2, eps, c1, c2);
        note_launches(1);
    }
}

}  // namespace mvgs
