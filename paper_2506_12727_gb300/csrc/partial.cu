// Pixel samples for thread-efficient partial rendering (Sec. 5.1.1, Alg. 3).
//
// The paper sub-samples, for every tile, the pixels each viewpoint renders and
// hands the rasterizer an index array per (tile, viewpoint).  The selection
// rule is not given; here view v renders pixel (x, y) when its cell
// (cx, cy) = (x / cell_w, y / cell_h) has
//     slot(cx, cy) = floor(group * (h >> 32) / 2^32) == v mod group,
//     h = SplitMix64 output number (2^32 cy + cx + 1) of the stream seeded
//         with `seed` (Steele, Lea & Flood, OOPSLA 2014)
// (1 x 1 cells: pixel by pixel; cells of a warp's strip keep the samples of a
// run together),
// so views v, v + group, ... take the same pixels and, for views of one
// resolution, any `group` consecutive views split every pixel position
// between them exactly once (the merged image of Fig. 3c).  Each tile's
// samples are stored in raster order as CSR: s_off[t] .. s_off[t + 1] index
// s_pix, the pixel index ly * tile_w + lx inside the tile.
#include "kernels.h"

namespace mvgs {
namespace {

__device__ __forceinline__ bool sampled(unsigned long long seed, int x, int y, int group, int cw, int ch, int v) {
    return sample_slot(seed, x / cw, y / ch, group) == v % group;
}

struct TileGeom {
    int v, x0, y0, w, h;  // view, pixel origin, extent inside the image
};

__device__ __forceinline__ TileGeom tile_geom(const DevCam* cams, int V, long long gt, int tw, int th) {
    TileGeom g;
    g.v = find_view(cams, V, gt);
    const DevCam& c = cams[g.v];
    const long long local = gt - c.tile_base;
    g.x0 = (int)(local % c.tiles_x) * tw;
    g.y0 = (int)(local / c.tiles_x) * th;
    g.w = min(tw, c.W - g.x0);
    g.h = min(th, c.H - g.y0);
    return g;
}

// One block per tile: number of samples.
__global__ void sample_count_kernel(const DevCam* __restrict__ cams, int V, int tw, int th, int group, int cw, int ch,
                                    unsigned long long seed, int* __restrict__ counts) {
    const long long gt = blockIdx.x;
    const TileGeom g = tile_geom(cams, V, gt, tw, th);
    int n = 0;
    for (int i = threadIdx.x; i < tw * th; i += blockDim.x) {
        const int lx = i % tw, ly = i / tw;
        if (lx < g.w && ly < g.h && sampled(seed, g.x0 + lx, g.y0 + ly, group, cw, ch, g.v)) n++;
    }
    __shared__ int warp_n[32];
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0) warp_n[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += warp_n[w];
        counts[gt] = t;
    }
}

// One block per tile: the samples in raster order.
__global__ void sample_fill_kernel(const DevCam* __restrict__ cams, int V, int tw, int th, int group, int cw, int ch,
                                   unsigned long long seed, const long long* __restrict__ s_off,
                                   uint16_t* __restrict__ s_pix) {
    const long long gt = blockIdx.x;
    const TileGeom g = tile_geom(cams, V, gt, tw, th);
    __shared__ int warp_n[32];
    __shared__ int base;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    long long out = s_off[gt];
    for (int i0 = 0; i0 < tw * th; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        const int lx = i % tw, ly = i / tw;
        const bool take =
            i < tw * th && lx < g.w && ly < g.h && sampled(seed, g.x0 + lx, g.y0 + ly, group, cw, ch, g.v);
        const unsigned bal = __ballot_sync(0xffffffffu, take);
        if (lane == 0) warp_n[w] = __popc(bal);
        __syncthreads();
        int before = base;
        for (int u = 0; u < w; u++) before += warp_n[u];
        if (take) s_pix[out + before + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)i;
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int u = 0; u < nw; u++) t += warp_n[u];
            base += t;
        }
        __syncthreads();
    }
}

// Runs of `run` samples per tile, counted in the blend's tile order.
__global__ void chunk_count_kernel(const uint32_t* __restrict__ order, const long long* __restrict__ s_off,
                                   long long tiles, int run, int* __restrict__ counts) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= tiles) return;
    const uint32_t t = order[i];
    const long long n = s_off[t + 1] - s_off[t];
    counts[i] = (int)((n + run - 1) / run);
}

__global__ void chunk_map_kernel(const long long* __restrict__ chunk_off, long long tiles, long long cap,
                                 int* __restrict__ map) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= tiles) return;
    const long long e = chunk_off[i + 1] < cap ? chunk_off[i + 1] : cap;
    for (long long c = chunk_off[i]; c < e; c++) map[c] = (int)i;
}

__global__ void samples_to_mask_kernel(const DevCam* __restrict__ cams, int V, int tw, int th,
                                       const long long* __restrict__ s_off, const uint16_t* __restrict__ s_pix,
                                       uint8_t* __restrict__ mask) {
    const long long gt = blockIdx.x;
    const TileGeom g = tile_geom(cams, V, gt, tw, th);
    const DevCam& c = cams[g.v];
    const long long e = s_off[gt + 1];
    for (long long i = s_off[gt] + threadIdx.x; i < e; i += blockDim.x) {
        const int li = s_pix[i];
        const int lx = li % tw, ly = li / tw;
        if (lx < g.w && ly < g.h) mask[c.pix_base + (long long)(g.y0 + ly) * c.W + g.x0 + lx] = 1;
    }
}

}  // namespace
}  // namespace mvgs

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
namespace mvgs {

size_t sample_temp_bytes(long long tiles) {
    return ((size_t)(tiles > 0 ? tiles : 1) * sizeof(int) + 255) / 256 * 256 + scan_temp_bytes((uint64_t)tiles);
}

void launch_partial_samples(const DevCam* cams, int V, long long tiles, int tw, int th, int group, int cw, int ch,
                            unsigned long long seed, long long* s_off, uint16_t* s_pix, void* tmp, cudaStream_t s) {
    if (tiles <= 0) return;
    int* counts = static_cast<int*>(tmp);
    void* scan_tmp = static_cast<char*>(tmp) + ((size_t)tiles * sizeof(int) + 255) / 256 * 256;
    sample_count_kernel<<<(unsigned)tiles, 256, 0, s>>>(cams, V, tw, th, group, cw, ch, seed, counts);
    scan_i32_to_i64(counts, s_off, (uint64_t)tiles, scan_tmp, s);
    sample_fill_kernel<<<(unsigned)tiles, 256, 0, s>>>(cams, V, tw, th, group, cw, ch, seed, s_off, s_pix);
    note_launches(2);
}

size_t chunk_temp_bytes(long long tiles) { return sample_temp_bytes(tiles); }

void launch_sample_chunks(const uint32_t* order, const long long* s_off, long long tiles, int run,
                          long long* chunk_off, int* chunk_map, long long map_cap, void* tmp, cudaStream_t s) {
    if (tiles <= 0) return;
    int* counts = static_cast<int*>(tmp);
    void* scan_tmp = static_cast<char*>(tmp) + ((size_t)tiles * sizeof(int) + 255) / 256 * 256;
    const unsigned blocks = (unsigned)((tiles + 255) / 256);
    chunk_count_kernel<<<blocks, 256, 0, s>>>(order, s_off, tiles, run, counts);
    scan_i32_to_i64(counts, chunk_off, (uint64_t)tiles, scan_tmp, s);
    chunk_map_kernel<<<blocks, 256, 0, s>>>(chunk_off, tiles, map_cap, chunk_map);
    note_launches(2);
}

void launch_samples_to_mask(const DevCam* cams, int V, long long tiles, long long pixels, int tw, int th,
                            const long long* s_off, const uint16_t* s_pix, uint8_t* mask, cudaStream_t s) {
    if (tiles <= 0) return;
    cudaMemsetAsync(mask, 0, (size_t)pixels, s);
    samples_to_mask_kernel<<<(unsigned)tiles, 256, 0, s>>>(cams, V, tw, th, s_off, s_pix, mask);
    note_launches(1);
}

}  // namespace mvgs
