// Key duplication, exclusive scans, stable LSD radix sort and tile ranges.
//
// The supplement ("Rasterization in multi-view training") sorts duplicated
// (tile, viewpoint, depth) keys so each (tile, view) list is depth ordered.
// Here the same order is reached in two cheaper sorts: the visible records
// are first sorted by depth (32-bit keys, one entry per record), then
// duplicated per covered tile in that order, and the duplicated entries are
// sorted stably on the global (view, tile) id alone -- ceil(log2(tiles)) bits
// instead of 32 + that.  Stability keeps depth order, and equal depths keep
// the record order, which is Gaussian-major, so ties inside a tile list are
// broken by Gaussian index.
#include "kernels.h"

namespace mvgs {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// exclusive scan (reduce, spine, downsweep)
// ---------------------------------------------------------------------------
constexpr int SC_THREADS = 256;
constexpr int SC_ITEMS = 16;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;
constexpr int SPINE_THREADS = 1024;

// Exclusive scan across the block of one value per thread.  `buf` holds
// at least 33 elements of shared memory.  Returns the thread's exclusive
// prefix and the block total.
template <class T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* buf, T& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) buf[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? buf[lane] : T(0);
        T wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(kFull, wi, o);
            if (lane >= o) wi += y;
        }
        buf[lane] = wi - w;
        if (lane == 31) buf[32] = wi;
    }
    __syncthreads();
    T res = inc - v + buf[warp];
    total = buf[32];
    __syncthreads();
    return res;
}

template <class Tin, class Tout>
struct LoadDirect {
    const Tin* in;
    __device__ __forceinline__ Tout operator()(uint64_t i) const { return (Tout)in[i]; }
};

template <class Tout>
struct LoadGather {
    const uint32_t* in;
    const uint32_t* idx;
    __device__ __forceinline__ Tout operator()(uint64_t i) const { return (Tout)in[idx[i]]; }
};

template <class Load, class T>
__global__ void __launch_bounds__(SC_THREADS) scan_reduce_kernel(Load ld, uint64_t n, T* partials) {
    __shared__ T buf[33];
    const uint64_t base = (uint64_t)blockIdx.x * SC_TILE;
    T s = 0;
#pragma unroll 4
    for (int i = threadIdx.x; i < SC_TILE; i += SC_THREADS) {
        const uint64_t idx = base + i;
        if (idx < n) s += ld(idx);
    }
    T total;
    block_exclusive_scan<T>(s, buf, total);
    if (threadIdx.x == 0) partials[blockIdx.x] = total;
}

template <class T>
__global__ void __launch_bounds__(SPINE_THREADS) scan_spine_kernel(T* partials, uint64_t nb, T* total_out) {
    __shared__ T buf[33];
    T carry = 0;
    for (uint64_t start = 0; start < nb; start += SPINE_THREADS) {
        const uint64_t i = start + threadIdx.x;
        const T v = i < nb ? partials[i] : T(0);
        T tot;
        const T ex = block_exclusive_scan<T>(v, buf, tot);
        if (i < nb) partials[i] = ex + carry;
        carry += tot;
    }
    if (threadIdx.x == 0 && total_out) *total_out = carry;
}

__device__ __forceinline__ int pad_index(int i) { return i + (i >> 5); }

template <class Load, class T>
__global__ void __launch_bounds__(SC_THREADS) scan_down_kernel(Load ld, uint64_t n, const T* partials, T* out) {
    __shared__ T tile[SC_TILE + SC_TILE / 32];
    __shared__ T buf[33];
    const uint64_t base = (uint64_t)blockIdx.x * SC_TILE;
    for (int i = threadIdx.x; i < SC_TILE; i += SC_THREADS) {
        const uint64_t idx = base + i;
        tile[pad_index(i)] = idx < n ? ld(idx) : T(0);
    }
    __syncthreads();
    T local[SC_ITEMS];
    T sum = 0;
#pragma unroll
    for (int k = 0; k < SC_ITEMS; k++) {
        local[k] = tile[pad_index(threadIdx.x * SC_ITEMS + k)];
        sum += local[k];
    }
    T total;
    T run = block_exclusive_scan<T>(sum, buf, total) + partials[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SC_ITEMS; k++) {
        tile[pad_index(threadIdx.x * SC_ITEMS + k)] = run;
        run += local[k];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SC_TILE; i += SC_THREADS) {
        const uint64_t idx = base + i;
        if (idx < n) out[idx] = tile[pad_index(i)];
    }
}

uint64_t ceil_div_u64(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

template <class Load, class T>
void scan_impl(Load ld, T* out, uint64_t n, T* total_out, void* tmp, cudaStream_t s) {
    if (n == 0) {
        if (total_out) cudaMemsetAsync(total_out, 0, sizeof(T), s);
        return;
    }
    const uint64_t nb = ceil_div_u64(n, SC_TILE);
    T* partials = static_cast<T*>(tmp);
    scan_reduce_kernel<Load, T><<<(unsigned)nb, SC_THREADS, 0, s>>>(ld, n, partials);
    scan_spine_kernel<T><<<1, SPINE_THREADS, 0, s>>>(partials, nb, total_out);
    scan_down_kernel<Load, T><<<(unsigned)nb, SC_THREADS, 0, s>>>(ld, n, partials, out);
    note_launches(3);
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of (uint32 key, uint32 value), 8-bit digits
// ---------------------------------------------------------------------------
constexpr int RS_THREADS = 256;  // == number of digit values
constexpr int RS_ITEMS = 16;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_SEG = RS_ITEMS * 32;  // contiguous keys per warp
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

// Per-block digit histogram, stored digit-major so that one exclusive scan of
// the whole table gives every block's first output position per digit.
__global__ void __launch_bounds__(RS_THREADS) rs_upsweep(const uint32_t* __restrict__ keys, uint64_t n, int shift,
                                                        uint32_t* __restrict__ counts, uint32_t nblocks) {
    __shared__ uint32_t hist[RS_WARPS * 256];
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) hist[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t base = (uint64_t)blockIdx.x * RS_TILE + warp * RS_SEG + lane;
#pragma unroll
    for (int j = 0; j < RS_ITEMS; j++) {
        const uint64_t idx = base + (uint64_t)j * 32;
        if (idx < n) atomicAdd(&hist[warp * 256 + ((keys[idx] >> shift) & 0xffu)], 1u);
    }
    __syncthreads();
    uint32_t sum = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; w++) sum += hist[w * 256 + threadIdx.x];
    counts[(uint64_t)threadIdx.x * nblocks + blockIdx.x] = sum;
}

// Stable scatter.  Warp w ranks the keys of its contiguous segment in index
// order (32 per round, lanes in order); equal digits inside a round are found
// with one ballot per digit bit.  Warps are then offset by the counts of the
// warps before them, and the block by the scanned table.
__global__ void __launch_bounds__(RS_THREADS) rs_downsweep(const uint32_t* __restrict__ kin,
                                                          const uint32_t* __restrict__ vin,
                                                          uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                          uint64_t n, int shift, const uint32_t* __restrict__ offsets,
                                                          uint32_t nblocks) {
    __shared__ uint32_t whist[RS_WARPS * 256];
    __shared__ uint32_t boff[256];
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) whist[i] = 0;
    boff[threadIdx.x] = offsets[(uint64_t)threadIdx.x * nblocks + blockIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const uint64_t base = (uint64_t)blockIdx.x * RS_TILE + warp * RS_SEG + lane;
    uint32_t k[RS_ITEMS], v[RS_ITEMS], lr[RS_ITEMS];
#pragma unroll
    for (int j = 0; j < RS_ITEMS; j++) {
        const uint64_t idx = base + (uint64_t)j * 32;
        const bool ok = idx < n;
        k[j] = ok ? kin[idx] : 0u;
        v[j] = ok ? vin[idx] : 0u;
    }
    uint32_t* wh = whist + warp * 256;
#pragma unroll
    for (int j = 0; j < RS_ITEMS; j++) {
        const bool ok = base + (uint64_t)j * 32 < n;
        const uint32_t d = (k[j] >> shift) & 0xffu;
        uint32_t peers = __ballot_sync(kFull, ok);
#pragma unroll
        for (int b = 0; b < 8; b++) {
            const uint32_t bit = (d >> b) & 1u;
            const uint32_t bb = __ballot_sync(kFull, bit);
            peers &= bit ? bb : ~bb;
        }
        const uint32_t rank = __popc(peers & lt);
        const uint32_t before = wh[d];
        __syncwarp();
        if (ok && rank == 0) wh[d] = before + __popc(peers);
        __syncwarp();
        lr[j] = before + rank;
    }
    __syncthreads();
    {
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; w++) {
            const uint32_t c = whist[w * 256 + threadIdx.x];
            whist[w * 256 + threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < RS_ITEMS; j++) {
        if (base + (uint64_t)j * 32 < n) {
            const uint32_t d = (k[j] >> shift) & 0xffu;
            const uint32_t pos = boff[d] + wh[d] + lr[j];
            kout[pos] = k[j];
            vout[pos] = v[j];
        }
    }
}

// ---------------------------------------------------------------------------
// duplication and tile ranges
// ---------------------------------------------------------------------------
constexpr int DUP_THREADS = 256;
constexpr int DUP_CHUNK = 2048;

// Block b emits keys [b*CHUNK, (b+1)*CHUNK).  Each key finds its record by
// a binary search over the (shared-memory) offsets of the records that cover
// the chunk; consecutive threads write consecutive keys.
__global__ void __launch_bounds__(DUP_THREADS) duplicate_kernel(const uint32_t* __restrict__ order,
                                                               const unsigned long long* __restrict__ off,
                                                               uint64_t R, uint64_t K, const short4* __restrict__ rect,
                                                               const int* __restrict__ rec_v,
                                                               const DevCam* __restrict__ cams, uint32_t tiles,
                                                               uint32_t* __restrict__ keys,
                                                               uint32_t* __restrict__ vals) {
    __shared__ unsigned long long s_off[DUP_CHUNK + 1];
    __shared__ unsigned long long s_lo;
    __shared__ int s_n;
    const uint64_t k0 = (uint64_t)blockIdx.x * DUP_CHUNK;
    const uint64_t k1 = K < k0 + DUP_CHUNK ? K : k0 + DUP_CHUNK;
    if (threadIdx.x == 0) {
        // last record r with off[r] <= k0, then last with off[r] <= k1 - 1
        uint64_t lo = 0, hi = R - 1;
        while (lo < hi) {
            const uint64_t mid = (lo + hi + 1) >> 1;
            if (off[mid] <= k0) lo = mid; else hi = mid - 1;
        }
        uint64_t lo2 = lo;
        hi = R - 1;
        while (lo2 < hi) {
            const uint64_t mid = (lo2 + hi + 1) >> 1;
            if (off[mid] <= k1 - 1) lo2 = mid; else hi = mid - 1;
        }
        s_lo = lo;
        // records with no tile share an offset with the next record, so a
        // chunk can span more records than keys; those chunks search globally
        s_n = lo2 - lo + 1 <= (uint64_t)DUP_CHUNK ? (int)(lo2 - lo + 1) : -1;
    }
    __syncthreads();
    const uint64_t rlo = s_lo;
    const int nr = s_n;
    if (nr > 0) {
        for (int i = threadIdx.x; i <= nr; i += DUP_THREADS) s_off[i] = off[rlo + i];  // off has R + 1 entries
    }
    __syncthreads();
    for (uint64_t k = k0 + threadIdx.x; k < k1; k += DUP_THREADS) {
        uint64_t r;
        unsigned long long first;
        if (nr > 0) {
            int lo = 0, hi = nr - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_off[mid] <= k) lo = mid; else hi = mid - 1;
            }
            r = rlo + lo;
            first = s_off[lo];
        } else {
            uint64_t lo = 0, hi = R - 1;
            while (lo < hi) {
                const uint64_t mid = (lo + hi + 1) >> 1;
                if (off[mid] <= k) lo = mid; else hi = mid - 1;
            }
            r = lo;
            first = off[lo];
        }
        const uint32_t rec = order[r];
        const uint32_t j = (uint32_t)(k - first);
        const short4 rc = rect[rec];
        const uint32_t w = (uint32_t)max(rc.z - rc.x, 1);
        const uint32_t tx = rc.x + j % w, ty = rc.y + j / w;
        const DevCam& cam = cams[rec_v[rec]];
        const long long t = cam.tile_base + (long long)ty * cam.tiles_x + tx;
        keys[k] = (uint32_t)(t < (long long)tiles ? t : (long long)tiles - 1);  // in range even for a bad record
        vals[k] = rec;
    }
}

__global__ void tile_ranges_kernel(const uint32_t* __restrict__ keys, uint64_t K, long long* __restrict__ ranges,
                                   uint32_t tiles) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K) return;
    const uint32_t t = keys[i];
    if (t >= tiles) return;
    if (i == 0 || keys[i - 1] != t) ranges[2 * (uint64_t)t] = (long long)i;
    if (i == K - 1 || keys[i + 1] != t) ranges[2 * (uint64_t)t + 1] = (long long)(i + 1);
}

}  // namespace

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
size_t scan_temp_bytes(uint64_t n) { return (ceil_div_u64(n, SC_TILE) + 1) * sizeof(unsigned long long); }

void scan_i32_to_i64(const int* in, long long* out, uint64_t n, void* tmp, cudaStream_t s) {
    scan_impl(LoadDirect<int, long long>{in}, out, n, out + n, tmp, s);
}

void scan_u32_to_u64(const uint32_t* in, unsigned long long* out, uint64_t n, void* tmp, cudaStream_t s) {
    scan_impl(LoadDirect<uint32_t, unsigned long long>{in}, out, n, out + n, tmp, s);
}

void scan_gather_u32_to_u64(const uint32_t* in, const uint32_t* idx, unsigned long long* out, uint64_t n, void* tmp,
                            cudaStream_t s) {
    scan_impl(LoadGather<unsigned long long>{in, idx}, out, n, out + n, tmp, s);
}

static uint64_t radix_blocks(uint64_t n) { return ceil_div_u64(n, RS_TILE); }

size_t radix_temp_bytes(uint64_t n) {
    const uint64_t nb = radix_blocks(n > 0 ? n : 1);
    const size_t counts = ((256 * nb * sizeof(uint32_t)) + 255) / 256 * 256;
    return counts + scan_temp_bytes(256 * nb);
}

void radix_sort_pairs(uint32_t* keys_a, uint32_t* vals_a, uint32_t* keys_b, uint32_t* vals_b, uint32_t* vals_out,
                      uint32_t** keys_sorted, uint64_t n, int bits, void* tmp, cudaStream_t s) {
    *keys_sorted = keys_a;
    if (n == 0) return;
    const int passes = (bits + 7) / 8;
    if (passes == 0) {
        cudaMemcpyAsync(vals_out, vals_a, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
        return;
    }
    const uint64_t nb = radix_blocks(n);
    uint32_t* counts = static_cast<uint32_t*>(tmp);
    void* scan_tmp = static_cast<char*>(tmp) + ((256 * nb * sizeof(uint32_t)) + 255) / 256 * 256;
    uint32_t *kin = keys_a, *vin = vals_a, *kout = keys_b, *vout = vals_b;
    for (int p = 0; p < passes; p++) {
        if (p == passes - 1) vout = vals_out;
        rs_upsweep<<<(unsigned)nb, RS_THREADS, 0, s>>>(kin, n, 8 * p, counts, (uint32_t)nb);
        scan_impl(LoadDirect<uint32_t, uint32_t>{counts}, counts, 256 * nb, (uint32_t*)nullptr, scan_tmp, s);
        rs_downsweep<<<(unsigned)nb, RS_THREADS, 0, s>>>(kin, vin, kout, vout, n, 8 * p, counts, (uint32_t)nb);
        note_launches(2);
        uint32_t* nk = kin;
        uint32_t* nv = vin;
        kin = kout;
        vin = vout;
        kout = nk;
        vout = (nv == vals_a || nv == vals_b) ? nv : vals_a;
    }
    *keys_sorted = kin;
}

void launch_duplicate(const uint32_t* order, const unsigned long long* tile_off, uint64_t R, uint64_t K,
                      const short4* rect, const int* rec_v, const DevCam* cams, long long tiles, uint32_t* keys,
                      uint32_t* vals, cudaStream_t s) {
    if (K == 0 || R == 0) return;
    duplicate_kernel<<<(unsigned)ceil_div_u64(K, DUP_CHUNK), DUP_THREADS, 0, s>>>(order, tile_off, R, K, rect, rec_v,
                                                                                  cams, (uint32_t)tiles, keys, vals);
    note_launches(1);
}

void launch_tile_ranges(const uint32_t* sorted_keys, uint64_t K, long long* ranges, long long tiles,
                        cudaStream_t s) {
    cudaMemsetAsync(ranges, 0, (size_t)tiles * 2 * sizeof(long long), s);
    if (K == 0) return;
    tile_ranges_kernel<<<(unsigned)ceil_div_u64(K, 256), 256, 0, s>>>(sorted_keys, K, ranges, (uint32_t)tiles);
    note_launches(1);
}

}  // namespace mvgs
