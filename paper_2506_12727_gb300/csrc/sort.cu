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
#include <cstddef>

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

struct LoadMasked {
    const int* in;
    int mask;
    __device__ __forceinline__ long long operator()(uint64_t i) const { return (long long)(in[i] & mask); }
};

template <class Tout>
struct LoadGather {
    const uint32_t* in;
    const uint32_t* idx;
    __device__ __forceinline__ Tout operator()(uint64_t i) const { return (Tout)in[idx[i]]; }
};

template <class Load, class T>
__global__ void __launch_bounds__(SC_THREADS) scan_reduce_kernel(Load ld, Count cn, T* partials) {
    __shared__ T buf[33];
    const uint64_t n = cn.get();
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
__global__ void __launch_bounds__(SPINE_THREADS) scan_spine_kernel(T* partials, uint64_t nb, T* total_out,
                                                                   T* end_out, Count cn) {
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
    if (threadIdx.x == 0 && end_out) end_out[cn.get()] = carry;
}

__device__ __forceinline__ int pad_index(int i) { return i + (i >> 5); }

template <class Load, class T>
__global__ void __launch_bounds__(SC_THREADS) scan_down_kernel(Load ld, Count cn, const T* partials, T* out) {
    __shared__ T tile[SC_TILE + SC_TILE / 32];
    __shared__ T buf[33];
    const uint64_t n = cn.get();
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

// Exclusive scan of ld(0 .. n); the total goes to out[n] when write_end, and
// to *total_out when given.
template <class Load, class T>
void scan_impl(Load ld, T* out, Count n, bool write_end, T* total_out, void* tmp, cudaStream_t s) {
    if (n.max == 0) {
        if (total_out) cudaMemsetAsync(total_out, 0, sizeof(T), s);
        if (write_end) cudaMemsetAsync(out, 0, sizeof(T), s);
        return;
    }
    const uint64_t nb = ceil_div_u64(n.max, SC_TILE);
    T* partials = static_cast<T*>(tmp);
    scan_reduce_kernel<Load, T><<<(unsigned)nb, SC_THREADS, 0, s>>>(ld, n, partials);
    scan_spine_kernel<T><<<1, SPINE_THREADS, 0, s>>>(partials, nb, total_out, write_end ? out : nullptr, n);
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

struct RankSmem {
    uint32_t whist[RS_WARPS * 256];  // per-warp digit counts, then per-warp prefixes
    uint32_t boff[256];              // first output position of each digit of the block
    uint32_t dstart[256];            // first block-local position of each digit
    uint32_t scan_buf[33];
    uint32_t skeys[RS_TILE];         // keys in block-local sorted order
    uint32_t svals[RS_TILE];         // values in block-local sorted order
};

// How a pass stores its output.  A two-pass sort of keys of at most 16 bits
// whose values fit beside the high key bits in one word packs the first pass's
// output: word = (key >> 8) << vb | value (vb value bits); the second pass
// sorts these words on bits [vb, 32) and writes word & (2^vb - 1).  The first
// pass of such a sort reads its keys as 16-bit words.
enum PassMode { kPlain = 0, kPackOut = 1, kPackIn = 2 };

// Stable rank of the block's keys (held in registers, warp w owning the
// contiguous segment [w*SEG, (w+1)*SEG) in rounds of 32 lanes) and scatter:
// first into shared memory in block-local digit order, then to global memory
// in runs of consecutive positions per digit.  Equal digits inside a round are
// found with one ballot per digit bit.  Values are fetched after the ranking
// (get_val(block-local index)), so they do not occupy registers during it.
// MODE kPackOut writes packed words to kout (shift 0); kPackIn takes the
// values from the packed words and writes them to vout (shift vb).
template <bool WRITE_KEYS, int NB, int MODE, class GetVal>
__device__ __forceinline__ void rank_and_scatter(RankSmem& sm, const uint32_t (&k)[RS_ITEMS], uint64_t n, int shift,
                                                 const uint32_t* __restrict__ offsets, uint32_t nblocks,
                                                 uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                 GetVal get_val, const uint32_t* __restrict__ gsrc,
                                                 uint32_t* __restrict__ gout, int vb) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const uint64_t block0 = (uint64_t)blockIdx.x * RS_TILE;
    const int local0 = warp * RS_SEG + lane;
    const uint64_t base = block0 + local0;
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) sm.whist[i] = 0;
    sm.boff[threadIdx.x] = offsets[(uint64_t)threadIdx.x * nblocks + blockIdx.x];
    __syncthreads();
    uint32_t* wh = sm.whist + warp * 256;
    uint32_t lr[RS_ITEMS];
#pragma unroll
    for (int j = 0; j < RS_ITEMS; j++) {
        const bool ok = base + (uint64_t)j * 32 < n;
        const uint32_t d = (k[j] >> shift) & 0xffu;
        uint32_t peers = __ballot_sync(kFull, ok);
#pragma unroll
        for (int b = 0; b < NB; b++) {  // digit bits above NB are zero in this pass
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
    // values are read before the barrier that precedes the scatter, so a
    // source may keep them in the staging the scatter overwrites
    uint32_t vv[RS_ITEMS];
    if (MODE != kPackIn) {
#pragma unroll
        for (int j = 0; j < RS_ITEMS; j++) vv[j] = base + (uint64_t)j * 32 < n ? get_val(local0 + j * 32) : 0u;
    }
    __syncthreads();
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; w++) {
        const uint32_t c = sm.whist[w * 256 + threadIdx.x];
        sm.whist[w * 256 + threadIdx.x] = run;
        run += c;
    }
    uint32_t total;
    sm.dstart[threadIdx.x] = block_exclusive_scan<uint32_t>(run, sm.scan_buf, total);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < RS_ITEMS; j++) {
        if (base + (uint64_t)j * 32 < n) {
            const uint32_t d = (k[j] >> shift) & 0xffu;
            const uint32_t lp = sm.dstart[d] + wh[d] + lr[j];
            sm.skeys[lp] = k[j];
            if (MODE != kPackIn) sm.svals[lp] = vv[j];
        }
    }
    __syncthreads();
    const int cnt = (int)(n - block0 < (uint64_t)RS_TILE ? n - block0 : (uint64_t)RS_TILE);
    for (int i = threadIdx.x; i < cnt; i += RS_THREADS) {
        const uint32_t key = sm.skeys[i];
        const uint32_t d = (key >> shift) & 0xffu;
        const uint32_t pos = sm.boff[d] + (uint32_t)i - sm.dstart[d];
        if (MODE == kPackOut) {
            kout[pos] = (key >> 8) << vb | sm.svals[i];
        } else if (MODE == kPackIn) {
            vout[pos] = key & ((1u << vb) - 1u);
        } else {
            vout[pos] = sm.svals[i];
            if (WRITE_KEYS) kout[pos] = key;
            if (gout) gout[pos] = gsrc[sm.svals[i]];
        }
    }
}

// Per-block digit histogram, stored digit-major so that one exclusive scan of
// the whole table gives every block's first output position per digit.
__global__ void __launch_bounds__(RS_THREADS) rs_upsweep(const uint32_t* __restrict__ keys, Count cn, int shift,
                                                        uint32_t* __restrict__ counts, uint32_t nblocks) {
    __shared__ uint32_t hist[RS_WARPS * 256];
    const uint64_t n = cn.get();
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

// vin == nullptr: the values are the keys' positions (an identity
// permutation, generated instead of read).  gout != nullptr: also writes
// gout[pos] = gsrc[value] (a per-element array carried into sorted order).
// The same table for a pass whose digits take at most 32 values (the tile
// sort's last pass over the tile ids' high bits): each lane counts into its
// own column of a per-warp table (digit-major, lane-minor: a lane's updates
// hit its own bank, and are plain read-modify-writes, not atomics, since no
// other lane touches the column), then a skewed sweep sums the columns.
// Shared-memory atomics from 32 lanes on a handful of digits serialise.
__global__ void __launch_bounds__(RS_THREADS) rs_upsweep_narrow(const uint32_t* __restrict__ keys, Count cn, int shift,
                                                               uint32_t mask, uint32_t* __restrict__ counts,
                                                               uint32_t nblocks) {
    __shared__ uint32_t cnt[RS_WARPS][32 * 32];
    __shared__ uint32_t wsum[RS_WARPS][32];
    const uint64_t n = cn.get();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* c = cnt[warp];
    for (int i = lane; i < 32 * 32; i += 32) c[i] = 0;
    __syncwarp();
    const uint64_t base = (uint64_t)blockIdx.x * RS_TILE + warp * RS_SEG + lane;
#pragma unroll
    for (int j = 0; j < RS_ITEMS; j++) {
        const uint64_t idx = base + (uint64_t)j * 32;
        if (idx < n) c[((keys[idx] >> shift) & mask) * 32 + lane] += 1u;
    }
    __syncwarp();
    // lane d sums digit d's column, starting at a different lane per digit
    uint32_t sum = 0;
#pragma unroll 8
    for (int i = 0; i < 32; i++) sum += c[lane * 32 + ((i + lane) & 31)];
    wsum[warp][lane] = sum;
    __syncthreads();
    uint32_t total = 0;
    if (threadIdx.x < 32) {
#pragma unroll
        for (int w = 0; w < RS_WARPS; w++) total += wsum[w][threadIdx.x];
    }
    counts[(uint64_t)threadIdx.x * nblocks + blockIdx.x] = threadIdx.x < 32 ? total : 0u;
}

// NB: significant bits of this pass's digit (8, or fewer in a last pass over
// the high bits of keys narrower than a whole number of digits); MODE and vb:
// see PassMode.
template <bool WRITE_KEYS, int NB = 8, int MODE = kPlain>
__global__ void __launch_bounds__(RS_THREADS, 3) rs_downsweep(const uint32_t* __restrict__ kin,
                                                             const uint32_t* __restrict__ vin,
                                                             uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                             Count cn, int shift,
                                                             const uint32_t* __restrict__ offsets, uint32_t nblocks,
                                                             const uint32_t* __restrict__ gsrc = nullptr,
                                                             uint32_t* __restrict__ gout = nullptr, int vb = 0) {
    __shared__ RankSmem sm;
    const uint64_t n = cn.get();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t block0 = (uint64_t)blockIdx.x * RS_TILE;
    if (block0 >= n) return;  // a block past the keys (capturable mode)
    const uint64_t base = block0 + warp * RS_SEG + lane;
    uint32_t k[RS_ITEMS];
#pragma unroll
    for (int j = 0; j < RS_ITEMS; j++) {
        const uint64_t idx = base + (uint64_t)j * 32;
        // kPackOut reads the 16-bit keys of a two-pass sort
        k[j] = idx >= n ? 0u : MODE == kPackOut ? (uint32_t)reinterpret_cast<const uint16_t*>(kin)[idx] : kin[idx];
    }
    rank_and_scatter<WRITE_KEYS, NB, MODE>(
        sm, k, n, shift, offsets, nblocks, kout, vout,
        [&](int local) { return vin ? vin[block0 + local] : (uint32_t)(block0 + local); }, gsrc, gout, vb);
}

// ---------------------------------------------------------------------------
// duplication: one (tile, record) entry per tile a record's rectangle covers,
// in the order of the depth-sorted records (rectangle tiles row-major).  Key
// index k belongs to the record r with off[r] <= k < off[r+1].  Each block
// emits one radix tile of entries and the histogram of their first digit, so
// the first radix pass needs no separate histogram sweep.
// ---------------------------------------------------------------------------
struct DupSrc {
    const uint32_t* order;             // records by depth
    const unsigned long long* off;     // [R + 1] exclusive scan of tiles in that order
    Count R;
    const unsigned long long* desc;    // tile descriptors (pack_tile_desc), record order
    const DevCam* cams;
    uint32_t tiles;
};

// Index of the record holding entry k: a binary search over the offsets of
// the records that cover the block (staged in shared memory, relative to k0),
// or over all offsets when they did not fit.
__device__ __forceinline__ uint64_t dup_record(const DupSrc& src, const int* s_off, uint64_t rlo, int nr, uint64_t k0,
                                               uint64_t k) {
    if (nr > 0) {
        const int kk = (int)(k - k0);
        int lo = 0, hi = nr - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= kk) lo = mid; else hi = mid - 1;
        }
        return rlo + lo;
    }
    uint64_t lo = 0, hi = src.R.get() - 1;
    while (lo < hi) {
        const uint64_t mid = (lo + hi + 1) >> 1;
        if (src.off[mid] <= k) lo = mid; else hi = mid - 1;
    }
    return lo;
}

constexpr int DUP_ITEMS = RS_ITEMS;  // consecutive entries per thread
constexpr int DUP_MAXR = 1024;       // records a block stages in shared memory

// first[b] = the record holding entry b * TILE, for every radix block b:
// each record fills the blocks whose first entry it holds, so no block has to
// search for its records; the block after the last entry gets R - 1.
__global__ void block_starts_kernel(const unsigned long long* __restrict__ off, Count Rc, uint32_t nblocks,
                                    uint32_t* __restrict__ first) {
    const uint64_t R = Rc.get();
    const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r == 0) {
        const uint64_t end = (off[R] + RS_TILE - 1) / RS_TILE;
        first[end < nblocks ? end : nblocks] = (uint32_t)(R - 1);
    }
    if (r >= R) return;
    const uint64_t b0 = (off[r] + RS_TILE - 1) / RS_TILE;
    const uint64_t b1 = (off[r + 1] + RS_TILE - 1) / RS_TILE;  // exclusive
    for (uint64_t b = b0; b < b1 && b < nblocks; b++) first[b] = (uint32_t)r;
}

// K16: keys stored as 16-bit words (tile ids below 2^16; see PassMode).
template <bool K16>
__global__ void __launch_bounds__(RS_THREADS, 4) dup_hist_kernel(DupSrc src, const uint32_t* __restrict__ first_rec,
                                                             Count Kc, uint32_t* __restrict__ keys,
                                                             uint32_t* __restrict__ vals,
                                                             uint32_t* __restrict__ counts, uint32_t nblocks) {
    __shared__ uint32_t hist[RS_WARPS * 256];
    // the block's record offsets and records (ids and tile descriptors,
    // gathered once by all threads together: the loads are independent, so
    // they are all in flight at once); after the generation the same bytes
    // stage the block's entries for coalesced stores
    constexpr int OFF_BYTES = (RS_TILE + 4) * 4;
    constexpr int RAW_BYTES = OFF_BYTES + DUP_MAXR * 20;
    static_assert(RAW_BYTES >= RS_TILE * 8, "entry staging");
    __shared__ __align__(16) unsigned char s_raw[RAW_BYTES];
    int* s_off = reinterpret_cast<int*>(s_raw);
    short4* s_rect = reinterpret_cast<short4*>(s_raw + OFF_BYTES);
    uint32_t* s_rec = reinterpret_cast<uint32_t*>(s_raw + OFF_BYTES + DUP_MAXR * 8);
    uint32_t* s_base = s_rec + DUP_MAXR;
    int* s_tx = reinterpret_cast<int*>(s_base + DUP_MAXR);
    const uint64_t K = Kc.get();
    const uint64_t k0 = (uint64_t)blockIdx.x * RS_TILE;
    if (k0 >= K) {  // a block past the entries (capturable mode): empty histogram
        counts[(uint64_t)threadIdx.x * nblocks + blockIdx.x] = 0u;
        return;
    }
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) hist[i] = 0;
    // records [rlo, rlo + nr) hold this block's entries (the next block's
    // first record may start inside it); a record without tiles shares its
    // offset with the next, so they can outnumber the entries: then search
    // all offsets instead
    const uint64_t rlo = first_rec[blockIdx.x];
    const uint64_t rhi = first_rec[blockIdx.x + 1];
    const int nr = rhi - rlo + 1 <= (uint64_t)RS_TILE ? (int)(rhi - rlo + 1) : -1;
    for (int i = threadIdx.x; i <= nr; i += RS_THREADS) s_off[i] = (int)((long long)src.off[rlo + i] - (long long)k0);
    const bool staged = nr > 0 && nr <= DUP_MAXR;
    if (staged) {
        for (int i = threadIdx.x; i < nr; i += RS_THREADS) {
            const uint32_t rec = src.order[rlo + i];
            const unsigned long long d = src.desc[rec];
            const DevCam& c = src.cams[tile_desc_view(d)];
            s_rec[i] = rec;
            s_rect[i] = tile_desc_rect(d);
            s_base[i] = (uint32_t)c.tile_base;
            s_tx[i] = c.tiles_x;
        }
    }
    __syncthreads();
    // record rr: id, rectangle, view tile base, tiles per row, end of its
    // entries relative to the block's first entry (32-bit arithmetic in the
    // walk: tile ids and entry positions are below 2^32)
    auto load = [&](uint64_t rr, uint32_t& rec, short4& rc, uint32_t& base, int& txs, uint32_t& rend) {
        if (staged) {
            const int li = (int)(rr - rlo);
            rec = s_rec[li];
            rc = s_rect[li];
            base = s_base[li];
            txs = s_tx[li];
            rend = (uint32_t)s_off[li + 1];
        } else {
            rec = src.order[rr];
            const unsigned long long d = src.desc[rec];
            rc = tile_desc_rect(d);
            const DevCam& c = src.cams[tile_desc_view(d)];
            base = (uint32_t)c.tile_base;
            txs = c.tiles_x;
            rend = (uint32_t)(src.off[rr + 1] - k0);
        }
    };
    uint32_t* wh = hist + (threadIdx.x >> 5) * 256;
    const uint32_t cnt_l = (uint32_t)(K - k0 < (uint64_t)RS_TILE ? K - k0 : (uint64_t)RS_TILE);
    const uint32_t first_l = (uint32_t)threadIdx.x * DUP_ITEMS;
    const uint32_t tmax = src.tiles - 1u;
    uint32_t kk[DUP_ITEMS], vv[DUP_ITEMS];
#pragma unroll
    for (int i = 0; i < DUP_ITEMS; i++) kk[i] = vv[i] = 0u;
    if (first_l < cnt_l) {
        const uint64_t first = k0 + first_l;
        uint64_t r = dup_record(src, s_off, rlo, nr, k0, first);
        uint32_t rend, rec, base;
        short4 rc;
        int txs;
        load(r, rec, rc, base, txs, rend);
        int w = max(rc.z - rc.x, 1);
        const uint64_t rstart = staged ? k0 + (uint64_t)(long long)s_off[r - rlo] : src.off[r];
        const uint32_t j = (uint32_t)(first - rstart);
        int tx = rc.x + (int)(j % (uint32_t)w), ty = rc.y + (int)(j / (uint32_t)w);
#pragma unroll
        for (int i = 0; i < DUP_ITEMS; i++) {
            const uint32_t l = first_l + i;
            if (l < cnt_l) {
                while (l >= rend) {  // next record (skipping any without tiles)
                    r++;
                    load(r, rec, rc, base, txs, rend);
                    w = max(rc.z - rc.x, 1);
                    tx = rc.x;
                    ty = rc.y;
                }
                const uint32_t t = base + (uint32_t)ty * (uint32_t)txs + (uint32_t)tx;
                const uint32_t key = t < tmax ? t : tmax;
                kk[i] = key;
                vv[i] = rec;
                atomicAdd(&wh[key & 0xffu], 1u);
                if (++tx == rc.x + w) {
                    tx = rc.x;
                    ty++;
                }
            }
        }
    }
    // stage the entries, then store them coalesced.  Thread t's quads of
    // 32-bit words go to slots 4t + ((q + t/2) & 3), its pairs of 8 16-bit
    // keys to 2t + ((q + t/4) & 1): the eight threads of a 128-byte phase hit
    // distinct banks.
    __syncthreads();
    uint4* sv = reinterpret_cast<uint4*>(s_raw);
    uint4* sk = sv + RS_TILE / 4;
    const int t = threadIdx.x;
#pragma unroll
    for (int q = 0; q < DUP_ITEMS / 4; q++)
        sv[4 * t + ((q + (t >> 1)) & 3)] = make_uint4(vv[4 * q], vv[4 * q + 1], vv[4 * q + 2], vv[4 * q + 3]);
    if (K16) {
#pragma unroll
        for (int q = 0; q < DUP_ITEMS / 8; q++) {
            const uint32_t* h = kk + 8 * q;
            sk[2 * t + ((q + (t >> 2)) & 1)] = make_uint4(h[0] | h[1] << 16, h[2] | h[3] << 16, h[4] | h[5] << 16,
                                                          h[6] | h[7] << 16);
        }
    } else {
#pragma unroll
        for (int q = 0; q < DUP_ITEMS / 4; q++)
            sk[4 * t + ((q + (t >> 1)) & 3)] = make_uint4(kk[4 * q], kk[4 * q + 1], kk[4 * q + 2], kk[4 * q + 3]);
    }
    __syncthreads();
    const uint64_t cnt = K - k0 < (uint64_t)RS_TILE ? K - k0 : (uint64_t)RS_TILE;
    for (int L = t; L < RS_TILE / 4; L += RS_THREADS) {  // values, 4 per quad
        const int owner = L >> 2;
        const uint4 a = sv[4 * owner + (((L & 3) + (owner >> 1)) & 3)];
        const uint64_t e = (uint64_t)L * 4;
        if (e + 4 <= cnt) {
            reinterpret_cast<uint4*>(vals + k0)[L] = a;
        } else {
            const uint32_t va[4] = {a.x, a.y, a.z, a.w};
            for (int i = 0; i < 4 && e + i < cnt; i++) vals[k0 + e + i] = va[i];
        }
    }
    constexpr int KPER = K16 ? 8 : 4;  // keys per quad
    for (int L = t; L < RS_TILE / KPER; L += RS_THREADS) {
        const int owner = K16 ? L >> 1 : L >> 2;
        const uint4 a = K16 ? sk[2 * owner + (((L & 1) + (owner >> 2)) & 1)]
                            : sk[4 * owner + (((L & 3) + (owner >> 1)) & 3)];
        const uint64_t e = (uint64_t)L * KPER;
        if (e + KPER <= cnt) {
            if (K16) reinterpret_cast<uint4*>(reinterpret_cast<uint16_t*>(keys) + k0)[L] = a;
            else reinterpret_cast<uint4*>(keys + k0)[L] = a;
        } else {
            const uint32_t ka[4] = {a.x, a.y, a.z, a.w};
            for (int i = 0; i < KPER && e + i < cnt; i++) {
                if (K16) reinterpret_cast<uint16_t*>(keys)[k0 + e + i] = (uint16_t)(ka[i >> 1] >> (16 * (i & 1)));
                else keys[k0 + e + i] = ka[i];
            }
        }
    }
    uint32_t sum = 0;
#pragma unroll
    for (int w2 = 0; w2 < RS_WARPS; w2++) sum += hist[w2 * 256 + threadIdx.x];
    counts[(uint64_t)threadIdx.x * nblocks + blockIdx.x] = sum;
}

// ---------------------------------------------------------------------------
// per-tile list lengths from the records' rectangles (2D difference counts),
// so the tile ranges need no pass over the sorted keys
// ---------------------------------------------------------------------------
__global__ void rect_diff_kernel(const short4* __restrict__ rect, const int* __restrict__ rec_v, Count Rc,
                                 const DevCam* __restrict__ cams, int* __restrict__ diff) {
    const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= Rc.get()) return;
    const short4 rc = rect[r];
    if (rc.z <= rc.x || rc.w <= rc.y) return;
    const DevCam& cam = cams[rec_v[r]];
    const long long W1 = cam.tiles_x + 1;
    int* d = diff + cam.diff_base;
    atomicAdd(d + rc.y * W1 + rc.x, 1);
    atomicAdd(d + rc.y * W1 + rc.z, -1);
    atomicAdd(d + rc.w * W1 + rc.x, -1);
    atomicAdd(d + rc.w * W1 + rc.z, 1);
}

// The same difference grid accumulated in shared memory: each block adds the
// corners of a contiguous chunk of records into its own copy of the grid of
// all views (no contention between blocks), then writes it out as one partial
// grid; sum_parts_kernel adds the partial grids.  Same-address atomics in L2
// serialise when many small rectangles share corners; shared-memory atomics
// spread over 32 banks per SM do not.
constexpr int RD_PARTS = 304;      // partial grids (2 per SM on 152 SMs)
constexpr int RD_THREADS = 512;
constexpr long long RD_MAX_CELLS = 54 * 1024;  // 216 KB of int counters

__global__ void __launch_bounds__(RD_THREADS)
rect_diff_smem_kernel(const short4* __restrict__ rect, const int* __restrict__ rec_v, Count Rc,
                      const DevCam* __restrict__ cams, int cells, int* __restrict__ parts) {
    extern __shared__ int grid[];
    const uint64_t R = Rc.get();
    for (int c = threadIdx.x; c < cells; c += blockDim.x) grid[c] = 0;
    __syncthreads();
    const uint64_t chunk = (R + gridDim.x - 1) / gridDim.x;
    const uint64_t r0 = (uint64_t)blockIdx.x * chunk;
    const uint64_t r1 = r0 + chunk < R ? r0 + chunk : R;
    for (uint64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        const short4 rc = rect[r];
        if (rc.z <= rc.x || rc.w <= rc.y) continue;
        const DevCam& cam = cams[rec_v[r]];
        const int W1 = cam.tiles_x + 1;
        int* d = grid + cam.diff_base;
        atomicAdd(d + rc.y * W1 + rc.x, 1);
        atomicAdd(d + rc.y * W1 + rc.z, -1);
        atomicAdd(d + rc.w * W1 + rc.x, -1);
        atomicAdd(d + rc.w * W1 + rc.z, 1);
    }
    __syncthreads();
    int* out = parts + (size_t)blockIdx.x * cells;
    for (int c = threadIdx.x; c < cells; c += blockDim.x) out[c] = grid[c];
}

__global__ void sum_parts_kernel(const int* __restrict__ parts, int cells, int nparts, int* __restrict__ diff) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cells) return;
    int acc = 0;
    for (int p = 0; p < nparts; p++) acc += parts[(size_t)p * cells + c];
    diff[c] = acc;
}

// One block per view: prefix sums along rows, then along columns, give the
// number of records covering each tile.
__global__ void diff_to_counts_kernel(const DevCam* __restrict__ cams, int* __restrict__ diff,
                                      uint32_t* __restrict__ counts) {
    const DevCam& cam = cams[blockIdx.x];
    const int W1 = cam.tiles_x + 1, H1 = cam.tiles_y + 1;
    int* d = diff + cam.diff_base;
    for (int y = threadIdx.x; y < H1; y += blockDim.x) {
        int run = 0;
        for (int x = 0; x < W1; x++) {
            run += d[y * W1 + x];
            d[y * W1 + x] = run;
        }
    }
    __syncthreads();
    for (int x = threadIdx.x; x < W1; x += blockDim.x) {
        int run = 0;
        for (int y = 0; y < H1; y++) {
            run += d[y * W1 + x];
            d[y * W1 + x] = run;
        }
    }
    __syncthreads();
    const int n = cam.tiles_x * cam.tiles_y;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        counts[cam.tile_base + i] = (uint32_t)d[(i / cam.tiles_x) * W1 + (i % cam.tiles_x)];
}

// Sort key of a tile for the blend's processing order: longest lists first.
// Blend processing order: tiles by decreasing list length, in 256 length
// classes (8 per octave: the exponent and three mantissa bits of length + 1),
// tile id order inside a class; the persistent blend kernels take the longest
// lists first so that no heavy tile is left for the end of the queue.  One
// block sorts all tiles by counting in shared memory (one launch instead of a
// radix sort's ten).
constexpr int TO_THREADS = 1024;
constexpr int TO_WARPS = TO_THREADS / 32;

__device__ __forceinline__ uint32_t length_class(long long len) {
    const unsigned long long v = (unsigned long long)(len > 0 ? len : 0) + 1ull;
    const int e = 63 - __clzll((long long)v);
    const uint32_t m = e >= 3 ? (uint32_t)(v >> (e - 3)) & 7u : (uint32_t)(v << (3 - e)) & 7u;
    const uint32_t b = 8u * (uint32_t)e + m;  // grows with the length
    return 255u - (b < 255u ? b : 255u);      // 0: the longest lists
}

__global__ void __launch_bounds__(TO_THREADS) tile_order_kernel(const long long* __restrict__ ranges, long long tiles,
                                                                uint32_t* __restrict__ order) {
    __shared__ uint32_t off[256];                // per class: next output position
    __shared__ uint32_t wcnt[TO_WARPS][256];     // per warp and class, within a chunk
    __shared__ uint32_t buf[33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    auto cls = [&](long long t) { return length_class(ranges[2 * t + 1] - ranges[2 * t]); };
    if (threadIdx.x < 256) off[threadIdx.x] = 0;
    __syncthreads();
    for (long long t = threadIdx.x; t < tiles; t += TO_THREADS) atomicAdd(&off[cls(t)], 1u);
    __syncthreads();
    uint32_t total;
    const uint32_t c0 = threadIdx.x < 256 ? off[threadIdx.x] : 0u;
    const uint32_t ex = block_exclusive_scan<uint32_t>(c0, buf, total);
    if (threadIdx.x < 256) off[threadIdx.x] = ex;
    __syncthreads();
    // stable scatter, chunk by chunk in tile order: rank inside the warp by
    // matching classes, then add the counts of the warps before
    for (long long base = 0; base < tiles; base += TO_THREADS) {
        const long long t = base + threadIdx.x;
        const bool valid = t < tiles;
        const uint32_t c = valid ? cls(t) : 256u;
        const uint32_t peers = __match_any_sync(kFull, c);
        for (int i = lane; i < 256; i += 32) wcnt[warp][i] = 0;
        __syncwarp();
        if (valid && (peers & lt) == 0) wcnt[warp][c] = (uint32_t)__popc(peers);
        __syncthreads();
        if (threadIdx.x < 256) {
            uint32_t run = off[threadIdx.x];
            for (int w = 0; w < TO_WARPS; w++) {
                const uint32_t n = wcnt[w][threadIdx.x];
                wcnt[w][threadIdx.x] = run;
                run += n;
            }
            off[threadIdx.x] = run;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = wcnt[warp][c] + (uint32_t)__popc(peers & lt);
            if ((long long)pos < tiles) order[pos] = (uint32_t)t;
        }
        __syncthreads();
    }
}

// Ranges are clamped to the entries that were generated (all of them unless
// a capturable call ran out of key capacity).
__global__ void ranges_kernel(const unsigned long long* __restrict__ starts, long long tiles, Count Kc,
                              long long* __restrict__ ranges) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= tiles) return;
    const unsigned long long K = Kc.get();
    ranges[2 * t] = (long long)(starts[t] < K ? starts[t] : K);
    ranges[2 * t + 1] = (long long)(starts[t + 1] < K ? starts[t + 1] : K);
}

}  // namespace

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
size_t scan_temp_bytes(uint64_t n) { return (ceil_div_u64(n, SC_TILE) + 1) * sizeof(unsigned long long); }

void scan_i32_to_i64(const int* in, long long* out, uint64_t n, void* tmp, cudaStream_t s) {
    scan_impl(LoadDirect<int, long long>{in}, out, n, true, (long long*)nullptr, tmp, s);
}

void scan_masked_i32_to_i64(const int* in, int mask, long long* out, uint64_t n, void* tmp, cudaStream_t s) {
    scan_impl(LoadMasked{in, mask}, out, n, true, (long long*)nullptr, tmp, s);
}

void scan_u32_to_u64(const uint32_t* in, unsigned long long* out, uint64_t n, void* tmp, cudaStream_t s) {
    scan_impl(LoadDirect<uint32_t, unsigned long long>{in}, out, n, true, (unsigned long long*)nullptr, tmp, s);
}

void scan_u32_to_u64_count(const uint32_t* in, unsigned long long* out, Count n, unsigned long long* total,
                           void* tmp, cudaStream_t s) {
    scan_impl(LoadDirect<uint32_t, unsigned long long>{in}, out, n, true, total, tmp, s);
}

void scan_gather_u32_to_u64(const uint32_t* in, const uint32_t* idx, unsigned long long* out, Count n,
                            unsigned long long* total, void* tmp, cudaStream_t s) {
    scan_impl(LoadGather<unsigned long long>{in, idx}, out, n, true, total, tmp, s);
}

static uint64_t radix_blocks(uint64_t n) { return ceil_div_u64(n, RS_TILE); }

size_t radix_temp_bytes(uint64_t n) {
    const uint64_t nb = radix_blocks(n > 0 ? n : 1);
    const size_t counts = ((256 * nb * sizeof(uint32_t)) + 255) / 256 * 256;
    return counts + (scan_temp_bytes(256 * nb) + 255) / 256 * 256;
}

size_t tile_sort_temp_bytes(uint64_t K) {
    return radix_temp_bytes(K) + ((radix_blocks(K > 0 ? K : 1) + 1) * sizeof(uint32_t) + 255) / 256 * 256;
}

namespace {
// One radix pass: histogram, scan, scatter.
template <class Up, class Down>
void radix_pass(uint64_t n, void* tmp, cudaStream_t s, Up up, Down down) {
    const uint64_t nb = radix_blocks(n);
    uint32_t* counts = static_cast<uint32_t*>(tmp);
    void* scan_tmp = static_cast<char*>(tmp) + ((256 * nb * sizeof(uint32_t)) + 255) / 256 * 256;
    up((unsigned)nb, counts);
    scan_impl(LoadDirect<uint32_t, uint32_t>{counts}, counts, Count(256 * nb), false, (uint32_t*)nullptr, scan_tmp, s);
    down((unsigned)nb, counts);
    note_launches(2);
}
}  // namespace

void radix_sort_pairs(const uint32_t* keys0, const uint32_t* vals0, uint32_t* keys_a, uint32_t* vals_a,
                      uint32_t* keys_b, uint32_t* vals_b, uint32_t* vals_out, Count n, int bits, void* tmp,
                      cudaStream_t s, const uint32_t* gather_src, uint32_t* gather_out) {
    if (n.max == 0) return;
    const int passes = (bits + 7) / 8 > 0 ? (bits + 7) / 8 : 1;
    // pass 0 reads (keys0, vals0); later passes ping-pong b -> a -> b ...
    const uint32_t* kin = keys0;
    const uint32_t* vin = vals0;
    for (int p = 0; p < passes; p++) {
        const bool last = p == passes - 1;
        uint32_t* kout = (p & 1) ? keys_a : keys_b;
        uint32_t* vout = last ? vals_out : ((p & 1) ? vals_a : vals_b);
        const int shift = 8 * p;
        const uint32_t* gs = last ? gather_src : nullptr;
        uint32_t* go = last ? gather_out : nullptr;
        radix_pass(
            n.max, tmp, s,
            [&](unsigned nb, uint32_t* counts) { rs_upsweep<<<nb, RS_THREADS, 0, s>>>(kin, n, shift, counts, nb); },
            [&](unsigned nb, uint32_t* counts) {
                if (last)
                    rs_downsweep<false><<<nb, RS_THREADS, 0, s>>>(kin, vin, kout, vout, n, shift, counts, nb, gs, go);
                else
                    rs_downsweep<true><<<nb, RS_THREADS, 0, s>>>(kin, vin, kout, vout, n, shift, counts, nb);
            });
        kin = kout;
        vin = vout;
    }
}

void tile_sort(const uint32_t* order, const unsigned long long* tile_off, Count R, Count K,
               const unsigned long long* desc, const DevCam* cams, long long tiles, int bits, uint32_t* keys_a,
               uint32_t* vals_a, uint32_t* keys_b, uint32_t* vals_b, uint32_t* vals_out, void* tmp, cudaStream_t s) {
    if (K.max == 0 || R.max == 0) return;
    // the radix pass uses the front of tmp; the block starts go behind it
    uint32_t* first_rec = reinterpret_cast<uint32_t*>(static_cast<char*>(tmp) + radix_temp_bytes(K.max));
    const DupSrc src{order, tile_off, R, desc, cams, (uint32_t)tiles};
    const int passes = bits > 8 ? (bits + 7) / 8 : 1;
    // record ids take vb bits; two passes whose second digit fits beside them
    // in one word run packed (PassMode)
    int vb = 1;
    while (vb < 32 && (R.max - 1) >> vb) vb++;
    const bool packed = passes == 2 && (bits - 8) + vb <= 32;
    uint32_t *kin = keys_a, *vin = vals_a, *kout = keys_b, *vout = vals_b;
    for (int p = 0; p < passes; p++) {
        const bool last = p == passes - 1;
        if (last) vout = vals_out;
        const int shift = packed && last ? vb : 8 * p;
        const int hi = bits - 8 * p;  // significant bits of this pass's digit
        radix_pass(
            K.max, tmp, s,
            [&](unsigned nb, uint32_t* counts) {
                // pass 0 writes the entries and the histogram of their first digit
                if (p == 0) {
                    block_starts_kernel<<<(unsigned)ceil_div_u64(R.max, 256), 256, 0, s>>>(tile_off, R, nb, first_rec);
                    if (packed)
                        dup_hist_kernel<true><<<nb, RS_THREADS, 0, s>>>(src, first_rec, K, keys_a, vals_a, counts, nb);
                    else
                        dup_hist_kernel<false><<<nb, RS_THREADS, 0, s>>>(src, first_rec, K, keys_a, vals_a, counts, nb);
                    note_launches(1);
                } else if (hi <= 5) {
                    rs_upsweep_narrow<<<nb, RS_THREADS, 0, s>>>(kin, K, shift, (1u << hi) - 1u, counts, nb);
                } else {
                    rs_upsweep<<<nb, RS_THREADS, 0, s>>>(kin, K, shift, counts, nb);
                }
            },
            [&](unsigned nb, uint32_t* counts) {
                if (packed && !last)
                    rs_downsweep<true, 8, kPackOut><<<nb, RS_THREADS, 0, s>>>(kin, vin, kout, nullptr, K, shift, counts,
                                                                               nb, nullptr, nullptr, vb);
                else if (packed && hi <= 5)
                    rs_downsweep<false, 5, kPackIn><<<nb, RS_THREADS, 0, s>>>(kin, nullptr, nullptr, vout, K, shift,
                                                                               counts, nb, nullptr, nullptr, vb);
                else if (packed)
                    rs_downsweep<false, 8, kPackIn><<<nb, RS_THREADS, 0, s>>>(kin, nullptr, nullptr, vout, K, shift,
                                                                               counts, nb, nullptr, nullptr, vb);
                else if (last && hi <= 5)
                    rs_downsweep<false, 5><<<nb, RS_THREADS, 0, s>>>(kin, vin, kout, vout, K, shift, counts, nb);
                else if (last) rs_downsweep<false><<<nb, RS_THREADS, 0, s>>>(kin, vin, kout, vout, K, shift, counts, nb);
                else rs_downsweep<true><<<nb, RS_THREADS, 0, s>>>(kin, vin, kout, vout, K, shift, counts, nb);
            });
        uint32_t* nk = kin;
        uint32_t* nv = vin;
        kin = kout;
        vin = vout;
        kout = nk;
        vout = nv;
    }
}

size_t tile_order_temp_bytes(long long) { return 256; }

void tile_order(const long long* ranges, long long tiles, uint32_t* order, void*, cudaStream_t s) {
    if (tiles <= 0) return;
    tile_order_kernel<<<1, TO_THREADS, 0, s>>>(ranges, tiles, order);
    note_launches(1);
}

static long long diff_cells(const DevCam* host_cams, int V) {
    long long cells = 0;
    for (int v = 0; v < V; v++) cells += (long long)(host_cams[v].tiles_x + 1) * (host_cams[v].tiles_y + 1);
    return cells;
}

size_t tile_count_temp_bytes(const DevCam* host_cams, int V, long long tiles) {
    const long long cells = diff_cells(host_cams, V);
    const size_t a = ((size_t)cells * sizeof(int) + 255) / 256 * 256;
    const size_t b = ((size_t)tiles * sizeof(uint32_t) + 255) / 256 * 256;
    const size_t c = ((size_t)(tiles + 1) * sizeof(unsigned long long) + 255) / 256 * 256;
    const size_t d = cells <= RD_MAX_CELLS ? (size_t)RD_PARTS * a : 0;
    return a + b + c + d + scan_temp_bytes((uint64_t)tiles);
}

void tile_ranges_from_rects(const short4* rect, const int* rec_v, Count R, Count K, const DevCam* cams,
                            const DevCam* host_cams, int V, long long tiles, long long* ranges, void* tmp,
                            cudaStream_t s) {
    const long long cells = diff_cells(host_cams, V);
    const size_t a = ((size_t)cells * sizeof(int) + 255) / 256 * 256;
    char* base = static_cast<char*>(tmp);
    int* diff = reinterpret_cast<int*>(base);
    base += a;
    uint32_t* counts = reinterpret_cast<uint32_t*>(base);
    base += ((size_t)tiles * sizeof(uint32_t) + 255) / 256 * 256;
    unsigned long long* starts = reinterpret_cast<unsigned long long*>(base);
    base += ((size_t)(tiles + 1) * sizeof(unsigned long long) + 255) / 256 * 256;
    if (cells <= RD_MAX_CELLS) {
        int* parts = reinterpret_cast<int*>(base);
        base += (size_t)RD_PARTS * a;
        const size_t smem = (size_t)cells * sizeof(int);
        // raise the kernel's shared-memory limit once per device, to the
        // largest size used (not at every call: the call may be captured)
        static thread_local int raised[64] = {0};
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev < 64 && raised[dev] < (int)(RD_MAX_CELLS * sizeof(int))) {
            cudaFuncSetAttribute(rect_diff_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(RD_MAX_CELLS * sizeof(int)));
            raised[dev] = (int)(RD_MAX_CELLS * sizeof(int));
        }
        rect_diff_smem_kernel<<<RD_PARTS, RD_THREADS, smem, s>>>(rect, rec_v, R, cams, (int)cells, parts);
        sum_parts_kernel<<<(unsigned)ceil_div_u64((uint64_t)cells, 256), 256, 0, s>>>(parts, (int)cells, RD_PARTS,
                                                                                       diff);
        note_launches(2);
    } else {
        cudaMemsetAsync(diff, 0, (size_t)cells * sizeof(int), s);
        if (R.max > 0) {
            rect_diff_kernel<<<(unsigned)ceil_div_u64(R.max, 256), 256, 0, s>>>(rect, rec_v, R, cams, diff);
            note_launches(1);
        }
    }
    diff_to_counts_kernel<<<V, 256, 0, s>>>(cams, diff, counts);
    scan_u32_to_u64(counts, starts, (uint64_t)tiles, base, s);
    ranges_kernel<<<(unsigned)ceil_div_u64((uint64_t)tiles, 256), 256, 0, s>>>(starts, tiles, K, ranges);
    note_launches(2);
}

}  // namespace mvgs
