// sort.cu -- binning of projected Gaussians into (tile, depth)-ordered pairs.
//
// The order required is that of a stable sort by the 64-bit key
// (global tile << 32) | depth bits with ties broken by record index ("sorted
// Gaussians along the ray", Supp. D.2).  It is produced in two cheaper stages:
//   1. the visible records (radius > 0), compacted in index order, are sorted
//      once by their 32-bit depth with a stable LSD radix sort, giving the
//      records in depth order;
//   2. every visible record emits one (tile, record) pair per overlapped
//      tile, in depth order, and a stable LSD radix sort on the tile bits
//      alone puts the pairs in tile order while keeping depth order inside a
//      tile.
// Each LSD pass counts the digits of every CTA's contiguous segment, scans
// the counts and scatters stably; the grid is the number of CTAs resident at
// once.  The last pass of the pair sort writes the renderer's ids and block
// masks and the tile ranges (from the tile boundaries it sees), so no kernel
// reads the pair list only to find ranges.  Every kernel reads its element
// count from device memory and runs on a grid fixed by the capacities, so the
// sequence needs no host synchronisation and can be captured.
#include <algorithm>

#include "gs_internal.cuh"
#include "gs_kernels.h"

namespace gs {

constexpr int kSortBlocks = 512;  // fixed grid of the segmented kernels
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;  // 2048 elements per block round

// ---------------------------------------------------------------------------
// block-wide exclusive scan (blockDim.x a multiple of 32, <= 1024)

template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T x, T &total, T *smem /* >= 32 */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T inc = x;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) smem[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? smem[lane] : T(0);
        T wi = w;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < nw) smem[lane] = wi - w;  // exclusive prefix of warp totals
        if (lane == nw - 1) smem[32] = wi;
    }
    __syncthreads();
    T res = smem[warp] + inc - x;
    total = smem[32];
    __syncthreads();
    return res;
}

// Contiguous segment of [0, count) owned by this block, a multiple of kSortTile.
__device__ __forceinline__ void block_segment(long long count, long long &beg, long long &end) {
    const long long seg = ceil_div(ceil_div(count, (long long)gridDim.x), (long long)kSortTile) * kSortTile;
    beg = min(count, (long long)blockIdx.x * seg);
    end = min(count, beg + seg);
}

// ---------------------------------------------------------------------------
// stage 0: stable compaction of the visible records with their depth key

__global__ void __launch_bounds__(kSortThreads) k_visible_count(const int *__restrict__ radius, long long nrec,
                                                                 unsigned long long *__restrict__ blk) {
    griddep_wait();
    __shared__ unsigned long long sm[33];
    long long beg, end;
    block_segment(nrec, beg, end);
    unsigned long long c = 0;
    for (long long i = beg + threadIdx.x; i < end; i += kSortThreads) c += radius[i] > 0;
    unsigned long long total;
    block_exclusive_scan<unsigned long long>(c, total, sm);
    if (threadIdx.x == 0) blk[blockIdx.x] = total;
}

// The per-block sums' exclusive prefix for this block and their total, summed by the block
// itself from the kSortBlocks counts (no separate scan launch; integer sums, order-free).
__device__ __forceinline__ void block_prefix(const unsigned long long *__restrict__ blk, unsigned long long &prefix,
                                             unsigned long long &total, unsigned long long *sm) {
    unsigned long long a = 0, b = 0;
    for (int i = threadIdx.x; i < kSortBlocks; i += blockDim.x) {
        const unsigned long long x = blk[i];
        b += x;
        if (i < (int)blockIdx.x) a += x;
    }
    unsigned long long ta, tb;
    block_exclusive_scan<unsigned long long>(a, ta, sm);
    block_exclusive_scan<unsigned long long>(b, tb, sm);
    prefix = ta;
    total = tb;
}

// Writes the visible records in index order with their depth keys; block 0 stores the count.
__global__ void __launch_bounds__(kSortThreads) k_visible_compact(const int *__restrict__ radius,
                                                                   const float4 *__restrict__ rgbd, long long nrec,
                                                                   const unsigned long long *__restrict__ blk,
                                                                   uint32_t *__restrict__ key, uint32_t *__restrict__ val,
                                                                   int *__restrict__ counts) {
    griddep_wait();
    __shared__ unsigned long long sm[33];
    long long beg, end;
    block_segment(nrec, beg, end);
    unsigned long long run, all;
    block_prefix(blk, run, all, sm);
    if (blockIdx.x == 0 && threadIdx.x == 0) counts[0] = (int)min(all, (unsigned long long)0x7fffffff);
    for (long long base = beg; base < end; base += kSortThreads) {
        const long long i = base + threadIdx.x;
        const bool f = i < end && radius[i] > 0;
        unsigned long long total;
        const unsigned long long off = block_exclusive_scan<unsigned long long>(f ? 1ull : 0ull, total, sm);
        if (f) {
            key[run + off] = __float_as_uint(rgbd[i].w);  // depth > near > 0: uint order = float order
            val[run + off] = (uint32_t)i;
        }
        run += total;
    }
}

// ---------------------------------------------------------------------------
// stable LSD radix pass (u32 keys with u32 values), digit of `bits` <= 8 bits
// at `shift`; element count read from *count.  Three kernels: per-CTA digit
// counts of its contiguous segment, their scan (digit-major), and the
// scatter.  The grid is the number of CTAs resident at once (four per SM), so
// every CTA walks one segment in rounds of 4096 elements with no second wave.

constexpr int kRxThreads = 256;
constexpr int kRxItems = 16;
constexpr int kRxRound = kRxThreads * kRxItems;  // 4096 elements per CTA round
constexpr int kRxWarps = kRxThreads / 32;
constexpr int kRxCtasPerSm = 4;
constexpr int kRxBlocks = 148 * kRxCtasPerSm;
constexpr int kRxScanThreads = 608;             // >= kRxBlocks, a multiple of 32

struct RxPass {
    const uint32_t *kin, *vin;
    uint32_t *kout, *vout;  // kout null: keys are not needed after this pass
    const int *count;       // element count (device)
    long long cap;          // capacity of kout / vout / masks (elements)
    int shift, bits;
    long long key_div;      // > 0: the key is value / key_div (a record's view), kin unused
    int nblocks;            // CTAs of the count and scatter kernels (kRxBlocks)
    uint32_t *hist;         // [256][kRxBlocks] per-CTA digit counts, then their scan
    uint32_t *dtotal;       // [256] digit totals
    uint8_t *masks;         // last pass of the pair sort: block masks (key >> 24) ...
    int2 *ranges;           // ... and tile ranges (INT_MAX - first, end) by atomic max
};

__device__ __forceinline__ void rx_segment(long long n, long long &beg, long long &end) {
    const long long seg = ceil_div(ceil_div(n, (long long)gridDim.x), (long long)kRxRound) * kRxRound;
    beg = min(n, (long long)blockIdx.x * seg);
    end = min(n, beg + seg);
}

__device__ __forceinline__ uint32_t rx_key(const RxPass &a, long long i, uint32_t v) {
    return a.key_div > 0 ? (uint32_t)v / (uint32_t)a.key_div : a.kin[i];
}

__global__ void __launch_bounds__(kRxThreads) k_rx_count(RxPass a) {
    griddep_wait();
    __shared__ uint32_t h[kRxWarps][256];
    const int radix = 1 << a.bits;
    const uint32_t mask = radix - 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = lane; i < 256; i += 32) h[warp][i] = 0;
    __syncthreads();
    long long beg, end;
    rx_segment(*a.count, beg, end);
    for (long long i = beg + threadIdx.x; i < end; i += kRxThreads) {
        const uint32_t v = a.key_div > 0 ? a.vin[i] : 0u;
        atomicAdd(&h[warp][(rx_key(a, i, v) >> a.shift) & mask], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < radix; d += kRxThreads) {
        uint32_t c = 0;
        #pragma unroll
        for (int w = 0; w < kRxWarps; ++w) c += h[w][d];
        a.hist[d * kRxBlocks + blockIdx.x] = c;
    }
}

// One CTA per digit: exclusive scan of the digit's per-CTA counts.
__global__ void __launch_bounds__(kRxScanThreads) k_rx_scan(RxPass a) {
    griddep_wait();
    __shared__ uint32_t sm[33];
    const int d = blockIdx.x;
    const bool in = (int)threadIdx.x < a.nblocks;
    const uint32_t x = in ? a.hist[d * kRxBlocks + threadIdx.x] : 0u;
    uint32_t total;
    const uint32_t ex = block_exclusive_scan<uint32_t>(x, total, sm);
    if (in) a.hist[d * kRxBlocks + threadIdx.x] = ex;
    if (threadIdx.x == 0) a.dtotal[d] = total;
}

// The stable scatter.  Each warp ranks its 512 consecutive elements of a
// round per digit (lanes holding the same digit take consecutive ranks after
// the warp's earlier ones), the warps' counts are scanned per digit, the
// round is reordered by digit in shared memory and written out in digit runs.
__global__ void __launch_bounds__(kRxThreads, kRxCtasPerSm) k_rx_scatter(RxPass a) {
    griddep_wait();
    __shared__ uint32_t s_base[256];    // output position of this CTA's next element of each digit
    __shared__ uint32_t s_dstart[257];  // first local slot of each digit in the current round
    __shared__ uint32_t s_whist[kRxWarps][256];
    __shared__ uint32_t s_key[kRxRound];
    __shared__ uint32_t s_val[kRxRound];
    __shared__ uint32_t sm[33];
    const int radix = 1 << a.bits;
    const uint32_t mask = radix - 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int dd = threadIdx.x;  // one thread per digit (radix <= 256 = blockDim)
    {
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan<uint32_t>(dd < radix ? a.dtotal[dd] : 0u, tot, sm);
        if (dd < radix) s_base[dd] = ex + a.hist[dd * kRxBlocks + blockIdx.x];
    }
    long long beg, end;
    rx_segment(*a.count, beg, end);
    for (long long tb = beg; tb < end; tb += kRxRound) {
        const int n_round = (int)min((long long)kRxRound, end - tb);
        for (int i = lane; i < 256; i += 32) s_whist[warp][i] = 0;
        __syncwarp();
        // keys now, values only when they are placed (fewer live registers)
        uint32_t k[kRxItems], rk[kRxItems];
        #pragma unroll
        for (int r = 0; r < kRxItems; ++r) {
            const int li = warp * (32 * kRxItems) + r * 32 + lane;
            const bool valid = li < n_round;
            k[r] = valid ? rx_key(a, tb + li, a.key_div > 0 ? a.vin[tb + li] : 0u) : 0xffffffffu;
        }
        #pragma unroll
        for (int r = 0; r < kRxItems; ++r) {
            const int li = warp * (32 * kRxItems) + r * 32 + lane;
            const bool valid = li < n_round;
            const uint32_t d = (k[r] >> a.shift) & mask;
            // lanes holding the same digit: all `bits` ballots agree (cheaper than a
            // match on digits of high entropy)
            uint32_t peers = __ballot_sync(0xffffffffu, valid);
            for (int b = 0; b < a.bits; ++b) {
                const uint32_t bal = __ballot_sync(0xffffffffu, (d >> b) & 1u);
                peers &= ((d >> b) & 1u) ? bal : ~bal;
            }
            const int leader = valid ? __ffs(peers) - 1 : 0;
            uint32_t base = 0;
            if (valid && lane == leader) {
                base = s_whist[warp][d];
                s_whist[warp][d] = base + __popc(peers);
            }
            base = __shfl_sync(0xffffffffu, base, leader);
            rk[r] = valid ? base + __popc(peers & lt) : 0xffffffffu;
        }
        __syncthreads();
        uint32_t cnt = 0;
        if (dd < radix) {
            #pragma unroll
            for (int w = 0; w < kRxWarps; ++w) {
                const uint32_t c = s_whist[w][dd];
                s_whist[w][dd] = cnt;
                cnt += c;
            }
        }
        {
            uint32_t tot;
            const uint32_t ex = block_exclusive_scan<uint32_t>(dd < radix ? cnt : 0u, tot, sm);
            if (dd < radix) s_dstart[dd] = ex;
            if (dd == 0) s_dstart[radix] = (uint32_t)n_round;
        }
        __syncthreads();
        #pragma unroll
        for (int r = 0; r < kRxItems; ++r) {
            if (rk[r] != 0xffffffffu) {
                const int li = warp * (32 * kRxItems) + r * 32 + lane;
                const uint32_t d = (k[r] >> a.shift) & mask;
                const uint32_t slot = s_dstart[d] + s_whist[warp][d] + rk[r];
                s_key[slot] = k[r];
                s_val[slot] = a.vin[tb + li];
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n_round; i += kRxThreads) {
            const uint32_t key = s_key[i];
            const uint32_t d = (key >> a.shift) & mask;
            const long long pos = (long long)s_base[d] + i - s_dstart[d];
            if (pos >= a.cap) continue;  // cannot happen with consistent counts
            a.vout[pos] = s_val[i];
            if (a.kout) a.kout[pos] = key;
            if (a.masks) {
                a.masks[pos] = (uint8_t)(key >> 24);
                // tile ranges: a round's elements of one digit are sorted by the lower
                // bits already, so a tile's elements are adjacent within the digit's run
                const uint32_t tile = key & 0xffffffu;
                const bool first = (uint32_t)i == s_dstart[d] || (s_key[i - 1] & 0xffffffu) != tile;
                const bool last = (uint32_t)i + 1 == s_dstart[d + 1] || (s_key[i + 1] & 0xffffffu) != tile;
                if (first) atomicMax(&a.ranges[tile].x, 0x7fffffff - (int)pos);
                if (last) atomicMax(&a.ranges[tile].y, (int)(pos + 1));
            }
        }
        __syncthreads();
        if (dd < radix) s_base[dd] += s_dstart[dd + 1] - s_dstart[dd];
        __syncthreads();
    }
}

static void rx_pass(RxPass a, cudaStream_t s) {
    // one wave of CTAs, but no more than a round of kRxRound elements each at the capacity
    a.nblocks = (int)std::min<long long>(kRxBlocks, std::max(1ll, ceil_div(a.cap, (long long)kRxRound)));
    launch_pdl(k_rx_count, a.nblocks, kRxThreads, 0, s, a);
    launch_pdl(k_rx_scan, 1 << a.bits, (a.nblocks + 31) / 32 * 32, 0, s, a);  // a thread per counting CTA
    launch_pdl(k_rx_scatter, a.nblocks, kRxThreads, 0, s, a);
}

// ---------------------------------------------------------------------------
// stage 2: pair emission in depth-rank order

__global__ void __launch_bounds__(kSortThreads) k_tiles_count(const uint32_t *__restrict__ sorted_rec,
                                                               const int *__restrict__ touched,
                                                               const int *__restrict__ counts,
                                                               unsigned long long *__restrict__ blk) {
    griddep_wait();
    __shared__ unsigned long long sm[33];
    long long beg, end;
    block_segment(counts[0], beg, end);
    unsigned long long c = 0;
    for (long long r = beg + threadIdx.x; r < end; r += kSortThreads) c += (unsigned)touched[sorted_rec[r]];
    unsigned long long total;
    block_exclusive_scan<unsigned long long>(c, total, sm);
    if (threadIdx.x == 0) blk[blockIdx.x] = total;
}

// Exclusive offsets of the sorted visible records' pair slots: off[r] for
// r < V and off[V] = total pairs.
__global__ void __launch_bounds__(kSortThreads) k_tiles_offsets(const uint32_t *__restrict__ sorted_rec,
                                                                 const int *__restrict__ touched,
                                                                 const int *__restrict__ counts,
                                                                 const unsigned long long *__restrict__ blk,
                                                                 uint32_t *__restrict__ off, int *counts_out,
                                                                 long long max_pairs, int *__restrict__ status) {
    griddep_wait();
    __shared__ unsigned long long sm[33];
    const long long V = counts[0];
    long long beg, end;
    block_segment(V, beg, end);
    unsigned long long run, all;
    block_prefix(blk, run, all, sm);
    // the pair total: counts[2] = needed, counts[1] = pairs or 0 on overflow; read by later kernels
    const int t32 = (int)min(all, (unsigned long long)0x7fffffff);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        counts_out[2] = t32;
        const bool ok = all <= (unsigned long long)max_pairs;
        counts_out[1] = ok ? t32 : 0;
        if (!ok && status) atomicOr(status, 1 << GS_ERR_CAPACITY);
    }
    for (long long base = beg; base < end; base += kSortThreads) {
        const long long r = base + threadIdx.x;
        const int tt = r < end ? touched[sorted_rec[r]] : 0;
        unsigned long long total;
        const unsigned long long o = run + block_exclusive_scan<unsigned long long>((unsigned long long)tt, total, sm);
        if (r < end) off[r] = (uint32_t)o;
        run += total;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) off[V] = (uint32_t)t32;
}

constexpr int kBigRecord = 128;  // records overlapping more tiles are emitted by a whole CTA

// Pair emission, one warp per 32 consecutive sorted records.  The warp writes
// the slots of its records with at most kBigRecord tiles, 32 at a time: each
// lane finds the record owning its slot by a binary search over the lanes'
// running slot counts (shuffles), then the slot's tile in that record's
// rectangle (row-major) and the mask of the tile's 8x4 blocks the Gaussian
// can reach.  key = tile | mask << 24 (the LSD sort orders on the tile bits
// only, the mask rides along), value = the record (emission follows the depth
// order, so the stable tile partition keeps it without a rank).  Larger records go to a
// list for k_emit_big, so no warp is left with a near-camera Gaussian's
// thousands of tiles.
__device__ __forceinline__ void emit_one(uint32_t o, uint32_t record, int i, int x0, int y0, int w, int toff, int gw,
                                         const Reach &rb, const ViewTable &vt,
                                         uint32_t *__restrict__ pkey, uint32_t *__restrict__ pval) {
    // i / w through a float reciprocal (i < 2^24, w < 2^16), then one exact correction step
    int qt = (int)(((float)i + 0.5f) * __frcp_rn((float)w));
    qt -= (qt * w > i) ? 1 : 0;
    qt += ((qt + 1) * w <= i) ? 1 : 0;
    const int ty = y0 + qt, tx = x0 + (i - qt * w);
    const uint32_t m = block_mask_of(rb, tx * vt.tile_w, ty * vt.tile_h, vt.tile_w);
    pkey[o] = (uint32_t)(toff + ty * gw + tx) | (m << 24);
    pval[o] = record;
}

__global__ void __launch_bounds__(256) k_emit_pairs(const uint32_t *__restrict__ sorted_rec,
                                                     const uint32_t *__restrict__ off,
                                                     const int *__restrict__ radius,
                                                     const float2 *__restrict__ xy, const float4 *__restrict__ co,
                                                     long long ld, ViewTable vt, float alpha_min,
                                                     int *__restrict__ counts, uint32_t *__restrict__ big,
                                                     uint32_t *__restrict__ pkey, uint32_t *__restrict__ pval) {
    griddep_wait();
    if (counts[1] == 0) return;  // nothing to emit, or overflow
    const long long V = counts[0];
    const int lane = threadIdx.x & 31;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long r0 = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; r0 < V;
         r0 += nwarps * 32) {
        const long long r = r0 + lane;
        const bool valid = r < V;
        uint32_t my_off = 0, my_rec = 0;
        int x0 = 0, y0 = 0, w = 1, toff = 0, gw = 1, n_small = 0;
        Reach rb;  // the record's alpha >= alpha_min box, computed once per record
        rb.cx = rb.cy = rb.ex = rb.ey = 0.0f;
        rb.any = false;
        rb.all = false;
        if (valid) {
            const uint32_t rec = sorted_rec[r];
            my_rec = rec;
            my_off = off[r];
            const int nt = (int)(off[r + 1] - my_off);
            if (nt > kBigRecord) {
                big[atomicAdd(&counts[3], 1)] = (uint32_t)r;
            } else {
                const ViewDesc &c = vt.v[(int)(rec / ld)];
                const float2 p = xy[rec];
                rb = reach_box(p, co[rec], alpha_min);
                const Rect rc = tile_rect(p.x, p.y, radius[rec], vt.tile_w, vt.tile_h, c.GW, c.GH);
                x0 = rc.x0; y0 = rc.y0; w = rc.x1 - rc.x0; toff = c.tile_offset; gw = c.GW;
                n_small = nt;
            }
        }
        const int flags = (rb.any ? 1 : 0) | (rb.all ? 2 : 0);
        // running count of small-record slots over the lanes
        int inc = n_small;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        const int excl = inc - n_small;
        const int total = __shfl_sync(0xffffffffu, inc, 31);
        for (int cb = 0; cb < total; cb += 32) {
            const int c = cb + lane;
            // owner: the last lane j with excl_j <= c (lanes with no small slots never win a tie
            // because their excl equals the next lane's)
            int j = 0;
            #pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int cand = j + step;
                const int ecand = __shfl_sync(0xffffffffu, excl, cand & 31);
                if (cand < 32 && ecand <= c) j = cand;
            }
            // skip back over lanes with no small slots that share the same excl
            const int ej = __shfl_sync(0xffffffffu, excl, j);
            const uint32_t oj = __shfl_sync(0xffffffffu, my_off, j);
            const uint32_t recj = __shfl_sync(0xffffffffu, my_rec, j);
            const int jx0 = __shfl_sync(0xffffffffu, x0, j), jy0 = __shfl_sync(0xffffffffu, y0, j);
            const int jw = __shfl_sync(0xffffffffu, w, j), jtoff = __shfl_sync(0xffffffffu, toff, j);
            const int jgw = __shfl_sync(0xffffffffu, gw, j), jn = __shfl_sync(0xffffffffu, n_small, j);
            Reach jr;
            jr.cx = __shfl_sync(0xffffffffu, rb.cx, j); jr.cy = __shfl_sync(0xffffffffu, rb.cy, j);
            jr.ex = __shfl_sync(0xffffffffu, rb.ex, j); jr.ey = __shfl_sync(0xffffffffu, rb.ey, j);
            const int jf = __shfl_sync(0xffffffffu, flags, j);
            jr.any = jf & 1;
            jr.all = (jf & 2) != 0;
            if (c < total && c - ej < jn) {
                const int i = c - ej;
                emit_one(oj + (uint32_t)i, recj, i, jx0, jy0, jw, jtoff, jgw, jr, vt, pkey, pval);
            }
        }
    }
}

// The records with more than kBigRecord tiles, one CTA each (grid-stride).
__global__ void __launch_bounds__(256) k_emit_big(const uint32_t *__restrict__ sorted_rec,
                                                   const uint32_t *__restrict__ off, const int *__restrict__ radius,
                                                   const float2 *__restrict__ xy, const float4 *__restrict__ co,
                                                   long long ld, ViewTable vt, float alpha_min,
                                                   const int *__restrict__ counts, const uint32_t *__restrict__ big,
                                                   uint32_t *__restrict__ pkey, uint32_t *__restrict__ pval) {
    griddep_wait();
    if (counts[1] == 0) return;
    const int nbig = counts[3];
    for (int b = blockIdx.x; b < nbig; b += gridDim.x) {
        const uint32_t r = big[b];
        const uint32_t rec = sorted_rec[r];
        const uint32_t o0 = off[r];
        const int nt = (int)(off[r + 1] - o0);
        const ViewDesc &c = vt.v[(int)(rec / ld)];
        const float2 p = xy[rec];
        const float4 q = co[rec];
        const Rect rc = tile_rect(p.x, p.y, radius[rec], vt.tile_w, vt.tile_h, c.GW, c.GH);
        const Reach rb = reach_box(p, q, alpha_min);
        for (int i = threadIdx.x; i < nt; i += blockDim.x)
            emit_one(o0 + (uint32_t)i, rec, i, rc.x0, rc.y0, rc.x1 - rc.x0, c.tile_offset, c.GW, rb, vt, pkey, pval);
    }
}

// Without a tile pass (one tile in all): ids and masks straight from the
// emitted pairs, which are already in order, and the one tile's range (in
// the encoding the range fix-up of k_tile_hist expects).
__global__ void __launch_bounds__(256) k_unpack_pairs(const uint32_t *__restrict__ pkey,
                                                       const uint32_t *__restrict__ pval, const int *__restrict__ counts,
                                                       int *__restrict__ ids, uint8_t *__restrict__ masks,
                                                       int2 *__restrict__ ranges) {
    griddep_wait();
    const long long P = counts[1];
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        ids[p] = (int)pval[p];
        masks[p] = (uint8_t)(pkey[p] >> 24);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && P > 0) ranges[0] = make_int2(0x7fffffff, (int)P);
}

// ---------------------------------------------------------------------------
// render schedule: tiles by descending pair count (log2 buckets), so the
// compositing kernels start the longest tiles first and their chains overlap
// the many short tiles instead of trailing them.

// The last sort pass leaves each tile's range as (INT_MAX - first, end),
// both accumulated by atomic max over a zeroed array (end 0: no pair);
// this pass turns them into [first, end), empty tiles into (0, 0).
__global__ void __launch_bounds__(256) k_tile_hist(int2 *__restrict__ ranges, int total_tiles,
                                                    unsigned int *__restrict__ bucket) {
    griddep_wait();
    __shared__ unsigned int h[33];
    if (threadIdx.x < 33) h[threadIdx.x] = 0;
    __syncthreads();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total_tiles; t += gridDim.x * blockDim.x) {
        int2 r = ranges[t];
        r = r.y > 0 ? make_int2(0x7fffffff - r.x, r.y) : make_int2(0, 0);
        ranges[t] = r;
        const unsigned c = (unsigned)(r.y - r.x);
        atomicAdd(&h[c ? 32 - __clz(c) : 0], 1u);  // 0 for empty, 1 + floor(log2 c) otherwise
    }
    __syncthreads();
    if (threadIdx.x < 33 && h[threadIdx.x]) atomicAdd(&bucket[threadIdx.x], h[threadIdx.x]);
}

// cursors: bucket 32 (longest) first

// Tiles into their length class's run of the schedule, longest classes first: each block
// forms the classes' starts from the 33 counts itself (bucket[0..32]); bucket[64 + c] are the
// cursors within the classes.
__global__ void __launch_bounds__(256) k_tile_scatter(const int2 *__restrict__ ranges, int total_tiles,
                                                       unsigned int *__restrict__ bucket, int *__restrict__ order) {
    griddep_wait();
    __shared__ unsigned int start[33];
    if (threadIdx.x == 0) {
        unsigned int run = 0;
        for (int b = 32; b >= 0; --b) {
            start[b] = run;
            run += bucket[b];
        }
    }
    __syncthreads();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total_tiles; t += gridDim.x * blockDim.x) {
        const int2 r = ranges[t];
        const unsigned c = (unsigned)(r.y - r.x);
        const int b = c ? 32 - __clz(c) : 0;
        order[start[b] + atomicAdd(&bucket[64 + b], 1u)] = t;
    }
}

// ---------------------------------------------------------------------------
// host side

struct SortWs {
    unsigned long long *blk;
    unsigned int *bucket;
    uint32_t *hist, *dtotal;
    uint32_t *dk0, *dv0, *dk1, *dv1, *off, *big;
    uint32_t *pk0, *pv0, *pk1, *pv1;
    size_t bytes;
};

static SortWs carve(void *base, long long nrec, long long max_pairs) {
    SortWs w;
    size_t off = 0;
    char *b = (char *)base;
    auto take = [&](size_t bytes) {
        char *p = b ? b + off : nullptr;
        off = align_up(off + bytes, 256);
        return p;
    };
    w.blk = (unsigned long long *)take(sizeof(unsigned long long) * (kSortBlocks + 1));
    w.bucket = (unsigned int *)take(sizeof(unsigned int) * 128);  // 33 class counts, 33 cursors at 64
    w.hist = (uint32_t *)take(sizeof(uint32_t) * 256 * kRxBlocks);
    w.dtotal = (uint32_t *)take(sizeof(uint32_t) * 256);
    w.dk0 = (uint32_t *)take(sizeof(uint32_t) * nrec);
    w.dv0 = (uint32_t *)take(sizeof(uint32_t) * nrec);
    w.dk1 = (uint32_t *)take(sizeof(uint32_t) * nrec);
    w.dv1 = (uint32_t *)take(sizeof(uint32_t) * nrec);
    w.off = (uint32_t *)take(sizeof(uint32_t) * (nrec + 1));
    w.big = (uint32_t *)take(sizeof(uint32_t) * (nrec + 1));
    w.pk0 = (uint32_t *)take(sizeof(uint32_t) * max_pairs);
    w.pv0 = (uint32_t *)take(sizeof(uint32_t) * max_pairs);
    w.pk1 = (uint32_t *)take(sizeof(uint32_t) * max_pairs);
    w.pv1 = (uint32_t *)take(sizeof(uint32_t) * max_pairs);
    w.bytes = off;
    return w;
}

size_t sort_workspace_bytes(long long nrec, long long max_pairs) { return carve(nullptr, nrec, max_pairs).bytes; }

// LSD radix sort of (k, v) on bits [0, total_bits) by ping-pong, in passes of
// equal width <= 8.  The last pass writes its values into final_v when given
// and, with masks set, the block masks and tile ranges instead of the keys.
// Returns the buffer pair holding the result (0: k0/v0, 1: k1/v1) when
// final_v is null.
static int radix_sort(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, const int *count, long long cap,
                      int total_bits, uint32_t *hist, uint32_t *dtotal, cudaStream_t s, uint32_t *final_v = nullptr,
                      uint8_t *masks = nullptr, int2 *ranges = nullptr) {
    if (total_bits <= 0) return 0;
    const int passes = (total_bits + 7) / 8;
    const int width = (total_bits + passes - 1) / passes;
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        const int shift = p * width;
        const bool last = p == passes - 1;
        RxPass a;
        a.kin = cur ? k1 : k0;
        a.vin = cur ? v1 : v0;
        a.kout = last ? nullptr : (cur ? k0 : k1);
        a.vout = (last && final_v) ? final_v : (cur ? v0 : v1);
        a.count = count;
        a.cap = cap;
        a.shift = shift;
        a.bits = std::min(width, total_bits - shift);
        a.key_div = 0;
        a.hist = hist;
        a.dtotal = dtotal;
        a.masks = last ? masks : nullptr;
        a.ranges = last ? ranges : nullptr;
        rx_pass(a, s);
        cur ^= 1;
    }
    return cur;
}

size_t key_sort_scratch_bytes() {
    return align_up(sizeof(uint32_t) * 256 * kRxBlocks, 256) + align_up(sizeof(uint32_t) * 256, 256);
}

void launch_key_sort(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, const int *count, long long cap,
                     int bits, void *scratch, uint32_t *final_v, cudaStream_t s) {
    uint32_t *hist = (uint32_t *)scratch;
    uint32_t *dtotal = (uint32_t *)((char *)scratch + align_up(sizeof(uint32_t) * 256 * kRxBlocks, 256));
    radix_sort(k0, v0, k1, v1, count, cap, bits, hist, dtotal, s, final_v);
}

cudaError_t launch_sort(const int *radius, const int *touched, const float2 *xy, const float4 *co, const float4 *rgbd,
                        long long nrec, long long ld, const ViewTable &vt, float alpha_min, int *gauss_ids,
                        int2 *tile_ranges, uint8_t *block_mask, int *tile_order, int *counts, long long max_pairs,
                        void *ws, int *status, cudaStream_t s) {
    SortWs w = carve(ws, nrec, max_pairs);
    cudaError_t e = cudaMemsetAsync(counts, 0, 4 * sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(tile_ranges, 0, sizeof(int2) * (size_t)vt.total_tiles, s);
    if (e != cudaSuccess) return e;

    // stage 1: visible records sorted by depth, then stably by view: records in
    // (view, depth) order, so the emission below gathers one view's records at
    // a time (an L2-sized working set)
    launch_pdl(k_visible_count, kSortBlocks, kSortThreads, 0, s, radius, nrec, w.blk);
    launch_pdl(k_visible_compact, kSortBlocks, kSortThreads, 0, s, radius, rgbd, nrec, w.blk, w.dk0, w.dv0, counts);
    const int dres = radix_sort(w.dk0, w.dv0, w.dk1, w.dv1, counts + 0, nrec, 32, w.hist, w.dtotal, s);
    const uint32_t *sorted_rec = dres ? w.dv1 : w.dv0;
    if (vt.n_views > 1) {
        int view_bits = 0;
        while ((1 << view_bits) < vt.n_views) ++view_bits;
        RxPass a;
        a.kin = nullptr;
        a.vin = sorted_rec;
        a.kout = nullptr;
        a.vout = dres ? w.dv0 : w.dv1;
        a.count = counts + 0;
        a.cap = nrec;
        a.shift = 0;
        a.bits = view_bits;
        a.key_div = ld;
        a.hist = w.hist;
        a.dtotal = w.dtotal;
        a.masks = nullptr;
        a.ranges = nullptr;
        rx_pass(a, s);
        sorted_rec = a.vout;
    }

    // stage 2: pairs in depth order, then a stable partition by tile
    launch_pdl(k_tiles_count, kSortBlocks, kSortThreads, 0, s, sorted_rec, touched, counts, w.blk);
    launch_pdl(k_tiles_offsets, kSortBlocks, kSortThreads, 0, s, sorted_rec, touched, counts, w.blk, w.off, counts,
               max_pairs, status);
    launch_pdl(k_emit_pairs, 148 * 16, 256, 0, s, sorted_rec, w.off, radius, xy, co, ld, vt, alpha_min, counts, w.big, w.pk0,
                                          w.pv0);
    launch_pdl(k_emit_big, 148 * 4, 256, 0, s, sorted_rec, w.off, radius, xy, co, ld, vt, alpha_min, counts, w.big, w.pk0,
                                       w.pv0);
    int tile_bits = 0;
    while ((1ll << tile_bits) < (long long)vt.total_tiles) ++tile_bits;
    if (tile_bits > 0) {
        radix_sort(w.pk0, w.pv0, w.pk1, w.pv1, counts + 1, max_pairs, tile_bits, w.hist, w.dtotal, s,
                   (uint32_t *)gauss_ids, block_mask, tile_ranges);
    } else {
        launch_pdl(k_unpack_pairs, 148 * 8, 256, 0, s, w.pk0, w.pv0, counts, gauss_ids, block_mask, tile_ranges);
    }
    e = cudaMemsetAsync(w.bucket, 0, sizeof(unsigned int) * 128, s);
    if (e != cudaSuccess) return e;
    const int tb = (int)std::min<long long>(ceil_div(vt.total_tiles, 256), 148 * 4);
    launch_pdl(k_tile_hist, tb, 256, 0, s, tile_ranges, vt.total_tiles, w.bucket);
    launch_pdl(k_tile_scatter, tb, 256, 0, s, tile_ranges, vt.total_tiles, w.bucket, tile_order);
    return cudaGetLastError();
}

}  // namespace gs
